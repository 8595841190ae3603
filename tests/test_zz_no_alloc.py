"""md_neighbours_noalloc: the neighbour list for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc (code running inside another framework's allocator, or
code that must not grow its device footprint after start-up).  This entry point keeps its
working memory in a fixed-size array inside the library and writes into arrays the caller
owns.  Its result must equal the list that md_build_neighbours builds (compared as sets),
on two calls in a row, the first on a larger system so that stale scratch would show.
The file is named so that pytest collects it last.
"""
import ctypes as C
import dataclasses

import numpy as np
import pytest

from paper_1107_2619_gb300 import inputs as I, md

pytestmark = pytest.mark.gpu

MAX_ATOMS = md.MD_NOALLOC_MAX_ATOMS


@pytest.fixture(scope="module")
def noalloc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1107_2619_gb300 import build
    build.build()
    f = md.lib().md_neighbours_noalloc
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_double, C.c_int32, C.c_void_p, C.c_void_p,
                  C.c_void_p]
    return f


def _rows(count, nl):
    return [tuple(sorted(nl[i, :count[i]].tolist())) for i in range(count.shape[0])]


def _call(f, w, k_max, stream):
    import torch
    n = w.n_atoms
    pos = torch.from_numpy(np.ascontiguousarray(w.pos)).cuda()
    count = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    nl = torch.full((n, k_max), -7, dtype=torch.int32, device="cuda")
    box = np.ascontiguousarray(w.box, dtype=np.float64)
    torch.cuda.synchronize()
    st = f(pos.data_ptr(), n, box.ctypes.data, w.potential.r_cut + w.skin, k_max, count.data_ptr(),
           nl.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    return st, count.cpu().numpy(), nl.cpu().numpy()


def test_noalloc_list_equals_md_build_neighbours_on_two_calls(noalloc):
    import torch
    stream = torch.cuda.Stream()
    for w in (I.bcc_fe_c(14, seed=41), I.bcc_fe(10, seed=42)):
        st, cn, ln = _call(noalloc, w, w.k_max, stream)
        assert st == md.MD_OK
        with md.System(w, precision="mixed") as s:
            s.build_neighbours()
            cg, lg = s.neighbours()
        assert np.array_equal(cn, cg)
        assert _rows(cn, ln) == _rows(cg, lg)
        assert np.all(ln[np.arange(w.k_max)[None, :] >= cn[:, None]] == -1)


def test_noalloc_rejects_sizes_beyond_its_capacity(noalloc):
    box = np.array([1000.0, 1000.0, 1000.0])
    st = noalloc(None, MAX_ATOMS + 1, box.ctypes.data, 4.0, 16, None, None, None)
    assert st == md.MD_ERR_CAPACITY
    st = noalloc(None, 10, box.ctypes.data, 1.0, 16, None, None, None)   # 1000^3 cells > capacity
    assert st == md.MD_ERR_CAPACITY


def test_noalloc_unwrapped_positions_equal_md_build_neighbours(noalloc):
    """Positions outside the box (atoms moved by whole and half box lengths, and by several
    boxes): both entry points take d = r_j - r_i from the coordinates as given and its minimum
    image, so the lists are the same sets."""
    import torch
    w = I.bcc_fe(9, seed=43)
    pos = w.pos.copy()
    n = pos.shape[0]
    shift = np.zeros_like(pos)
    idx = np.arange(n)
    shift[idx % 5 == 1] += w.box * np.array([1.0, 0.0, -1.0])
    shift[idx % 5 == 2] += w.box * np.array([-3.0, 2.0, 1.0])
    shift[idx % 7 == 3] += 0.5 * w.box
    shift[idx % 11 == 4] -= 0.5 * w.box * np.array([1.0, 1.0, 0.0])
    wu = dataclasses.replace(w, pos=pos + shift)
    stream = torch.cuda.Stream()
    st, cn, ln = _call(noalloc, wu, wu.k_max, stream)
    assert st == md.MD_OK
    with md.System(wu, precision="fp64") as s:
        s.build_neighbours()
        cg, lg = s.neighbours()
    assert np.array_equal(cn, cg)
    assert _rows(cn, ln) == _rows(cg, lg)


def test_noalloc_row_overflow_reports_count_and_fills_rows(noalloc):
    """k_max below the longest row: MD_ERR_NBR_OVERFLOW, the true counts, and each cut row
    holds k_max listed neighbours."""
    import torch
    w = I.bcc_fe(8, seed=44)
    k_small = 10                      # bcc Fe has about 14 neighbours inside r_cut + skin
    stream = torch.cuda.Stream()
    st, cn, ln = _call(noalloc, w, k_small, stream)
    assert st == md.MD_ERR_NBR_OVERFLOW
    with md.System(w, precision="fp64") as s:
        s.build_neighbours()
        cg, lg = s.neighbours()
    assert np.array_equal(cn, cg)
    assert (cn > k_small).any()
    full = [set(lg[i, :cg[i]].tolist()) for i in range(w.n_atoms)]
    for i in range(w.n_atoms):
        got = ln[i, :min(cn[i], k_small)]
        assert np.all(got >= 0)
        assert set(got.tolist()) <= full[i]
        assert len(set(got.tolist())) == got.size
        if cn[i] < k_small:
            assert np.all(ln[i, cn[i]:] == -1)


def test_noalloc_rejects_a_box_thinner_than_three_cells(noalloc):
    import torch
    w = I.bcc_fe(6, seed=45)
    r_list = w.potential.r_cut + w.skin
    box = np.array([w.box[0], 2.9 * r_list, w.box[2]])
    pos = torch.from_numpy(np.ascontiguousarray(w.pos)).cuda()
    count = torch.zeros(w.n_atoms, dtype=torch.int32, device="cuda")
    nl = torch.zeros((w.n_atoms, w.k_max), dtype=torch.int32, device="cuda")
    st = noalloc(pos.data_ptr(), w.n_atoms, box.ctypes.data, r_list, w.k_max, count.data_ptr(), nl.data_ptr(),
                 None)
    assert st == md.MD_ERR_BOX
    huge = np.array([1e300, 1e300, 1e300])
    st = noalloc(pos.data_ptr(), w.n_atoms, huge.ctypes.data, r_list, w.k_max, count.data_ptr(), nl.data_ptr(),
                 None)
    assert st == md.MD_ERR_CAPACITY
