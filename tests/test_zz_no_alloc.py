"""md_neighbours_noalloc: the neighbour list for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc (code running inside another framework's allocator, or
code that must not grow its device footprint after start-up).  This entry point keeps its
working memory in a fixed-size array inside the library and writes into arrays the caller
owns.  Its result must equal the list that md_build_neighbours builds (compared as sets),
on two calls in a row, the first on a larger system so that stale scratch would show.
The file is named so that pytest collects it last.
"""
import ctypes as C

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
