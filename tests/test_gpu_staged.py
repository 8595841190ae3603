"""Group walks of the mixed-precision step kernel (MD_PASSES_STAGED, MD_PASSES_CELLS,
MD_PASSES_HALF) against the FP64 oracle.

The walks read each atom's neighbours from a shared-memory copy of its cell group's
neighbourhood: the staged walk through a 16-bit copy of its list row, the cell walk (no Verlet
list) by testing every staged atom of the 27 cells around its own, the half walk through the
half row (j > i) with the neighbour's share summed per stage slot (Newton's third law); a pair
missed or counted twice by the half walk, or a share added to the wrong slot, breaks the force
and energy parity as surely as a wrong position.  A wrong local index, a
missed periodic shift, a stencil cell staged from the wrong place or a candidate range off by a
cell changes a force by far more than the mixed bound, so element-wise force parity at the final
positions of a trajectory checks the staging, the local lists written by both list builds (the
stand-alone rebuild before the first step and the step kernel's own rebuild phases), the
candidate ranges and the group slot tables.

Workloads: fcc Cu (Sutton-Chen knot tables, 5,000 knots, held in shared memory) with Gaussian
displacements, on 3 x 3 x 3 link cells (stencils that wrap onto the same cell twice), 4^3 cells,
a non-cubic 6 x 3 x 4 grid, and the same grid with half the sites empty (about 26 atoms per
cell, so that groups span several cells and the last group of a row is shorter).
"""
import numpy as np
import pytest

import oracle
from mixed_bound import assert_mixed_forces
from paper_1107_2619_gb300 import inputs as I, md

pytestmark = pytest.mark.gpu

# Forces: the bound derived per atom (tests/mixed_bound.py), which covers the group walks' FP32
# periodic shift of the staged coordinates, with the longest sequential sum (lanes=1).
MIXED_PE_TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1107_2619_gb300 import build
    build.build()


def _case(name):
    if name == "cu7":
        return I.fcc_cu(7, seed=21, sigma=0.05, temperature=600.0)
    if name == "cu10":
        return I.fcc_cu(10, seed=22, sigma=0.05)
    if name == "cu_rect":
        w = I.fcc_cu(7, seed=23)
        pos, box = I.replicate(I.FCC_BASIS, (13, 8, 9), 3.615)
        pos = I.gaussian_displace(pos, 0.05, 23)
        n = len(pos)
        sp = np.zeros(n, np.int32)
        vel = I.maxwell_boltzmann(w.potential.masses[sp], 300.0, 23)
        return I.Workload(name="fcc Cu 13x8x9", pos=pos, vel=vel, species=sp, box=box, potential=w.potential,
                          skin=w.skin, k_max=w.k_max, dt_fs=w.dt_fs, steps=1, temperature=300.0)
    if name == "cu_dilute":   # every other atom removed at random: about 26 atoms per cell
        w = _case("cu_rect")
        keep = np.sort(np.random.default_rng(25).permutation(w.n_atoms)[: w.n_atoms // 2])
        return I.Workload(**{**w.__dict__, "name": "fcc Cu 13x8x9, half the sites empty", "pos": w.pos[keep],
                             "vel": w.vel[keep], "species": w.species[keep]})
    raise ValueError(name)


@pytest.mark.parametrize("walk,lanes", [("staged", 1), ("staged", 2), ("staged", 4), ("staged", 8),
                                        ("cells", 1), ("cells", 4), ("half", 1), ("half", 4), ("half", 8)])
@pytest.mark.parametrize("case", ["cu7", "cu10", "cu_rect", "cu_dilute"])
def test_group_walk_steps_match_the_oracle(case, walk, lanes):
    w = _case(case)
    n_steps = 12
    ref = oracle.run_vv(w.pos, w.vel, w.species, w.potential.masses, w.box, w.potential, w.dt_fs, n_steps,
                        w.skin, w.k_max)
    with md.System(w, precision="mixed", lanes_per_atom=lanes, passes=walk) as s:
        p = s.passes()
        assert p["walk"] == walk and p["groups"] > 0 and 1 <= p["cells_per_group"] <= 8
        # at least two stage buffers (the next group staged by bulk copies while one is computed)
        assert p["stage_buffers"] >= 2
        if case == "cu_dilute" and walk != "half":
            assert p["cells_per_group"] >= 4   # groups of several cells, the row's last one shorter
        s.step(n_steps)
        p = s.passes()
        assert p["active"] == 1 and 0 < p["last_max"] <= p["capacity"]
        pos, f, e, img = s.positions(), s.forces(), s.energy(), s.get(md.MD_GET_IMAGE)
    assert np.abs(pos - ref["pos"]).max() < 1e-5
    assert abs(e["pe"] - ref["energies"][-1, 0]) <= MIXED_PE_TOL * abs(ref["energies"][-1, 0])
    # the last force pass of the step kernel (staged) at the GPU's own final positions
    assert_mixed_forces(w, pos, f, img, pe=e["pe"], pe_tol=MIXED_PE_TOL)


@pytest.mark.parametrize("walk", ["staged", "cells", "half"])
def test_group_walk_rebuild_phases_inside_the_step_kernel(walk):
    """Rebuilds every 3 steps: the group slot tables (and local lists) of the step kernel's own
    rebuild phases, then steps that use them; those rebuilds write no global list rows (the cell
    walk no list at all), so the list is built again, at the current positions, when it is asked
    for."""
    w = _case("cu10")
    ref = oracle.run_vv(w.pos, w.vel, w.species, w.potential.masses, w.box, w.potential, w.dt_fs, 14,
                        w.skin, w.k_max, rebuild_every=3)
    with md.System(w, precision="mixed", rebuild_every=3, passes=walk) as s:
        s.step(14)
        e = s.energy()
        assert s.passes()["active"] == 1
        pos, f, img = s.positions(), s.forces(), s.get(md.MD_GET_IMAGE)
        counts = s.get(md.MD_GET_NBR_COUNT)
    assert e["n_rebuilds"] >= 4
    assert np.abs(pos - ref["pos"]).max() < 1e-5
    assert_mixed_forces(w, pos, f, img)
    ref_counts = oracle.neighbours(pos, w.box, w.potential.r_cut + w.skin, w.k_max, "brute")[0]
    assert np.array_equal(counts, ref_counts)


@pytest.mark.parametrize("walk", ["staged", "cells", "half"])
def test_group_and_list_walks_differ_in_rounding_only(walk):
    w = _case("cu_rect")
    with md.System(w, precision="mixed", lanes_per_atom=4, passes=walk) as a, \
            md.System(w, precision="mixed", lanes_per_atom=4, passes="list") as b:
        assert a.passes()["walk"] == walk and b.passes()["walk"] == "list"
        a.step(10)
        b.step(10)
        assert b.passes()["active"] == 0
        fa, fb = a.forces(), b.forces()
        pa, pb = a.positions(), b.positions()
        assert np.abs(pa - pb).max() < 1e-6
        ia, ib = a.get(md.MD_GET_IMAGE), b.get(md.MD_GET_IMAGE)
        ea, eb = a.energy(), b.energy()
    assert_mixed_forces(w, pa, fa, ia, lanes=4)
    assert_mixed_forces(w, pb, fb, ib, lanes=4)
    assert abs(ea["pe"] - eb["pe"]) <= MIXED_PE_TOL * abs(eb["pe"])


def test_auto_takes_the_list_walk():
    with md.System(_case("cu7"), precision="mixed") as s:
        s.step(2)
        p = s.passes()
        assert p["walk"] == "list" and p["active"] == 0


@pytest.mark.parametrize("walk", ["staged", "cells", "half"])
@pytest.mark.parametrize("precision,name", [("fp64", "cu7"), ("mixed", "fe")])
def test_group_walk_where_it_does_not_apply_is_an_argument_error(precision, name, walk):
    if precision == "fp64" and walk == "half":
        pytest.skip("on the FP64 path 'half' is the half list over the full list (tests/test_gpu_pairs.py)")
    w = _case("cu7") if name == "cu7" else I.bcc_fe(8, seed=3)
    with pytest.raises(md.MDError) as ex:
        md.System(w, precision=precision, passes=walk)
    assert ex.value.status == md.MD_ERR_ARG


@pytest.mark.parametrize("walk", ["staged", "cells", "half"])
def test_overfull_group_falls_back_to_the_list_walk_and_back(walk):
    """Squeeze the crystal into half of the box along y (twice the density): the groups whose
    3-cell-high neighbourhood lies inside the dense half hold about twice the atoms the stage
    was sized for, so the build marks them and the step kernel walks the list; a state at the
    original density restores the group walk."""
    w = I.fcc_cu(13, seed=24, sigma=0.02)
    k_max = 400   # the squeezed half has twice the neighbours
    squeezed = w.pos.copy()
    squeezed[:, 1] = np.mod(squeezed[:, 1], w.box[1]) * 0.5
    with md.System(w, precision="mixed", lanes_per_atom=8, passes=walk, k_max=k_max) as s:
        s.step(1)
        assert s.passes()["active"] == 1
        s.set_state(pos=squeezed, vel=np.zeros_like(squeezed))
        s.step(1)
        p = s.passes()
        assert p["last_max"] > p["capacity"] and p["active"] == 0
        pos, f, img = s.positions(), s.forces(), s.get(md.MD_GET_IMAGE)
        wk = I.Workload(**{**w.__dict__, "k_max": k_max})
        assert_mixed_forces(wk, pos, f, img, lanes=8)
        s.set_state(pos=w.pos, vel=w.vel)
        s.step(2)
        assert s.passes()["active"] == 1
        pos, f, img = s.positions(), s.forces(), s.get(md.MD_GET_IMAGE)
    assert_mixed_forces(wk, pos, f, img)


@pytest.mark.parametrize("walk", ["staged", "cells", "half"])
def test_bounded_staging_waits_report_timeout_and_recover(walk):
    """Failure detection without a fault: block 0's staging producer releases no cell group, its
    consumers' bounded mbarrier waits run out, the call returns MD_ERR_TIMEOUT, and the context
    then steps as a fresh one does (the half walk to the run-to-run spread of its FP32 shared
    atomic sums)."""
    w = _case("cu10")
    with md.System(w, precision="mixed", lanes_per_atom=4, passes=walk) as s, \
            md.System(w, precision="mixed", lanes_per_atom=4, passes=walk) as ref:
        s.eam_forces()
        assert s.passes()["active"] == 1
        assert md.md_selftest_timeout(s.ctx) == md.MD_ERR_TIMEOUT
        s.set_state(pos=w.pos, vel=w.vel)
        s.step(6)
        ref.step(6)
        tol = 1e-7 if walk == "half" else 1e-9
        assert np.abs(s.positions() - ref.positions()).max() < tol
        assert abs(s.energy()["pe"] - ref.energy()["pe"]) <= tol * abs(ref.energy()["pe"])
