"""CUDA path (through the C ABI) against the FP64 oracle, on the same seeded inputs.

Bars: neighbour lists bit-exact as sets; FP64 forces, energies and virial within 1e-10
relative (max-norm); the mixed path within its stated bound (below); trajectories of
velocity Verlet within 1e-9 Å after 100 steps; edge cases and device-detected errors.
"""
import numpy as np
import pytest

import oracle
from mixed_bound import assert_mixed_forces
from paper_1107_2619_gb300 import inputs as I, md

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
# Mixed path: every force component within the bound derived per atom from the potential and
# the configuration (tests/mixed_bound.py: the exact share of the FP32 coordinates plus the FP32
# arithmetic of the pair terms and their sums).  PE is summed in FP64 from FP32 per-pair terms.
MIXED_PE_TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1107_2619_gb300 import build
    build.build()


def _rows(count, nl):
    return [tuple(sorted(nl[i, :count[i]].tolist())) for i in range(count.shape[0])]


def _ragged_box(seed):
    """bcc Fe on a non-cubic 7 x 8 x 9 replication, 7 atoms removed (1,001 atoms: a ragged
    tail for every block size), strong displacements and atoms unwrapped by whole boxes."""
    pos, box = I.replicate(I.BCC_BASIS, (7, 8, 9), 2.8665)
    pos = I.gaussian_displace(pos, 0.15, seed)
    keep = np.ones(len(pos), bool)
    keep[[3, 50, 111, 400, 401, 800, 1007]] = False
    pos = pos[keep]
    pos[::4] += box * np.array([2.0, -1.0, 5.0])     # unwrapped images
    n = len(pos)
    pot = I.fs_fe_analytic()
    vel = I.maxwell_boltzmann(pot.masses[np.zeros(n, np.int32)], 300.0, seed)
    return I.Workload(name="ragged", pos=pos, vel=vel, species=np.zeros(n, np.int32),
                      box=box, potential=pot, skin=0.3, k_max=48, dt_fs=1.0, steps=1, temperature=300.0)


def _near_cutoff(seed=9):
    """Pairs placed so that |r_ij| sits within a few ulps of r_list (random directions)."""
    pot = I.fs_fe_analytic()
    rl = pot.r_cut + 0.3
    box = np.array([40.0, 40.0, 40.0])
    u = I.random_uniform(seed, 6, 4000).reshape(-1, 4)
    pos = []
    for k in range(300):
        c = 4.0 + (np.array([k % 6, (k // 6) % 6, k // 36]) * 6.5)
        v = u[k, :3] - 0.5
        v /= np.linalg.norm(v)
        d = rl * (1.0 + (k % 9 - 4) * 2.0 ** -52)
        pos += [c, c + d * v]
    pos = np.array(pos)
    return I.Workload(name="near", pos=pos, vel=np.zeros_like(pos), species=np.zeros(len(pos), np.int32),
                      box=box, potential=pot, skin=0.3, k_max=16, dt_fs=1.0, steps=1, temperature=0.0)


def _workload(name):
    if name == "fe2k":
        return I.bcc_fe(10, seed=1)
    if name == "fe_tables":
        return I.bcc_fe(10, seed=11, tables=True)
    if name == "cu2k":
        return I.fcc_cu(8, seed=2, sigma=0.03)
    if name == "fec":
        return I.bcc_fe_c(10, seed=4)
    if name == "random":
        return _ragged_box(seed=7)
    if name == "near":
        return _near_cutoff()
    if name == "fe_knots":
        return I.bcc_fe(10, seed=13, potential=I.fe_knots())
    if name == "fec_knots":
        import dataclasses
        return dataclasses.replace(I.bcc_fe_c(10, seed=14), potential=I.fe_c_knots())
    raise ValueError(name)


def _gpu_system(w, precision="fp64", **kw):
    return md.System(w, precision=precision, **kw)


# --------------------------------------------------------------------------- neighbour lists
@pytest.mark.parametrize("name", ["fe2k", "cu2k", "fec", "random", "near"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_neighbour_sets_bit_exact(name, precision):
    w = _workload(name)
    with _gpu_system(w, precision) as s:
        s.build_neighbours()
        cg, lg = s.neighbours()
    co, lo, m = oracle.neighbours(w.pos, w.box, w.potential.r_cut + w.skin, w.k_max, "brute")
    assert m <= w.k_max
    assert np.array_equal(cg, co)
    assert _rows(cg, lg) == _rows(co, lo)
    assert np.all(lg[np.arange(w.k_max)[None, :] >= cg[:, None]] == -1)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_neighbour_sets_bit_exact_for_every_cell_remainder(precision):
    """Link cells of 25..56 atoms, built by warp-wide lane groups: after the first 32 atoms of a cell
    the last 1..16 take 32, 16, 8, 4 or 2 lanes each (more than 16 take one each)."""
    w = I.cell_count_gas(np.tile(np.arange(25, 57), 2))
    with _gpu_system(w, precision) as s:
        s.build_neighbours()
        cg, lg = s.neighbours()
    co, lo, m = oracle.neighbours(w.pos, w.box, w.potential.r_cut + w.skin, w.k_max, "brute")
    assert m <= w.k_max
    assert np.array_equal(cg, co)
    assert _rows(cg, lg) == _rows(co, lo)
    assert np.all(lg[np.arange(w.k_max)[None, :] >= cg[:, None]] == -1)


# --------------------------------------------------------------------------- FP64 parity
@pytest.mark.parametrize("name", ["fe2k", "fe_tables", "cu2k", "fec", "random", "fe_knots", "fec_knots"])
def test_fp64_forces_energies_virial_match_oracle(name):
    w = _workload(name)
    ref = oracle.forces(w.pos, w.species, w.box, w.potential, skin=w.skin, k_max=w.k_max, method="brute")
    with _gpu_system(w) as s:
        pe = s.eam_forces()
        f = s.forces()
        rho = s.get(md.MD_GET_RHO)
        dF = s.get(md.MD_GET_DF)
        ea = s.get(md.MD_GET_EATOM)
        e = s.energy()
    fs = np.abs(ref["force"]).max()
    assert np.abs(f - ref["force"]).max() <= FP64_TOL * fs
    assert abs(pe - ref["pe"]) <= FP64_TOL * abs(ref["pe"])
    assert abs(e["pe"] - ref["pe"]) <= FP64_TOL * abs(ref["pe"])
    assert np.abs(rho - ref["rho"]).max() <= FP64_TOL * np.abs(ref["rho"]).max()
    assert np.abs(dF - ref["dF"]).max() <= FP64_TOL * np.abs(ref["dF"]).max()
    assert np.abs(ea - ref["e_atom"]).max() <= FP64_TOL * np.abs(ref["e_atom"]).max()
    ws = np.abs(ref["virial"]).max()
    assert np.abs(e["virial"] - ref["virial"]).max() <= FP64_TOL * ws
    k = oracle.kinetic(w.vel, w.species, w.potential.masses)
    assert abs(e["ke"] - k["ke"]) <= FP64_TOL * max(k["ke"], 1e-300)
    p = oracle.pressure_gpa(k["kin_tensor"], ref["virial"], w.box)
    assert abs(e["pressure_gpa"] - p) <= FP64_TOL * max(abs(p), ws / np.prod(w.box) * 160.2)


@pytest.mark.parametrize("name", ["fe2k", "fe_tables", "cu2k", "fec", "fe_knots", "fec_knots"])
def test_mixed_forces_within_bound(name):
    w = _workload(name)
    ref = oracle.forces(w.pos, w.species, w.box, w.potential, skin=w.skin, k_max=w.k_max, method="brute")
    with _gpu_system(w, "mixed") as s:
        pe = s.eam_forces()
        f = s.forces()
        rho = s.get(md.MD_GET_RHO)
        img = s.get(md.MD_GET_IMAGE)
    assert_mixed_forces(w, w.pos, f, img, pe=pe, pe_tol=MIXED_PE_TOL)
    assert np.abs(rho - ref["rho"]).max() <= 1e-5 * np.abs(ref["rho"]).max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_knot_sums_step_like_the_oracle(precision):
    """Explicit knot sums through the persistent step kernel: 20 steps against the oracle."""
    w = _workload("fec_knots")
    ref = oracle.run_vv(w.pos, w.vel, w.species, w.potential.masses, w.box, w.potential, w.dt_fs, 20,
                        w.skin, w.k_max, strain_rate_zz=w.strain_rate_zz)
    with _gpu_system(w, precision) as s:
        s.step(20)
        pos = s.positions()
        e = s.energy()
    tol = 1e-9 if precision == "fp64" else 1e-5
    assert np.abs(pos - ref["pos"]).max() < tol
    assert abs(e["pe"] - ref["energies"][-1, 0]) <= (1e-10 if precision == "fp64" else 1e-6) * abs(ref["energies"][-1, 0])


@pytest.mark.parametrize("lanes", [1, 4])
def test_two_species_tables_step_like_the_oracle(lanes):
    """Fe-C two-species tables (the Fe-Fe table in shared memory, the C rows from global memory)
    through the persistent step kernel under the strain ramp: 20 steps against the oracle, and
    the last force pass at the GPU's final positions."""
    w = _workload("fec")
    ref = oracle.run_vv(w.pos, w.vel, w.species, w.potential.masses, w.box, w.potential, w.dt_fs, 20,
                        w.skin, w.k_max, strain_rate_zz=w.strain_rate_zz)
    with _gpu_system(w, "mixed", lanes_per_atom=lanes) as s:
        s.step(20)
        pos, f, e, img = s.positions(), s.forces(), s.energy(), s.get(md.MD_GET_IMAGE)
    assert np.abs(pos - ref["pos"]).max() < 1e-5
    assert abs(e["pe"] - ref["energies"][-1, 0]) <= MIXED_PE_TOL * abs(ref["energies"][-1, 0])
    assert_mixed_forces(w, pos, f, img, box=np.array(e["box"]), lanes=lanes, pe=e["pe"], pe_tol=MIXED_PE_TOL)


def test_unwrapped_images_give_the_same_forces():
    w = I.bcc_fe(10, seed=12)
    shifted = I.Workload(**{**w.__dict__, "pos": w.pos + w.box * np.array([3.0, -7.0, 1.0])})
    with _gpu_system(w) as a, _gpu_system(shifted) as b:
        a.eam_forces()
        b.eam_forces()
        fa, fb = a.forces(), b.forces()
    assert np.abs(fa - fb).max() <= FP64_TOL * np.abs(fa).max()


# --------------------------------------------------------------------------- dynamics
def test_fp64_trajectory_matches_oracle_fe2k():
    """The 2,000-atom bcc Fe workload: 100 velocity-Verlet steps of 1 fs (FP64)."""
    w = I.bcc_fe(10, seed=1)
    ref = oracle.run_vv(w.pos, w.vel, w.species, w.potential.masses, w.box, w.potential, w.dt_fs, 100,
                        w.skin, w.k_max)
    with _gpu_system(w) as s:
        pes, kes = [], []
        for _ in range(100):
            s.step(1)
            e = s.energy()
            pes.append(e["pe"])
            kes.append(e["ke"])
        pos, vel = s.positions(), s.velocities()
        e = s.energy()
    scale = abs(ref["energies"][:, 0]).max()
    assert np.abs(np.array(pes) - ref["energies"][:, 0]).max() <= FP64_TOL * scale
    assert np.abs(np.array(kes) - ref["energies"][:, 1]).max() <= FP64_TOL * scale
    assert np.abs(pos - ref["pos"]).max() < 1e-9
    assert np.abs(vel - ref["vel"]).max() < 1e-11
    assert e["n_rebuilds"] == ref["n_rebuilds"]
    assert np.abs(e["momentum"]).max() < 1e-9


def test_mixed_nve_energy_is_conserved():
    w = I.bcc_fe(10, seed=13)
    with _gpu_system(w, "mixed") as s:
        s.eam_forces()
        e0 = s.energy()
        tes = []
        for _ in range(20):
            s.step(10)
            tes.append(s.energy()["te"])
    tes = np.array(tes)
    assert np.abs(tes - e0["te"]).max() < 2e-3 * e0["ke"]


def test_strain_ramp_matches_oracle():
    w = I.bcc_fe(10, seed=14, tables=True)
    w.strain_rate_zz = -1.0e9
    ref = oracle.run_vv(w.pos, w.vel, w.species, w.potential.masses, w.box, w.potential, w.dt_fs, 30,
                        w.skin, w.k_max, strain_rate_zz=w.strain_rate_zz)
    with _gpu_system(w) as s:
        s.step(30)
        e = s.energy()
        pos = s.positions()
    assert np.array_equal(e["box"], ref["box"])
    assert np.abs(pos - ref["pos"]).max() < 1e-9
    assert abs(e["pe"] - ref["energies"][-1, 0]) <= FP64_TOL * abs(ref["energies"][-1, 0])


def test_scheduled_rebuilds_and_determinism():
    w = I.bcc_fe(10, seed=15)
    with _gpu_system(w, "mixed", rebuild_every=5) as a, _gpu_system(w, "mixed", rebuild_every=5) as b:
        a.step(20)
        b.step(20)
        ea = a.energy()
        assert ea["n_rebuilds"] >= 5
        assert np.array_equal(a.positions(), b.positions())
        assert np.array_equal(a.velocities(), b.velocities())
        assert ea["te"] == b.energy()["te"]


def test_state_round_trip_continues_bitwise():
    """Checkpoint/restart (§4.1.3): read the state, write it back, continue; no drift in bits."""
    w = I.bcc_fe(10, seed=16)
    with _gpu_system(w) as a, _gpu_system(w) as b:
        a.step(10)
        pos, vel, f = a.positions(), a.velocities(), a.forces()
        a.set_state(pos, vel, f)
        a.step(10)
        b.step(20)
        assert np.array_equal(a.positions(), b.positions())
        assert np.array_equal(a.velocities(), b.velocities())


def test_device_inputs_match_host_inputs():
    w = I.bcc_fe(10, seed=17)
    with _gpu_system(w) as a, _gpu_system(w, device_inputs=True) as b:
        a.eam_forces()
        b.eam_forces()
        assert np.array_equal(a.forces(), b.forces())


@pytest.mark.parametrize("device", [False, True, "pinned"])
def test_step_io_equals_the_separate_calls(device):
    """md_step_io (state in, steps, state out, energies; one synchronisation) against
    md_set_state + md_step + md_get x3 + md_energy: bitwise equal, host buffers (pageable: copies
    through a device stage; pinned: read and written by the device directly), device buffers,
    and with the same buffers as inputs and outputs."""
    torch = pytest.importorskip("torch")
    w = I.fcc_cu(8, seed=31, sigma=0.03)
    with _gpu_system(w, "mixed") as a, _gpu_system(w, "mixed") as b:
        a.eam_forces()
        b.eam_forces()
        p, v, f = a.positions(), a.velocities(), a.forces()
        for _ in range(3):   # three round trips, as a host-side driver would do them
            b.set_state(p, v, f)
            b.step(4)
            p2, v2, f2, e2 = b.positions(), b.velocities(), b.forces(), b.energy()
            if device == "pinned":
                bufs = [torch.from_numpy(x.copy()).pin_memory() for x in (p, v, f)]
                e1 = a.step_io(4, *bufs, *bufs)
                p1, v1, f1 = (t.numpy() for t in bufs)
            elif device:
                bufs = [torch.from_numpy(x.copy()).cuda() for x in (p, v, f)]
                e1 = a.step_io(4, *bufs, *bufs)
                torch.cuda.synchronize()
                p1, v1, f1 = (t.cpu().numpy() for t in bufs)
            else:
                p1, v1, f1 = p.copy(), v.copy(), f.copy()
                e1 = a.step_io(4, p1, v1, f1, p1, v1, f1)
            assert np.array_equal(p1, p2) and np.array_equal(v1, v2) and np.array_equal(f1, f2)
            assert e1["pe"] == e2["pe"] and e1["ke"] == e2["ke"] and e1["step"] == e2["step"]
            p, v, f = p1, v1, f1
        e = a.step_io(0, pos_out=p1)   # no steps: the copies only
        assert np.array_equal(p1, a.positions()) and e["pe"] == a.energy()["pe"]


@pytest.mark.parametrize("offset", [0, 1])
def test_step_io_pinned_ragged_and_unaligned(offset):
    """The direct pinned-buffer copies move each block's range in 16-byte pieces when the buffer
    is 16-byte aligned, 8-byte pieces when it is not (offset 1: the arrays start one double into a
    pinned allocation): 2,047 atoms (15 full blocks of 128 and a last one of 127, an odd number of
    doubles), bitwise against the separate calls."""
    import dataclasses
    torch = pytest.importorskip("torch")
    w = I.fcc_cu(8, seed=33, sigma=0.03)
    w = dataclasses.replace(w, pos=w.pos[:-1].copy(), vel=w.vel[:-1].copy(), species=w.species[:-1].copy())
    n = w.pos.shape[0]
    assert n % 128 == 127
    with _gpu_system(w, "fp64") as a, _gpu_system(w, "fp64") as b:
        a.eam_forces()
        b.eam_forces()
        p, v, f = a.positions(), a.velocities(), a.forces()
        bufs = []
        for x in (p, v, f):
            t = torch.empty(3 * n + offset, dtype=torch.float64).pin_memory()
            view = t[offset:].view(n, 3)
            view.copy_(torch.from_numpy(x))
            bufs.append(view)
        assert all((t.data_ptr() % 16 == 0) == (offset == 0) for t in bufs)
        for _ in range(2):
            b.set_state(p, v, f)
            b.step(3)
            p2, v2, f2, e2 = b.positions(), b.velocities(), b.forces(), b.energy()
            e1 = a.step_io(3, *bufs, *bufs)
            p1, v1, f1 = (t.numpy().copy() for t in bufs)
            assert np.array_equal(p1, p2) and np.array_equal(v1, v2) and np.array_equal(f1, f2)
            assert e1["pe"] == e2["pe"] and e1["ke"] == e2["ke"]
            p, v, f = p1, v1, f1


# --------------------------------------------------------------------------- edge cases
def test_empty_and_single_atom_systems():
    pot = I.fs_fe_analytic()
    box = np.array([20.0, 20.0, 20.0])
    empty = I.Workload(name="empty", pos=np.zeros((0, 3)), vel=np.zeros((0, 3)), species=np.zeros(0, np.int32),
                       box=box, potential=pot, skin=0.3, k_max=8, dt_fs=1.0, steps=1, temperature=0.0)
    with _gpu_system(empty) as s:
        assert s.eam_forces() == 0.0
        s.step(3)
        e = s.energy()
        assert e["pe"] == 0.0 and e["ke"] == 0.0
    one = I.Workload(name="one", pos=np.array([[1.0, 2.0, 3.0]]), vel=np.array([[0.01, 0.02, -0.03]]),
                     species=np.zeros(1, np.int32), box=box, potential=pot, skin=0.3, k_max=8, dt_fs=2.0,
                     steps=1, temperature=0.0)
    with _gpu_system(one) as s:
        s.step(50)
        assert np.allclose(s.positions(), [[1.0 + 1.0, 2.0 + 2.0, 3.0 - 3.0]], rtol=0, atol=1e-12)


def test_overflow_is_reported():
    w = I.bcc_fe(10, seed=18)
    with _gpu_system(w, k_max=8) as s:
        with pytest.raises(md.MDError) as ei:
            s.eam_forces()
        assert ei.value.status == md.MD_ERR_NBR_OVERFLOW


def test_strict_skin_is_reported():
    w = I.bcc_fe(10, seed=19)
    with _gpu_system(w, strict_skin=True) as s:
        s.step(2)
        pos = s.positions()
        pos[3] += 0.2          # teleport one atom by more than skin/2
        s.set_state(pos=pos)
        with pytest.raises(md.MDError) as ei:
            s.step(1)
        assert ei.value.status == md.MD_ERR_SKIN


def test_coincident_atoms_are_reported_non_finite():
    w = I.bcc_fe(8, seed=20)
    w.pos[5] = w.pos[6]
    with _gpu_system(w) as s:
        with pytest.raises(md.MDError) as ei:
            s.eam_forces()
        assert ei.value.status == md.MD_ERR_NONFINITE


# --------------------------------------------------------------------------- full size
def test_full_size_cu500k_forces_and_lists():
    """fcc Cu 50^3 = 500,000 atoms, Sutton-Chen 5,000-knot tables, in the benchmark's
    configuration: every force (FP64 and mixed) and every neighbour set against the oracle."""
    w = I.fcc_cu(50, seed=2, sigma=0.05)   # displaced: the perfect lattice has zero forces
    ref = oracle.forces(w.pos, w.species, w.box, w.potential, skin=w.skin, k_max=w.k_max, method="cells")
    fs = np.abs(ref["force"]).max()
    with _gpu_system(w) as s:
        pe = s.eam_forces()
        f = s.forces()
        cg, lg = s.neighbours()
    assert np.array_equal(cg, ref["count"])
    lg.sort(axis=1)
    lo = np.where(ref["list"] < 0, np.iinfo(np.int32).max, ref["list"])
    lg = np.where(lg < 0, np.iinfo(np.int32).max, lg)
    lo.sort(axis=1)
    lg.sort(axis=1)
    assert np.array_equal(lg, lo)
    assert np.abs(f - ref["force"]).max() <= FP64_TOL * fs
    assert abs(pe - ref["pe"]) <= FP64_TOL * abs(ref["pe"])
    with _gpu_system(w, "mixed") as s:
        pe32 = s.eam_forces()
        f32 = s.forces()
        img = s.get(md.MD_GET_IMAGE)
    ratio, _ = assert_mixed_forces(w, w.pos, f32, img, pe=pe32, pe_tol=MIXED_PE_TOL)
    print(f"Cu 500k mixed: largest error / derived bound = {ratio:.3f}")


def test_full_size_cu500k_step_kernel_as_benchmarked():
    """The benchmark's launch: fcc Cu 500,000 atoms, mixed, the autotuner's lane count, one
    persistent launch of 30 steps (list rebuilds inside it); the forces of its last force pass
    at its own final positions, and its energies, against the oracle."""
    w = I.fcc_cu(50, seed=2)
    with _gpu_system(w, "mixed") as s:
        s.eam_forces()
        lanes = s.tune()
        s.step(30)
        e = s.energy()
        pos, f, img = s.positions(), s.forces(), s.get(md.MD_GET_IMAGE)
    assert e["n_rebuilds"] >= 1
    ratio, _ = assert_mixed_forces(w, pos, f, img, lanes=lanes, pe=e["pe"], pe_tol=MIXED_PE_TOL)
    print(f"Cu 500k step kernel: largest error / derived bound = {ratio:.3f}")


# --------------------------------------------------------------------------- lanes per atom
@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["fec", "cu2k"])   # two species; one species (table in shared memory)
def test_every_lane_count_matches_oracle(lanes, precision, case):
    w = _workload(case)
    ref = oracle.forces(w.pos, w.species, w.box, w.potential, skin=w.skin, k_max=w.k_max, method="brute")
    fs = np.abs(ref["force"]).max()
    with _gpu_system(w, precision, lanes_per_atom=lanes) as s:
        pe = s.eam_forces()
        f = s.forces()
        img = s.get(md.MD_GET_IMAGE)
        s.step(5)
        e = s.energy()
    if precision == "fp64":
        assert np.abs(f - ref["force"]).max() <= FP64_TOL * fs
        assert abs(pe - ref["pe"]) <= FP64_TOL * abs(ref["pe"])
    else:
        assert_mixed_forces(w, w.pos, f, img, lanes=lanes, pe=pe, pe_tol=MIXED_PE_TOL)
    assert np.isfinite(e["te"])


def test_autotuner_picks_a_valid_lane_count_and_stays_exact():
    w = _workload("cu2k")
    ref = oracle.forces(w.pos, w.species, w.box, w.potential, skin=w.skin, k_max=w.k_max, method="brute")
    with _gpu_system(w) as s:
        lanes = s.tune()
        assert lanes in (1, 2, 4, 8, 16, 32)
        s.eam_forces()
        f = s.forces()
    assert np.abs(f - ref["force"]).max() <= FP64_TOL * np.abs(ref["force"]).max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_autotuner_trial_steps_leave_the_state_unchanged(precision):
    w = _workload("cu2k")
    with _gpu_system(w, precision) as s:
        s.eam_forces()
        s.step(3)
        before = [s.positions(), s.velocities(), s.forces()]
        e0 = s.energy()
        s.tune()
        after = [s.positions(), s.velocities(), s.forces()]
        e1 = s.energy()
        for a, b in zip(before, after):
            assert np.array_equal(a, b)
        assert e1["step"] == e0["step"] and e1["n_rebuilds"] == e0["n_rebuilds"]
        s.step(2)
        assert np.isfinite(s.energy()["te"])


# --------------------------------------------------------------------------- persistent step
def test_graph_replay_equals_direct_launch():
    w = I.bcc_fe(10, seed=21)
    with _gpu_system(w, "mixed") as a, _gpu_system(w, "mixed") as b:
        b.set_graph(True)
        for _ in range(3):
            a.step(7)
            b.step(7)
        assert np.array_equal(a.positions(), b.positions())
        assert a.energy()["te"] == b.energy()["te"]


def test_profile_stamps_cover_the_phases():
    w = I.fcc_cu(10, seed=22)
    with _gpu_system(w, "mixed", rebuild_every=3) as s:
        s.eam_forces()
        s.set_profiling(True)
        s.step(9)
        p = s.profile()
    assert p["n_density"] == 9 and p["n_force"] == 9
    assert p["ms_density"] > 0 and p["ms_force"] > 0 and p["ms_rebuild"] > 0


def test_bounded_barrier_wait_reports_timeout_and_recovers():
    """Failure detection without a fault: one block withholds a barrier arrival, the others'
    bounded wait runs out, the call returns MD_ERR_TIMEOUT and the context stays usable."""
    w = I.bcc_fe(10, seed=23)
    ref = oracle.forces(w.pos, w.species, w.box, w.potential, skin=w.skin, k_max=w.k_max)
    with _gpu_system(w) as s:
        s.eam_forces()
        assert md.md_selftest_timeout(s.ctx) == md.MD_ERR_TIMEOUT
        s.set_state(pos=w.pos, vel=w.vel)
        s.eam_forces()
        assert np.abs(s.forces() - ref["force"]).max() <= FP64_TOL * np.abs(ref["force"]).max()
        s.step(3)


def _replicas(seeds, sizes, temps):
    ws = []
    for seed, n, t in zip(seeds, sizes, temps):
        ws.append(I.bcc_fe(n, seed=seed, temperature=t))
    return ws


def test_batch_of_replicas_matches_replicas_alone():
    ws = _replicas([3001, 3002, 3003], [6, 9, 7], [300.0, 900.0, 600.0])
    with md.Batch(ws, precision="fp64") as b:
        b.step(20)
        pos_b = b.positions()
        per = b.replica_energies()
        tot = b.energy()
    off = np.concatenate([[0], np.cumsum([w.n_atoms for w in ws])])
    pe_sum = 0.0
    for r, w in enumerate(ws):
        with _gpu_system(w) as s:
            s.step(20)
            e = s.energy()
            assert np.abs(pos_b[off[r]:off[r + 1]] - s.positions()).max() < 1e-9
        assert abs(per[r]["pe"] - e["pe"]) <= FP64_TOL * abs(e["pe"])
        assert abs(per[r]["ke"] - e["ke"]) <= 1e-9 * e["ke"]
        assert abs(per[r]["temperature"] - e["temperature"]) <= 1e-9 * e["temperature"]
        pe_sum += e["pe"]
    assert abs(tot["pe"] - pe_sum) <= FP64_TOL * abs(pe_sum)


def test_batch_against_oracle_trajectories():
    ws = _replicas([3011, 3012], [6, 8], [1200.0, 300.0])
    with md.Batch(ws, precision="fp64") as b:
        b.step(30)
        pos_b = b.positions()
    off = np.concatenate([[0], np.cumsum([w.n_atoms for w in ws])])
    for r, w in enumerate(ws):
        ref = oracle.run_vv(w.pos, w.vel, w.species, w.potential.masses, w.box, w.potential, w.dt_fs, 30,
                            w.skin, w.k_max)
        assert np.abs(pos_b[off[r]:off[r + 1]] - ref["pos"]).max() < 1e-9


def test_full_size_fe_c_forces_and_strain_steps():
    """bcc Fe 128^3 + 0.1 % C (4,198,498 atoms), two-species tables, in the benchmark's
    configuration: every force (FP64 and mixed) against the oracle, then strained steps."""
    w = I.bcc_fe_c(128, seed=4)
    assert w.n_atoms == 2 * 128 ** 3 + 4194
    ref = oracle.forces(w.pos, w.species, w.box, w.potential, skin=w.skin, k_max=w.k_max, method="cells")
    fs = np.abs(ref["force"]).max()
    with _gpu_system(w) as s:
        pe = s.eam_forces()
        f = s.forces()
        cg = s.get(md.MD_GET_NBR_COUNT)
    assert np.array_equal(cg, ref["count"])
    assert np.abs(f - ref["force"]).max() <= FP64_TOL * fs
    assert abs(pe - ref["pe"]) <= FP64_TOL * abs(ref["pe"])
    with _gpu_system(w, "mixed") as s:
        pe32 = s.eam_forces()
        f32 = s.forces()
        img = s.get(md.MD_GET_IMAGE)
        ratio, _ = assert_mixed_forces(w, w.pos, f32, img, pe=pe32, pe_tol=MIXED_PE_TOL)
        print(f"Fe-C 4.2M mixed: largest error / derived bound = {ratio:.3f}")
        s.step(20)
        e = s.energy()
    assert abs(e["box"][2] - w.box[2] * (1 - 1e-6) ** 20) < 1e-9 * w.box[2]
    assert np.isfinite(e["te"])
