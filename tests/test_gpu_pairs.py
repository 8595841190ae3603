"""The FP64 half list (md_config.passes = MD_PASSES_HALF on the FP64 path: every pair computed once
from the full list's entries j > i, the neighbour's share added with FP64 atomics, §3.2.2)
against the oracle at the FP64 bars: forces, energies, virial and rho within 1e-10, trajectories
within 1e-9 Å, at every lane count, FS analytic and tables, with rebuilds, under the
predictor-corrector and the thermostat, in a batch, at full size as benchmarked; and the rows it
reorders still hold the same neighbour sets."""
import numpy as np
import pytest

import oracle
from paper_1107_2619_gb300 import inputs as I, md

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1107_2619_gb300 import build
    build.build()


def _sys(w, **kw):
    return md.System(w, precision="fp64", passes="half", **kw)


@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("case", ["cu", "fe"])
def test_forces_energies_virial_match_oracle(lanes, case):
    w = I.fcc_cu(8, seed=2, sigma=0.03) if case == "cu" else I.bcc_fe(10, seed=12)
    ref = oracle.forces(w.pos, w.species, w.box, w.potential, skin=w.skin, k_max=w.k_max, method="brute")
    with _sys(w, lanes_per_atom=lanes) as s:
        pe = s.eam_forces()
        f, e, rho = s.forces(), s.energy(), s.get(md.MD_GET_RHO)
        assert s.passes()["walk"] == "half"
        cnt, nl = s.neighbours()
    fs = np.abs(ref["force"]).max()
    assert np.abs(f - ref["force"]).max() <= TOL * fs
    assert abs(pe - ref["pe"]) <= TOL * abs(ref["pe"])
    assert np.abs(rho - ref["rho"]).max() <= TOL * np.abs(ref["rho"]).max()
    assert np.abs(e["virial"] - ref["virial"]).max() <= TOL * np.abs(ref["virial"]).max()
    assert np.array_equal(cnt, ref["count"])
    assert [sorted(nl[i, :cnt[i]].tolist()) for i in range(w.n_atoms)] == \
        [sorted(ref["list"][i, :cnt[i]].tolist()) for i in range(w.n_atoms)]


@pytest.mark.parametrize("integrator", ["verlet", "pc3"])
def test_trajectory_with_rebuilds_matches_oracle(integrator):
    w = I.bcc_fe(10, seed=1)
    n = 100
    run = oracle.run_vv if integrator == "verlet" else oracle.run_pc3
    ref = run(w.pos, w.vel, w.species, w.potential.masses, w.box, w.potential, w.dt_fs, n, w.skin, w.k_max,
              rebuild_every=10)
    with _sys(w, rebuild_every=10, integrator=integrator) as s:
        s.step(n)
        pos, e = s.positions(), s.energy()
    assert e["n_rebuilds"] >= 10
    assert np.abs(pos - ref["pos"]).max() < 1e-9
    assert abs(e["pe"] - ref["energies"][-1, 0]) <= TOL * abs(ref["energies"][-1, 0])


def test_thermostat_matches_oracle():
    ws = [I.bcc_fe(6, seed=3300, temperature=300.0)]
    with md.System(ws[0], precision="fp64", passes="half") as s:
        s.set_thermostat(900.0, tau_fs=40.0)
        s.eam_forces()
        q = s.thermostat()[0, 2]
        s.step(40)
        pos = s.positions()
    ref = oracle.run_nvt(ws[0].pos, ws[0].vel, ws[0].species, ws[0].potential.masses, ws[0].box, ws[0].potential, 1.0,
                         40, 0.3, 32, 900.0, q)
    assert np.abs(pos - ref["pos"]).max() < 1e-8


def test_batch_of_replicas_matches_oracle():
    ws = [I.bcc_fe(5 + r, seed=3400 + r, temperature=300.0 + 400.0 * r) for r in range(3)]
    with md.Batch(ws, precision="fp64", passes="half") as b:
        b.step(30)
        pos = b.positions()
    o = np.concatenate([[0], np.cumsum([w.n_atoms for w in ws])])
    for r, w in enumerate(ws):
        ref = oracle.run_vv(w.pos, w.vel, w.species, w.potential.masses, w.box, w.potential, w.dt_fs, 30, w.skin,
                            w.k_max)
        assert np.abs(pos[o[r]:o[r + 1]] - ref["pos"]).max() < 1e-9, r


def test_full_size_cu500k_step_kernel_as_benchmarked():
    """fcc Cu 500,000 atoms, FP64 half list, tuned lanes, one launch of 30 steps with rebuilds:
    the last force pass at the final positions and the energies against the oracle."""
    w = I.fcc_cu(50, seed=2)
    with _sys(w) as s:
        s.eam_forces()
        s.tune()
        s.step(30)
        e = s.energy()
        pos, f = s.positions(), s.forces()
    assert e["n_rebuilds"] >= 1
    ref = oracle.forces(pos, w.species, w.box, w.potential, skin=w.skin, k_max=w.k_max, method="cells")
    assert np.abs(f - ref["force"]).max() <= TOL * np.abs(ref["force"]).max()
    assert abs(e["pe"] - ref["pe"]) <= TOL * abs(ref["pe"])


def test_combinations_it_does_not_take():
    for w in (I.bcc_fe_c(6, seed=8), I.bcc_fe(6, seed=9, potential=I.fe_knots())):   # two species; knot sums
        with pytest.raises(md.MDError) as ex:
            _sys(w)
        assert ex.value.status == md.MD_ERR_ARG
