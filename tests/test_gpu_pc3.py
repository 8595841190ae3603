"""The third-order predictor-corrector (§2.3; md.h MD_INTEGRATOR_PC3) in the persistent step
kernel against the oracle's orc_run_pc3: FP64 trajectories (one call, split calls that carry
the third-derivative term across, list rebuilds inside the launch, a batch of replicas), the
mixed path within its trajectory tolerance, the restart at md_set_state, the paper's energy
behaviour on the GPU (linear drift, while velocity Verlet stays bounded), and the combinations
it does not take."""
import numpy as np
import pytest

import oracle
from paper_1107_2619_gb300 import inputs as I, md

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1107_2619_gb300 import build
    build.build()


def _ref(w, n, **kw):
    return oracle.run_pc3(w.pos, w.vel, w.species, w.potential.masses, w.box, w.potential, w.dt_fs, n, w.skin,
                          w.k_max, **kw)


@pytest.mark.parametrize("split", [(100,), (37, 63)])
def test_fp64_trajectory_matches_oracle(split):
    """bcc Fe 2,000 atoms, FP64, 100 steps of 1 fs in one md_step call or two (the third-derivative
    term carried from one call to the next)."""
    w = I.bcc_fe(10, seed=1)
    ref = _ref(w, 100)
    with md.System(w, precision="fp64", integrator="pc3") as s:
        for n in split:
            s.step(n)
        pos, vel, f, e = s.positions(), s.velocities(), s.forces(), s.energy()
    assert np.abs(pos - ref["pos"]).max() < 1e-9
    assert np.abs(vel - ref["vel"]).max() < 1e-11
    assert np.abs(f - ref["force"]).max() <= 1e-9 * np.abs(ref["force"]).max()
    assert abs(e["pe"] - ref["energies"][-1, 0]) <= 1e-10 * abs(ref["energies"][-1, 0])
    assert abs(e["ke"] - ref["energies"][-1, 1]) <= 1e-9 * ref["energies"][-1, 1]


def test_fp64_tables_with_scheduled_rebuilds_match_oracle():
    """fcc Cu tables (the derivative cache of the force pass), rebuilds every 4 steps inside one
    launch of 24 steps."""
    w = I.fcc_cu(8, seed=2, sigma=0.03)
    ref = _ref(w, 24, rebuild_every=4)
    with md.System(w, precision="fp64", integrator="pc3", rebuild_every=4) as s:
        s.step(24)
        pos, e = s.positions(), s.energy()
    assert e["n_rebuilds"] >= 6
    assert np.abs(pos - ref["pos"]).max() < 1e-9
    assert abs(e["pe"] - ref["energies"][-1, 0]) <= 1e-10 * abs(ref["energies"][-1, 0])


def test_fp64_batch_replicas_match_oracle():
    ws = [I.bcc_fe(5 + r, seed=3100 + r, temperature=300.0 + 400.0 * r) for r in range(3)]
    with md.Batch(ws, precision="fp64", integrator="pc3") as b:
        b.step(30)
        pos = b.positions()
    o = np.concatenate([[0], np.cumsum([w.n_atoms for w in ws])])
    for r, w in enumerate(ws):
        assert np.abs(pos[o[r]:o[r + 1]] - _ref(w, 30)["pos"]).max() < 1e-9, r


def test_mixed_trajectory_within_its_tolerance():
    w = I.fcc_cu(8, seed=4, sigma=0.03)
    ref = _ref(w, 30)
    with md.System(w, precision="mixed", integrator="pc3") as s:
        s.step(30)
        pos, e = s.positions(), s.energy()
    assert np.abs(pos - ref["pos"]).max() < 1e-5
    assert abs(e["pe"] - ref["energies"][-1, 0]) <= 1e-6 * abs(ref["energies"][-1, 0])


def test_set_state_restarts_the_predictor():
    """After md_set_state the third-derivative term is zero: the continuation equals the oracle
    started afresh (gear3 = 0) from that state with its forces."""
    w = I.bcc_fe(8, seed=6, temperature=600.0)
    with md.System(w, precision="fp64", integrator="pc3") as s:
        s.step(20)
        p, v = s.positions(), s.velocities()
        s.set_state(p, v)
        s.step(20)
        pos = s.positions()
    ref = _ref(I.Workload(**{**w.__dict__, "pos": p, "vel": v}), 20)
    assert np.abs(pos - ref["pos"]).max() < 1e-9


def test_energy_drifts_linearly_while_verlet_stays_bounded():
    """The paper's integration-error comparison on the GPU: bcc Fe 8^3 cells on lattice sites with
    1,800 K of kinetic energy, dt = 2 fs, FP64: over steps 1,000-4,000 the predictor-corrector's
    total energy follows a line (R^2 > 0.95) and velocity Verlet's has no trend beyond its own
    scatter."""
    w = I.bcc_fe(8, seed=5, temperature=1800.0, sigma=0.0, dt_fs=2.0)
    te = {}
    for integ in ("pc3", "verlet"):
        with md.System(w, precision="fp64", integrator=integ) as s:
            s.step(1000)
            e = []
            for _ in range(60):
                s.step(50)
                e.append(s.energy()["te"])
        te[integ] = np.array(e)
    t = np.arange(60.0)
    ca = np.polyfit(t, te["pc3"], 1)
    fit = np.polyval(ca, t)
    r2 = 1.0 - ((te["pc3"] - fit) ** 2).sum() / ((te["pc3"] - te["pc3"].mean()) ** 2).sum()
    drift = abs(ca[0]) * t[-1]
    trend_vv = abs(np.polyfit(t, te["verlet"], 1)[0]) * t[-1]
    assert r2 > 0.95 and drift > 0.0
    assert trend_vv < max(np.std(te["verlet"]), 1e-12) * 2.0 and trend_vv < 0.25 * drift


def test_combinations_it_does_not_take():
    w = I.bcc_fe(6, seed=7)
    strained = I.Workload(**{**w.__dict__, "strain_rate_zz": -1e9})
    with pytest.raises(md.MDError) as ex:
        md.System(strained, precision="fp64", integrator="pc3")
    assert ex.value.status == md.MD_ERR_ARG
    cu = I.fcc_cu(7, seed=8)
    with pytest.raises(md.MDError) as ex:
        md.System(cu, precision="mixed", integrator="pc3", passes="staged")
    assert ex.value.status == md.MD_ERR_ARG
    with md.System(w, precision="fp64", integrator="pc3") as s:
        with pytest.raises(md.MDError) as ex:
            s.set_thermostat(300.0, tau_fs=50.0)
        assert ex.value.status == md.MD_ERR_STATE
