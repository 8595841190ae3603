"""GPU parity of the Nose-Hoover thermostat (NVTp) with the oracle: FP64 trajectories and
thermostat state, a batch of replicas at different temperatures, infinite thermal inertia =
NVE bit for bit, the conserved extended energy in mixed precision, graph replay."""
import numpy as np
import pytest

import oracle
from paper_1107_2619_gb300 import inputs as I
from paper_1107_2619_gb300 import md

pytestmark = pytest.mark.gpu
KB = I.KB_EV_PER_K


def test_library_sets_q_from_tau():
    w = I.bcc_fe(5, seed=3)
    with md.System(w, precision="fp64") as s:
        s.set_thermostat(900.0, tau_fs=40.0)
        q = s.thermostat()[0, 2]
    assert abs(q - (3 * w.n_atoms - 3) * KB * 900.0 * 40.0 ** 2) <= 1e-14 * q


def test_fp64_nvt_trajectory_matches_oracle():
    w = I.bcc_fe(5, seed=3, temperature=300.0, sigma=0.05)
    T = 900.0
    with md.System(w, precision="fp64") as s:
        s.set_thermostat(T, tau_fs=40.0)
        s.eam_forces()
        q = s.thermostat()[0, 2]
        ref = oracle.run_nvt(w.pos, w.vel, w.species, w.potential.masses, w.box, w.potential, 1.0, 60, 0.3, 32, T,
                             q)
        s.step(60)
        pos, vel = s.positions(), s.velocities()
        th = s.thermostat()[0]
        e = s.energy()
    assert np.abs(pos - ref["pos"]).max() < 1e-8
    assert np.abs(vel - ref["vel"]).max() < 1e-9
    assert abs(th[0] - ref["pi"]) <= 1e-9 * max(abs(ref["pi"]), 1e-6)
    assert abs(th[1] - ref["xi"]) <= 1e-9 * max(abs(ref["xi"]), 1e-6)
    assert abs(th[3] - ref["energies"][-1, 2]) <= 1e-9 * abs(ref["energies"][-1, 2])
    assert abs(e["ke"] - ref["energies"][-1, 1]) <= 1e-9 * ref["energies"][-1, 1]


def test_batch_replicas_each_follow_their_own_thermostat():
    temps = [300.0, 700.0, 1200.0]
    ws = [I.bcc_fe(5 + r % 2, seed=60 + r, temperature=400.0, sigma=0.05) for r in range(3)]
    with md.Batch(ws, precision="fp64") as b:
        b.set_thermostat(temps, tau_fs=30.0)
        b.eam_forces()
        qs = b.thermostat()[:, 2]
        b.step(40)
        pos, th = b.positions(), b.thermostat()
    for r, (w, T, q) in enumerate(zip(ws, temps, qs)):
        ref = oracle.run_nvt(w.pos, w.vel, w.species, w.potential.masses, w.box, w.potential, 1.0, 40, 0.3, 32, T, q)
        o = b.offsets
        assert np.abs(pos[o[r]:o[r + 1]] - ref["pos"]).max() < 1e-8
        assert abs(th[r, 0] - ref["pi"]) <= 1e-9 * max(abs(ref["pi"]), 1e-6)
        assert abs(th[r, 3] - ref["energies"][-1, 2]) <= 1e-9 * abs(ref["energies"][-1, 2])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_infinite_thermal_inertia_is_nve(precision):
    w = I.bcc_fe(6, seed=4, temperature=600.0)
    with md.System(w, precision=precision) as a, md.System(w, precision=precision) as b:
        a.set_thermostat(600.0, tau_fs=1e20)
        for s in (a, b):
            s.eam_forces()
            s.step(25)
        assert np.array_equal(a.positions(), b.positions())
        assert np.array_equal(a.velocities(), b.velocities())


def test_mixed_nvt_conserves_extended_energy_and_reaches_target():
    w = I.fcc_cu(8, seed=9, temperature=300.0, n_knots=5000)
    T = 700.0
    with md.System(w, precision="mixed") as s:
        s.set_thermostat(T, tau_fs=50.0)
        s.eam_forces()
        h0 = s.thermostat()[0, 3]
        temps, hs = [], []
        for _ in range(30):
            s.step(50)
            temps.append(s.energy()["temperature"])
            hs.append(s.thermostat()[0, 3])
    assert np.abs(np.array(hs) - h0).max() / w.n_atoms < 2e-4
    assert abs(np.mean(temps[10:]) - T) < 0.05 * T


def test_thermostat_graph_replay_and_switch_off():
    w = I.bcc_fe(6, seed=5, temperature=300.0)
    with md.System(w, precision="mixed") as a, md.System(w, precision="mixed") as b:
        for s in (a, b):
            s.set_thermostat(900.0, tau_fs=40.0)
            s.eam_forces()
        b.set_graph(True)
        for _ in range(3):
            a.step(10)
            b.step(10)
        assert np.array_equal(a.positions(), b.positions())
        for s in (a, b):
            md.md_set_thermostat(s.ctx, False)
            e0 = s.energy()
            s.step(40)
            assert abs(s.energy()["te"] - e0["te"]) / w.n_atoms < 1e-4   # NVE again
