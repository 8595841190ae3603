"""Pins of the oracle's third-order predictor-corrector (§2.3; orc_run_pc3) against what the
mathematics and the paper fix, not against itself:

- free atoms move exactly in straight lines;
- started from a consistent Taylor vector (the third-derivative term taken from finite
  differences of the accelerations along an independent, fine velocity-Verlet trajectory), the
  error against that trajectory falls by at least 10x per halving of the time step (high order),
  and started with a zero third derivative (the start-up error) by about 4x (second order);
- in NVE the total energy drifts linearly with the number of steps while velocity Verlet's
  stays bounded (the paper's comparison of the two integrators, §5).
"""
import numpy as np

import oracle
from paper_1107_2619_gb300 import inputs as I


def _fe(seed=3, T=600.0, sigma=0.08, n=5):
    return I.bcc_fe(n, seed=seed, temperature=T, sigma=sigma)


def test_free_atoms_move_in_straight_lines():
    pot = I.fs_fe_analytic()
    pos = np.array([[1.0, 2.0, 3.0], [10.0, 10.0, 10.0], [1.0, 15.0, 4.0]])   # > r_cut apart
    vel = np.array([[0.01, -0.02, 0.005], [0.0, 0.03, -0.01], [-0.02, 0.0, 0.0]])
    sp = np.zeros(3, np.int32)
    box = np.array([20.0, 20.0, 20.0])
    out = oracle.run_pc3(pos, vel, sp, pot.masses, box, pot, 2.0, 50, 0.3, 8)
    assert np.abs(out["force"]).max() == 0.0
    assert np.allclose(out["pos"], pos + 100.0 * vel, rtol=0, atol=1e-12)
    assert np.array_equal(out["vel"], vel)
    assert np.abs(out["gear3"]).max() == 0.0


def _consistent_start(w, t0=5.0, h=0.125, dtf=1.0 / 64):
    """State at t0 of a fine velocity-Verlet trajectory and the third derivative of the position
    there, b = da/dt, by central differences of the accelerations at t0 +- h."""
    def state(t):
        return oracle.run_vv(w.pos, w.vel, w.species, w.potential.masses, w.box, w.potential, dtf,
                             int(round(t / dtf)), w.skin, w.k_max)

    s0, sp, sm = state(t0), state(t0 + h), state(t0 - h)
    acc = lambda s: s["force"] / (w.potential.masses[w.species][:, None] * ACC_UNIT)
    b = (acc(sp) - acc(sm)) / (2.0 * h)
    return s0["pos"], s0["vel"], b


# (eV/Å)/amu in Å/fs^2 is 1 / ACC_UNIT: amu (Å/fs)^2 in eV (CODATA 2018)
ACC_UNIT = 1.66053906660e-27 * 1.0e10 / 1.602176634e-19


def test_error_order_from_a_consistent_start_and_from_a_zero_third_derivative():
    w = _fe()
    x0, v0, b = _consistent_start(w)
    T = 40.0
    ref = oracle.run_vv(x0, v0, w.species, w.potential.masses, w.box, w.potential, 1.0 / 128, int(T * 128),
                        w.skin, w.k_max)
    err, err0 = [], []
    for dt in (2.0, 1.0, 0.5):
        n = int(round(T / dt))
        a = oracle.run_pc3(x0, v0, w.species, w.potential.masses, w.box, w.potential, dt, n, w.skin, w.k_max,
                           gear3=dt ** 3 / 6.0 * b)
        z = oracle.run_pc3(x0, v0, w.species, w.potential.masses, w.box, w.potential, dt, n, w.skin, w.k_max)
        err.append(np.abs(a["pos"] - ref["pos"]).max())
        err0.append(np.abs(z["pos"] - ref["pos"]).max())
    assert err[0] / err[1] > 10.0 and err[1] / err[2] > 8.0, err
    assert 3.0 < err0[0] / err0[1] < 5.5 and 3.0 < err0[1] / err0[2] < 5.5, err0
    assert err[0] < 0.1 * err0[0]


def test_nve_energy_drifts_linearly_while_verlet_stays_bounded():
    """bcc Fe 8^3 cells (1,024 atoms) started on the lattice sites at 1,800 K with dt = 2 fs, as in
    the paper's integration-error experiment: over steps 1,000-4,000 the predictor-corrector's
    total energy follows a straight line (R^2 > 0.95, its change over the window more than 20x the
    scatter about the line), while velocity Verlet's total energy fluctuates about a level: its
    trend over the window is smaller than its own scatter and under a quarter of the
    predictor-corrector's drift."""
    w = I.bcc_fe(8, seed=5, temperature=1800.0, sigma=0.0)
    args = (w.species, w.potential.masses, w.box, w.potential, 2.0, 4000, w.skin, w.k_max)
    ea = oracle.run_pc3(w.pos, w.vel, *args)["energies"].sum(axis=1)[1000:]
    eb = oracle.run_vv(w.pos, w.vel, *args)["energies"].sum(axis=1)[1000:]
    t = np.arange(ea.size, dtype=np.float64)
    ca = np.polyfit(t, ea, 1)
    fit = np.polyval(ca, t)
    r2 = 1.0 - ((ea - fit) ** 2).sum() / ((ea - ea.mean()) ** 2).sum()
    drift = abs(ca[0]) * t[-1]
    assert r2 > 0.95, r2
    assert drift > 20.0 * np.std(ea - fit), (drift, np.std(ea - fit))
    trend_vv = abs(np.polyfit(t, eb, 1)[0]) * t[-1]
    assert trend_vv < np.std(eb) and trend_vv < 0.25 * drift, (trend_vv, np.std(eb), drift)
