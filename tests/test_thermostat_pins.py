"""Pins of the oracle's Nose-Hoover thermostat (NVTp) to facts outside it (CPU only): the
extended energy H' = KE + U + Q pi^2/2 + g k T xi is conserved with an O(dt^2) error, a
thermostat of infinite inertia is plain velocity Verlet (bit for bit), the integrator is time
reversible, and the kinetic temperature settles at the target."""
import numpy as np
import pytest

import oracle
from paper_1107_2619_gb300 import inputs as I

KB = 8.617333262e-5


def _fe(T=300.0, seed=3):
    return I.bcc_fe(5, seed=seed, temperature=T, sigma=0.05)


def _q(n, T, tau_fs):
    return (3 * n - 3) * KB * T * tau_fs ** 2


def test_extended_energy_is_conserved_with_dt2_error():
    w = _fe()
    T = 900.0
    q = _q(w.n_atoms, T, 40.0)
    dev = {}
    for dt in (1.0, 0.5):
        steps = int(round(100 / dt))
        r = oracle.run_nvt(w.pos, w.vel, w.species, w.potential.masses, w.box, w.potential, dt, steps, 0.3, 32, T, q)
        h = r["energies"][:, 2]
        dev[dt] = np.abs(h - h[0]).max()
        # the thermostat does work: the plain total energy is not conserved
        te = r["energies"][:, 0] + r["energies"][:, 1]
        assert np.abs(te - te[0]).max() > 20 * dev[dt]
    # the run heats 300 K -> ~1300 K (total energy changes by 0.3 eV/atom); H' moves < 1e-4 eV/atom
    assert dev[1.0] / w.n_atoms < 1e-4
    assert 3.5 < dev[1.0] / dev[0.5] < 4.5


def test_infinite_thermal_inertia_is_plain_velocity_verlet():
    w = _fe()
    a = oracle.run_nvt(w.pos, w.vel, w.species, w.potential.masses, w.box, w.potential, 1.0, 30, 0.3, 32, 900.0,
                       1e40)
    b = oracle.run_vv(w.pos, w.vel, w.species, w.potential.masses, w.box, w.potential, 1.0, 30, 0.3, 32,
                      rebuild_every=1)
    assert np.array_equal(a["pos"], b["pos"]) and np.array_equal(a["vel"], b["vel"])


def test_thermostat_is_time_reversible():
    w = _fe()
    T = 900.0
    q = _q(w.n_atoms, T, 40.0)
    r = oracle.run_nvt(w.pos, w.vel, w.species, w.potential.masses, w.box, w.potential, 1.0, 60, 0.3, 32, T, q)
    back = oracle.run_nvt(r["pos"], -r["vel"], w.species, w.potential.masses, w.box, w.potential, 1.0, 60, 0.3, 32,
                          T, q, pi=-r["pi"], xi=r["xi"], force=r["force"])
    assert np.abs(back["pos"] - w.pos).max() < 1e-8
    assert abs(back["pi"]) < 1e-10


def test_temperature_settles_at_the_target():
    w = _fe(T=300.0)
    T = 800.0
    q = _q(w.n_atoms, T, 30.0)
    r = oracle.run_nvt(w.pos, w.vel, w.species, w.potential.masses, w.box, w.potential, 1.0, 3000, 0.3, 32, T, q)
    ke = r["energies"][1000:, 1]
    t_mean = (2.0 * ke / ((3 * w.n_atoms - 3) * KB)).mean()
    assert abs(t_mean - T) < 0.06 * T
