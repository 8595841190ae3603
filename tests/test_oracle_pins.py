"""Pins of the FP64 oracle to facts outside itself (CPU only).

Each test checks the oracle against something the paper, the literature or the
mathematics fixes: fitted cohesive energies, the paper's time unit, lattice
geometry, finite differences of Eq. (1), brute-force neighbour sets, Newton's
third law, the virial theorem, velocity-Verlet energy conservation with its
O(dt^2) error, time reversibility and the affine strain boundary condition.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1107_2619_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split()
                vals[k] = float(v)
    return vals


def total_energy(pos, w, pot=None, box=None, k_max=200):
    pot = pot or w.potential
    box = w.box if box is None else box
    return oracle.forces(pos, w.species, box, pot, skin=0.3, k_max=k_max, method="brute")["pe"]


# --------------------------------------------------------------------------- lattice energies
def test_fs_fe_cohesive_energy_equilibrium_and_coordination():
    g = golden("fs_fe_bcc.txt")
    w = I.bcc_fe(6, seed=1, sigma=0.0, a=g["lattice_a_angstrom"])
    out = oracle.forces(w.pos, w.species, w.box, w.potential)
    e = out["pe"] / w.n_atoms
    assert abs(e - g["cohesive_energy_ev_per_atom"]) < 5e-6
    assert np.all(out["count"] == int(g["neighbours_per_atom"]))
    assert np.abs(out["force"]).max() < 1e-12          # every atom is a centre of inversion
    # the fit's lattice parameter is an equilibrium: zero static pressure
    p = oracle.pressure_gpa(np.zeros((3, 3)), out["virial"], w.box)
    assert abs(p) < 1e-3


def _shell_sum(f, basis, a, rc, m=6):
    g = np.arange(-m, m + 1, dtype=np.float64)
    cells = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    pts = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a
    r = np.sqrt((pts * pts).sum(axis=1))
    r = r[(r > 1e-9) & (r < rc)]
    return float(f(r).sum())


def test_sutton_chen_constants_give_cu_cohesive_energy():
    # infinite-range lattice sums of the analytic Sutton-Chen form (pins the constants)
    g = golden("sutton_chen_cu.txt")
    p = I.SC_CU
    a = g["lattice_a_angstrom"]
    big = 12 * a
    v = _shell_sum(lambda r: p["eps"] * (p["a"] / r) ** p["n"], I.FCC_BASIS, a, big, m=13)
    rho = _shell_sum(lambda r: (p["a"] / r) ** p["m"], I.FCC_BASIS, a, big, m=13)
    e = 0.5 * v - p["eps"] * p["c"] * math.sqrt(rho)
    assert abs(e - g["cohesive_energy_ev_per_atom"]) < g["abs_tol"]


def test_sc_cu_tables_lattice_energy_vs_shell_sums():
    """Oracle (knot tables, link cells, Eq. 1) vs closed-form shell sums of the shifted analytic forms."""
    g = golden("sutton_chen_cu.txt")
    w = I.fcc_cu(5, seed=2, temperature=0.0)
    out = oracle.forces(w.pos, w.species, w.box, w.potential, k_max=176, method="brute")
    assert np.all(out["count"] == int(g["neighbours_per_atom_2a_plus_0.3"]))
    p = I.SC_CU
    rc = w.potential.r_cut
    V = lambda r: p["eps"] * (p["a"] / r) ** 9
    dV = lambda r: -9 * p["eps"] * (p["a"] / r) ** 9 / r
    P = lambda r: (p["a"] / r) ** 6
    dP = lambda r: -6 * (p["a"] / r) ** 6 / r
    Vs = lambda r: V(r) - V(rc) - (r - rc) * dV(rc)
    Ps = lambda r: P(r) - P(rc) - (r - rc) * dP(rc)
    v = _shell_sum(Vs, I.FCC_BASIS, 3.615, rc)
    rho = _shell_sum(Ps, I.FCC_BASIS, 3.615, rc)
    e = 0.5 * v - p["eps"] * p["c"] * math.sqrt(rho)
    assert abs(out["pe"] / w.n_atoms - e) < 1e-9 * abs(e)
    assert np.abs(out["force"]).max() < 1e-10


def test_time_unit_matches_paper():
    g = golden("units.txt")
    # one atom of 1 amu at 1 Å/fs: KE = m v^2 / 2 in eV equals tau^2/2 with tau in fs
    ke = oracle.kinetic(np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 0.0]]), np.zeros(2, np.int32),
                        np.array([1.0]))["ke"]
    tau_s = math.sqrt(2.0 * ke) * 1e-15
    assert abs(tau_s - g["time_unit_seconds"]) < g["rel_tol"] * g["time_unit_seconds"]


# --------------------------------------------------------------------------- neighbour sets
def _rows(count, nl):
    return [tuple(sorted(nl[i, :count[i]].tolist())) for i in range(count.shape[0])]


@pytest.mark.parametrize("cells,n", [((3, 3, 3), 300), ((3, 4, 5), 700), ((5, 3, 4), 1)])
def test_link_cells_equal_brute_force(cells, n):
    rl = 3.7
    box = np.array(cells, dtype=np.float64) * (rl + 0.013)
    u = I.random_uniform(11, n, 3 * n).reshape(n, 3)
    pos = u * box
    # unwrap some atoms by whole box lengths: the sets must not change
    pos[::3] += box * np.array([1.0, -2.0, 3.0])
    c1, l1, m1 = oracle.neighbours(pos, box, rl, 128, "brute")
    c2, l2, m2 = oracle.neighbours(pos, box, rl, 128, "cells")
    assert m1 <= 128 and m1 == m2
    assert np.array_equal(c1, c2)
    assert _rows(c1, l1) == _rows(c2, l2)


def test_cell_count_gas_fills_its_cells_as_prescribed_and_its_lists_agree():
    """The list case for warp-wide lane groups: every link cell holds its prescribed count (each of
    25..56 twice), so every remainder after a first 32 atoms occurs; on it the link-cell oracle
    equals the brute-force definition."""
    counts = np.tile(np.arange(25, 57), 2)
    w = I.cell_count_gas(counts)
    rl = w.potential.r_cut + w.skin
    assert int(np.floor(w.box[0] / rl)) == 4
    width = w.box / 4
    c = np.floor(w.pos / width).astype(int)
    assert c.min() >= 0 and c.max() <= 3
    frac = w.pos / width - c
    assert frac.min() >= 0.019 and frac.max() <= 0.981
    assert np.array_equal(np.bincount(c[:, 0] + 4 * c[:, 1] + 16 * c[:, 2], minlength=64), counts)
    assert set((counts - 32)[(counts > 32) & (counts <= 48)]) == set(range(1, 17))
    c1, l1, m1 = oracle.neighbours(w.pos, w.box, rl, w.k_max, "brute")
    c2, l2, m2 = oracle.neighbours(w.pos, w.box, rl, w.k_max, "cells")
    assert m1 <= w.k_max and m1 == m2
    assert np.array_equal(c1, c2)
    assert _rows(c1, l1) == _rows(c2, l2)


def test_neighbour_cutoff_is_strict_and_empty_box():
    box = np.array([20.0, 20.0, 20.0])
    pos = np.array([[1.0, 1.0, 1.0], [5.0, 1.0, 1.0], [1.0, 4.999999999, 1.0]])
    c, nl, _ = oracle.neighbours(pos, box, 4.0, 8, "brute")
    assert c.tolist() == [1, 0, 1]      # |r| == r_list exactly is not a neighbour
    # minimum image across the boundary
    pos = np.array([[0.5, 1.0, 1.0], [19.0, 1.0, 1.0]])
    c, nl, _ = oracle.neighbours(pos, box, 4.0, 8, "brute")
    assert c.tolist() == [1, 1]
    c, nl, m = oracle.neighbours(np.zeros((0, 3)), box, 4.0, 8, "cells")
    assert c.shape == (0,) and m == 0


# --------------------------------------------------------------------------- forces
def _displaced(kind):
    if kind == "fs":
        return I.bcc_fe(5, seed=21, sigma=0.08)
    if kind == "fs_tables":
        return I.bcc_fe(5, seed=22, sigma=0.08, tables=True)
    if kind == "cu":
        return I.fcc_cu(5, seed=23, n_knots=5000, sigma=0.08)
    if kind == "fec":
        w = I.bcc_fe_c(5, seed=24)
        w.potential  # two species with asymmetric densities
        return w
    if kind == "knots":
        return I.bcc_fe(5, seed=25, sigma=0.08, potential=I.fe_knots())
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["fs", "fs_tables", "cu", "fec", "knots"])
def test_forces_are_minus_energy_gradient(kind):
    w = _displaced(kind)
    if kind == "fec":
        # place two C atoms: 0.1% of 250 rounds to 0, so add them by hand on octahedral sites
        sites, _ = I.replicate(I.BCC_OCTA_BASIS, (5, 5, 5), 2.8665)
        pos = np.concatenate([w.pos, sites[[3, 401]] + 0.03])
        w = I.Workload(name="fec", pos=pos, vel=np.zeros_like(pos),
                       species=np.concatenate([w.species, np.ones(2, np.int32)]), box=w.box,
                       potential=w.potential, skin=0.3, k_max=64, dt_fs=1.0, steps=1, temperature=0)
    out = oracle.forces(w.pos, w.species, w.box, w.potential, k_max=200, method="brute")
    h = 1e-5
    idx = [0, 7, w.n_atoms // 2, w.n_atoms - 1]
    for i in idx:
        for c in range(3):
            p1 = w.pos.copy(); p1[i, c] += h
            p2 = w.pos.copy(); p2[i, c] -= h
            fd = -(total_energy(p1, w) - total_energy(p2, w)) / (2 * h)
            assert abs(fd - out["force"][i, c]) < 2e-7 + 1e-7 * abs(fd), (i, c, fd, out["force"][i, c])
    # Newton's third law: the total force vanishes up to summation rounding
    fsum = np.abs(out["force"].sum(axis=0)).max()
    assert fsum < 1e-12 * np.abs(out["force"]).sum()


def test_explicit_knot_sums_equal_their_hermite_tables():
    """The 15-term Fe potential evaluated term by term (kind 4) and through cubic-Hermite tables
    of the same sums (kind 2, orc_table): two independent code paths agree to the tables'
    interpolation error."""
    w = I.bcc_fe(6, seed=26, sigma=0.1, potential=I.fe_knots())
    a = oracle.forces(w.pos, w.species, w.box, I.fe_knots())
    b = oracle.forces(w.pos, w.species, w.box, I.fe_knot_tables())
    assert np.abs(a["force"] - b["force"]).max() < 1e-6
    assert abs(a["pe"] - b["pe"]) < 1e-10 * abs(a["pe"])
    assert np.array_equal(a["count"], b["count"])
    # and the fit is an iron: near the FS cohesive energy at the FS lattice parameter
    g = golden("fs_fe_bcc.txt")
    w0 = I.bcc_fe(6, seed=1, sigma=0.0, a=g["lattice_a_angstrom"], potential=I.fe_knots())
    e = oracle.forces(w0.pos, w0.species, w0.box, w0.potential)["pe"] / w0.n_atoms
    assert abs(e - g["cohesive_energy_ev_per_atom"]) < 0.01


def test_half_list_equals_full_list_two_species():
    w = I.bcc_fe_c(10, seed=25)        # 2000 Fe + 2 C
    assert (w.species == 1).sum() == 2
    full = oracle.forces(w.pos, w.species, w.box, w.potential, k_max=64)
    half_f, half_pe = oracle.eam_forces_half(w.pos, w.species, w.box, w.potential, full["count"],
                                             full["list"])
    scale = np.abs(full["force"]).max()
    assert np.abs(half_f - full["force"]).max() < 1e-12 * max(scale, 1.0)
    assert abs(half_pe - full["pe"]) < 1e-12 * abs(full["pe"])


def test_tables_reproduce_analytic_fs():
    wa = I.bcc_fe(6, seed=26, sigma=0.08)
    wt = I.bcc_fe(6, seed=26, sigma=0.08, tables=True)
    a = oracle.forces(wa.pos, wa.species, wa.box, wa.potential)
    t = oracle.forces(wt.pos, wt.species, wt.box, wt.potential)
    assert np.abs(a["force"] - t["force"]).max() < 1e-6
    assert abs(a["pe"] - t["pe"]) < 1e-8 * abs(a["pe"])


def test_virial_pressure_equals_minus_dU_dV():
    w = I.bcc_fe(6, seed=27, sigma=0.08)
    out = oracle.forces(w.pos, w.species, w.box, w.potential)
    p_vir = oracle.pressure_gpa(np.zeros((3, 3)), out["virial"], w.box)
    h = 1e-6
    up = total_energy(w.pos * (1 + h), w, box=w.box * (1 + h))
    dn = total_energy(w.pos * (1 - h), w, box=w.box * (1 - h))
    vol = float(np.prod(w.box))
    dUdV = (up - dn) / (vol * ((1 + h) ** 3 - (1 - h) ** 3))
    p_fd = -dUdV * 160.21766208
    assert abs(p_vir - p_fd) < 1e-5 * max(1.0, abs(p_fd))


# --------------------------------------------------------------------------- dynamics
def test_initial_temperature_exact_and_zero_momentum():
    w = I.bcc_fe(10, seed=1)
    k = oracle.kinetic(w.vel, w.species, w.potential.masses)
    assert abs(k["temperature"] - 300.0) < 1e-9
    assert np.abs(k["momentum"]).max() < 1e-12


def _nve(w, dt, steps):
    r = oracle.run_vv(w.pos, w.vel, w.species, w.potential.masses, w.box, w.potential, dt, steps,
                      w.skin, w.k_max)
    e = r["energies"].sum(axis=1)
    return r, e


def test_velocity_verlet_conserves_energy_with_dt2_error():
    w = I.bcc_fe(6, seed=28, temperature=600.0)
    r1, e1 = _nve(w, 1.0, 200)
    r2, e2 = _nve(w, 0.5, 400)
    dev1 = np.abs(e1 - e1.mean()).max()
    dev2 = np.abs(e2 - e2.mean()).max()
    ke = r1["energies"][:, 1].mean()
    assert dev1 < 1e-3 * ke                         # bounded fluctuation
    assert 2.5 < dev1 / dev2 < 6.0                  # second-order integrator: error ~ dt^2
    # no linear drift: first and last quarter agree within the fluctuation
    q = len(e1) // 4
    assert abs(e1[:q].mean() - e1[-q:].mean()) < dev1
    k = oracle.kinetic(r1["vel"], w.species, w.potential.masses)
    assert np.abs(k["momentum"]).max() < 1e-10      # NVEp: total momentum stays zero (§2.1.1)


def test_velocity_verlet_is_time_reversible():
    w = I.bcc_fe(6, seed=29, temperature=300.0)
    f = oracle.run_vv(w.pos, w.vel, w.species, w.potential.masses, w.box, w.potential, 1.0, 60, w.skin,
                      w.k_max)
    b = oracle.run_vv(f["pos"], -f["vel"], w.species, w.potential.masses, w.box, w.potential, 1.0, 60,
                      w.skin, w.k_max, force=f["force"])
    assert np.abs(b["pos"] - w.pos).max() < 1e-9
    assert np.abs(-b["vel"] - w.vel).max() < 1e-10


def test_free_atoms_move_ballistically():
    box = np.array([40.0, 40.0, 40.0])
    pos = np.array([[1.0, 2.0, 3.0], [21.0, 22.0, 23.0]])
    vel = np.array([[0.01, -0.02, 0.03], [0.0, 0.05, -0.01]])
    pot = I.fs_fe_analytic()
    r = oracle.run_vv(pos, vel, np.zeros(2, np.int32), pot.masses, box, pot, 2.0, 50, 0.3, 8)
    assert np.allclose(r["pos"], pos + 100.0 * vel, rtol=0, atol=1e-12)


def test_strain_ramp_keeps_fractional_coordinates():
    w = I.bcc_fe(6, seed=30, sigma=0.0, temperature=0.0)
    rate = -1.0e9
    r = oracle.run_vv(w.pos, w.vel, w.species, w.potential.masses, w.box, w.potential, 1.0, 10, w.skin,
                      w.k_max, strain_rate_zz=rate)
    s = (1.0 + rate * 1e-15) ** 10
    assert abs(r["box"][2] - w.box[2] * s) < 1e-12 * w.box[2]
    assert np.allclose(r["pos"][:, 2] / r["box"][2], w.pos[:, 2] / w.box[2], rtol=0, atol=1e-13)
    assert np.allclose(r["pos"][:, :2], w.pos[:, :2], rtol=0, atol=1e-13)
