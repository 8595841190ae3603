"""Seeded synthetic inputs for the EAM hot path.

This module produces only inputs: lattices (the paper's unit cell x replication
construction, §4.1.2), random displacements and velocities (§2.5), potential
parameter sets and the knot tables sampled from them.  The same arrays feed the
CUDA library, the FP64 oracle, the tests and the benchmark.  It holds none of the
hot path's arithmetic (no neighbour search, no density or force sums, no
integration).

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based generator,
so a draw depends only on (seed, stream, index) and is identical on every machine.
Normal deviates use the Box-Muller transform.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# ---------------------------------------------------------------------------
# Physical constants (CODATA 2018) and the paper's unit system (§2.7: Å, amu, eV,
# time in sqrt(amu Å^2 / eV) ~ 1.018e-14 s, user time in fs, temperature in K).
# ---------------------------------------------------------------------------
KB_EV_PER_K = 8.617333262e-5
AMU_KG = 1.66053906660e-27
EV_J = 1.602176634e-19
# kinetic energy of 1 amu moving at 1 Å/fs, in eV
MVV_TO_EV = AMU_KG * 1.0e10 / EV_J

MASS_AMU = {26: 55.847, 29: 63.546, 6: 12.011}   # Fe (paper §5.1 system file), Cu, C

# ---------------------------------------------------------------------------
# SplitMix64 as a counter-based generator
# ---------------------------------------------------------------------------
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def random_u64(seed: int, stream: int, n: int) -> np.ndarray:
    """n 64-bit words; word k is mix(key + (k+1)*gamma) with key = mix(seed, stream)."""
    with np.errstate(over="ignore"):
        key = _mix64(np.array([(seed * 0x100000001B3 + stream * 0x9E3779B97F4A7C15 + 1)
                               & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
        k = np.arange(1, n + 1, dtype=np.uint64)
        return _mix64(key + k * _GAMMA)


def random_uniform(seed: int, stream: int, n: int) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits."""
    return (random_u64(seed, stream, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def random_normal(seed: int, stream: int, n: int) -> np.ndarray:
    """Standard normal deviates by Box-Muller on pairs of uniforms."""
    m = (n + 1) // 2
    u = random_uniform(seed, stream, 2 * m)
    u1, u2 = u[0::2], u[1::2]
    rad = np.sqrt(-2.0 * np.log(1.0 - u1))
    z = np.empty(2 * m)
    z[0::2] = rad * np.cos(2.0 * math.pi * u2)
    z[1::2] = rad * np.sin(2.0 * math.pi * u2)
    return z[:n]


# ---------------------------------------------------------------------------
# Lattices: a unit cell replicated nx x ny x nz times (§4.1.2, §5.1)
# ---------------------------------------------------------------------------
BCC_BASIS = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5]])
FCC_BASIS = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
# octahedral interstices of bcc: 3 face centres + 3 edge midpoints per conventional cell
BCC_OCTA_BASIS = np.array([[0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5],
                           [0.5, 0.0, 0.0], [0.0, 0.5, 0.0], [0.0, 0.0, 0.5]])


def replicate(basis: np.ndarray, cells, a: float):
    """Positions (N,3) in Å, ordered x fastest then y then z, basis innermost; box lengths."""
    nx, ny, nz = cells
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    origin = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    pos = (origin[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a
    box = np.array([nx * a, ny * a, nz * a], dtype=np.float64)
    return pos, box


def gaussian_displace(pos: np.ndarray, sigma: float, seed: int, stream: int = 1) -> np.ndarray:
    """Random displacement of every coordinate (the paper's `dsp`, §2.5), Gaussian here."""
    return pos + sigma * random_normal(seed, stream, pos.size).reshape(pos.shape)


def maxwell_boltzmann(masses: np.ndarray, temperature: float, seed: int, stream: int = 2) -> np.ndarray:
    """Velocities (N,3) in Å/fs: Gaussian draw, zero total momentum, then scaled so that
    the kinetic temperature with 3N-3 degrees of freedom is exactly `temperature` (§2.1.2, §2.5)."""
    n = masses.shape[0]
    sigma = np.sqrt(KB_EV_PER_K * temperature / (masses * MVV_TO_EV))
    v = random_normal(seed, stream, 3 * n).reshape(n, 3) * sigma[:, None]
    v -= (masses[:, None] * v).sum(axis=0) / masses.sum()
    if temperature <= 0.0 or n < 2:
        return np.zeros_like(v)
    ke = 0.5 * MVV_TO_EV * float((masses[:, None] * v * v).sum())
    t_now = 2.0 * ke / ((3 * n - 3) * KB_EV_PER_K)
    return v * math.sqrt(temperature / t_now)


# ---------------------------------------------------------------------------
# Potential parameter sets
# ---------------------------------------------------------------------------
# Finnis-Sinclair bcc Fe: phi(r) = (r-d)^2 + beta (r-d)^3 / d  (r < d),
# V(r) = (r-c)^2 (c0 + c1 r + c2 r^2)  (r < c), F(rho) = -A sqrt(rho).
FS_FE = dict(d=3.569745, c=3.40, A=1.828905, beta=1.8, c0=1.2371147, c1=-0.3592185, c2=-0.0385607)
# Sutton-Chen Cu (Sutton & Chen 1990): V = eps (a/r)^n, phi = (a/r)^m, F = -eps c sqrt(rho)
SC_CU = dict(eps=1.2382e-2, c=39.432, a=3.61, n=9, m=6)

POT_FS_ANALYTIC = 1
POT_TABLES = 2
POT_SURROGATE = 3
POT_KNOTS = 4


@dataclasses.dataclass
class Potential:
    """A potential as data.  kind 1: single-species analytic FS (coefficients `fs`).
    kind 2: knot tables; `tables` holds, for each table, n_knots values followed by
    n_knots slopes, in the order V[a][b] (a,b < ns), phi[a][b] (density at an atom of
    species a due to a neighbour of species b), F[a].  r-tables span [r_min, r_cut],
    F-tables span [rho_min, rho_max]; knots are uniform."""
    kind: int
    atomic_numbers: np.ndarray
    masses: np.ndarray
    r_cut: float
    fs: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(7))
    n_knots: int = 0
    r_min: float = 0.0
    rho_min: float = 0.0
    rho_max: float = 0.0
    tables: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0))

    @property
    def n_species(self) -> int:
        return int(self.atomic_numbers.shape[0])


def fs_fe_analytic() -> Potential:
    p = FS_FE
    return Potential(kind=POT_FS_ANALYTIC, atomic_numbers=np.array([26], dtype=np.int32),
                     masses=np.array([MASS_AMU[26]]), r_cut=max(p["d"], p["c"]),
                     fs=np.array([p["d"], p["c"], p["A"], p["beta"], p["c0"], p["c1"], p["c2"]]))


def _sample(f, df, lo, hi, n):
    x = np.linspace(lo, hi, n)
    return np.concatenate([f(x), df(x)])


def _shifted(f, df, rc):
    """Shifted-force form: value and slope both vanish at rc."""
    frc, dfrc = f(rc), df(rc)
    return (lambda r: np.where(r < rc, f(r) - frc - (r - rc) * dfrc, 0.0),
            lambda r: np.where(r < rc, df(r) - dfrc, 0.0))


def sc_cu_tables(n_knots: int = 5000, lattice_a: float = 3.615, r_min: float = 1.0) -> Potential:
    """Sutton-Chen Cu sampled into cubic-Hermite knot tables, cutoff 2a (shifted-force)."""
    p = SC_CU
    rc = 2.0 * lattice_a
    eps, c, a, n, m = p["eps"], p["c"], p["a"], p["n"], p["m"]
    V, dV = _shifted(lambda r: eps * (a / r) ** n, lambda r: -n * eps * (a / r) ** n / r, rc)
    P, dP = _shifted(lambda r: (a / r) ** m, lambda r: -m * (a / r) ** m / r, rc)
    # density range: around the perfect-lattice value of the shifted phi
    pos, _ = replicate(FCC_BASIS, (1, 1, 1), lattice_a)
    rho0 = _lattice_sum(P, FCC_BASIS, lattice_a, rc)
    rho_min, rho_max = rho0 / 20.0, 2.0 * rho0
    F = lambda x: -eps * c * np.sqrt(x)
    dF = lambda x: -0.5 * eps * c / np.sqrt(x)
    tables = np.concatenate([_sample(V, dV, r_min, rc, n_knots), _sample(P, dP, r_min, rc, n_knots),
                             _sample(F, dF, rho_min, rho_max, n_knots)])
    return Potential(kind=POT_TABLES, atomic_numbers=np.array([29], dtype=np.int32),
                     masses=np.array([MASS_AMU[29]]), r_cut=rc, n_knots=n_knots, r_min=r_min,
                     rho_min=rho_min, rho_max=rho_max, tables=tables)


def _fs_fe_funcs():
    p = FS_FE
    d, cc, beta = p["d"], p["c"], p["beta"]
    c0, c1, c2 = p["c0"], p["c1"], p["c2"]
    phi = lambda r: np.where(r < d, (r - d) ** 2 + beta * (r - d) ** 3 / d, 0.0)
    dphi = lambda r: np.where(r < d, 2 * (r - d) + 3 * beta * (r - d) ** 2 / d, 0.0)
    V = lambda r: np.where(r < cc, (r - cc) ** 2 * (c0 + c1 * r + c2 * r * r), 0.0)
    dV = lambda r: np.where(r < cc, 2 * (r - cc) * (c0 + c1 * r + c2 * r * r)
                            + (r - cc) ** 2 * (c1 + 2 * c2 * r), 0.0)
    return V, dV, phi, dphi


def fs_fe_tables(n_knots: int = 5000, r_min: float = 1.0) -> Potential:
    """The analytic FS Fe potential sampled into knot tables (same cutoff)."""
    V, dV, P, dP = _fs_fe_funcs()
    rc = max(FS_FE["d"], FS_FE["c"])
    A = FS_FE["A"]
    rho_min, rho_max = 0.3, 14.0
    F = lambda x: -A * np.sqrt(x)
    dF = lambda x: -0.5 * A / np.sqrt(x)
    tables = np.concatenate([_sample(V, dV, r_min, rc, n_knots), _sample(P, dP, r_min, rc, n_knots),
                             _sample(F, dF, rho_min, rho_max, n_knots)])
    return Potential(kind=POT_TABLES, atomic_numbers=np.array([26], dtype=np.int32),
                     masses=np.array([MASS_AMU[26]]), r_cut=rc, n_knots=n_knots, r_min=r_min,
                     rho_min=rho_min, rho_max=rho_max, tables=tables)


def _knot_sum(coef, knots):
    """The paper's cubic-spline knot-sum form f(r) = sum_k a_k (r_k - r)^3 H(r_k - r) (§3.1.1)."""
    coef = np.asarray(coef, dtype=np.float64)
    knots = np.asarray(knots, dtype=np.float64)

    def f(r):
        r = np.asarray(r, dtype=np.float64)[..., None]
        s = np.clip(knots - r, 0.0, None)
        return (coef * s ** 3).sum(axis=-1)

    def df(r):
        r = np.asarray(r, dtype=np.float64)[..., None]
        s = np.clip(knots - r, 0.0, None)
        return (-3.0 * coef * s ** 2).sum(axis=-1)

    return f, df


def _fe_knot_fit():
    """A Finnis-Sinclair-like Fe as 15 cubic knot terms (§3.1.1 form): 8 for V on knots evenly in
    2.3..c, 7 for phi evenly in 2.1..d, coefficients from a least-squares fit of FS Fe's V and phi
    on 1.8..d (the 15-term cubic-spline iron of the paper's scaling tests, §5.1)."""
    V, _, P, _ = _fs_fe_funcs()
    d, cc = FS_FE["d"], FS_FE["c"]
    r = np.linspace(1.8, d, 600)
    rkv, rkp = np.linspace(2.3, cc, 8), np.linspace(2.1, d, 7)
    basis = lambda rk: np.clip(rk[None, :] - r[:, None], 0.0, None) ** 3
    av = np.linalg.lstsq(basis(rkv), V(r), rcond=None)[0]
    ap = np.linalg.lstsq(basis(rkp), P(r), rcond=None)[0]
    return (av, rkv), (ap, rkp)


def fe_knots() -> Potential:
    """bcc Fe potential given as explicit cubic knot sums (kind 4): V and phi = sum_k c_k (r_k - r)^3
    for r < r_k, F = -A sqrt(rho).  `tables` = V (8 coefficients, 8 radii), phi (the same, the
    8th term zero), then A.  r_cut = the largest knot."""
    (av, rkv), (ap, rkp) = _fe_knot_fit()
    K = 8
    ap8, rkp8 = np.concatenate([ap, [0.0]]), np.concatenate([rkp, [rkp[-1]]])
    tables = np.concatenate([av, rkv, ap8, rkp8, [FS_FE["A"]]])
    return Potential(kind=POT_KNOTS, atomic_numbers=np.array([26], dtype=np.int32),
                     masses=np.array([MASS_AMU[26]]), r_cut=float(max(rkv.max(), rkp.max())), n_knots=K,
                     tables=tables)


def fe_knot_tables(n_knots: int = 5000, r_min: float = 1.0) -> Potential:
    """The same 15-term Fe potential sampled into cubic-Hermite knot tables (kind 2)."""
    (av, rkv), (ap, rkp) = _fe_knot_fit()
    V, dV = _knot_sum(av, rkv)
    P, dP = _knot_sum(ap, rkp)
    rc = float(max(rkv.max(), rkp.max()))
    A = FS_FE["A"]
    rho_min, rho_max = 0.3, 14.0
    tables = np.concatenate([_sample(V, dV, r_min, rc, n_knots), _sample(P, dP, r_min, rc, n_knots),
                             _sample(lambda x: -A * np.sqrt(x), lambda x: -0.5 * A / np.sqrt(x), rho_min, rho_max,
                                     n_knots)])
    return Potential(kind=POT_TABLES, atomic_numbers=np.array([26], dtype=np.int32),
                     masses=np.array([MASS_AMU[26]]), r_cut=rc, n_knots=n_knots, r_min=r_min,
                     rho_min=rho_min, rho_max=rho_max, tables=tables)


def fe_c_knots(seed: int = 4) -> Potential:
    """Two-species Fe-C as explicit knot sums (kind 4): Fe-Fe is the 15-term Fe fit, the terms with
    C are the seeded knot sums of fe_c_tables (same seed, same draws).  K = 8 terms per function."""
    (av, rkv), (ap, rkp) = _fe_knot_fit()
    u = random_uniform(seed, 7, 64)
    K = 8

    def pad(c, r):
        c, r = list(c), list(r)
        return np.array(c + [0.0] * (K - len(c))), np.array(r + [r[-1]] * (K - len(r)))

    V = {(0, 0): (av, rkv),
         (0, 1): pad([0.9 + 0.2 * u[0], 0.05 + 0.05 * u[1], 0.01 * u[2]], [1.9, 2.6, 3.5]),
         (1, 1): pad([1.0 + 0.2 * u[3], 0.02 * u[4]], [2.2, 3.5])}
    V[(1, 0)] = V[(0, 1)]
    P = {(0, 0): pad(ap, rkp),
         (0, 1): pad([0.30 + 0.1 * u[5], 0.02 + 0.02 * u[6]], [2.4, 3.5]),
         (1, 0): pad([0.25 + 0.1 * u[7], 0.02 + 0.02 * u[8]], [2.6, 3.5]),
         (1, 1): pad([0.05 + 0.02 * u[9]], [3.5])}
    parts = [np.concatenate(V[(a, b)]) for a in range(2) for b in range(2)]
    parts += [np.concatenate(P[(a, b)]) for a in range(2) for b in range(2)]
    parts.append(np.array([FS_FE["A"], 1.0 + 0.3 * u[10]]))
    rc = max(FS_FE["d"], FS_FE["c"], 3.5)
    return Potential(kind=POT_KNOTS, atomic_numbers=np.array([26, 6], dtype=np.int32),
                     masses=np.array([MASS_AMU[26], MASS_AMU[6]]), r_cut=float(rc), n_knots=K,
                     tables=np.concatenate(parts))


def fe_c_tables(seed: int = 4, n_knots: int = 5000, r_min: float = 1.0) -> Potential:
    """Two-species Fe-C tables: Fe-Fe is FS Fe; every term involving C is a seeded knot sum
    with knots <= 3.5 Å (repulsive Fe-C and C-C cores, positive densities).  V is symmetric."""
    V_ff, dV_ff, P_ff, dP_ff = _fs_fe_funcs()
    rc = max(FS_FE["d"], FS_FE["c"])
    u = random_uniform(seed, 7, 64)
    # Fe-C pair: repulsive, knots at 1.9..3.5
    V_fc = _knot_sum([0.9 + 0.2 * u[0], 0.05 + 0.05 * u[1], 0.01 * u[2]], [1.9, 2.6, 3.5])
    V_cc = _knot_sum([1.0 + 0.2 * u[3], 0.02 * u[4]], [2.2, 3.5])
    P_fc = _knot_sum([0.30 + 0.1 * u[5], 0.02 + 0.02 * u[6]], [2.4, 3.5])   # density at Fe from C
    P_cf = _knot_sum([0.25 + 0.1 * u[7], 0.02 + 0.02 * u[8]], [2.6, 3.5])   # density at C from Fe
    P_cc = _knot_sum([0.05 + 0.02 * u[9]], [3.5])
    A_c = 1.0 + 0.3 * u[10]
    A = FS_FE["A"]
    rho_min, rho_max = 0.3, 14.0
    F_fe = (lambda x: -A * np.sqrt(x), lambda x: -0.5 * A / np.sqrt(x))
    F_c = (lambda x: -A_c * np.sqrt(x), lambda x: -0.5 * A_c / np.sqrt(x))
    r_tab = lambda fd: _sample(fd[0], fd[1], r_min, rc, n_knots)
    Vs = [[(V_ff, dV_ff), V_fc], [V_fc, V_cc]]
    Ps = [[(P_ff, dP_ff), P_fc], [P_cf, P_cc]]
    parts = [r_tab(Vs[a][b]) for a in range(2) for b in range(2)]
    parts += [r_tab(Ps[a][b]) for a in range(2) for b in range(2)]
    parts += [_sample(F_fe[0], F_fe[1], rho_min, rho_max, n_knots),
              _sample(F_c[0], F_c[1], rho_min, rho_max, n_knots)]
    return Potential(kind=POT_TABLES, atomic_numbers=np.array([26, 6], dtype=np.int32),
                     masses=np.array([MASS_AMU[26], MASS_AMU[6]]), r_cut=rc, n_knots=n_knots,
                     r_min=r_min, rho_min=rho_min, rho_max=rho_max, tables=np.concatenate(parts))


def _lattice_sum(f, basis, a, rc):
    """Sum of f over all neighbours of the atom at the origin in the infinite lattice (r < rc)."""
    m = int(math.ceil(rc / a)) + 1
    g = np.arange(-m, m + 1, dtype=np.float64)
    cells = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    pts = ((cells[:, None, :] + basis[None, :, :]).reshape(-1, 3)) * a
    r = np.sqrt((pts * pts).sum(axis=1))
    r = r[(r > 1e-9) & (r < rc)]
    return float(f(r).sum())


# ---------------------------------------------------------------------------
# Workloads shaped like the paper's (bcc Fe cubes 2n^3, §5.1) and the larger ones
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    name: str
    pos: np.ndarray            # (N,3) Å, unwrapped
    vel: np.ndarray            # (N,3) Å/fs
    species: np.ndarray        # (N,) int32 index into potential species
    box: np.ndarray            # (3,) orthorhombic box lengths Å
    potential: Potential
    skin: float
    k_max: int
    dt_fs: float
    steps: int
    temperature: float
    strain_rate_zz: float = 0.0   # 1/s, applied each step

    @property
    def n_atoms(self) -> int:
        return int(self.pos.shape[0])


def bcc_fe(n: int, seed: int, temperature: float = 300.0, sigma: float = 0.05, tables: bool = False,
           steps: int = 100, dt_fs: float = 1.0, a: float = 2.8665, cells=None, potential=None) -> Workload:
    cells = cells or (n, n, n)
    pos, box = replicate(BCC_BASIS, cells, a)
    pos = gaussian_displace(pos, sigma, seed)
    pot = potential if potential is not None else (fs_fe_tables() if tables else fs_fe_analytic())
    species = np.zeros(pos.shape[0], dtype=np.int32)
    vel = maxwell_boltzmann(pot.masses[species], temperature, seed)
    return Workload(name=f"bcc Fe {cells[0]}x{cells[1]}x{cells[2]}", pos=pos, vel=vel, species=species,
                    box=box, potential=pot, skin=0.3, k_max=32, dt_fs=dt_fs, steps=steps,
                    temperature=temperature)


def fcc_cu(n: int, seed: int, temperature: float = 300.0, n_knots: int = 5000, steps: int = 1000,
           dt_fs: float = 2.0, a: float = 3.615, sigma: float = 0.0) -> Workload:
    pos, box = replicate(FCC_BASIS, (n, n, n), a)
    if sigma > 0.0:
        pos = gaussian_displace(pos, sigma, seed)
    pot = sc_cu_tables(n_knots=n_knots, lattice_a=a)
    species = np.zeros(pos.shape[0], dtype=np.int32)
    vel = maxwell_boltzmann(pot.masses[species], temperature, seed)
    return Workload(name=f"fcc Cu {n}x{n}x{n}", pos=pos, vel=vel, species=species, box=box,
                    potential=pot, skin=0.3, k_max=176, dt_fs=dt_fs, steps=steps, temperature=temperature)


def cell_count_gas(counts, cells: int = 4, seed: int = 5, skin: float = 0.3, k_max: int = 320) -> Workload:
    """Cu atoms (the Sutton-Chen tables' r_cut) in a cubic box of cells^3 link cells, each edge
    cells x 1.01 r_list long, link cell c (x fastest) holding counts[c] atoms at uniform random
    positions inside it, at least 2 % of its width from its faces; zero velocities.  A neighbour
    list case only: atoms may sit arbitrarily close together."""
    counts = np.asarray(counts, dtype=np.int64)
    assert counts.shape == (cells ** 3,)
    pot = sc_cu_tables(n_knots=500)
    w = 1.01 * (pot.r_cut + skin)
    u = random_uniform(seed, 12, 3 * int(counts.sum())).reshape(-1, 3)
    c = np.repeat(np.arange(cells ** 3), counts)
    corner = np.stack([c % cells, (c // cells) % cells, c // (cells * cells)], axis=1) * w
    pos = corner + w * (0.02 + 0.96 * u)
    n = pos.shape[0]
    return Workload(name=f"gas {cells}^3 cells", pos=pos, vel=np.zeros_like(pos),
                    species=np.zeros(n, dtype=np.int32), box=np.full(3, cells * w), potential=pot,
                    skin=skin, k_max=k_max, dt_fs=2.0, steps=1, temperature=0.0)


def bcc_fe_c(n: int, seed: int, temperature: float = 600.0, c_fraction: float = 0.001,
             steps: int = 200, dt_fs: float = 1.0, a: float = 2.8665,
             strain_rate_zz: float = -1.0e9) -> Workload:
    """bcc Fe with round(c_fraction * N_Fe) C atoms on distinct, seeded octahedral sites."""
    fe, box = replicate(BCC_BASIS, (n, n, n), a)
    sites, _ = replicate(BCC_OCTA_BASIS, (n, n, n), a)
    n_c = int(round(c_fraction * fe.shape[0]))
    keys = random_u64(seed, 3, sites.shape[0])
    chosen = np.sort(np.argsort(keys, kind="stable")[:n_c])
    pos = np.concatenate([fe, sites[chosen]])
    species = np.concatenate([np.zeros(fe.shape[0], np.int32), np.ones(n_c, np.int32)])
    pos = gaussian_displace(pos, 0.05, seed)
    pot = fe_c_tables(seed=seed)
    vel = maxwell_boltzmann(pot.masses[species], temperature, seed)
    return Workload(name=f"bcc Fe-C {n}^3 + {n_c} C", pos=pos, vel=vel, species=species, box=box,
                    potential=pot, skin=0.3, k_max=40, dt_fs=dt_fs, steps=steps,
                    temperature=temperature, strain_rate_zz=strain_rate_zz)


def replica_recipe(n_replicas: int = 256, seed: int = 3000):
    """Sizes and temperatures of the uneven-replica workload: replica r is bcc Fe of 2 n_r^3 atoms
    with n_r ~ U{10..30} and T_r ~ U[300, 1200] K, drawn from stream 11 of `seed` (the first
    256 draws give the sizes, the next 256 the temperatures); its own seed is seed + r."""
    u = random_uniform(seed, 11, 512)
    sizes = (10 + np.floor(u[:256] * 21)).astype(int)[:n_replicas]
    temps = (300.0 + 900.0 * u[256:])[:n_replicas]
    return sizes, temps


def fe_replicas(indices=None, n_replicas: int = 256, seed: int = 3000):
    """Workloads of the replicas `indices` (default all) of replica_recipe, and their temperatures."""
    sizes, temps = replica_recipe(n_replicas, seed)
    idx = range(n_replicas) if indices is None else indices
    ws = [bcc_fe(int(sizes[r]), seed=seed + r, temperature=float(temps[r])) for r in idx]
    return ws, np.array([temps[r] for r in idx])


# ----------------------------------------------------------------------------- surrogate
# Radial-basis descriptor and network shape of the learned per-atom energy: 32 Gaussians of
# width 0.1 Å centred evenly on 1.5-3.6 Å, cosine cutoff at 4.0 Å, list radius 4.3 Å; a
# 32-64-64-1 network.
SUR_FE = dict(nb=32, h1=64, h2=64, mu0=1.5, dmu=2.1 / 31.0, width=0.1, rd=4.0, skin=0.3, k_max=48)


def sur_n_params(spec=SUR_FE) -> int:
    nb, h1, h2 = spec["nb"], spec["h1"], spec["h2"]
    return h1 * nb + h1 + h2 * h1 + h2 + h2 + 1


def sur_init_weights(seed: int, spec=SUR_FE, scale: float = 1.0) -> np.ndarray:
    """Seeded Glorot-uniform weights, zero biases, packed W1 [h1][nb], b1, W2 [h2][h1], b2, w3, b3."""
    nb, h1, h2 = spec["nb"], spec["h1"], spec["h2"]
    parts = []
    for s, (fan_out, fan_in) in enumerate([(h1, nb), (h2, h1), (1, h2)]):
        lim = scale * np.sqrt(6.0 / (fan_in + fan_out))
        w = (2.0 * random_uniform(seed, 40 + s, fan_out * fan_in) - 1.0) * lim
        parts += [w, np.zeros(fan_out)]
    return np.concatenate(parts)


def surrogate_potential(spec=SUR_FE) -> Potential:
    """The potential record of a surrogate context: Fe mass, range = descriptor cutoff."""
    return Potential(kind=POT_SURROGATE, atomic_numbers=np.array([26], dtype=np.int32),
                     masses=np.array([MASS_AMU[26]]), r_cut=float(spec["rd"]))


def as_surrogate(w: Workload, spec=SUR_FE) -> Workload:
    """The same atoms with the surrogate's potential record, list skin and capacity."""
    return dataclasses.replace(w, potential=surrogate_potential(spec), skin=float(spec["skin"]),
                               k_max=int(spec["k_max"]), name=w.name + " (surrogate)")
