"""The mixed path's binary16 table coefficients, bounded on the CPU.

With one species, the mixed force pass evaluates the t-derivative of each table cubic,
c1 + t (2 c2 + 3 c3 t), with 2 c2 and 3 c3 rounded to binary16 after scaling each function's pair
by a power of two that puts the larger magnitude in [2^14, 2^15).  Here the pair terms of the
force (gradient of Eq. (1)) are evaluated from the tables' Hermite knots (value and slope at each
knot) over every pair of a thermal Cu state, once exactly and once with those coefficients
rounded, and the difference of the summed forces is held to the binary16 share of the derived
mixed bound (tests/mixed_bound.py), which must itself be a small part of the whole bound.
"""
import numpy as np

import oracle
from mixed_bound import U16
from paper_1107_2619_gb300 import inputs as I


def _cubic_rows(tab, n, h):
    """Cubic of each knot interval in t = (r - r_k) / h from the Hermite data (y_k, y'_k)."""
    y, s = tab[:n], tab[n:]
    y1, s1 = np.append(y[1:], y[-1]), np.append(s[1:], s[-1])
    return np.stack([y, h * s, 3.0 * (y1 - y) - h * (2.0 * s + s1), 2.0 * (y - y1) + h * (s + s1)], axis=1)


def _binary16(a2, a3):
    e = np.floor(np.log2(max(np.abs(a2).max(), np.abs(a3).max()))) - 14
    q = lambda a: (a / 2.0 ** e).astype(np.float32).astype(np.float16).astype(np.float64) * 2.0 ** e
    return q(a2), q(a3)


def _pair_forces(w, dF, rows_v, rows_p, h, rounded):
    pot = w.potential
    count, nl, _ = oracle.neighbours(w.pos, w.box, pot.r_cut + w.skin, w.k_max, "brute")
    i = np.repeat(np.arange(w.n_atoms), count)
    j = nl[nl >= 0]
    d = w.pos[j] - w.pos[i]
    d -= w.box * np.rint(d / w.box)
    r = np.sqrt((d * d).sum(axis=1))
    keep = r < pot.r_cut
    i, j, d, r = i[keep], j[keep], d[keep], r[keep]
    x = (r - pot.r_min) / h
    k = np.floor(x).astype(int)
    t = x - k

    def deriv(rows):
        a2, a3 = 2.0 * rows[:, 2], 3.0 * rows[:, 3]
        if rounded:
            a2, a3 = _binary16(a2, a3)
        return (rows[k, 1] + t * (a2[k] + a3[k] * t)) / h

    g = (deriv(rows_v) + (dF[i] + dF[j]) * deriv(rows_p)) / r
    f = np.zeros((w.n_atoms, 3))
    np.add.at(f, i, g[:, None] * d)
    return f


def test_binary16_derivative_coefficients_within_their_share_of_the_derived_bound():
    w = I.fcc_cu(8, seed=2, sigma=0.08)
    pot = w.potential
    n = pot.n_knots
    h = (pot.r_cut - pot.r_min) / (n - 1)
    rows_v = _cubic_rows(pot.tables[:2 * n], n, h)
    rows_p = _cubic_rows(pot.tables[2 * n:4 * n], n, h)
    ref = oracle.forces(w.pos, w.species, w.box, pot, skin=w.skin, k_max=w.k_max, method="brute")
    fmax = np.abs(ref["force"]).max()
    exact = _pair_forces(w, ref["dF"], rows_v, rows_p, h, rounded=False)
    # the pair model is the oracle's force: the bound below is about the rounding alone
    assert np.abs(exact - ref["force"]).max() <= 1e-10 * fmax
    rounded = _pair_forces(w, ref["dF"], rows_v, rows_p, h, rounded=True)
    err = np.abs(rounded - exact).max(axis=1)
    share = U16 * oracle.eam_error_scales(w.pos, w.species, w.box, pot, ref["count"], ref["list"], ref["dF"])["c"]
    assert 0.0 < err.max() and np.all(err <= share)
    assert err.max() <= 2e-5 and share.max() <= 1e-4


def test_binary16_scaling_bound_over_any_dynamic_range():
    """The scale puts the largest magnitude in [2^14, 2^15): every coefficient is then within
    2^-11 of itself (times 1 + 2^-12 for the rounding to FP32 on the way), or within 2^-25 of the
    scale where it underflows, over twelve decades of magnitude."""
    u = I.random_uniform(41, 1, 200000)
    a = np.sign(u - 0.5) * 10.0 ** (-12.0 * I.random_uniform(41, 2, 200000))
    a2, a3 = _binary16(a[:100000], a[100000:])
    q = np.concatenate([a2, a3])
    scale = 2.0 ** (np.floor(np.log2(np.abs(a).max())) - 14)
    assert 2.0 ** 14 <= np.abs(a).max() / scale < 2.0 ** 15
    err = np.abs(q - a)
    rel = 2.0 ** -11 * (1.0 + 2.0 ** -12)
    assert np.all(err <= np.maximum(rel * np.abs(a), 2.0 ** -25 * scale))
    normal = np.abs(a) >= 2.0 ** -14 * scale
    assert normal.sum() > 50000 and np.all(err[normal] <= rel * np.abs(a[normal]))
