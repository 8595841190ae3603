"""The error bound of the mixed-precision force pass, derived per atom from the potential and
the configuration (no fitted constant).

The mixed path (md.h MD_PREC_MIXED) evaluates the pair terms of Eq. (1)'s gradient in FP32 from
FP32 copies of the coordinates, wrapped into the periodic image of the last list build.  Its
force on atom i differs from the FP64 oracle's by at most, to first order in the FP32 unit
roundoff u = 2^-24:

  C_i   the coordinates' rounding, computed EXACTLY: the oracle's force at the FP32 coordinates
        the passes read (md_get MD_GET_IMAGE) in the box rounded to FP32 (the periodic shifts
        of the FP32 minimum image), minus its force at the FP64 positions;
  12 u q_i   the FP32 evaluation of r: r^2 (3 roundings), the reciprocal square root (<= 2 ulp),
        r = r^2 / sqrt(r^2) (1), the subtraction of the periodic shift (<= 3 u of r at the
        shortest pair) and the knot index (2): a relative change of r of at most 12 u, whose
        effect on the force is at most 12 u q_i (q_i: r |d/dr| of every pair term);
  B_i   atoms within r_list + skin of a box face only: a pair that crosses the face is formed
        from coordinates on opposite sides, as x_j - x_i of size ~L rounded to FP32 before the
        periodic shift (the minimum image of the list walk; the group walks instead add the
        stencil's shift to a coordinate, a rounding of the same size): up to half an ulp of
        L + r_list + skin per component, i.e. a change of the separation of at most
        sqrt(3) ulp / 2, relative sqrt(3) ulp / (2 r_min) of r and of its direction, hence
        B_i = (q_i + m_i) sqrt(3) ulp / (2 r_min);
  (9 + n_i + log2 T + K_t) u m_i   the FP32 pair term (F' rounded to FP32, the derivative
        cubic, the combination, the scaling by 1/r: 9 roundings of each term's size) and its
        recursive summation over n_i = ceil(K_i / T) list entries per lane, then log2 T lane
        sums (m_i: the sum of the absolute terms; K_t: the terms of an explicit knot sum, whose
        sum of absolute terms is then taken as its size);
  12 u e_i   the density sum: every phi term (and its r) within 12 u, summed error-free, moves
        F' by F'' times that (e_i);
  2^-11 c_i   with knot tables, the quadratic and cubic coefficients of the derivative cubic
        held as scaled binary16 (unit roundoff 2^-11): per pair at most 2^-11 (|2 c2| + |3 c3|) / h
        of V' on the pair's interval, plus |F'_i| and |F'_j| times that of phi'_ab and phi'_ba
        (c_i: their sum over the pairs).

The bound is per atom and per force component (every term bounds a vector norm).
"""
import math

import numpy as np

import oracle

U32 = 2.0 ** -24


U16 = 2.0 ** -11


def mixed_force_bound(w, pos, image, box=None, lanes=1):
    """Per-atom bound (N,) on |F_mixed - F_oracle| (any component) at positions `pos` (FP64,
    caller order), where `image` is the context's MD_GET_IMAGE at those positions; `box` the
    current box (default w.box); `lanes` the lanes per atom of the force pass (1 when unknown:
    the longest sequential sum; the group walks' shared-memory sums are no longer)."""
    box = np.asarray(w.box if box is None else box, np.float64)
    pot = w.potential
    ref = oracle.forces(pos, w.species, box, pot, skin=w.skin, k_max=w.k_max, method="cells")
    box32 = box.astype(np.float32).astype(np.float64)
    rnd = oracle.forces(np.asarray(image, np.float64), w.species, box32, pot, skin=w.skin, k_max=w.k_max,
                        method="cells")
    C = np.abs(rnd["force"] - ref["force"]).max(axis=1)
    sc = oracle.eam_error_scales(pos, w.species, box, pot, ref["count"], ref["list"], ref["dF"])
    rc = float(pot.r_cut)
    d = []
    for i in range(min(len(pos), 4096)):          # the shortest pair distance of a sample
        c = ref["count"][i]
        if c:
            dv = pos[ref["list"][i, :c]] - pos[i]
            dv -= box * np.rint(dv / box)
            d.append(np.sqrt((dv ** 2).sum(axis=1)).min())
    r_lo = min(d) if d else rc
    k_in = ref["count"].astype(np.float64)
    n_seq = np.ceil(k_in / max(1, int(lanes)))
    k_terms = float(pot.n_knots) if int(pot.kind) == 4 else 0.0
    arith = U32 * (12.0 * sc["q"] + (9.0 + n_seq + math.log2(max(1, int(lanes))) + k_terms) * sc["m"]
                   + 12.0 * sc["e"])
    b16 = U16 * sc["c"]
    reach = rc + 2.0 * float(w.skin)
    img = np.asarray(image, np.float64)
    near = np.any((img < reach) | (img > box - reach), axis=1)
    top = float(np.max(box)) + reach
    ulp = 2.0 ** (math.floor(math.log2(top)) - 23)
    edge = np.where(near, (sc["q"] + sc["m"]) * math.sqrt(3.0) * ulp / (2.0 * r_lo), 0.0)
    return C + arith + b16 + edge, ref


def assert_mixed_forces(w, pos, f_gpu, image, box=None, lanes=1, pe=None, pe_tol=1e-6):
    """Every component of every mixed force within its atom's derived bound; returns the ratio
    of the largest error to the bound of its atom (for the record) and the oracle's result."""
    bound, ref = mixed_force_bound(w, pos, image, box, lanes)
    err = np.abs(np.asarray(f_gpu) - ref["force"]).max(axis=1)
    bad = np.nonzero(err > bound)[0]
    assert bad.size == 0, (f"{bad.size} atoms outside the derived bound; worst atom {bad[0]}: "
                           f"error {err[bad[0]]:.3e} > bound {bound[bad[0]]:.3e}")
    if pe is not None:
        assert abs(pe - ref["pe"]) <= pe_tol * abs(ref["pe"])
    return float((err / np.maximum(bound, 1e-300)).max()), ref
