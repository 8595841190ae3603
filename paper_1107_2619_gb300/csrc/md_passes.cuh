// Per-item device functions of the two EAM passes (the two sums of Eq. (1)), FP64 and mixed.
// An item is one lane of one atom: item g -> atom i = g / T, lane g % T.  Every lane of a
// warp must call an item function in the same iteration (the lane sums use shuffles), so
// callers iterate over a range rounded up to whole warps and pass items past the end too.
//
//   density:  rho_i = sum_j phi_{s_i s_j}(r_ij);  F_i = F(rho_i), F'_i;  pass-2 copy of (r_i, F'_i)
//   force:    f_i = sum_j [V'(r) + F'_i phi'_{s_i s_j}(r) + F'_j phi'_{s_j s_i}(r)] d / r, d = r_j - r_i,
//             then (optionally) the second half kick v += (dt/2) f/m and the FP64 partial sums.
// Mixed precision: pair and density terms FP32 from FP32 wrapped coordinates, density sum
// error-free in an FP32 (hi, lo) pair rounded to FP64 before F(rho); F, F', kick, sums FP64.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <type_traits>

#include "md_df.cuh"
#include "md_eam_common.cuh"
#include "md_phases.cuh"

namespace mdk {
namespace ps {

using namespace eam;

__device__ __forceinline__ float mi32(float d, float L, float invL) { return fmaf(-L, rintf(d * invL), d); }
// The FP64 passes' minimum image, for separations of coordinates kept in one periodic image of
// the box (|d| < 3L/2): d - L rint(d / L) as one subtraction of L with the sign of d, or of 0,
// chosen and signed on the bit patterns in integer registers (|d| > L/2, L/2 by the exponent
// field), so that the FP64 pipe does the one subtraction only.  Where |d / L| rounds to exactly
// 1/2 the choice may differ from rint's, but such a pair is L/2 apart, far beyond r_list, either
// way.
__device__ __forceinline__ double mi64s(double d, double L, double &shift) {
    const long long b = __double_as_longlong(d);
    const bool far = (b & 0x7FFFFFFFFFFFFFFFLL) > __double_as_longlong(L) - (1LL << 52);
    const long long sL = __double_as_longlong(L) | (b & (long long)0x8000000000000000ULL);   // L, sign of d
    shift = far ? __longlong_as_double(sL) : 0.0;
    return d - shift;
}
__device__ __forceinline__ double mi64(double d, double L, double) {
    double s;
    return mi64s(d, L, s);
}
// The image shift s = d_raw - d of one pair (zero off the box boundary), for the virial.
template <typename WRAP>
__device__ __forceinline__ double sep64s(double d, double L, double &s) {
    if (WRAP::value) return mi64s(d, L, s);
    s = 0.0;
    return d;
}

// The pair walk's virial (energy steps).  With d = x_j - x_i - s (s the image shift) and -g d
// the neighbour's share, sum over pairs d_a (-g d)_b equals sum over atoms x_a F_b (the kick
// phase adds it, from the force on each atom) minus sum over pairs s_a (-g d)_b, which only pairs
// across the box boundary have: so each pair adds nothing, and those six products only where s
// is not zero.
__device__ __forceinline__ void virial_shift(double sx, double sy, double sz, double ngx, double ngy, double ngz,
                                             double &wxx, double &wyy, double &wzz, double &wyz, double &wxz,
                                             double &wxy) {
    if (((unsigned long long)(__double_as_longlong(sx) | __double_as_longlong(sy) | __double_as_longlong(sz))) << 1) {
        wxx = fma(-sx, ngx, wxx);
        wyy = fma(-sy, ngy, wyy);
        wzz = fma(-sz, ngz, wzz);
        wyz = fma(-sy, ngz, wyz);
        wxz = fma(-sx, ngz, wxz);
        wxy = fma(-sx, ngy, wxy);
    }
}

// A knot row's cubic at t, continued linearly below the first knot (cubic() with `below`): there
// c2 and c3 are taken as 0, chosen in integer registers, so the linear branch costs no second
// evaluation on the FP64 pipe (fma(t, 0, 0) = 0 and fma(t, 0, c1) = c1 exactly).
__device__ __forceinline__ double cubic64(double t, const double4_32a &c, bool below) {
    const double c2 = below ? 0.0 : c.z, c3 = below ? 0.0 : c.w;
    return fma(t, fma(t, fma(t, c3, c2), c.y), c.x);
}

// The minimum image of a separation, or the separation itself for an atom whose link cell was not
// on the box boundary at the last build (A.wrap) while the FP32 positions stay in the image of
// that build (A.image_fixed: no strain ramp): none of its list entries is then a periodic image,
// |d| < L/2, rint(d / L) = 0 and the minimum image returns d unchanged, so skipping it changes no
// bit.  WRAP is a compile-time tag (std::true_type / std::false_type).
template <typename WRAP>
__device__ __forceinline__ float sep32(float d, float L, float invL) {
    return WRAP::value ? mi32(d, L, invL) : d;
}
template <typename WRAP>
__device__ __forceinline__ double sep64(double d, double L, double invL) {
    return WRAP::value ? mi64(d, L, invL) : d;
}

// Whether the warp of atom i (lane: every lane of the warp calls it together) takes the minimum
// image: when any of its atoms needs it, all do (the same bits, and no divergence between the
// two walks inside a warp).
__device__ __forceinline__ bool needs_image(const Atoms &A, int i, bool live) {
    const bool w = live && (!A.image_fixed || ld_phase(A.wrap + i) != 0);
    return __any_sync(0xffffffffu, w);
}

// Knot-table row of a species pair: (V c0..c3, phi c0..c3) as 8 floats in one 32-byte load.
__device__ __forceinline__ void row32(const double4_32a *tab, size_t idx, float (&v)[4], float (&p)[4]) {
    const double4_32a d = tab[idx];
    unpack2(d.x, v[0], v[1]);
    unpack2(d.y, v[2], v[3]);
    unpack2(d.z, p[0], p[1]);
    unpack2(d.w, p[2], p[3]);
}

__device__ __forceinline__ float4 phi_half32(const double4_32a *tab, size_t idx) {
    return __ldg(reinterpret_cast<const float4 *>(tab + idx) + 1);
}

// The same rows from a copy of the table of species pair (0, 0) in the kernel's dynamic shared
// memory (SMT; rows of other pairs, idx >= nk, come from the global table).  The copy is split:
// nk float4 rows, then the nk rows of phi coefficients, so that the rows a warp reads at random
// spread over all eight 16-byte bank groups (interleaved V/phi rows would put every phi row in
// four of them).  The first nk rows hold the V coefficients with two species (vp_row) and, with
// one, the force pass's derivative rows (Pot::D32, read in pair_g32).
template <bool SMT, bool MULTI>
__device__ __forceinline__ float4 phi_row(const Pot &P, size_t idx) {
    if (SMT && (!MULTI || idx < (size_t)P.nk)) {
        extern __shared__ float4 sm_table_f4[];
        return sm_table_f4[P.smt_phi + idx];
    }
    return phi_half32(P.VP32, idx);
}

template <bool SMT, bool MULTI>
__device__ __forceinline__ void vp_row(const Pot &P, size_t idx, float (&v)[4], float (&p)[4]) {
    if (SMT && (!MULTI || idx < (size_t)P.nk)) {
        extern __shared__ float4 sm_table_f4[];
        const float4 a = sm_table_f4[idx], b = sm_table_f4[P.nk + idx];
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        p[0] = b.x; p[1] = b.y; p[2] = b.z; p[3] = b.w;
        return;
    }
    row32(P.VP32, idx, v, p);
}

// The pair (2 c2, 3 c3) of a derivative row, packed as two binary16 values scaled by 1/s.
__device__ __forceinline__ float2 dtab_pair(float packed) {
    const unsigned u = __float_as_uint(packed);
    return make_float2(__half2float(__ushort_as_half((unsigned short)(u & 0xffffu))),
                       __half2float(__ushort_as_half((unsigned short)(u >> 16))));
}
// d/dt of a table cubic from its derivative row: c1 + t (2 c2 + 3 c3 t); below r_min the linear
// extension (c1).
__device__ __forceinline__ float dtab(float c1, float2 a, float s, float t, bool below) {
    return below ? c1 : fmaf(s * t, fmaf(t, a.y, a.x), c1);
}

// ======================================================================= mixed precision
// List entries between r_cut and r_list (the skin shell, about a tenth of a Cu row) contribute
// nothing; MD_TABLE_SKIP=1 skips their table-row loads (the loads are predicated, the
// arithmetic is not).
#ifndef MD_TABLE_SKIP
#define MD_TABLE_SKIP 1
#endif
// phi_{s_i s_j}(r) of one pair at separation d = (dx, dy, dz); 0 at or beyond r_cut (no branch,
// so the loads of the next pair can issue early).  viol counts table lookups below r_min.
template <int KIND, bool MULTI, bool SMT>
__device__ __forceinline__ float rho_term32(const Pot &P, int si, int sj, float dx, float dy, float dz,
                                            unsigned &viol) {
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const bool inside = r2 < P.rc2f;
    const float r = r2 * rsqrtf(r2);
    float phi;
    if (KIND == MD_POT_FS_ANALYTIC) {
        phi = fs_phi<float>(P.fsf, P.bdf, r);
    } else if (KIND == MD_POT_KNOTS) {
        float d;
        phi = knot_sum<float, float2>(P.K32 + (size_t)(P.ns * P.ns + si * P.ns + sj) * P.nkt, P.nkt, r, d);
    } else {
        float t, d;
        bool below;
        const int kr = knot_row((r - P.r_minf) * P.inv_drf, P.nk, t, below);
        viol += (below && inside) ? 1u : 0u;
        float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
        if (!MD_TABLE_SKIP || inside) c = phi_row<SMT, MULTI>(P, (size_t)(si * P.ns + sj) * P.nk + kr);
        phi = cubic(t, c.x, c.y, c.z, c.w, below, d);
    }
    return inside ? phi : 0.f;
}

// Per-atom sums of the force pass: force, and on the energy step the pair energy and virial.
struct Acc32 {
    float fx = 0.f, fy = 0.f, fz = 0.f, ep = 0.f;
    float wxx = 0.f, wyy = 0.f, wzz = 0.f, wyz = 0.f, wxz = 0.f, wxy = 0.f;
};

// The scalar of one pair of the force pass: g = [V'(r) + F'_i phi'_{s_i s_j}(r) + F'_j phi'_{s_j s_i}(r)] / r
// (the force on i is g d, d = r_j - r_i) and V(r), both zero at or beyond r_cut (no branch).
template <int KIND, bool MULTI, bool SMT, bool ENERGY = true>
__device__ __forceinline__ float pair_g32(const Pot &P, int si, int sj, float Fpi, float Fpj, float r2, float &V,
                                          unsigned &viol) {
    const bool inside = r2 < P.rc2f;
    const float rinv = rsqrtf(r2);
    const float r = r2 * rinv;
    float gg;
    if (KIND == MD_POT_FS_ANALYTIC) {
        float dV;
        V = fs_V<float>(P.fsf, r, dV);
        gg = fmaf(Fpi + Fpj, fs_dphi<float>(P.fsf, P.bdf, r), dV);
    } else if (KIND == MD_POT_KNOTS) {
        const int nn = P.ns * P.ns;
        float dVk, dab;
        V = knot_sum<float, float2>(P.K32 + (size_t)(si * P.ns + sj) * P.nkt, P.nkt, r, dVk);
        knot_sum<float, float2>(P.K32 + (size_t)(nn + si * P.ns + sj) * P.nkt, P.nkt, r, dab);
        if (MULTI) {
            float dba;
            knot_sum<float, float2>(P.K32 + (size_t)(nn + sj * P.ns + si) * P.nkt, P.nkt, r, dba);
            gg = fmaf(Fpi, dab, fmaf(Fpj, dba, dVk));
        } else {
            gg = fmaf(Fpi + Fpj, dab, dVk);
        }
    } else {
        float t;
        bool below;
        const int kr = knot_row((r - P.r_minf) * P.inv_drf, P.nk, t, below);
        viol += (below && inside) ? 1u : 0u;
        float dVk, dab, gk;
        if constexpr (SMT && !MULTI && MD_DTABLE) {
            // one row per pair: the derivative row in shared memory; V(r) itself only on the energy
            // step, with c0 from a small global table
            extern __shared__ float4 sm_table_f4[];
            float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
            if (!MD_TABLE_SKIP || inside) d = sm_table_f4[kr];
            const float2 av = dtab_pair(d.z);
            dVk = dtab(d.x, av, P.dsv, t, below);
            dab = dtab(d.y, dtab_pair(d.w), P.dsp, t, below);
            V = 0.f;
            if (ENERGY) {   // V = c0 + t (c1 + t (c2 + t c3)), c2 and c3 from the derivative row
                const float c0 = inside ? __ldg(P.V0 + kr) : 0.f;
                const float c2 = 0.5f * P.dsv * av.x, c3 = (1.f / 3.f) * P.dsv * av.y;
                V = below ? fmaf(t, d.x, c0) : fmaf(t, fmaf(t, fmaf(t, c3, c2), d.x), c0);
            }
            gk = fmaf(Fpi + Fpj, dab, dVk);
            gg = gk * P.inv_drf;
            V = inside ? V : 0.f;
            return inside ? gg * rinv : 0.f;
        }
        float cv[4] = {0.f, 0.f, 0.f, 0.f}, cp[4] = {0.f, 0.f, 0.f, 0.f};
        if (!MD_TABLE_SKIP || inside) vp_row<SMT, MULTI>(P, (size_t)(si * P.ns + sj) * P.nk + kr, cv, cp);
        V = cubic(t, cv[0], cv[1], cv[2], cv[3], below, dVk);
        cubic(t, cp[0], cp[1], cp[2], cp[3], below, dab);
        if (MULTI) {
            float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
            if (!MD_TABLE_SKIP || inside) c = phi_row<SMT, MULTI>(P, (size_t)(sj * P.ns + si) * P.nk + kr);
            float dba;
            cubic(t, c.x, c.y, c.z, c.w, below, dba);
            gk = fmaf(Fpi, dab, fmaf(Fpj, dba, dVk));
        } else {
            gk = fmaf(Fpi + Fpj, dab, dVk);
        }
        gg = gk * P.inv_drf;
    }
    V = inside ? V : 0.f;
    return inside ? gg * rinv : 0.f;
}

// One pair of the force pass along d = (dx, dy, dz) = r_j - r_i, added to atom i's sums: the
// force g d, and on the energy step V(r)/2 and the virial -g d (x) d / 2.
template <int KIND, bool MULTI, bool ENERGY, bool SMT>
__device__ __forceinline__ void pair32(const Pot &P, int si, int sj, float Fpi, float Fpj, float dx, float dy,
                                       float dz, Acc32 &a, unsigned &viol) {
    float V;
    const float gr =
        pair_g32<KIND, MULTI, SMT, ENERGY>(P, si, sj, Fpi, Fpj, fmaf(dx, dx, fmaf(dy, dy, dz * dz)), V, viol);
    a.fx = fmaf(gr, dx, a.fx);
    a.fy = fmaf(gr, dy, a.fy);
    a.fz = fmaf(gr, dz, a.fz);
    if (ENERGY) {
        a.ep = fmaf(0.5f, V, a.ep);
        const float hg = -0.5f * gr;
        a.wxx = fmaf(hg * dx, dx, a.wxx);
        a.wyy = fmaf(hg * dy, dy, a.wyy);
        a.wzz = fmaf(hg * dz, dz, a.wzz);
        a.wyz = fmaf(hg * dy, dz, a.wyz);
        a.wxz = fmaf(hg * dx, dz, a.wxz);
        a.wxy = fmaf(hg * dx, dy, a.wxy);
    }
}

// End of the density pass for atom i (lane 0 after the lane sum): rho, F(rho), F'(rho) and the
// pass-2 copy (position, F').
__device__ __forceinline__ void density32_finish(const Atoms &A, const Pot &P, int i, int si, const float4 &pi,
                                                 float hi, float lo) {
    const double rho = (double)hi + (double)lo;
    double dF;
    const double F = embed64(P, si, rho, dF, A.flags);
    A.rho[i] = rho;
    A.dF[i] = dF;
    A.e_atom[i] = F;
    A.p2f[i] = make_float4(pi.x, pi.y, pi.z, (float)dF);
}

// Lane sums of the force-pass accumulators over the T lanes of an atom.
template <int T, bool ENERGY>
__device__ __forceinline__ void lane_sum_acc(Acc32 &a) {
    a.fx = lane_sum<T>(a.fx);
    a.fy = lane_sum<T>(a.fy);
    a.fz = lane_sum<T>(a.fz);
    if (ENERGY) {
        a.ep = lane_sum<T>(a.ep);
        a.wxx = lane_sum<T>(a.wxx); a.wyy = lane_sum<T>(a.wyy); a.wzz = lane_sum<T>(a.wzz);
        a.wyz = lane_sum<T>(a.wyz); a.wxz = lane_sum<T>(a.wxz); a.wxy = lane_sum<T>(a.wxy);
    }
}

// End of the force pass for atom i: the force, the second half kick and the FP64 partial sums.
template <bool ENERGY>
__device__ __forceinline__ void force32_finish(const Atoms &A, int i, const Acc32 &a, double half_dt, int motion,
                                               double (&part)[kPartials]) {
    A.force[i] = make_double4_32a(a.fx, a.fy, a.fz, 0.0);
    if (!isfinite(a.fx + a.fy + a.fz)) atomicOr(&A.flags->error, FLAG_NONFINITE);
    double4_32a v = A.vel[i];
    finish_motion(A, i, v, a.fx, a.fy, a.fz, half_dt, motion);
    if (ENERGY) {
        const double e = A.e_atom[i] + (double)a.ep;
        A.e_atom[i] = e;
        const double m = 1.0 / (kMvv2e * v.w);
        part[0] += e;
        part[1] += m * fma(v.x, v.x, fma(v.y, v.y, v.z * v.z));
        part[2] += a.wxx; part[3] += a.wyy; part[4] += a.wzz;
        part[5] += a.wyz; part[6] += a.wxz; part[7] += a.wxy;
        part[8] += m * v.x; part[9] += m * v.y; part[10] += m * v.z;
    }
}

template <int T, int KIND, bool MULTI, bool SMT = false>
__device__ __forceinline__ void density32_item(const Atoms &A, const Pot &P, const Box *boxes, long long g) {
    const int i = (int)(g / T), lane = (int)(g & (T - 1));
    const bool live = i < A.n;
    float hi = 0.f, lo = 0.f;
    float4 pi = make_float4(0.f, 0.f, 0.f, 0.f);
    int si = 0;
    const bool wrap = needs_image(A, i, live);
    if (live) {
        const Box &B = boxes[ph::replica_of(A, i)];
        const float Lx = B.Lf[0], Ly = B.Lf[1], Lz = B.Lf[2];
        const float ix = B.invLf[0], iy = B.invLf[1], iz = B.invLf[2];
        pi = A.posf[i];
        si = MULTI ? __float_as_int(pi.w) : 0;
        const int cnt = min(A.count[i], A.k_max);
        const NbrRow row = nbr_row(A, i);
        unsigned viol = 0;
        auto walk = [&](auto wrap) {
            using W = decltype(wrap);
            auto term = [&](const float4 &pj) -> float {
                return rho_term32<KIND, MULTI, SMT>(P, si, MULTI ? __float_as_int(pj.w) : 0,
                                                    sep32<W>(pj.x - pi.x, Lx, ix), sep32<W>(pj.y - pi.y, Ly, iy),
                                                    sep32<W>(pj.z - pi.z, Lz, iz), viol);
            };
            // two neighbours per iteration, software-pipelined: the positions of the next iteration
            // and the list entries of the one after are loaded before this iteration's terms are
            // computed, so the dependent loads of one neighbour overlap the arithmetic of others
            auto entry = [&](int q) { return q < cnt ? ld_phase(row.ptr(q)) : i; };
            int k = lane;
            float4 p0 = ld_phase(A.posf + entry(k)), p1 = ld_phase(A.posf + entry(k + T));
            int n0 = entry(k + 2 * T), n1 = entry(k + 3 * T);
            for (; k + T < cnt; k += 2 * T) {
                const float4 q0 = ld_phase(A.posf + n0), q1 = ld_phase(A.posf + n1);
                n0 = entry(k + 4 * T);
                n1 = entry(k + 5 * T);
                const float a0 = term(p0), a1 = term(p1);
                two_sum_add(hi, lo, a0);
                two_sum_add(hi, lo, a1);
                p0 = q0;
                p1 = q1;
            }
            if (k < cnt) two_sum_add(hi, lo, term(p0));
        };
        if (wrap) walk(std::true_type{});
        else walk(std::false_type{});
        if (viol) atomicAdd(&A.flags->range_violations, (unsigned long long)viol);
    }
    lane_sum_df<T>(hi, lo);
    if (live && lane == 0) density32_finish(A, P, i, si, pi, hi, lo);
}

// Returns the atom index for the lane that finished atom i (lane 0 of a live atom), else -1.
template <int T, int KIND, bool MULTI, bool ENERGY, bool SMT = false>
__device__ __forceinline__ int force32_item(const Atoms &A, const Pot &P, const Box *boxes, long long g,
                                            double half_dt, int motion, double (&part)[kPartials]) {
    const int i = (int)(g / T), lane = (int)(g & (T - 1));
    const bool live = i < A.n;
    Acc32 a;
    const bool wrap = needs_image(A, i, live);
    if (live) {
        const Box &B = boxes[ph::replica_of(A, i)];
        const float Lx = B.Lf[0], Ly = B.Lf[1], Lz = B.Lf[2];
        const float ix = B.invLf[0], iy = B.invLf[1], iz = B.invLf[2];
        const float4 pi = A.p2f[i];
        const int si = MULTI ? A.spec[i] : 0;
        const int cnt = min(A.count[i], A.k_max);
        const NbrRow row = nbr_row(A, i);
        unsigned viol = 0;
        auto walk = [&](auto wrap) {
            using W = decltype(wrap);
            auto pair = [&](int j, const float4 &pj) {
                pair32<KIND, MULTI, ENERGY, SMT>(P, si, MULTI ? ld_phase(A.spec + j) : 0, pi.w, pj.w,
                                                 sep32<W>(pj.x - pi.x, Lx, ix), sep32<W>(pj.y - pi.y, Ly, iy),
                                                 sep32<W>(pj.z - pi.z, Lz, iz), a, viol);
            };
            // two neighbours per iteration; the list entries of the next iteration are loaded before
            // this iteration's positions are used (one dependent load less on the critical path)
            int k = lane;
            int j0 = k < cnt ? ld_phase(row.ptr(k)) : 0, j1 = k + T < cnt ? ld_phase(row.ptr(k + T)) : 0;
            for (; k + T < cnt; k += 2 * T) {
                const float4 p0 = ld_phase(A.p2f + j0), p1 = ld_phase(A.p2f + j1);
                const int ja = j0, jb = j1, kn = k + 2 * T;
                j0 = kn < cnt ? ld_phase(row.ptr(kn)) : 0;
                j1 = kn + T < cnt ? ld_phase(row.ptr(kn + T)) : 0;
                pair(ja, p0);
                pair(jb, p1);
            }
            if (k < cnt) pair(j0, ld_phase(A.p2f + j0));
        };
        if (wrap) walk(std::true_type{});
        else walk(std::false_type{});
        if (viol) atomicAdd(&A.flags->range_violations, (unsigned long long)viol);
    }
    lane_sum_acc<T, ENERGY>(a);
    if (!(live && lane == 0)) return -1;
    force32_finish<ENERGY>(A, i, a, half_dt, motion, part);
    return i;
}

// ======================================================================= FP64
// energy (one species, derivative cache kept): the pair energies 1/2 V(r) of the atom are summed
// here too, into E_i, and the force pass adds only the virial.
template <int T, int KIND, bool MULTI>
__device__ __forceinline__ void density64_item(const Atoms &A, const Pot &P, const Box *boxes, long long g,
                                               bool energy = false) {
    const int i = (int)(g / T), lane = (int)(g & (T - 1));
    const bool live = i < A.n;
    double rho = 0.0, ep = 0.0;
    double4_32a pi = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    int si = 0;
    const bool wrap = needs_image(A, i, live);
    if (live) {
        const Box &B = boxes[ph::replica_of(A, i)];
        pi = ld_phase(A.posd + i);
        si = MULTI ? A.spec[i] : 0;
        const int cnt = min(A.count[i], A.k_max);
        const NbrRow row = nbr_row(A, i);
        // one species: keep (V'/r, phi'/r) of every entry for the force passes without energies
        const bool keep = !MULTI && A.dcache != nullptr;
        const DRow drow = dcache_row(A, i);
        auto walk = [&](auto wrapt) {
            using W = decltype(wrapt);
            for (int k = lane; k < cnt; k += T) {
                const int j = ld_phase(row.ptr(k));
                const double4_32a pj = ld_phase(A.posd + j);
                const double dx = sep64<W>(pj.x - pi.x, B.L[0], B.invL[0]);
                const double dy = sep64<W>(pj.y - pi.y, B.L[1], B.invL[1]);
                const double dz = sep64<W>(pj.z - pi.z, B.L[2], B.invL[2]);
                const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
                if (!inside64(r2, P.rc2)) {
                    if (keep) *drow.ptr(k) = make_double2(0.0, 0.0);
                    continue;
                }
                const double rinv = rsqrt64(r2);
                const double r = r2 * rinv;
                if (KIND == MD_POT_FS_ANALYTIC) {
                    rho += fs_phi<double>(P.fs, P.bd, r);
                    if (keep) {
                        double dV;
                        const double V = fs_V<double>(P.fs, r, dV);
                        if (energy) ep = fma(0.5, V, ep);
                        *drow.ptr(k) = make_double2(dV * rinv, fs_dphi<double>(P.fs, P.bd, r) * rinv);
                    }
                } else if (KIND == MD_POT_KNOTS) {
                    const int sj = MULTI ? (int)pj.w : 0;
                    double d;
                    rho += knot_sum<double, double2>(P.K64 + (size_t)(P.ns * P.ns + si * P.ns + sj) * P.nkt, P.nkt, r, d);
                    if (keep) {
                        double dV;
                        const double V = knot_sum<double, double2>(P.K64, P.nkt, r, dV);
                        if (energy) ep = fma(0.5, V, ep);
                        *drow.ptr(k) = make_double2(dV * rinv, d * rinv);
                    }
                } else {
                    const int sj = MULTI ? (int)pj.w : 0;
                    double t, d;
                    bool below;
                    const int kr = knot_row64(fma(r, P.inv_dr, P.xneg), P.nk, t, below);
                    if (below) atomicAdd(&A.flags->range_violations, 1ull);
                    const size_t ab = ((size_t)(si * P.ns + sj) * P.nk + kr) * 2;
                    const double4_32a c = P.VP64[ab + 1];
                    rho += cubic(t, c.x, c.y, c.z, c.w, below, d);
                    if (keep) {   // r-derivatives from the interval's derivative rows (inv_dr folded in)
                        const double4_32a dv = P.D64[2 * kr], dp = P.D64[2 * kr + 1];
                        const double dV = below ? dv.x : fma(t, fma(dv.z, t, dv.y), dv.x);
                        const double dphi = below ? dp.x : fma(t, fma(dp.z, t, dp.y), dp.x);
                        *drow.ptr(k) = make_double2(dV * rinv, dphi * rinv);
                        if (energy) {
                            const double4_32a cv = P.VP64[ab];
                            double dd;
                            ep = fma(0.5, cubic(t, cv.x, cv.y, cv.z, cv.w, below, dd), ep);
                        }
                    }
                }
            }
        };
        if (wrap) walk(std::true_type{});
        else walk(std::false_type{});
    }
    rho = lane_sum<T>(rho);
    if (energy) ep = lane_sum<T>(ep);
    if (live && lane == 0) {
        double dF;
        const double F = embed64(P, si, rho, dF, A.flags);
        A.rho[i] = rho;
        A.dF[i] = dF;
        A.e_atom[i] = F + ep;
        A.p2d[i] = make_double4_32a(pi.x, pi.y, pi.z, dF);
    }
}

// The FP64 force pass from the derivative cache of the density pass (one species): per entry the
// separation, then f_i += [V'/r + (F'_i + F'_j) phi'/r] d, the same terms as the full evaluation
// below in another order of rounding.  With ENERGY the virial is added (the pair energies were
// summed into E_i by the density pass of the same step), while the force takes the same
// operations as without, so that a run does not depend on which of its steps evaluate energies.
template <int T, int KIND, bool ENERGY>
__device__ __forceinline__ int force64_cached_item(const Atoms &A, const Pot &P, const Box *boxes, long long g,
                                                   double half_dt, int motion, double (&part)[kPartials]) {
    const int i = (int)(g / T), lane = (int)(g & (T - 1));
    const bool live = i < A.n;
    double fx = 0.0, fy = 0.0, fz = 0.0, ep = 0.0;
    double wxx = 0.0, wyy = 0.0, wzz = 0.0, wyz = 0.0, wxz = 0.0, wxy = 0.0;
    const bool wrap = needs_image(A, i, live);
    if (live) {
        const Box &B = boxes[ph::replica_of(A, i)];
        const double4_32a pi = A.p2d[i];
        const double Fpi = pi.w;
        const int cnt = min(A.count[i], A.k_max);
        const NbrRow row = nbr_row(A, i);
        const DRow drow = dcache_row(A, i);
        auto walk = [&](auto wrapt) {
            using W = decltype(wrapt);
            for (int k = lane; k < cnt; k += T) {
                const int j = ld_phase(row.ptr(k));
                const double4_32a pj = ld_phase(A.p2d + j);
                const double2 e = ld_phase(drow.ptr(k));
                const double dx = sep64<W>(pj.x - pi.x, B.L[0], B.invL[0]);
                const double dy = sep64<W>(pj.y - pi.y, B.L[1], B.invL[1]);
                const double dz = sep64<W>(pj.z - pi.z, B.L[2], B.invL[2]);
                const double gr = fma(Fpi + pj.w, e.y, e.x);
                fx = fma(gr, dx, fx);
                fy = fma(gr, dy, fy);
                fz = fma(gr, dz, fz);
                if (ENERGY) {   // the pair energies are in E_i already (density pass)
                    const double hg = -0.5 * gr;
                    wxx = fma(hg * dx, dx, wxx);
                    wyy = fma(hg * dy, dy, wyy);
                    wzz = fma(hg * dz, dz, wzz);
                    wyz = fma(hg * dy, dz, wyz);
                    wxz = fma(hg * dx, dz, wxz);
                    wxy = fma(hg * dx, dy, wxy);
                }
            }
        };
        if (wrap) walk(std::true_type{});
        else walk(std::false_type{});
    }
    fx = lane_sum<T>(fx);
    fy = lane_sum<T>(fy);
    fz = lane_sum<T>(fz);
    if (ENERGY) {
        ep = lane_sum<T>(ep);
        wxx = lane_sum<T>(wxx); wyy = lane_sum<T>(wyy); wzz = lane_sum<T>(wzz);
        wyz = lane_sum<T>(wyz); wxz = lane_sum<T>(wxz); wxy = lane_sum<T>(wxy);
    }
    if (!(live && lane == 0)) return -1;
    A.force[i] = make_double4_32a(fx, fy, fz, 0.0);
    if (!isfinite(fx + fy + fz)) atomicOr(&A.flags->error, FLAG_NONFINITE);
    double4_32a v = A.vel[i];
    finish_motion(A, i, v, fx, fy, fz, half_dt, motion);
    if (ENERGY) {
        const double e = A.e_atom[i] + ep;
        A.e_atom[i] = e;
        const double m = 1.0 / (kMvv2e * v.w);
        part[0] += e;
        part[1] += m * fma(v.x, v.x, fma(v.y, v.y, v.z * v.z));
        part[2] += wxx; part[3] += wyy; part[4] += wzz;
        part[5] += wyz; part[6] += wxz; part[7] += wxy;
        part[8] += m * v.x; part[9] += m * v.y; part[10] += m * v.z;
    }
    return i;
}

template <int T, int KIND, bool MULTI, bool ENERGY>
__device__ __forceinline__ int force64_item(const Atoms &A, const Pot &P, const Box *boxes, long long g,
                                            double half_dt, int motion, double (&part)[kPartials]) {
    if constexpr (!MULTI) {
        if (A.dcache) return force64_cached_item<T, KIND, ENERGY>(A, P, boxes, g, half_dt, motion, part);
    }
    const int i = (int)(g / T), lane = (int)(g & (T - 1));
    const bool live = i < A.n;
    double fx = 0.0, fy = 0.0, fz = 0.0, ep = 0.0;
    double wxx = 0.0, wyy = 0.0, wzz = 0.0, wyz = 0.0, wxz = 0.0, wxy = 0.0;
    const bool wrap = needs_image(A, i, live);
    if (live) {
        const Box &B = boxes[ph::replica_of(A, i)];
        const double4_32a pi = A.p2d[i];
        const double Fpi = pi.w;
        const int si = MULTI ? A.spec[i] : 0;
        const int cnt = min(A.count[i], A.k_max);
        const NbrRow row = nbr_row(A, i);
        auto walk = [&](auto wrapt) {
            using W = decltype(wrapt);
            for (int k = lane; k < cnt; k += T) {
                const int j = ld_phase(row.ptr(k));
                const double4_32a pj = ld_phase(A.p2d + j);
                const double dx = sep64<W>(pj.x - pi.x, B.L[0], B.invL[0]);
                const double dy = sep64<W>(pj.y - pi.y, B.L[1], B.invL[1]);
                const double dz = sep64<W>(pj.z - pi.z, B.L[2], B.invL[2]);
                const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
                if (!inside64(r2, P.rc2)) continue;
                const double rinv = rsqrt64(r2);
                const double r = r2 * rinv;
                const double Fpj = pj.w;
                double V, gg;
                if (KIND == MD_POT_FS_ANALYTIC) {
                    double dV;
                    V = fs_V<double>(P.fs, r, dV);
                    gg = fma(Fpi + Fpj, fs_dphi<double>(P.fs, P.bd, r), dV);
                } else if (KIND == MD_POT_KNOTS) {
                    const int sj = MULTI ? ld_phase(A.spec + j) : 0;
                    const int nn = P.ns * P.ns;
                    double dVk, dab;
                    V = knot_sum<double, double2>(P.K64 + (size_t)(si * P.ns + sj) * P.nkt, P.nkt, r, dVk);
                    knot_sum<double, double2>(P.K64 + (size_t)(nn + si * P.ns + sj) * P.nkt, P.nkt, r, dab);
                    if (MULTI) {
                        double dba;
                        knot_sum<double, double2>(P.K64 + (size_t)(nn + sj * P.ns + si) * P.nkt, P.nkt, r, dba);
                        gg = fma(Fpi, dab, fma(Fpj, dba, dVk));
                    } else {
                        gg = fma(Fpi + Fpj, dab, dVk);
                    }
                } else {
                    const int sj = MULTI ? ld_phase(A.spec + j) : 0;
                    double t;
                    bool below;
                    const int kr = knot_row64(fma(r, P.inv_dr, P.xneg), P.nk, t, below);
                    if (below) atomicAdd(&A.flags->range_violations, 1ull);
                    const size_t ab = ((size_t)(si * P.ns + sj) * P.nk + kr) * 2;
                    const double4_32a cv = P.VP64[ab], cp = P.VP64[ab + 1];
                    double dVk, dab;
                    V = cubic(t, cv.x, cv.y, cv.z, cv.w, below, dVk);
                    cubic(t, cp.x, cp.y, cp.z, cp.w, below, dab);
                    double gk;
                    if (MULTI) {
                        const double4_32a cb = P.VP64[((size_t)(sj * P.ns + si) * P.nk + kr) * 2 + 1];
                        double dba;
                        cubic(t, cb.x, cb.y, cb.z, cb.w, below, dba);
                        gk = fma(Fpi, dab, fma(Fpj, dba, dVk));
                    } else {
                        gk = fma(Fpi + Fpj, dab, dVk);
                    }
                    gg = gk * P.inv_dr;
                }
                const double gr = gg * rinv;
                fx = fma(gr, dx, fx);
                fy = fma(gr, dy, fy);
                fz = fma(gr, dz, fz);
                if (ENERGY) {
                    ep = fma(0.5, V, ep);
                    const double hg = -0.5 * gr;
                    wxx = fma(hg * dx, dx, wxx);
                    wyy = fma(hg * dy, dy, wyy);
                    wzz = fma(hg * dz, dz, wzz);
                    wyz = fma(hg * dy, dz, wyz);
                    wxz = fma(hg * dx, dz, wxz);
                    wxy = fma(hg * dx, dy, wxy);
                }
            }
        };
        if (wrap) walk(std::true_type{});
        else walk(std::false_type{});
    }
    fx = lane_sum<T>(fx);
    fy = lane_sum<T>(fy);
    fz = lane_sum<T>(fz);
    if (ENERGY) {
        ep = lane_sum<T>(ep);
        wxx = lane_sum<T>(wxx); wyy = lane_sum<T>(wyy); wzz = lane_sum<T>(wzz);
        wyz = lane_sum<T>(wyz); wxz = lane_sum<T>(wxz); wxy = lane_sum<T>(wxy);
    }
    if (!(live && lane == 0)) return -1;
    A.force[i] = make_double4_32a(fx, fy, fz, 0.0);
    if (!isfinite(fx + fy + fz)) atomicOr(&A.flags->error, FLAG_NONFINITE);
    double4_32a v = A.vel[i];
    finish_motion(A, i, v, fx, fy, fz, half_dt, motion);
    if (ENERGY) {
        const double e = A.e_atom[i] + ep;
        A.e_atom[i] = e;
        const double m = 1.0 / (kMvv2e * v.w);
        part[0] += e;
        part[1] += m * fma(v.x, v.x, fma(v.y, v.y, v.z * v.z));
        part[2] += wxx; part[3] += wyy; part[4] += wzz;
        part[5] += wyz; part[6] += wxz; part[7] += wxy;
        part[8] += m * v.x; part[9] += m * v.y; part[10] += m * v.z;
    }
    return i;
}

// ======================================================================= FP64, each pair once
// The half list of §3.2.2 taken from the full list: atom i handles only its entries j > i (cell
// order; the rows are partitioned at every build so that these come first, cup[i] of them),
// computes the pair term once and adds the neighbour's share to FP64 accumulators with atomic
// adds (Newton's third law).  The density pass leaves each atom's own share in rho and
// the neighbours' shares in rho_acc (on an energy step the pair energies, 1/2 V to each atom, in
// e_acc); F(rho) follows in a phase of its own (pairs_embed64) once every share is in, the force
// pass likewise leaves its own share in force and the others' in
// f_acc, and the kick follows in a phase of its own (pairs_kick64).  The per-entry derivative
// cache holds the entries j > i only.  The order of the atomic adds, and so the last bits of the
// sums, varies from run to run.  One species.
template <int T, int KIND>
__device__ __forceinline__ void density64_pairs_item(const Atoms &A, const Pot &P, const Box *boxes, long long g,
                                                     bool energy = false) {
    const int i = (int)(g / T), lane = (int)(g & (T - 1));
    const bool live = i < A.n;
    double rho = 0.0, ep = 0.0;
    const bool wrap = needs_image(A, i, live);
    if (live) {
        const Box &B = boxes[ph::replica_of(A, i)];
        const double4_32a pi = ld_phase(A.posd + i);
        const int cnt = ld_phase(A.cup + i);
        const NbrRow row = nbr_row(A, i);
        const DRow drow = dcache_row(A, i);
        auto walk = [&](auto wrapt) {
            using W = decltype(wrapt);
            for (int k = lane; k < cnt; k += T) {
                const int j = ld_phase(row.ptr(k));
                const double4_32a pj = ld_phase(A.posd + j);
                const double dx = sep64<W>(pj.x - pi.x, B.L[0], B.invL[0]);
                const double dy = sep64<W>(pj.y - pi.y, B.L[1], B.invL[1]);
                const double dz = sep64<W>(pj.z - pi.z, B.L[2], B.invL[2]);
                const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
                if (!inside64(r2, P.rc2)) {
                    *drow.ptr(k) = make_double2(0.0, 0.0);
                    continue;
                }
                const double rinv = rsqrt64(r2);
                const double r = r2 * rinv;
                double phi, dV, dphi, V = 0.0;
                if (KIND == MD_POT_FS_ANALYTIC) {
                    phi = fs_phi<double>(P.fs, P.bd, r);
                    V = fs_V<double>(P.fs, r, dV);
                    dphi = fs_dphi<double>(P.fs, P.bd, r);
                } else {
                    double t;
                    bool below;
                    const int kr = knot_row64(fma(r, P.inv_dr, P.xneg), P.nk, t, below);
                    if (below) atomicAdd(&A.flags->range_violations, 1ull);
                    const double4_32a c = P.VP64[(size_t)kr * 2 + 1];
                    phi = cubic64(t, c, below);
                    const double4_32a dv = P.D64[2 * kr], dp = P.D64[2 * kr + 1];
                    dV = below ? dv.x : fma(t, fma(dv.z, t, dv.y), dv.x);
                    dphi = below ? dp.x : fma(t, fma(dp.z, t, dp.y), dp.x);
                    if (energy) {
                        const double4_32a cv = P.VP64[(size_t)kr * 2];
                        V = cubic64(t, cv, below);
                    }
                }
                rho += phi;
                atomicAdd(A.rho_acc + j, phi);
                if (energy) {   // each atom of the pair gets half its pair energy
                    const double hV = half64(V);
                    ep += hV;
                    atomicAdd(A.e_acc + j, hV);
                }
                *drow.ptr(k) = make_double2(-dV * rinv, -dphi * rinv);   // negated (the force pass needs -g)
            }
        };
        if (wrap) walk(std::true_type{});
        else walk(std::false_type{});
    }
    rho = lane_sum<T>(rho);
    if (energy) ep = lane_sum<T>(ep);
    if (live && lane == 0) {
        A.rho[i] = rho;
        if (energy) atomicAdd(A.e_acc + i, ep);
    }
}

// After the pair density pass, per atom: rho = own share + the neighbours' shares; F, F'; the
// pass-2 copy; the accumulators cleared for the force pass.
__device__ __forceinline__ void pairs_embed64(const Atoms &A, const Pot &P, int i) {
    const double rho = A.rho[i] + A.rho_acc[i];
    double dF;
    const double F = embed64(P, 0, rho, dF, A.flags);
    A.rho[i] = rho;
    A.dF[i] = dF;
    A.e_atom[i] = F + A.e_acc[i];   // the pair energies (energy steps; else 0)
    A.e_acc[i] = 0.0;
    const double4_32a p = A.posd[i];
    A.p2d[i] = make_double4_32a(p.x, p.y, p.z, dF);
    A.rho_acc[i] = 0.0;
    A.f_acc[i] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
}

template <int T, int KIND, bool ENERGY>
__device__ __forceinline__ void force64_pairs_item(const Atoms &A, const Pot &P, const Box *boxes, long long g,
                                                   double (&part)[kPartials]) {
    const int i = (int)(g / T), lane = (int)(g & (T - 1));
    const bool live = i < A.n;
    double fx = 0.0, fy = 0.0, fz = 0.0, ep = 0.0;
    double wxx = 0.0, wyy = 0.0, wzz = 0.0, wyz = 0.0, wxz = 0.0, wxy = 0.0;
    const bool wrap = needs_image(A, i, live);
    if (live) {
        const Box &B = boxes[ph::replica_of(A, i)];
        const double4_32a pi = A.p2d[i];
        const int cnt = ld_phase(A.cup + i);
        const NbrRow row = nbr_row(A, i);
        const DRow drow = dcache_row(A, i);
        auto walk = [&](auto wrapt) {
            using W = decltype(wrapt);
            for (int k = lane; k < cnt; k += T) {
                const double2 e = ld_phase(drow.ptr(k));
                // beyond r_cut (the row's skin entries, at its end): nothing to add
                if ((__double_as_longlong(e.x) | __double_as_longlong(e.y)) == 0) continue;
                const int j = ld_phase(row.ptr(k));
                const double4_32a pj = ld_phase(A.p2d + j);
                double sx, sy, sz;
                const double dx = sep64s<W>(pj.x - pi.x, B.L[0], sx);
                const double dy = sep64s<W>(pj.y - pi.y, B.L[1], sy);
                const double dz = sep64s<W>(pj.z - pi.z, B.L[2], sz);
                // -g d, the neighbour's share, from the negated radial factors (no negation)
                const double ngr = fma(pi.w + pj.w, e.y, e.x);
                const double ngx = ngr * dx, ngy = ngr * dy, ngz = ngr * dz;
                fx -= ngx;
                fy -= ngy;
                fz -= ngz;
                if (ENERGY && W::value) virial_shift(sx, sy, sz, ngx, ngy, ngz, wxx, wyy, wzz, wyz, wxz, wxy);
                double *acc = reinterpret_cast<double *>(A.f_acc + j);
                atomicAdd(acc, ngx);
                atomicAdd(acc + 1, ngy);
                atomicAdd(acc + 2, ngz);
            }
        };
        if (wrap) walk(std::true_type{});
        else walk(std::false_type{});
    }
    fx = lane_sum<T>(fx);
    fy = lane_sum<T>(fy);
    fz = lane_sum<T>(fz);
    if (ENERGY) {
        ep = lane_sum<T>(ep);
        wxx = lane_sum<T>(wxx); wyy = lane_sum<T>(wyy); wzz = lane_sum<T>(wzz);
        wyz = lane_sum<T>(wyz); wxz = lane_sum<T>(wxz); wxy = lane_sum<T>(wxy);
    }
    if (!(live && lane == 0)) return;
    A.force[i] = make_double4_32a(fx, fy, fz, 0.0);
    if (ENERGY) {
        part[2] += wxx; part[3] += wyy; part[4] += wzz;
        part[5] += wyz; part[6] += wxz; part[7] += wxy;
    }
}

// ---- the pair walk with the warp's rows flattened (T >= kFlatLanes lanes per atom)
// The AW = 32 / T atoms of a warp are walked as one sequence of entries, so that every lane has an
// entry in every round but the last: first the entries j > i that lay inside r_cut at the build
// (cin[i] of them, at the front of each row), then the rest of the entries j > i (the skin at the
// build; their pair terms run only where the pair has since come inside r_cut).  Entry e of a
// segment belongs to atom a with off[a] <= e < off[a + 1].  A lane's entries belong to atoms in
// ascending order, so it keeps one running sum per quantity and adds it to its own slot of the
// warp's shared sums S[q][a][lane] when the atom changes (put_slot); the T lanes of each atom then
// add the 32 slots of that atom (and the butterfly of the per-atom walk).  S: this warp's
// kPairSlots(AW) doubles.
template <int AW>
struct FlatRows {
    int off[AW + 1];   // prefix counts of the segment's entries (the same in every lane)
    int lo[AW];        // first row entry of each atom's segment
    // Atom a (0 .. AW-1) of entry e, and the row entry k of e.
    __device__ __forceinline__ int atom(int e, int &k) const {
        int a = 0, base = 0, l = lo[0];
#pragma unroll
        for (int b = 1; b < AW; b++)
            if (e >= off[b]) {
                a = b;
                base = off[b];
                l = lo[b];
            }
        k = l + (e - base);
        return a;
    }
};

// Segment seg (0: [0, cin), 1: [cin, cup)) of the rows of the warp's atoms; c_in, c_up: atom
// i0 + lane's counts in lanes < AW (every lane calls).
template <int AW>
__device__ __forceinline__ FlatRows<AW> flat_rows(int c_in, int c_up, int seg) {
    FlatRows<AW> R;
    R.off[0] = 0;
#pragma unroll
    for (int b = 0; b < AW; b++) {
        const int ci = __shfl_sync(0xffffffffu, c_in, b), cu = __shfl_sync(0xffffffffu, c_up, b);
        R.lo[b] = seg == 0 ? 0 : ci;
        R.off[b + 1] = R.off[b] + (seg == 0 ? ci : cu - ci);
    }
    return R;
}

__host__ __device__ constexpr int kPairSlots(int aw) { return 3 * aw * 32; }
// The fewest lanes per atom that take the flattened walk (at most 32 / kFlatLanes atoms a warp).
constexpr int kFlatLanes = 4;

// A lane's running sum of one atom into its slot.  A lane's entries of an atom form one run in
// each segment and the slots start cleared, so the first segment stores the sum; the second adds
// it only where it is not zero (a bit-pattern test: the skin segment's sums mostly are).
__device__ __forceinline__ void put_slot(double *s, double v, int seg) {
    if (seg == 0) *s = v;
    else if ((unsigned long long)__double_as_longlong(v) << 1) *s += v;
}

// Atom a's sum of slot row q over the warp's 32 lanes, in the T lanes of atom a (butterfly).
template <int T>
__device__ __forceinline__ double flat_sum(const double *S, int q) {
    constexpr int AW = 32 / T;
    const int lane = threadIdx.x & 31, a = lane / T, l = lane & (T - 1);
    const double *row = S + (q * AW + a) * 32 + l;
    double x = row[0];
#pragma unroll
    for (int m = 1; m < 32 / T; m++) x += row[T * m];
    return lane_sum<T>(x);
}

template <int T, int KIND>
__device__ __forceinline__ void density64_pairs_flat(const Atoms &A, const Pot &P, const Box *boxes, long long g,
                                                     bool energy, double *S) {
    constexpr int AW = 32 / T;
    const int lane = (int)(g & 31);
    const int i0 = (int)(g >> 5) * AW;   // the warp's first atom
    const int me = i0 + lane / T;        // the atom whose sums this lane finishes
    const bool wrap = needs_image(A, me, me < A.n);
    int c_in = 0, c_up = 0;
    if (lane < AW && i0 + lane < A.n) {
        c_in = ld_phase(A.cin + i0 + lane);
        c_up = ld_phase(A.cup + i0 + lane);
    }
#pragma unroll
    for (int q = 0; q < 2 * AW; q++) S[q * 32 + lane] = 0.0;
    auto walk = [&](auto wrapt) {
        using W = decltype(wrapt);
        for (int seg = 0; seg < 2; seg++) {
            const FlatRows<AW> R = flat_rows<AW>(c_in, c_up, seg);
            int cur = -1, i = 0;
            double rho = 0.0, ep = 0.0;
            double4_32a pi = make_double4_32a(0.0, 0.0, 0.0, 0.0);
            NbrRow row{nullptr, 0};
            DRow drow{nullptr, 0};
            for (int e = lane; e < R.off[AW]; e += 32) {
                int k;
                const int a = R.atom(e, k);
                if (a != cur) {   // the next atom of this lane: flush the sums, load the atom
                    if (cur >= 0) {
                        put_slot(S + cur * 32 + lane, rho, seg);
                        if (energy) put_slot(S + (AW + cur) * 32 + lane, ep, seg);
                    }
                    cur = a;
                    rho = ep = 0.0;
                    i = i0 + a;
                    pi = ld_phase(A.posd + i);
                    row = nbr_row(A, i);
                    drow = dcache_row(A, i);
                }
                const int j = ld_phase(row.ptr(k));
                double2 *dc = drow.ptr(k);
                if (seg == 1) {
                    // the skin at the build: an FP32 test on the FP32 copies (same periodic image)
                    // drops the pairs still beyond r_cut before any FP64 work (rc2f_skin: r_cut^2
                    // plus 4x the bound on the FP32 error of r^2, as for the list build's band)
                    const float4 fi = ld_phase(A.posf + i), fj = ld_phase(A.posf + j);
                    float ex = fj.x - fi.x, ey = fj.y - fi.y, ez = fj.z - fi.z;
                    if (W::value) {
                        const Box &B = boxes[ph::replica_of(A, i)];
                        ex = fmaf(-B.Lf[0], rintf(ex * B.invLf[0]), ex);
                        ey = fmaf(-B.Lf[1], rintf(ey * B.invLf[1]), ey);
                        ez = fmaf(-B.Lf[2], rintf(ez * B.invLf[2]), ez);
                    }
                    if (fmaf(ex, ex, fmaf(ey, ey, ez * ez)) > P.rc2f_skin) {
                        *dc = make_double2(0.0, 0.0);
                        continue;
                    }
                }
                const double4_32a pj = ld_phase(A.posd + j);
                double dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
                if (W::value) {
                    const Box &B = boxes[ph::replica_of(A, i)];
                    dx = mi64(dx, B.L[0], B.invL[0]);
                    dy = mi64(dy, B.L[1], B.invL[1]);
                    dz = mi64(dz, B.L[2], B.invL[2]);
                }
                const double r2 = r2_split(dx, dy, dz);   // FP32 pieces, one FP64 addition
                if (!inside64(r2, P.rc2)) {
                    *dc = make_double2(0.0, 0.0);
                    continue;
                }
                const double rinv = rsqrt64(r2);
                const double r = r2 * rinv;
                double phi, dV, dphi, V = 0.0;
                if (KIND == MD_POT_FS_ANALYTIC) {
                    phi = fs_phi<double>(P.fs, P.bd, r);
                    V = fs_V<double>(P.fs, r, dV);
                    dphi = fs_dphi<double>(P.fs, P.bd, r);
                } else {
                    double t;
                    bool below;
                    const int kr = knot_row64(fma(r, P.inv_dr, P.xneg), P.nk, t, below);
                    if (below) atomicAdd(&A.flags->range_violations, 1ull);
                    const double4_32a c = P.VP64[(size_t)kr * 2 + 1];
                    phi = cubic64(t, c, below);
                    const double4_32a dv = P.D64[2 * kr], dp = P.D64[2 * kr + 1];
                    dV = below ? dv.x : fma(t, fma(dv.z, t, dv.y), dv.x);
                    dphi = below ? dp.x : fma(t, fma(dp.z, t, dp.y), dp.x);
                    if (energy) {
                        const double4_32a cv = P.VP64[(size_t)kr * 2];
                        V = cubic64(t, cv, below);
                    }
                }
                rho += phi;
                atomicAdd(A.rho_acc + j, phi);
                if (energy) {   // each atom of the pair gets half its pair energy
                    const double hV = half64(V);
                    ep += hV;
                    atomicAdd(A.e_acc + j, hV);
                }
                *dc = make_double2(-dV * rinv, -dphi * rinv);   // negated (the force pass needs -g)
            }
            if (cur >= 0) {
                put_slot(S + cur * 32 + lane, rho, seg);
                if (energy) put_slot(S + (AW + cur) * 32 + lane, ep, seg);
            }
        }
    };
    if (wrap) walk(std::true_type{});
    else walk(std::false_type{});
    __syncwarp();
    const double rho = flat_sum<T>(S, 0);
    const double ep = energy ? flat_sum<T>(S, 1) : 0.0;
    __syncwarp();   // S is free for the next item of this warp
    if (me < A.n && (lane & (T - 1)) == 0) {
        A.rho[me] = rho;
        if (energy) atomicAdd(A.e_acc + me, ep);
    }
}

template <int T, int KIND, bool ENERGY>
__device__ __forceinline__ void force64_pairs_flat(const Atoms &A, const Pot &P, const Box *boxes, long long g,
                                                   double (&part)[kPartials], double *S) {
    constexpr int AW = 32 / T;
    const int lane = (int)(g & 31);
    const int i0 = (int)(g >> 5) * AW;
    const int me = i0 + lane / T;
    const bool wrap = needs_image(A, me, me < A.n);
    int c_in = 0, c_up = 0;
    if (lane < AW && i0 + lane < A.n) {
        c_in = ld_phase(A.cin + i0 + lane);
        c_up = ld_phase(A.cup + i0 + lane);
    }
#pragma unroll
    for (int q = 0; q < 3 * AW; q++) S[q * 32 + lane] = 0.0;
    double wxx = 0.0, wyy = 0.0, wzz = 0.0, wyz = 0.0, wxz = 0.0, wxy = 0.0;
    auto walk = [&](auto wrapt) {
        using W = decltype(wrapt);
        for (int seg = 0; seg < 2; seg++) {
            const FlatRows<AW> R = flat_rows<AW>(c_in, c_up, seg);
            int cur = -1, i = 0;
            double fx = 0.0, fy = 0.0, fz = 0.0;
            double4_32a pi = make_double4_32a(0.0, 0.0, 0.0, 0.0);
            for (int e = lane; e < R.off[AW]; e += 32) {
                int k;
                const int a = R.atom(e, k);
                // the entry's radial factors and its neighbour index, both loaded before either is
                // used (one memory latency for the two)
                const double2 d = ld_phase(dcache_row(A, i0 + a).ptr(k));
                const int j = ld_phase(nbr_row(A, i0 + a).ptr(k));
                // beyond r_cut: nothing to add (the skin segment mostly ends here)
                if ((__double_as_longlong(d.x) | __double_as_longlong(d.y)) == 0) continue;
                if (a != cur) {   // the next atom of this lane: flush the sums, load the atom
                    if (cur >= 0) {
                        put_slot(S + cur * 32 + lane, fx, seg);
                        put_slot(S + (AW + cur) * 32 + lane, fy, seg);
                        put_slot(S + (2 * AW + cur) * 32 + lane, fz, seg);
                    }
                    cur = a;
                    fx = fy = fz = 0.0;
                    i = i0 + a;
                    pi = ld_phase(A.p2d + i);
                }
                const double4_32a pj = ld_phase(A.p2d + j);
                double dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z, sx = 0.0, sy = 0.0, sz = 0.0;
                if (W::value) {
                    const Box &B = boxes[ph::replica_of(A, i)];
                    dx = mi64s(dx, B.L[0], sx);
                    dy = mi64s(dy, B.L[1], sy);
                    dz = mi64s(dz, B.L[2], sz);
                }
                // -g d, the neighbour's share, from the negated radial factors (no negation)
                const double ngr = fma(pi.w + pj.w, d.y, d.x);
                const double ngx = ngr * dx, ngy = ngr * dy, ngz = ngr * dz;
                fx -= ngx;
                fy -= ngy;
                fz -= ngz;
                if (ENERGY && W::value) virial_shift(sx, sy, sz, ngx, ngy, ngz, wxx, wyy, wzz, wyz, wxz, wxy);
                double *acc = reinterpret_cast<double *>(A.f_acc + j);
                atomicAdd(acc, ngx);
                atomicAdd(acc + 1, ngy);
                atomicAdd(acc + 2, ngz);
            }
            if (cur >= 0) {
                put_slot(S + cur * 32 + lane, fx, seg);
                put_slot(S + (AW + cur) * 32 + lane, fy, seg);
                put_slot(S + (2 * AW + cur) * 32 + lane, fz, seg);
            }
        }
    };
    if (wrap) walk(std::true_type{});
    else walk(std::false_type{});
    if (ENERGY) {
        part[2] += wxx; part[3] += wyy; part[4] += wzz;
        part[5] += wyz; part[6] += wxz; part[7] += wxy;
    }
    __syncwarp();
    const double fx = flat_sum<T>(S, 0), fy = flat_sum<T>(S, 1), fz = flat_sum<T>(S, 2);
    __syncwarp();
    if (me < A.n && (lane & (T - 1)) == 0) A.force[me] = make_double4_32a(fx, fy, fz, 0.0);
}

// The pair walk's passes: the flattened rows for T >= kFlatLanes lanes per atom (S: this warp's
// kPairSlots(32 / T) doubles of shared memory), the per-atom rows otherwise.
template <int T, int KIND>
__device__ __forceinline__ void density64_pairs(const Atoms &A, const Pot &P, const Box *boxes, long long g,
                                                bool energy, double *S) {
    if constexpr (T >= kFlatLanes) density64_pairs_flat<T, KIND>(A, P, boxes, g, energy, S);
    else density64_pairs_item<T, KIND>(A, P, boxes, g, energy);
}
template <int T, int KIND, bool ENERGY>
__device__ __forceinline__ void force64_pairs(const Atoms &A, const Pot &P, const Box *boxes, long long g,
                                              double (&part)[kPartials], double *S) {
    if constexpr (T >= kFlatLanes) force64_pairs_flat<T, KIND, ENERGY>(A, P, boxes, g, part, S);
    else force64_pairs_item<T, KIND, ENERGY>(A, P, boxes, g, part);
}

// After the pair force pass, per atom: the force = own share + the neighbours' shares, then what
// follows it (the kick or the corrector), on the energy step the atom's energy and partial sums.
template <bool ENERGY>
__device__ __forceinline__ void pairs_kick64(const Atoms &A, int i, double half_dt, int motion,
                                             double (&part)[kPartials]) {
    const double4_32a own = A.force[i], acc = A.f_acc[i];
    const double fx = own.x + acc.x, fy = own.y + acc.y, fz = own.z + acc.z;
    A.force[i] = make_double4_32a(fx, fy, fz, 0.0);
    if (!isfinite(fx + fy + fz)) atomicOr(&A.flags->error, FLAG_NONFINITE);
    double4_32a v = A.vel[i];
    finish_motion(A, i, v, fx, fy, fz, half_dt, motion);
    if (ENERGY) {
        // the virial's per-atom part x_a F_b (virial_shift), x as the force pass took it
        const double4_32a x = A.p2d[i];
        part[2] = fma(x.x, fx, part[2]);
        part[3] = fma(x.y, fy, part[3]);
        part[4] = fma(x.z, fz, part[4]);
        part[5] = fma(x.y, fz, part[5]);
        part[6] = fma(x.x, fz, part[6]);
        part[7] = fma(x.x, fy, part[7]);
        const double e = A.e_atom[i];
        const double m = 1.0 / (kMvv2e * v.w);
        part[0] += e;
        part[1] += m * fma(v.x, v.x, fma(v.y, v.y, v.z * v.z));
        part[8] += m * v.x; part[9] += m * v.y; part[10] += m * v.z;
    }
}

// ======================================================================= double-float (MD_PREC_DF)
// One species, knot tables.  The separation of two atoms is formed from the double-float image
// coordinates (md_df.cuh; posx/p2x): the high parts lie within a factor of two of each other
// (Box::xoff), so their difference is exact, and so is the subtraction of the periodic shift
// L_hi; the low parts carry the rest.  Every later quantity of the pair term (r^2, 1/r by one
// Newton step from the FP32 estimate, r, the knot index and t, the cubic of phi and the
// derivatives of V and phi) is double-float; the quadratic and cubic coefficients enter in FP32
// where their share of the result is below 2^-40 of it.  rho is summed in double-float and F(rho)
// is taken in FP64.  The force pass combines the per-entry (V'/r, phi'/r) of the density pass with
// F' as in the FP64 path, in double-float.

template <typename W>
__device__ __forceinline__ df::F2 sep_df(float xjh, float xih, float xjl, float xil, float Lh, float Ll, float invL) {
    float dh = __fsub_rn(xjh, xih);   // exact: both within a factor of two (Box::xoff)
    float dl = __fsub_rn(xjl, xil);
    if (W::value) {
        const float k = rintf(__fmul_rn(dh, invL));
        dh = __fmaf_rn(-k, Lh, dh);    // exact (|dh| and |k Lh| within a factor of two)
        dl = __fmaf_rn(-k, Ll, dl);
    }
    // left unnormalised (|dl| <= ulp(xoff), which can exceed ulp(dh)): the products below take dh
    // and dl separately, and the square keeps the dl^2 term
    return df::make(dh, dl);
}

__device__ __forceinline__ df::F2 r2_df(df::F2 dx, df::F2 dy, df::F2 dz) {
    auto sq = [](df::F2 d) {   // d unnormalised: its low part may exceed ulp(d.h), so keep d.l^2
        df::F2 p = df::two_prod(d.h, d.h);
        p.l = __fmaf_rn(2.f * d.h, d.l, __fmaf_rn(d.l, d.l, p.l));
        return p;
    };
    return df::add(df::add(sq(dx), sq(dy)), sq(dz));
}

// 1/sqrt(r2) from the FP32 estimate and one Newton step in double-float, and r = r2 / sqrt(r2).
__device__ __forceinline__ void rinv_df(df::F2 r2, df::F2 &rinv, df::F2 &r) {
    const float y = rsqrtf(r2.h);
    const df::F2 q = df::mul(r2, df::two_prod(y, y));
    const float e = __fsub_rn(__fsub_rn(1.f, q.h), q.l);   // 1 - r2 y^2 (1 - q.h exact)
    rinv = df::fast_two_sum(y, __fmul_rn(0.5f * y, e));
    r = df::mul(r2, rinv);
}

// Knot interval and t of r (x = r inv_dr - r_min inv_dr); below r_min: row 0, t = x (negative).
__device__ __forceinline__ int knot_df(const Pot &P, df::F2 r, df::F2 &t, bool &below) {
    const df::F2 x = df::add(df::mul(r, df::make(P.idr_h, P.idr_l)), df::make(-P.x0_h, -P.x0_l));
    below = x.h < 0.f;
    int k = below ? 0 : min((int)x.h, P.nk - 1);
    t = below ? x : df::two_sum(__fsub_rn(x.h, (float)k), x.l);   // x.h - k exact
    return k;
}

// Value of the interval's cubic c0 + t (c1 + t (c2 + t c3)): r0 = (c0 hi, lo, c1 hi, lo), c2, c3.
__device__ __forceinline__ df::F2 cubic_df(df::F2 t, float4 r0, float c2, float c3, bool below) {
    const float q = below ? 0.f : __fmaf_rn(t.h, c3, c2);
    df::F2 u = df::two_prod(t.h, q);
    u.l = __fmaf_rn(t.l, q, u.l);
    const df::F2 w = df::add(df::make(r0.z, r0.w), u);
    return df::add(df::make(r0.x, r0.y), df::mul(t, w));
}

// r-derivative of the interval's cubic: d1 + t (d2 + t e3) with r1 = (d1 hi, lo, d2 hi, lo).
__device__ __forceinline__ df::F2 dcubic_df(df::F2 t, float4 r1, float e3, bool below) {
    if (below) return df::make(r1.x, r1.y);
    const df::F2 q = df::two_sum(r1.z, __fmaf_rn(t.h, e3, r1.w));
    df::F2 u = df::two_prod(t.h, q.h);
    u.l = __fmaf_rn(t.h, q.l, __fmaf_rn(t.l, q.h, u.l));
    return df::add(df::make(r1.x, r1.y), u);
}

template <int T>
__device__ __forceinline__ void density_df_item(const Atoms &A, const Pot &P, const Box *boxes, long long g,
                                                bool energy = false) {
    const int i = (int)(g / T), lane = (int)(g & (T - 1));
    const bool live = i < A.n;
    df::Acc rho_acc{0.f, 0.f}, e_acc{0.f, 0.f};
    float4 pih = make_float4(0.f, 0.f, 0.f, 0.f), pil = pih;
    const bool wrap = needs_image(A, i, live);
    if (live) {
        const Box &B = boxes[ph::replica_of(A, i)];
        pih = ld_phase(A.posx + 2 * (size_t)i);
        pil = ld_phase(A.posx + 2 * (size_t)i + 1);
        const int cnt = min(A.count[i], A.k_max);
        const NbrRow row = nbr_row(A, i);
        const DRow drow = dcache_row(A, i);
        auto walk = [&](auto wrapt) {
            using W = decltype(wrapt);
            for (int k = lane; k < cnt; k += T) {
                const int j = ld_phase(row.ptr(k));
                const float4 pjh = ld_phase(A.posx + 2 * (size_t)j), pjl = ld_phase(A.posx + 2 * (size_t)j + 1);
                const df::F2 dx = sep_df<W>(pjh.x, pih.x, pjl.x, pil.x, B.Lh[0], B.Ll[0], B.invLf[0]);
                const df::F2 dy = sep_df<W>(pjh.y, pih.y, pjl.y, pil.y, B.Lh[1], B.Ll[1], B.invLf[1]);
                const df::F2 dz = sep_df<W>(pjh.z, pih.z, pjl.z, pil.z, B.Lh[2], B.Ll[2], B.invLf[2]);
                const df::F2 r2 = r2_df(dx, dy, dz);
                float4 *dc = reinterpret_cast<float4 *>(drow.ptr(k));
                if (!(r2.h < P.rc2f)) {
                    *dc = make_float4(0.f, 0.f, 0.f, 0.f);
                    continue;
                }
                df::F2 rinv, r, t;
                rinv_df(r2, rinv, r);
                bool below;
                const int kr = knot_df(P, r, t, below);
                if (below) atomicAdd(&A.flags->range_violations, 1ull);
                const float4 *tx = P.TX + 4 * (size_t)kr;
                const float4 x1 = tx[1];
                df::acc_add(rho_acc, cubic_df(t, tx[0], x1.x, x1.y, below));
                const df::F2 dphi = dcubic_df(t, tx[2], x1.z, below);
                const df::F2 dV = dcubic_df(t, tx[3], x1.w, below);
                const df::F2 gV = df::mul(dV, rinv), gP = df::mul(dphi, rinv);
                *dc = make_float4(gV.h, gV.l, gP.h, gP.l);
                if (energy) {   // the pair energy 1/2 V(r) into E_i
                    const float4 v0 = P.TVx[2 * (size_t)kr], v1 = P.TVx[2 * (size_t)kr + 1];
                    const df::F2 V = cubic_df(t, v0, v1.x, v1.y, below);
                    df::acc_add(e_acc, df::make(0.5f * V.h, 0.5f * V.l));
                }
            }
        };
        if (wrap) walk(std::true_type{});
        else walk(std::false_type{});
    }
    const df::F2 rho = df::lane_sum<T>(df::acc_value(rho_acc));
    const df::F2 ep = energy ? df::lane_sum<T>(df::acc_value(e_acc)) : df::make(0.f);
    if (live && lane == 0) {
        const double rr = df::to_double(rho);
        double dF;
        const double F = embed64(P, 0, rr, dF, A.flags);
        A.rho[i] = rr;
        A.dF[i] = dF;
        A.e_atom[i] = F + df::to_double(ep);
        const df::F2 f2 = df::from_double(dF);
        A.p2x[2 * (size_t)i] = make_float4(pih.x, pih.y, pih.z, f2.h);
        A.p2x[2 * (size_t)i + 1] = make_float4(pil.x, pil.y, pil.z, f2.l);
    }
}

template <int T, bool ENERGY>
__device__ __forceinline__ int force_df_item(const Atoms &A, const Pot &P, const Box *boxes, long long g,
                                             double half_dt, int motion, double (&part)[kPartials]) {
    const int i = (int)(g / T), lane = (int)(g & (T - 1));
    const bool live = i < A.n;
    df::Acc ax{0.f, 0.f}, ay = ax, az = ax;
    df::F2 ep = df::make(0.f);
    df::F2 wv[6] = {ep, ep, ep, ep, ep, ep};
    const bool wrap = needs_image(A, i, live);
    if (live) {
        const Box &B = boxes[ph::replica_of(A, i)];
        const float4 pih = A.p2x[2 * (size_t)i], pil = A.p2x[2 * (size_t)i + 1];
        const df::F2 Fpi = df::make(pih.w, pil.w);
        const int cnt = min(A.count[i], A.k_max);
        const NbrRow row = nbr_row(A, i);
        const DRow drow = dcache_row(A, i);
        auto walk = [&](auto wrapt) {
            using W = decltype(wrapt);
            for (int k = lane; k < cnt; k += T) {
                const int j = ld_phase(row.ptr(k));
                const float4 pjh = ld_phase(A.p2x + 2 * (size_t)j), pjl = ld_phase(A.p2x + 2 * (size_t)j + 1);
                const float4 e = ld_phase(reinterpret_cast<const float4 *>(drow.ptr(k)));
                const df::F2 dx = sep_df<W>(pjh.x, pih.x, pjl.x, pil.x, B.Lh[0], B.Ll[0], B.invLf[0]);
                const df::F2 dy = sep_df<W>(pjh.y, pih.y, pjl.y, pil.y, B.Lh[1], B.Ll[1], B.invLf[1]);
                const df::F2 dz = sep_df<W>(pjh.z, pih.z, pjl.z, pil.z, B.Lh[2], B.Ll[2], B.invLf[2]);
                const df::F2 sF = df::add(Fpi, df::make(pjh.w, pjl.w));
                const df::F2 gr = df::add(df::make(e.x, e.y), df::mul(sF, df::make(e.z, e.w)));
                df::acc_add(ax, df::mul(gr, dx));
                df::acc_add(ay, df::mul(gr, dy));
                df::acc_add(az, df::mul(gr, dz));
                if (ENERGY) {   // the virial (the pair energies are in E_i: density pass)
                    const df::F2 hg = df::make(-0.5f * gr.h, -0.5f * gr.l);
                    const df::F2 hx = df::mul(hg, dx), hy = df::mul(hg, dy);
                    wv[0] = df::add(wv[0], df::mul(hx, dx));
                    wv[1] = df::add(wv[1], df::mul(hy, dy));
                    wv[2] = df::add(wv[2], df::mul(df::mul(hg, dz), dz));
                    wv[3] = df::add(wv[3], df::mul(hy, dz));
                    wv[4] = df::add(wv[4], df::mul(hx, dz));
                    wv[5] = df::add(wv[5], df::mul(hx, dy));
                }
            }
        };
        if (wrap) walk(std::true_type{});
        else walk(std::false_type{});
    }
    const df::F2 fx = df::lane_sum<T>(df::acc_value(ax)), fy = df::lane_sum<T>(df::acc_value(ay)),
                 fz = df::lane_sum<T>(df::acc_value(az));
    if (ENERGY) {
        ep = df::lane_sum<T>(ep);
#pragma unroll
        for (int q = 0; q < 6; q++) wv[q] = df::lane_sum<T>(wv[q]);
    }
    if (!(live && lane == 0)) return -1;
    const double Fx = df::to_double(fx), Fy = df::to_double(fy), Fz = df::to_double(fz);
    A.force[i] = make_double4_32a(Fx, Fy, Fz, 0.0);
    if (!isfinite(Fx + Fy + Fz)) atomicOr(&A.flags->error, FLAG_NONFINITE);
    double4_32a v = A.vel[i];
    finish_motion(A, i, v, Fx, Fy, Fz, half_dt, motion);
    if (ENERGY) {
        const double e = A.e_atom[i] + df::to_double(ep);
        A.e_atom[i] = e;
        const double m = 1.0 / (kMvv2e * v.w);
        part[0] += e;
        part[1] += m * fma(v.x, v.x, fma(v.y, v.y, v.z * v.z));
#pragma unroll
        for (int q = 0; q < 6; q++) part[2 + q] += df::to_double(wv[q]);
        part[8] += m * v.x; part[9] += m * v.y; part[10] += m * v.z;
    }
    return i;
}

// Precision-generic front ends.
// energy: the step's energies are wanted (the FP64 path with the derivative cache and the
// double-float path sum the pair energies in this pass; the mixed path in the force pass).
template <int PREC, int T, int KIND, bool MULTI, bool SMT = false>
__device__ __forceinline__ void density_item(const Atoms &A, const Pot &P, const Box *boxes, long long g,
                                             bool energy = false) {
    if constexpr (PREC == MD_PREC_DF) {
        if constexpr (KIND == MD_POT_TABLES && !MULTI) density_df_item<T>(A, P, boxes, g, energy);
    } else if constexpr (PREC == MD_PREC_FP64) {
        density64_item<T, KIND, MULTI>(A, P, boxes, g, energy);
    } else {
        density32_item<T, KIND, MULTI, SMT>(A, P, boxes, g);
    }
}

template <int PREC, int T, int KIND, bool MULTI, bool ENERGY, bool SMT = false>
__device__ __forceinline__ int force_item(const Atoms &A, const Pot &P, const Box *boxes, long long g,
                                          double half_dt, int motion, double (&part)[kPartials]) {
    if constexpr (PREC == MD_PREC_DF) {
        if constexpr (KIND == MD_POT_TABLES && !MULTI) return force_df_item<T, ENERGY>(A, P, boxes, g, half_dt, motion, part);
        return -1;
    } else if constexpr (PREC == MD_PREC_FP64) {
        return force64_item<T, KIND, MULTI, ENERGY>(A, P, boxes, g, half_dt, motion, part);
    } else {
        return force32_item<T, KIND, MULTI, ENERGY, SMT>(A, P, boxes, g, half_dt, motion, part);
    }
}

}  // namespace ps
}  // namespace mdk
