// Device helpers shared by the FP64 and mixed EAM passes (md_eam64.cu, md_eam32.cu).
//
// Work split: T lanes per atom (T a power of two dividing 32).  Lane l of atom i takes the
// neighbours k = l, l+T, l+2T, ... of i's list row (nbr[i*k_max + k]), so the T lanes read
// one contiguous stretch of the row; the lanes' partial sums are combined by a fixed
// butterfly of warp shuffles, so the result depends on T but not on scheduling.
#pragma once

#include <cuda_runtime.h>

#include "md_internal.cuh"

namespace mdk {
namespace eam {

// Conversions between FP64 and FP32 by the IEEE bit fields, in integer registers (the FP64 pipe,
// which the FP64 passes keep busy, also executes the conversion instructions): the exponent is
// rebiased by 1023 - 127 = 896 and the significand shifted by 29 bits.  f32_trunc: x >= 0 below
// the FP32 overflow threshold, rounded toward zero (relative error < 2^-23), and 0 below the
// normal FP32 range (so that coincident atoms still give 1/sqrt(0) = inf); f64_exact: f positive,
// normal or +inf, exact.
__device__ __forceinline__ float f32_trunc(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    return __uint_as_float(hi < (897u << 20) ? 0u : ((hi - (896u << 20)) << 3) | (lo >> 29));
}
__device__ __forceinline__ double f64_exact(float f) {
    const unsigned b = __float_as_uint(f);
    return b >= 0x7f800000u ? __hiloint2double(0x7ff00000, 0)
                            : __hiloint2double((int)((b >> 3) + (896u << 20)), (int)(b << 29));
}

// The rest x - f32_trunc(x) of a positive normal x, as FP32: its 29 low significand bits m, worth
// m 2^(E - 52), rounded to nearest (0 where m = 0 or E < -70, below which the exponent field
// would not hold it; the FP64 path's r^2 lie far inside).
__device__ __forceinline__ float f32_rest(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned m = lo & 0x1FFFFFFFu;
    const int E = (int)(hi >> 20) - 1023;
    const float mf = __uint2float_rn(m);
    return (m == 0u || E < -70) ? 0.f : __int_as_float(__float_as_int(mf) + (E - 52) * (1 << 23));
}
// f as a double, exact, any sign: 0 for |f| below the normal FP32 range, NaN for inf or NaN.
__device__ __forceinline__ double f64_of_f32(float f) {
    const unsigned b = __float_as_uint(f), mag = b & 0x7fffffffu;
    const double v = __hiloint2double((int)((b & 0x80000000u) | ((mag >> 3) + (896u << 20))), (int)(mag << 29));
    return mag >= 0x7f800000u ? __hiloint2double(0x7ff80000, 0) : (mag < 0x00800000u ? 0.0 : v);
}

// d = dh + dl for any sign: dh = d truncated to FP32, dl the rest rounded to FP32 (|dl| < 2^-23
// |dh|, relative rounding 2^-24), both on the bit fields in integer registers; 0 and 0 where |d|
// lies below FP32's normal range, and a NaN dh where |d| >= 2^128 or d is not finite.
__device__ __forceinline__ void split64(double d, float &dh, float &dl) {
    const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
    const unsigned mag = hi & 0x7fffffffu, sgn = hi & 0x80000000u;
    const bool tiny = mag < (897u << 20);
    const unsigned h = mag >= (1151u << 20) ? 0x7fc00000u : ((mag - (896u << 20)) << 3) | (lo >> 29);
    dh = __uint_as_float(tiny ? 0u : (sgn | h));
    const float r = f32_rest(__hiloint2double((int)mag, (int)lo));
    dl = tiny ? 0.f : __uint_as_float(__float_as_uint(r) | sgn);
}
// dx^2 + dy^2 + dz^2 from FP32 pieces: each square as Dekker's exact product of the high part
// plus the cross term 2 dh dl in FP32 (dl^2, below 2^-46 of the square, dropped), the three
// exact high products summed exactly by Knuth's two-sum and the small terms (at most 2^-21.7 of
// the sum) in FP32, then one FP64 addition.  Worst-case relative error 1.7e-13 (the six FP32
// roundings of the small terms, 2^-24 of them each, and the replaced and dropped parts of the
// squares), so that 1/r from it and rsqrt64 stays within 4e-13.
__device__ __forceinline__ double r2_split(double dx, double dy, double dz) {
    float xh, xl, yh, yl, zh, zl;
    split64(dx, xh, xl);
    split64(dy, yh, yl);
    split64(dz, zh, zl);
    const float px = __fmul_rn(xh, xh), py = __fmul_rn(yh, yh), pz = __fmul_rn(zh, zh);
    float e = __fmaf_rn(xh, xh, -px);   // the products' low parts and the cross terms
    e = __fadd_rn(e, __fmaf_rn(yh, yh, -py));
    e = __fadd_rn(e, __fmaf_rn(zh, zh, -pz));
    e = __fmaf_rn(__fmul_rn(2.f, xh), xl, e);
    e = __fmaf_rn(__fmul_rn(2.f, yh), yl, e);
    e = __fmaf_rn(__fmul_rn(2.f, zh), zl, e);
    float s = __fadd_rn(px, py);        // px + py + pz = s2 + c exactly
    float bb = __fsub_rn(s, px);
    float c = __fadd_rn(__fsub_rn(px, __fsub_rn(s, bb)), __fsub_rn(py, bb));
    const float s2 = __fadd_rn(s, pz);
    bb = __fsub_rn(s2, s);
    c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(s2, bb)), __fsub_rn(pz, bb)));
    return f64_of_f32(s2) + f64_of_f32(__fadd_rn(c, e));
}

// 1/sqrt(x), x positive: the FP32 estimate y (x truncated to FP32, then rsqrtf within 2 ulp:
// relative error eps <= 3.6e-7) and one Newton-Raphson step y + y e / 2, e = 1 - x y^2, which
// leaves (3/2) eps^2 <= 2e-13.  The step's correction is small, so it is formed in FP32 from
// exact pieces (Dekker's product y^2 = ph + pl; x = xf + xr split on its bit fields): 1 - xf ph
// by one FMA (|e| < 2^-20, so rounded to within 2^-44), the rest x y^2 - xf ph to about 2^-46,
// y e / 2 to 2^-24 of itself; e and the correction add at most 1e-13 to the relative error, <=
// 3e-13 in all, three orders of magnitude inside the 1e-10 parity of the FP64 path, for one FP64
// addition (the FP64 pipe bounds the FP64 passes).  Coincident atoms (x = 0) still give a
// non-finite value.
// MD_RSQRT64_STEPS=2: two Newton steps in FP64 instead, to FP64 rounding (~1e-16).
#ifndef MD_RSQRT64_STEPS
#define MD_RSQRT64_STEPS 1
#endif
__device__ __forceinline__ double rsqrt64(double x) {
#if MD_RSQRT64_STEPS >= 2
    // y / 2 by the exponent field (y is positive and normal, or +inf: then e is NaN either way)
    auto half = [](double y) { return __longlong_as_double(__double_as_longlong(y) - (1LL << 52)); };
    double y = f64_exact(rsqrtf(f32_trunc(x)));
    for (int s = 0; s < 2; s++) {
        const double e = fma(-x * y, y, 1.0);
        y = fma(half(y), e, y);
    }
    return y;
#else
    const float xf = f32_trunc(x), xr = f32_rest(x);
    const float y = rsqrtf(xf);
    const float ph = __fmul_rn(y, y), pl = __fmaf_rn(y, y, -ph);   // y^2 = ph + pl exactly
    const float a = __fmaf_rn(-xf, ph, 1.0f);                     // 1 - xf ph, one rounding
    const float b = __fmaf_rn(xf, pl, __fmul_rn(xr, ph));         // x y^2 - xf ph (xr pl dropped)
    const float h = __fmul_rn(__fmul_rn(0.5f, y), __fsub_rn(a, b));  // y e / 2
    return f64_exact(y) + f64_of_f32(h);
#endif
}

// Error-free FP32 accumulation (Knuth's TwoSum): hi + lo carries the exact running sum.
__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float x) {
    float s = hi + x;
    float bp = s - hi;
    float err = (hi - (s - bp)) + (x - bp);
    hi = s;
    lo += err;
}

__device__ __forceinline__ void unpack2(double d, float &a, float &b) {
    long long v = __double_as_longlong(d);
    a = __int_as_float((int)(v & 0xffffffffll));
    b = __int_as_float((int)(v >> 32));
}

// Interval of a uniform knot grid: x in knot units.  Returns the row and t in [0,1]
// (row nk-1 continues linearly); below the first knot returns row 0 with `below` set.
template <typename R>
__device__ __forceinline__ int knot_row(R x, int nk, R &t, bool &below) {
    below = !(x >= R(0));
    int k = (x < (R)(nk - 1)) ? (int)x : nk - 1;
    k = below ? 0 : k;
    t = below ? x : x - (R)k;
    return k;
}

// The FP64 passes' versions of the pair cut and of knot_row<double>, with the same results: the
// comparisons and the conversions between double and int act on the IEEE bit patterns in integer
// registers (non-negative doubles order as their bit patterns do), which leaves the FP64 pipe to
// the arithmetic.
// v / 2 by the exponent field (no FP64 operation); |v| below 2^-1021 (a subnormal half) gives 0.
__device__ __forceinline__ double half64(double v) {
    const long long b = __double_as_longlong(v);
    return (b & 0x7FF0000000000000LL) > (1LL << 52) ? __longlong_as_double(b - (1LL << 52)) : 0.0;
}
// r2 < rc2 for r2 >= 0 (or NaN, which is never inside) and rc2 > 0.
__device__ __forceinline__ bool inside64(double r2, double rc2) {
    return __double_as_longlong(r2) < __double_as_longlong(rc2);
}
// knot_row<double>(x, nk, t, below) for finite x < nk, which holds for every pair inside r_cut
// (the last knot): k = min(floor(x), nk - 1) from the significand, and t = x - floor(x) (exactly
// x - k, as x - k is exact) from the fraction's bits, normalised in integer registers, so that the
// knot interval and its coordinate take no FP64 operation.
__device__ __forceinline__ int knot_row64(double x, int nk, double &t, bool &below) {
    const long long b = __double_as_longlong(x);
    below = b < 0;   // x < 0 (x = -0 gives the same values either way)
    const int e = (int)((b >> 52) & 0x7ff) - 1023;   // x >= 1: floor(x) = significand >> (52 - e)
    const long long sig = (b & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;
    const int sh = 52 - min(max(e, 0), 52);           // bits below the binary point (e >= 0)
    const long long fb = sig & ((1LL << sh) - 1);     // the fraction, fb 2^(e - 52)
    const int p = 63 - __clzll(fb | 1);               // its leading bit
    const long long tb = ((long long)(1023 + e - 52 + p) << 52) | ((fb << (52 - p)) & 0xFFFFFFFFFFFFFLL);
    // e >= 31 (x >= 2^31: only a NaN or infinite x, from coincident atoms): the last row, and t = x
    // carries the non-finite value on
    const bool huge = e >= 31;
    const int k = e < 0 ? 0 : (huge ? nk - 1 : min((int)(sig >> sh), nk - 1));
    t = (below || e < 0 || huge) ? x : (fb == 0 ? 0.0 : __longlong_as_double(tb));
    return below ? 0 : k;
}

template <typename R>
__device__ __forceinline__ R cubic(R t, R c0, R c1, R c2, R c3, bool below, R &dydt) {
    if (below) {
        dydt = c1;
        return fma(t, c1, c0);
    }
    dydt = fma(t, fma(R(3) * c3, t, R(2) * c2), c1);
    return fma(t, fma(t, fma(t, c3, c2), c1), c0);
}

// ---- analytic Finnis-Sinclair pair functions (fs = d, c, A, beta, c0, c1, c2; bd = beta/d) ----
template <typename R>
__device__ __forceinline__ R fs_phi(const R *fs, R bd, R r) {
    R t = r - fs[0];
    return t < R(0) ? t * t * fma(bd, t, R(1)) : R(0);
}

template <typename R>
__device__ __forceinline__ R fs_dphi(const R *fs, R bd, R r) {
    R t = r - fs[0];
    return t < R(0) ? t * fma(R(3) * bd, t, R(2)) : R(0);
}

template <typename R>
__device__ __forceinline__ R fs_V(const R *fs, R r, R &dV) {
    R u = r - fs[1];
    if (!(u < R(0))) {
        dV = R(0);
        return R(0);
    }
    R q = fma(fma(fs[6], r, fs[5]), r, fs[4]);
    R dq = fma(R(2) * fs[6], r, fs[5]);
    dV = u * fma(u, dq, R(2) * q);
    return u * u * q;
}

// Explicit cubic knot sum f(r) = sum_q c_q (r_q - r)^3 for r < r_q (the generic potential files'
// form, §3.1.1) and df/dr; k[q] = (c_q, r_q).
template <typename R, typename R2>
__device__ __forceinline__ R knot_sum(const R2 *__restrict__ k, int n, R r, R &d) {
    R v = R(0), g = R(0);
    for (int q = 0; q < n; q++) {
        const R2 c = k[q];
        const R u = c.y > r ? c.y - r : R(0);
        const R cu2 = c.x * u * u;
        v = fma(cu2, u, v);
        g = fma(R(-3), cu2, g);
    }
    d = g;
    return v;
}

// F and F' in FP64 (one evaluation per atom, both precisions).
__device__ __forceinline__ double embed64(const Pot &P, int a, double rho, double &dF, Flags *flags) {
    if (P.kind == MD_POT_FS_ANALYTIC || P.kind == MD_POT_KNOTS) {
        const double Aa = P.kind == MD_POT_KNOTS ? P.A64[a] : P.fs[2];
        if (!(rho > 0.0)) {
            dF = 0.0;
            return 0.0;
        }
        double s = sqrt(rho);
        dF = -0.5 * Aa / s;
        return -Aa * s;
    }
    double x = (rho - P.rho_min) * P.inv_drho, t, d;
    bool below;
    int k = knot_row(x, P.nk, t, below);
    if (below || x > (double)(P.nk - 1)) atomicAdd(&flags->range_violations, 1ull);
    double4_32a c = P.F64[(size_t)a * P.nk + k];
    double F = cubic(t, c.x, c.y, c.z, c.w, below, d);
    dF = d * P.inv_drho;
    return F;
}

// Butterfly sum over the T lanes of an atom (all 32 lanes of the warp take part).
template <int T, typename V>
__device__ __forceinline__ V lane_sum(V x) {
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

template <int T>
__device__ __forceinline__ void lane_sum_df(float &hi, float &lo) {
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) {
        float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        two_sum_add(hi, lo, h2);
        lo += l2;
    }
}

// Per-block FP64 partial sums (fixed order), stored as out[q * stride + block]: every thread of
// the block (NT threads) must call it.
template <int NT = kThreads>
__device__ __forceinline__ void block_partials(double (&v)[kPartials], double *out, int stride) {
    __shared__ double sh[NT / 32][kPartials];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kPartials; q++) {
        double x = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[w][q] = x;
    }
    __syncthreads();
    if (threadIdx.x < kPartials) {
        double s = 0.0;
        for (int k = 0; k < NT / 32; k++) s += sh[k][threadIdx.x];
        out[(size_t)threadIdx.x * stride + blockIdx.x] = s;
    }
}

__device__ __forceinline__ void clear_rebuild_once(Flags *f) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (f->need_rebuild) f->n_rebuilds++;
        f->need_rebuild = 0;
    }
}

// Second half kick v += (dt/2 * f) * (acc/m) with the separately rounded operations of the
// definition, and the atom's kinetic/momentum partials (m = acc / v.w).
__device__ __forceinline__ void kick_and_partials(double4_32a &v, double fx, double fy, double fz,
                                                  double half_dt, bool kick) {
    if (kick) {
        v.x = __dadd_rn(v.x, __dmul_rn(__dmul_rn(half_dt, fx), v.w));
        v.y = __dadd_rn(v.y, __dmul_rn(__dmul_rn(half_dt, fy), v.w));
        v.z = __dadd_rn(v.z, __dmul_rn(__dmul_rn(half_dt, fz), v.w));
    }
}

// Gear's corrector coefficients of the third-order predictor-corrector for a second-order equation
// (four Taylor terms): position, velocity (scaled by dt), acceleration (1), third derivative.
constexpr double kPcPos = 1.0 / 6.0, kPcVel = 5.0 / 6.0, kPcJerk = 1.0 / 3.0;

// What follows atom i's force f: motion kMotionVerlet: the second half kick v += (dt/2) f/m;
// kMotionPC3: the corrector, D = (dt^2/2) f/m - g2 (g2 = the predicted acceleration term), then
// r += D/6, v += (5/6) D/dt, g3 += D/3 (the acceleration term becomes (dt^2/2) f/m, which the
// next predictor takes from the stored force).  v (in/out) is the atom's velocity record.
__device__ __forceinline__ void finish_motion(const Atoms &A, int i, double4_32a &v, double fx, double fy, double fz,
                                              double half_dt, int motion) {
    if (motion == kMotionVerlet) {
        kick_and_partials(v, fx, fy, fz, half_dt, true);
        A.vel[i] = v;
    } else if (motion == kMotionPC3) {
        const double dt = 2.0 * half_dt, h2 = 0.5 * dt * dt;
        const double4_32a q2 = A.g2[i];
        double4_32a q3 = A.g3[i], p = A.pos[i];
        const double Dx = __dsub_rn(__dmul_rn(__dmul_rn(h2, fx), v.w), q2.x);
        const double Dy = __dsub_rn(__dmul_rn(__dmul_rn(h2, fy), v.w), q2.y);
        const double Dz = __dsub_rn(__dmul_rn(__dmul_rn(h2, fz), v.w), q2.z);
        p.x = __dadd_rn(p.x, __dmul_rn(kPcPos, Dx));
        p.y = __dadd_rn(p.y, __dmul_rn(kPcPos, Dy));
        p.z = __dadd_rn(p.z, __dmul_rn(kPcPos, Dz));
        v.x = __dadd_rn(v.x, __ddiv_rn(__dmul_rn(kPcVel, Dx), dt));
        v.y = __dadd_rn(v.y, __ddiv_rn(__dmul_rn(kPcVel, Dy), dt));
        v.z = __dadd_rn(v.z, __ddiv_rn(__dmul_rn(kPcVel, Dz), dt));
        q3.x = __dadd_rn(q3.x, __dmul_rn(kPcJerk, Dx));
        q3.y = __dadd_rn(q3.y, __dmul_rn(kPcJerk, Dy));
        q3.z = __dadd_rn(q3.z, __dmul_rn(kPcJerk, Dz));
        A.pos[i] = p;
        A.vel[i] = v;
        A.g3[i] = q3;
    }
}

// Host-side grid size of a T-lanes-per-atom launch.
template <int T>
inline int blocks_for_lanes(long long n) {
    return (int)((n * T + kThreads - 1) / kThreads);
}

}  // namespace eam
}  // namespace mdk
