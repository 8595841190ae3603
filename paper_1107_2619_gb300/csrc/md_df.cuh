// Double-float arithmetic: a value held as the unevaluated sum hi + lo of two FP32 numbers
// (|lo| <= ulp(hi) / 2 when normalised), 48 significant bits.  The error-free transformations
// are Knuth's two-sum, Dekker's fast two-sum (|a| >= |b|) and the FMA form of the exact
// product (a b = p + fma(a, b, -p)); the operations built from them are the classical
// double-float add and multiply (Dekker 1971; the "sloppy" add, whose relative error is a few
// units of 2^-48 when the operands do not cancel).
//
// On GB300 the FP32 pipes run 64x the FP64 rate, so a pair term evaluated in double-float (about
// 150 FP32 operations) costs a fraction of the same term in FP64 (about 30 FP64 operations).
#pragma once

#include <cuda_runtime.h>

namespace mdk {
namespace df {

struct F2 {
    float h, l;
};

__device__ __forceinline__ F2 make(float h, float l = 0.f) { return F2{h, l}; }

// s + e = a + b exactly.
__device__ __forceinline__ F2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return F2{s, e};
}

// s + e = a + b exactly, for |a| >= |b| (or a = 0).
__device__ __forceinline__ F2 fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return F2{s, __fsub_rn(b, __fsub_rn(s, a))};
}

// p + e = a b exactly.
__device__ __forceinline__ F2 two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return F2{p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ F2 add(F2 a, F2 b) {
    const F2 s = two_sum(a.h, b.h);
    return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}

__device__ __forceinline__ F2 neg(F2 a) { return F2{-a.h, -a.l}; }

__device__ __forceinline__ F2 mul(F2 a, F2 b) {
    F2 p = two_prod(a.h, b.h);
    p.l = __fmaf_rn(a.h, b.l, p.l);
    p.l = __fmaf_rn(a.l, b.h, p.l);
    return fast_two_sum(p.h, p.l);
}

// a (double-float) times b (FP32).
__device__ __forceinline__ F2 mul_f(F2 a, float b) {
    F2 p = two_prod(a.h, b);
    p.l = __fmaf_rn(a.l, b, p.l);
    return fast_two_sum(p.h, p.l);
}

// Compensated accumulator of many terms: the running FP32 sum s and the FP32 sum e of the exact
// rounding errors of the additions and of the terms' low parts (normalised once, at the end).
struct Acc {
    float s, e;
};
__device__ __forceinline__ void acc_add(Acc &a, F2 x) {
    const F2 t = two_sum(a.s, x.h);
    a.s = t.h;
    a.e = __fadd_rn(a.e, __fadd_rn(t.l, x.l));
}
__device__ __forceinline__ F2 acc_value(Acc a) { return fast_two_sum(a.s, a.e); }

// Value as FP64 (exact: both parts convert exactly).
__device__ __forceinline__ double to_double(F2 a) { return (double)a.h + (double)a.l; }

// Nearest double-float of an FP64 value (hi rounded to FP32, then the remainder).
__host__ __device__ __forceinline__ F2 from_double(double x) {
    const float h = (float)x;
    return F2{h, (float)(x - (double)h)};
}

// Butterfly sum over the T lanes of an atom (every lane of the warp takes part).
template <int T>
__device__ __forceinline__ F2 lane_sum(F2 x) {
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) {
        F2 y;
        y.h = __shfl_xor_sync(0xffffffffu, x.h, o);
        y.l = __shfl_xor_sync(0xffffffffu, x.l, o);
        x = add(x, y);
    }
    return x;
}

}  // namespace df
}  // namespace mdk
