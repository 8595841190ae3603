// Per-atom state kernels: velocity-Verlet half kick + drift (§2.3), the strain-rate box
// update (§2.2), the skin displacement check (§3.2.1), the FP32 wrapped position copy, and
// the conversions between cell order and the caller's atom order.
#include <cuda_runtime.h>

#include "md_internal.cuh"

namespace mdk {

namespace {

__device__ __forceinline__ float wrap1(double x, double L, double invL) {
    return (float)(x - L * floor(x * invL));
}

__device__ __forceinline__ float4 wrapped(const double4_32a &p, const Box &B, int species) {
    return make_float4(wrap1(p.x, B.L[0], B.invL[0]), wrap1(p.y, B.L[1], B.invL[1]),
                       wrap1(p.z, B.L[2], B.invL[2]), __int_as_float(species));
}

// The box matrix times the strain matrix diag(1, 1, s): one thread, once per step.
__global__ void k_box_update(Box *box, double s) {
    Box b = *box;
    b.L[2] = __dmul_rn(b.L[2], s);
    b.invL[2] = 1.0 / b.L[2];
    b.Lf[2] = (float)b.L[2];
    b.invLf[2] = (float)b.invL[2];
    *box = b;
}

// v += (dt/2) F/m;  r += dt v;  [z *= s];  displacement since the list build vs skin/2.
// The FP64 operations are the separately rounded ones of the definition (no contraction).
template <bool STRAIN>
__global__ void __launch_bounds__(kThreads) k_kick_drift(Atoms A, double half_dt, double dt, double s,
                                                         double lim2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    const Box B = *A.box;
    double4_32a v = A.vel[i];
    const double4_32a f = A.force[i];
    double4_32a p = A.pos[i];
    v.x = __dadd_rn(v.x, __dmul_rn(__dmul_rn(half_dt, f.x), v.w));
    v.y = __dadd_rn(v.y, __dmul_rn(__dmul_rn(half_dt, f.y), v.w));
    v.z = __dadd_rn(v.z, __dmul_rn(__dmul_rn(half_dt, f.z), v.w));
    p.x = __dadd_rn(p.x, __dmul_rn(dt, v.x));
    p.y = __dadd_rn(p.y, __dmul_rn(dt, v.y));
    p.z = __dadd_rn(p.z, __dmul_rn(dt, v.z));
    if (STRAIN) p.z = __dmul_rn(p.z, s);
    A.vel[i] = v;
    A.pos[i] = p;
    const double4_32a r = A.ref[i];
    const double ex = __dsub_rn(p.x, r.x), ey = __dsub_rn(p.y, r.y), ez = __dsub_rn(p.z, r.z);
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
    if (d2 > lim2 || !(d2 == d2)) {
        A.flags->need_rebuild = 1;
        A.flags->skin_exceeded = 1;
    }
    A.posf[i] = wrapped(p, B, __float_as_int(A.posf[i].w));
}

__global__ void k_check_displacement(Atoms A, double lim2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    const double4_32a p = A.pos[i], r = A.ref[i];
    const double ex = __dsub_rn(p.x, r.x), ey = __dsub_rn(p.y, r.y), ez = __dsub_rn(p.z, r.z);
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
    if (d2 > lim2 || !(d2 == d2)) {
        A.flags->need_rebuild = 1;
        A.flags->skin_exceeded = 1;
    }
}

__global__ void k_wrap(Atoms A) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    A.posf[i] = wrapped(A.pos[i], *A.box, A.spec[i]);
}

__global__ void k_unsort_vec(Atoms A, const double4_32a *src, double *dst) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= A.n) return;
    const double4_32a v = src[k];
    const size_t o = 3 * (size_t)A.id[k];
    dst[o] = v.x;
    dst[o + 1] = v.y;
    dst[o + 2] = v.z;
}

__global__ void k_unsort_scalar(Atoms A, const double *src, double *dst) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= A.n) return;
    dst[A.id[k]] = src[k];
}

__global__ void k_unsort_int(Atoms A, const int32_t *src, int32_t *dst) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= A.n) return;
    dst[A.id[k]] = src[k];
}

__global__ void k_unsort_list(Atoms A, int32_t *dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    const int cnt = min(A.count[i], A.k_max);
    int32_t *row = dst + (size_t)A.id[i] * A.k_max;
    const int32_t *src = A.nbr + (size_t)i * A.k_max;
    for (int k = 0; k < A.k_max; k++)
        row[k] = k < cnt ? A.id[src[k]] : -1;
}

__global__ void k_sort_in_vec(Atoms A, const double *src, double4_32a *dst) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= A.n) return;
    const size_t o = 3 * (size_t)A.id[k];
    double4_32a v = dst[k];
    v.x = src[o];
    v.y = src[o + 1];
    v.z = src[o + 2];
    dst[k] = v;
}

}  // namespace

cudaError_t launch_box_update(Box *box, double scale_z, cudaStream_t s) {
    k_box_update<<<1, 1, 0, s>>>(box, scale_z);
    return cudaGetLastError();
}

cudaError_t launch_kick_drift(const Atoms &A, double half_dt, double dt, double strain_scale, double lim2,
                              cudaStream_t s) {
    if (A.n == 0) return cudaSuccess;
    const int nb = blocks_for(A.n, kThreads);
    if (strain_scale != 1.0)
        k_kick_drift<true><<<nb, kThreads, 0, s>>>(A, half_dt, dt, strain_scale, lim2);
    else
        k_kick_drift<false><<<nb, kThreads, 0, s>>>(A, half_dt, dt, strain_scale, lim2);
    return cudaGetLastError();
}

cudaError_t launch_check_displacement(const Atoms &A, double lim2, cudaStream_t s) {
    if (A.n == 0) return cudaSuccess;
    k_check_displacement<<<blocks_for(A.n, kThreads), kThreads, 0, s>>>(A, lim2);
    return cudaGetLastError();
}

cudaError_t launch_wrap(const Atoms &A, cudaStream_t s) {
    if (A.n == 0) return cudaSuccess;
    k_wrap<<<blocks_for(A.n, kThreads), kThreads, 0, s>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_unsort_vec(const Atoms &A, const double4_32a *src, double *dst, cudaStream_t s) {
    if (A.n == 0) return cudaSuccess;
    k_unsort_vec<<<blocks_for(A.n, kThreads), kThreads, 0, s>>>(A, src, dst);
    return cudaGetLastError();
}

cudaError_t launch_unsort_scalar(const Atoms &A, const double *src, double *dst, cudaStream_t s) {
    if (A.n == 0) return cudaSuccess;
    k_unsort_scalar<<<blocks_for(A.n, kThreads), kThreads, 0, s>>>(A, src, dst);
    return cudaGetLastError();
}

cudaError_t launch_unsort_int(const Atoms &A, const int32_t *src, int32_t *dst, cudaStream_t s) {
    if (A.n == 0) return cudaSuccess;
    k_unsort_int<<<blocks_for(A.n, kThreads), kThreads, 0, s>>>(A, src, dst);
    return cudaGetLastError();
}

cudaError_t launch_unsort_list(const Atoms &A, int32_t *dst, cudaStream_t s) {
    if (A.n == 0) return cudaSuccess;
    k_unsort_list<<<blocks_for(A.n, kThreads), kThreads, 0, s>>>(A, dst);
    return cudaGetLastError();
}

cudaError_t launch_sort_in_vec(const Atoms &A, const double *src, double4_32a *dst, cudaStream_t s) {
    if (A.n == 0) return cudaSuccess;
    k_sort_in_vec<<<blocks_for(A.n, kThreads), kThreads, 0, s>>>(A, src, dst);
    return cudaGetLastError();
}

}  // namespace mdk
