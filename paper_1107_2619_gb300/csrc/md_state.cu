// Per-atom state kernels outside the step: the skin displacement check (§3.2.1), the FP32
// position copy (in the image of the last list build), and the conversions between cell
// order and the caller's atom order.
#include <cuda_runtime.h>

#include "md_phases.cuh"

namespace mdk {

namespace {

__global__ void k_check_displacement(Atoms A, double lim2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    ph::check_displacement(A, i, lim2);
}

__global__ void k_wrap(Atoms A) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    A.posf[i] = ph::build_image(A.pos[i], A.ref[i], A.boxes[ph::replica_of(A, i)], A.spec[i]);
    if (A.posd) {
        const Box &B = A.boxes[ph::replica_of(A, i)];
        const double4_32a q = ph::build_image64(A.pos[i], A.ref[i], B);
        A.posd[i] = q;
        if (A.posx) ph::store_dfpos(A, i, q, B);
    }
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

// The coordinates the passes take: the FP32 copy (mixed path) or the FP64 copy (FP64 path), both
// in the periodic image of the last list build.
__global__ void k_unsort_image(Atoms A, double *dst) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= A.n) return;
    const size_t o = 3 * (size_t)A.id[k];
    if (A.posd) {
        const double4_32a v = A.posd[k];
        dst[o] = v.x;
        dst[o + 1] = v.y;
        dst[o + 2] = v.z;
    } else {
        const float4 v = A.posf[k];
        dst[o] = v.x;
        dst[o + 1] = v.y;
        dst[o + 2] = v.z;
    }
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
    const NbrRow src = nbr_row(A, i);
    for (int k = 0; k < A.k_max; k++) row[k] = k < cnt ? A.id[src[k]] : -1;
}

// The same two copies for a caller buffer in mapped pinned host memory, read and written by the
// device over the host link.  A block takes the caller's atoms c0 .. c0 + kThreads - 1, whose 3
// doubles each are one contiguous host range: it is moved in 16-byte pieces by consecutive
// threads (whole lines over the link; the range starts 16-byte aligned when the buffer does, as
// 24 kThreads is a multiple of 16), staged in shared memory, and each thread c reaches the
// cell-ordered slot rank[c] in device memory.  VEC = false: 8-byte pieces, for a buffer that is
// not 16-byte aligned.
template <bool VEC>
__device__ __forceinline__ void host_range_in(const double *src, double *sh, int c0, int nb) {
    const int m = 3 * nb;   // doubles of this block
    if (VEC) {
        const double2 *s2 = reinterpret_cast<const double2 *>(src + 3 * (size_t)c0);
        for (int q = threadIdx.x; q < m / 2; q += blockDim.x) reinterpret_cast<double2 *>(sh)[q] = s2[q];
        if ((m & 1) && threadIdx.x == 0) sh[m - 1] = src[3 * (size_t)c0 + m - 1];
    } else {
        for (int q = threadIdx.x; q < m; q += blockDim.x) sh[q] = src[3 * (size_t)c0 + q];
    }
}
template <bool VEC>
__device__ __forceinline__ void host_range_out(double *dst, const double *sh, int c0, int nb) {
    const int m = 3 * nb;
    if (VEC) {
        double2 *d2 = reinterpret_cast<double2 *>(dst + 3 * (size_t)c0);
        for (int q = threadIdx.x; q < m / 2; q += blockDim.x) d2[q] = reinterpret_cast<const double2 *>(sh)[q];
        if ((m & 1) && threadIdx.x == 0) dst[3 * (size_t)c0 + m - 1] = sh[m - 1];
    } else {
        for (int q = threadIdx.x; q < m; q += blockDim.x) dst[3 * (size_t)c0 + q] = sh[q];
    }
}

template <bool VEC>
__global__ void __launch_bounds__(kThreads) k_sort_in_mapped(Atoms A, const double *src, double4_32a *dst) {
    __shared__ __align__(16) double sh[3 * kThreads];
    const int c0 = blockIdx.x * kThreads, nb = min(kThreads, A.n - c0);
    host_range_in<VEC>(src, sh, c0, nb);
    __syncthreads();
    if ((int)threadIdx.x >= nb) return;
    const int k = A.rank[c0 + threadIdx.x];
    double4_32a v = dst[k];
    v.x = sh[3 * threadIdx.x];
    v.y = sh[3 * threadIdx.x + 1];
    v.z = sh[3 * threadIdx.x + 2];
    dst[k] = v;
}

template <bool VEC>
__global__ void __launch_bounds__(kThreads) k_unsort_mapped(Atoms A, const double4_32a *src, double *dst) {
    __shared__ __align__(16) double sh[3 * kThreads];
    const int c0 = blockIdx.x * kThreads, nb = min(kThreads, A.n - c0);
    if ((int)threadIdx.x < nb) {
        const double4_32a v = src[A.rank[c0 + threadIdx.x]];
        sh[3 * threadIdx.x] = v.x;
        sh[3 * threadIdx.x + 1] = v.y;
        sh[3 * threadIdx.x + 2] = v.z;
    }
    __syncthreads();
    host_range_out<VEC>(dst, sh, c0, nb);
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

// Per-replica sums in a fixed order, one block per replica: PE (E_i), sum m v^2, momentum.
__global__ void k_replica_sums(Atoms A, const int32_t *off, double *out) {
    __shared__ double sh[5][256];
    const int r = blockIdx.x;
    double q[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int k = off[r] + threadIdx.x; k < off[r + 1]; k += 256) {
        const double4_32a v = A.vel[k];
        const double m = 1.0 / (kMvv2e * v.w);
        q[0] += A.e_atom[k];
        q[1] += m * fma(v.x, v.x, fma(v.y, v.y, v.z * v.z));
        q[2] += m * v.x;
        q[3] += m * v.y;
        q[4] += m * v.z;
    }
    for (int c = 0; c < 5; c++) sh[c][threadIdx.x] = q[c];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < 5; c++) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 5) out[5 * r + threadIdx.x] = sh[threadIdx.x][0];
}

}  // namespace

cudaError_t launch_replica_sums(const Atoms &A, const int32_t *off, int n_rep, double *out, cudaStream_t s) {
    k_replica_sums<<<n_rep, 256, 0, s>>>(A, off, out);
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

cudaError_t launch_unsort_image(const Atoms &A, double *dst, cudaStream_t s) {
    if (A.n == 0) return cudaSuccess;
    k_unsort_image<<<blocks_for(A.n, kThreads), kThreads, 0, s>>>(A, dst);
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

cudaError_t launch_sort_in_mapped(const Atoms &A, const double *src, double4_32a *dst, cudaStream_t s) {
    if (A.n == 0) return cudaSuccess;
    if (reinterpret_cast<uintptr_t>(src) % 16 == 0)
        k_sort_in_mapped<true><<<blocks_for(A.n, kThreads), kThreads, 0, s>>>(A, src, dst);
    else
        k_sort_in_mapped<false><<<blocks_for(A.n, kThreads), kThreads, 0, s>>>(A, src, dst);
    return cudaGetLastError();
}

cudaError_t launch_unsort_mapped(const Atoms &A, const double4_32a *src, double *dst, cudaStream_t s) {
    if (A.n == 0) return cudaSuccess;
    if (reinterpret_cast<uintptr_t>(dst) % 16 == 0)
        k_unsort_mapped<true><<<blocks_for(A.n, kThreads), kThreads, 0, s>>>(A, src, dst);
    else
        k_unsort_mapped<false><<<blocks_for(A.n, kThreads), kThreads, 0, s>>>(A, src, dst);
    return cudaGetLastError();
}

}  // namespace mdk
