// FP64 EAM passes as stand-alone kernels (md_eam_forces, md_tune; arithmetic in
// md_passes.cuh), the deterministic energy reduction, and the precision dispatch.
#include <cuda_runtime.h>

#include "md_passes.cuh"

namespace mdk {

using namespace eam;

cudaError_t launch_density32(const Atoms &A, const Pot &P, int lanes, cudaStream_t s);
cudaError_t launch_density_df(const Atoms &A, const Pot &P, int lanes, cudaStream_t s);
cudaError_t launch_force_df(const Atoms &A, const Pot &P, int lanes, bool kick, bool energy, double half_dt,
                            cudaStream_t s);
cudaError_t launch_force32(const Atoms &A, const Pot &P, int lanes, bool kick, bool energy, double half_dt,
                           cudaStream_t s);

namespace {

template <int T, int KIND, bool MULTI>
__global__ void __launch_bounds__(kThreads) k_density64(Atoms A, Pot P) {
    clear_rebuild_once(A.flags);
    ps::density64_item<T, KIND, MULTI>(A, P, A.boxes, (long long)blockIdx.x * kThreads + threadIdx.x, true);
}

template <int T, int KIND, bool MULTI, bool ENERGY>
__global__ void __launch_bounds__(kThreads) k_force64(Atoms A, Pot P, double half_dt, int kick) {
    double part[kPartials];
#pragma unroll
    for (int q = 0; q < kPartials; q++) part[q] = 0.0;
    ps::force64_item<T, KIND, MULTI, ENERGY>(A, P, A.boxes, (long long)blockIdx.x * kThreads + threadIdx.x,
                                             half_dt, kick != 0, part);
    if (ENERGY) block_partials(part, A.partials, A.part_stride);
}

// The pair walk (A.pairs): each pair once, then the per-atom phase that needs every share.
template <int T, int KIND>
__global__ void __launch_bounds__(kThreads) k_density64_pairs(Atoms A, Pot P) {
    __shared__ double sums[T >= ps::kFlatLanes ? kThreads / 32 * ps::kPairSlots(32 / T) : 1];
    clear_rebuild_once(A.flags);
    ps::density64_pairs<T, KIND>(A, P, A.boxes, (long long)blockIdx.x * kThreads + threadIdx.x, true,
                                 sums + (T >= ps::kFlatLanes ? (threadIdx.x >> 5) * ps::kPairSlots(32 / T) : 0));
}

__global__ void __launch_bounds__(kThreads) k_embed64_pairs(Atoms A, Pot P) {
    const int i = blockIdx.x * kThreads + threadIdx.x;
    if (i < A.n) ps::pairs_embed64(A, P, i);
}

template <int T, int KIND, bool ENERGY>
__global__ void __launch_bounds__(kThreads) k_force64_pairs(Atoms A, Pot P) {
    double part[kPartials];
#pragma unroll
    for (int q = 0; q < kPartials; q++) part[q] = 0.0;
    __shared__ double sums[T >= ps::kFlatLanes ? kThreads / 32 * ps::kPairSlots(32 / T) : 1];
    ps::force64_pairs<T, KIND, ENERGY>(A, P, A.boxes, (long long)blockIdx.x * kThreads + threadIdx.x, part,
                                       sums + (T >= ps::kFlatLanes ? (threadIdx.x >> 5) * ps::kPairSlots(32 / T) : 0));
    if (ENERGY) block_partials(part, A.partials, A.part_stride);
}

// The per-atom phase after the pair force pass; its partial sums go to the block rows after the
// force pass's (virial) rows, and the reduction adds both sets.
template <bool ENERGY>
__global__ void __launch_bounds__(kThreads) k_finish64_pairs(Atoms A, double half_dt, int kick, int row0) {
    double part[kPartials];
#pragma unroll
    for (int q = 0; q < kPartials; q++) part[q] = 0.0;
    const int i = blockIdx.x * kThreads + threadIdx.x;
    if (i < A.n) ps::pairs_kick64<ENERGY>(A, i, half_dt, kick ? kMotionVerlet : kMotionNone, part);
    if (ENERGY) {
        Atoms B = A;
        B.partials = A.partials + row0;
        block_partials(part, B.partials, A.part_stride);
    }
}

// Deterministic final reduction of the per-block partials: one block per quantity, a fixed
// thread-to-row mapping (coalesced rows partials[q*stride + b]) and a fixed tree, so repeated
// runs give bitwise identical totals.
__global__ void k_reduce(const double *__restrict__ partials, int nblocks, int stride, double *out) {
    __shared__ double sh[512];
    const int q = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += 512) s += partials[(size_t)q * stride + b];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 256; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = sh[0];
}

template <int T>
void density_t(const Atoms &A, const Pot &P, cudaStream_t s) {
    const int nb = A.n > 0 ? blocks_for_lanes<T>(A.n) : 1;
    if (A.pairs) {
        if (P.kind == MD_POT_FS_ANALYTIC) k_density64_pairs<T, MD_POT_FS_ANALYTIC><<<nb, kThreads, 0, s>>>(A, P);
        else k_density64_pairs<T, MD_POT_TABLES><<<nb, kThreads, 0, s>>>(A, P);
        k_embed64_pairs<<<blocks_for(A.n > 0 ? A.n : 1, kThreads), kThreads, 0, s>>>(A, P);
        return;
    }
    if (P.kind == MD_POT_FS_ANALYTIC) k_density64<T, MD_POT_FS_ANALYTIC, false><<<nb, kThreads, 0, s>>>(A, P);
    else if (P.kind == MD_POT_KNOTS && P.ns == 1) k_density64<T, MD_POT_KNOTS, false><<<nb, kThreads, 0, s>>>(A, P);
    else if (P.kind == MD_POT_KNOTS) k_density64<T, MD_POT_KNOTS, true><<<nb, kThreads, 0, s>>>(A, P);
    else if (P.ns == 1) k_density64<T, MD_POT_TABLES, false><<<nb, kThreads, 0, s>>>(A, P);
    else k_density64<T, MD_POT_TABLES, true><<<nb, kThreads, 0, s>>>(A, P);
}

template <int T, bool ENERGY>
void force_te(const Atoms &A, const Pot &P, double half_dt, int kick, cudaStream_t s) {
    const int nb = blocks_for_lanes<T>(A.n);
    if (A.pairs) {   // the pair force pass, then the per-atom phase (partial rows after the pass's)
        if (P.kind == MD_POT_FS_ANALYTIC) k_force64_pairs<T, MD_POT_FS_ANALYTIC, ENERGY><<<nb, kThreads, 0, s>>>(A, P);
        else k_force64_pairs<T, MD_POT_TABLES, ENERGY><<<nb, kThreads, 0, s>>>(A, P);
        k_finish64_pairs<ENERGY><<<blocks_for(A.n > 0 ? A.n : 1, kThreads), kThreads, 0, s>>>(A, half_dt, kick, nb);
        return;
    }
    if (P.kind == MD_POT_FS_ANALYTIC)
        k_force64<T, MD_POT_FS_ANALYTIC, false, ENERGY><<<nb, kThreads, 0, s>>>(A, P, half_dt, kick);
    else if (P.kind == MD_POT_KNOTS && P.ns == 1)
        k_force64<T, MD_POT_KNOTS, false, ENERGY><<<nb, kThreads, 0, s>>>(A, P, half_dt, kick);
    else if (P.kind == MD_POT_KNOTS)
        k_force64<T, MD_POT_KNOTS, true, ENERGY><<<nb, kThreads, 0, s>>>(A, P, half_dt, kick);
    else if (P.ns == 1)
        k_force64<T, MD_POT_TABLES, false, ENERGY><<<nb, kThreads, 0, s>>>(A, P, half_dt, kick);
    else
        k_force64<T, MD_POT_TABLES, true, ENERGY><<<nb, kThreads, 0, s>>>(A, P, half_dt, kick);
}

template <int T>
void force_t(const Atoms &A, const Pot &P, bool kick, bool energy, double half_dt, cudaStream_t s) {
    if (energy) force_te<T, true>(A, P, half_dt, kick, s);
    else force_te<T, false>(A, P, half_dt, kick, s);
}

cudaError_t density64(const Atoms &A, const Pot &P, int lanes, cudaStream_t s) {
    switch (lanes) {
        case 1: density_t<1>(A, P, s); break;
        case 2: density_t<2>(A, P, s); break;
        case 4: density_t<4>(A, P, s); break;
        case 8: density_t<8>(A, P, s); break;
        case 16: density_t<16>(A, P, s); break;
        case 32: density_t<32>(A, P, s); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t force64(const Atoms &A, const Pot &P, int lanes, bool kick, bool energy, double half_dt,
                    cudaStream_t s) {
    if (A.n == 0) return cudaSuccess;
    switch (lanes) {
        case 1: force_t<1>(A, P, kick, energy, half_dt, s); break;
        case 2: force_t<2>(A, P, kick, energy, half_dt, s); break;
        case 4: force_t<4>(A, P, kick, energy, half_dt, s); break;
        case 8: force_t<8>(A, P, kick, energy, half_dt, s); break;
        case 16: force_t<16>(A, P, kick, energy, half_dt, s); break;
        case 32: force_t<32>(A, P, kick, energy, half_dt, s); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

int partial_blocks(int n, int lanes) {
    return n > 0 ? (int)(((long long)n * lanes + kThreads - 1) / kThreads) : 0;
}

cudaError_t launch_density(const Atoms &A, const Pot &P, int precision, int lanes, cudaStream_t s) {
    if (precision == MD_PREC_DF) return launch_density_df(A, P, lanes, s);
    return precision == MD_PREC_FP64 ? density64(A, P, lanes, s) : launch_density32(A, P, lanes, s);
}

cudaError_t launch_force(const Atoms &A, const Pot &P, int precision, int lanes, bool kick, bool energy,
                         double half_dt, cudaStream_t s) {
    if (precision == MD_PREC_DF) return launch_force_df(A, P, lanes, kick, energy, half_dt, s);
    return precision == MD_PREC_FP64 ? force64(A, P, lanes, kick, energy, half_dt, s)
                                     : launch_force32(A, P, lanes, kick, energy, half_dt, s);
}

cudaError_t launch_reduce(const Atoms &A, int nblocks, double *out, cudaStream_t s) {
    k_reduce<<<kPartials, 512, 0, s>>>(A.partials, nblocks, A.part_stride, out);
    return cudaGetLastError();
}

}  // namespace mdk
