// Double-float EAM passes (MD_PREC_DF) as stand-alone kernels (md_eam_forces, md_tune; arithmetic
// in md_passes.cuh): one species, knot tables.
#include <cuda_runtime.h>

#include "md_passes.cuh"

namespace mdk {

using namespace eam;

namespace {

template <int T>
__global__ void __launch_bounds__(kThreads) k_density_df(Atoms A, Pot P) {
    clear_rebuild_once(A.flags);
    ps::density_df_item<T>(A, P, A.boxes, (long long)blockIdx.x * kThreads + threadIdx.x, true);
}

template <int T, bool ENERGY>
__global__ void __launch_bounds__(kThreads) k_force_df(Atoms A, Pot P, double half_dt, int kick) {
    double part[kPartials];
#pragma unroll
    for (int q = 0; q < kPartials; q++) part[q] = 0.0;
    ps::force_df_item<T, ENERGY>(A, P, A.boxes, (long long)blockIdx.x * kThreads + threadIdx.x, half_dt,
                                 kick ? kMotionVerlet : kMotionNone, part);
    if (ENERGY) block_partials(part, A.partials, A.part_stride);
}

template <int T>
void density_t(const Atoms &A, const Pot &P, cudaStream_t s) {
    const int nb = A.n > 0 ? blocks_for_lanes<T>(A.n) : 1;
    k_density_df<T><<<nb, kThreads, 0, s>>>(A, P);
}

template <int T>
void force_t(const Atoms &A, const Pot &P, bool kick, bool energy, double half_dt, cudaStream_t s) {
    const int nb = A.n > 0 ? blocks_for_lanes<T>(A.n) : 1;
    if (energy) k_force_df<T, true><<<nb, kThreads, 0, s>>>(A, P, half_dt, kick);
    else k_force_df<T, false><<<nb, kThreads, 0, s>>>(A, P, half_dt, kick);
}

}  // namespace

cudaError_t launch_density_df(const Atoms &A, const Pot &P, int lanes, cudaStream_t s) {
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

cudaError_t launch_force_df(const Atoms &A, const Pot &P, int lanes, bool kick, bool energy, double half_dt,
                            cudaStream_t s) {
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

}  // namespace mdk
