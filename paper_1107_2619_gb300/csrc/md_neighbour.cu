// Link-cell binning and Verlet neighbour list (§3.2.1 of the MOLDY paper), as stand-alone
// kernels (used by md_build_neighbours and md_eam_forces; the step kernel runs the same
// per-item functions inside one persistent launch).
//
// Rebuild pipeline, all on the launching stream and all returning at once when the device
// flag `need_rebuild` is clear.  The per-atom and per-cell kernels loop over their items with a
// grid of at most 8 blocks per SM, so that a launch with nothing to do costs a few µs:
//   k_bin        wrapped fractional coordinate -> link cell; per-cell counter -> slot
//   k_scan_*     exclusive scan of the per-cell counts -> cell_start (3 phases)
//   k_scatter    order[cell_start[c] + slot] = atom; the stencil slot tables of the cell groups
//                (group walks)
//   k_cell_sort  stable order inside a cell: ascending caller atom id (deterministic)
//   k_gather / k_copyback   renumber every per-atom array into cell order
//   k_build_list full list: the 27 cells around each cell, |r_ij|^2 < r_list^2, a group of
//                lanes per cell (for the staged and half walks also as 16-bit stencil slots)
// Link cells are fixed in fractional coordinates and at least r_list wide, so every pair
// closer than r_list lies in adjacent cells (the hybrid NL-LCM of §3.2.1).
#include <cuda_runtime.h>

#include <algorithm>

#include "md_phases.cuh"

namespace mdk {

namespace {

constexpr int kScanThreads = 1024;

__global__ void k_set_rebuild(Flags *f) { f->need_rebuild = 1; }

__global__ void k_clear_rebuild(Flags *f) {
    if (f->need_rebuild) f->n_rebuilds++;
    f->need_rebuild = 0;
}

__device__ __forceinline__ long long gtid() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ long long gstride() { return (long long)gridDim.x * blockDim.x; }

__global__ void k_bin(Atoms A, Cells C) {
    if (!ph::rebuild_requested(A.flags)) return;
    for (long long i = gtid(); i < A.n; i += gstride()) ph::bin_atom(A, C, A.boxes, (int)i);
}

__global__ void k_scan_tiles(Cells C, const Flags *f) {
    __shared__ int ws[32];
    if (!ph::rebuild_requested(f)) return;
    ph::scan_tile_sum(C, blockIdx.x, ws);
}

__global__ void k_scan_top(Cells C, Flags *f) {
    __shared__ int ws[32];
    if (!ph::rebuild_requested(f)) return;
    if (threadIdx.x == 0) {  // k_scatter and k_build_list run later
        f->max_count = 0;
        f->tile_bad = 0;
        f->tile_max = 0;
    }
    ph::scan_top(C, ws);
}

__global__ void k_scan_apply(Cells C, const Flags *f) {
    __shared__ int ws[32];
    if (!ph::rebuild_requested(f)) return;
    ph::scan_apply(C, blockIdx.x, ws);
}

__global__ void k_scatter(Atoms A, Cells C) {
    if (!ph::rebuild_requested(A.flags)) return;
    for (long long i = gtid(); i < A.n; i += gstride()) ph::scatter_atom(A, C, (int)i);
    if (C.tile)
        for (long long g = gtid(); g < C.n_groups; g += gstride()) ph::group_table(C, (int)g, A.flags);
}

__global__ void k_cell_sort(Atoms A, Cells C) {
    if (!ph::rebuild_requested(A.flags)) return;
    const long long warps = gstride() >> 5;
    for (long long c = gtid() >> 5; c < C.ncell; c += warps)   // one warp per cell
        ph::sort_cell_warp(A, C, (int)c, threadIdx.x & 31);
}

__global__ void k_gather(Atoms A) {
    if (!ph::rebuild_requested(A.flags)) return;
    for (long long k = gtid(); k < A.n; k += gstride()) ph::gather_atom(A, (int)k);
}

__global__ void k_copyback(Atoms A) {
    if (!ph::rebuild_requested(A.flags)) return;
    for (long long k = gtid(); k < A.n; k += gstride()) ph::copyback_atom(A, A.boxes, (int)k);
}

template <int G, int LOCAL>
__global__ void __launch_bounds__(kThreads, 8) k_build_list(Atoms A, Cells C, double rl2, float band_lo,
                                                         float band_hi) {
    if (!ph::rebuild_requested(A.flags)) return;
    int m = ph::build_cells<G, LOCAL>(A, C, A.boxes, gtid() >> 5, gstride() >> 5, threadIdx.x & 31, rl2, band_lo, band_hi);
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(&A.flags->max_count, m);
}

template <int LOCAL>
void launch_build(const Atoms &A, const Cells &C, double rl2, float band_lo, float band_hi, int list_group, int nbl,
                  cudaStream_t s) {
    if (list_group == 4) k_build_list<4, LOCAL><<<nbl, kThreads, 0, s>>>(A, C, rl2, band_lo, band_hi);
    else if (list_group == 8) k_build_list<8, LOCAL><<<nbl, kThreads, 0, s>>>(A, C, rl2, band_lo, band_hi);
    else if (list_group == 16) k_build_list<16, LOCAL><<<nbl, kThreads, 0, s>>>(A, C, rl2, band_lo, band_hi);
    else k_build_list<32, LOCAL><<<nbl, kThreads, 0, s>>>(A, C, rl2, band_lo, band_hi);
}

int capped_blocks(long long items, int threads) {
    static int n_sm = 0;
    if (!n_sm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (n_sm <= 0) n_sm = 1;
    }
    return (int)std::max(1LL, std::min(blocks_for(items, threads) * 1LL, 8LL * n_sm));
}

}  // namespace

cudaError_t launch_set_rebuild(Flags *f, cudaStream_t s) {
    k_set_rebuild<<<1, 1, 0, s>>>(f);
    return cudaGetLastError();
}

cudaError_t launch_clear_rebuild(Flags *f, cudaStream_t s) {
    k_clear_rebuild<<<1, 1, 0, s>>>(f);
    return cudaGetLastError();
}

// FP64 pair walk: each row's entries j > i first (one warp per atom).
__global__ void k_partition_rows(Atoms A) {
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w < A.n) ph::partition_row_warp(A, A.boxes, (int)w, threadIdx.x & 31);
}

cudaError_t launch_rebuild(const Atoms &A, const Cells &C, double rl2, float band_lo, float band_hi,
                           int list_group, cudaStream_t s) {
    const int nb = capped_blocks(A.n, kThreads);
    const int ntiles = (C.ncell + kScanThreads * ph::kScanItems - 1) / (kScanThreads * ph::kScanItems);
    if (A.n > 0) k_bin<<<nb, kThreads, 0, s>>>(A, C);
    k_scan_tiles<<<ntiles, kScanThreads, 0, s>>>(C, A.flags);
    k_scan_top<<<1, kScanThreads, 0, s>>>(C, A.flags);
    k_scan_apply<<<ntiles, kScanThreads, 0, s>>>(C, A.flags);
    if (A.n > 0) {
        k_scatter<<<nb, kThreads, 0, s>>>(A, C);
        k_cell_sort<<<capped_blocks((long long)C.ncell * 32, kThreads), kThreads, 0, s>>>(A, C);
        k_gather<<<nb, kThreads, 0, s>>>(A);
        k_copyback<<<nb, kThreads, 0, s>>>(A);
        const int nbl = capped_blocks((long long)C.ncell * list_group, kThreads);
        if (C.tile == kWalkStaged) launch_build<1>(A, C, rl2, band_lo, band_hi, list_group, nbl, s);
        else if (C.tile == kWalkHalf) launch_build<2>(A, C, rl2, band_lo, band_hi, list_group, nbl, s);
        else launch_build<0>(A, C, rl2, band_lo, band_hi, list_group, nbl, s);
        if (A.pairs) k_partition_rows<<<(int)(((long long)A.n * 32 + kThreads - 1) / kThreads), kThreads, 0, s>>>(A);
    }
    return cudaGetLastError();
}

}  // namespace mdk
