// Link-cell binning and Verlet neighbour list (§3.2.1 of the MOLDY paper).
//
// Rebuild pipeline, all on the launching stream and all early-exiting when the device flag
// `need_rebuild` is clear (so a step can launch them unconditionally):
//   k_bin        wrapped fractional coordinate -> link cell; per-cell counter -> slot
//   k_scan_*     exclusive scan of the per-cell counts -> cell_start (3 phases)
//   k_scatter    order[cell_start[c] + slot] = atom
//   k_cell_sort  stable order inside a cell: ascending caller atom id (deterministic)
//   k_gather / k_copyback   renumber every per-atom array into cell order
//   k_build_list full list: the 27 cells around the atom's cell, |r_ij|^2 < r_list^2
// Link cells are fixed in fractional coordinates and at least r_list wide, so every pair
// closer than r_list lies in adjacent cells (the hybrid NL-LCM of §3.2.1).
#include <cuda_runtime.h>

#include "md_internal.cuh"

namespace mdk {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ bool rebuild_requested(const Flags *f) {
    return *reinterpret_cast<const volatile int32_t *>(&f->need_rebuild) != 0;
}

// Cell index along one edge from the wrapped fractional coordinate.
__device__ __forceinline__ int cell_coord(double x, double invL, int nc) {
    double s = x * invL;
    s = s - floor(s);
    int c = (int)(s * (double)nc);
    return min(max(c, 0), nc - 1);
}

__device__ __forceinline__ int cell_of_pos(const double4_32a &p, const Box &B, const Cells &C) {
    int cx = cell_coord(p.x, B.invL[0], C.nc[0]);
    int cy = cell_coord(p.y, B.invL[1], C.nc[1]);
    int cz = cell_coord(p.z, B.invL[2], C.nc[2]);
    return (cz * C.nc[1] + cy) * C.nc[0] + cx;
}

__device__ __forceinline__ float wrap1(double x, double L, double invL) {
    return (float)(x - L * floor(x * invL));
}

// Block-wide exclusive scan of one int per thread; returns the block total in `total`.
__device__ int block_exclusive_scan(int v, int *warp_sums, int &total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        warp_sums[lane] = s;
    }
    __syncthreads();
    int prefix = (w > 0 ? warp_sums[w - 1] : 0) + x - v;
    total = warp_sums[nw - 1];
    __syncthreads();
    return prefix;
}

__global__ void k_set_rebuild(Flags *f) { f->need_rebuild = 1; }

__global__ void k_clear_rebuild(Flags *f) {
    if (f->need_rebuild) f->n_rebuilds++;
    f->need_rebuild = 0;
}

__global__ void k_bin(Atoms A, Cells C) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n || !rebuild_requested(A.flags)) return;
    const Box B = *A.box;
    int c = cell_of_pos(A.pos[i], B, C);
    A.cell_of[i] = c;
    A.slot[i] = atomicAdd(&C.cell_count[c], 1);
}

__global__ void k_scan_tiles(Cells C, const Flags *f) {
    __shared__ int ws[32];
    if (!rebuild_requested(f)) return;
    int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++)
        if (base + k < C.ncell) s += C.cell_count[base + k];
    int total;
    block_exclusive_scan(s, ws, total);
    if (threadIdx.x == 0) C.tile_sums[blockIdx.x] = total;
}

__global__ void k_scan_top(Cells C, const Flags *f) {
    __shared__ int ws[32];
    if (!rebuild_requested(f)) return;
    if (threadIdx.x == 0) const_cast<Flags *>(f)->max_count = 0;  // k_build_list runs later
    int carry = 0;
    for (int base = 0; base < C.ntiles; base += kScanTile) {
        int idx = base + threadIdx.x * kScanItems;
        int v[kScanItems], s = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            v[k] = (idx + k < C.ntiles) ? C.tile_sums[idx + k] : 0;
            s += v[k];
        }
        int total;
        int pre = block_exclusive_scan(s, ws, total) + carry;
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            if (idx + k < C.ntiles) C.tile_sums[idx + k] = pre;
            pre += v[k];
        }
        carry += total;
    }
}

__global__ void k_scan_apply(Cells C, const Flags *f) {
    __shared__ int ws[32];
    if (!rebuild_requested(f)) return;
    int idx = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int v[kScanItems], s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        v[k] = (idx + k < C.ncell) ? C.cell_count[idx + k] : 0;
        s += v[k];
    }
    int total;
    int pre = block_exclusive_scan(s, ws, total) + C.tile_sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        if (idx + k < C.ncell) C.cell_start[idx + k] = pre;
        pre += v[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) C.cell_start[C.ncell] = pre;
}

__global__ void k_scatter(Atoms A, Cells C) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n || !rebuild_requested(A.flags)) return;
    A.order[C.cell_start[A.cell_of[i]] + A.slot[i]] = i;
}

// Inside each cell, order the atoms by caller id so that the renumbering (and with it every
// summation order) does not depend on the order of the counter increments in k_bin.
__global__ void k_cell_sort(Atoms A, Cells C) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C.ncell || !rebuild_requested(A.flags)) return;
    int s = C.cell_start[c], e = C.cell_start[c + 1];
    for (int a = s + 1; a < e; a++) {
        int v = A.order[a];
        int key = A.id[v];
        int b = a - 1;
        while (b >= s && A.id[A.order[b]] > key) {
            A.order[b + 1] = A.order[b];
            b--;
        }
        A.order[b + 1] = v;
    }
    C.cell_count[c] = 0;   // ready for the next build
}

__global__ void k_gather(Atoms A) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= A.n || !rebuild_requested(A.flags)) return;
    int o = A.order[k];
    A.pos_tmp[k] = A.pos[o];
    A.vel_tmp[k] = A.vel[o];
    A.force_tmp[k] = A.force[o];
    A.id_tmp[k] = A.id[o];
    A.spec_tmp[k] = A.spec[o];
}

__global__ void k_copyback(Atoms A) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= A.n || !rebuild_requested(A.flags)) return;
    const Box B = *A.box;
    double4_32a p = A.pos_tmp[k];
    A.pos[k] = p;
    A.ref[k] = p;
    A.vel[k] = A.vel_tmp[k];
    A.force[k] = A.force_tmp[k];
    int id = A.id_tmp[k], sp = A.spec_tmp[k];
    A.id[k] = id;
    A.spec[k] = sp;
    A.rank[id] = k;
    A.posf[k] = make_float4(wrap1(p.x, B.L[0], B.invL[0]), wrap1(p.y, B.L[1], B.invL[1]),
                            wrap1(p.z, B.L[2], B.invL[2]), __int_as_float(sp));
}

// The exact neighbour test: the same IEEE operations, in the same order and without
// contraction, as the definition d = r_j - r_i; d -= L*rint(d*(1/L)); r2 = (dx dx + dy dy) + dz dz.
__device__ __forceinline__ double mi_exact(double d, double L, double invL) {
    return __dsub_rn(d, __dmul_rn(L, rint(__dmul_rn(d, invL))));
}

__device__ __forceinline__ bool within_exact(const double4_32a &pi, const double4_32a &pj, const Box &B,
                                             double rl2) {
    double dx = mi_exact(__dsub_rn(pj.x, pi.x), B.L[0], B.invL[0]);
    double dy = mi_exact(__dsub_rn(pj.y, pi.y), B.L[1], B.invL[1]);
    double dz = mi_exact(__dsub_rn(pj.z, pi.z), B.L[2], B.invL[2]);
    double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return r2 < rl2;
}

// One thread per atom (cell order).  Candidates are screened with FP32 wrapped coordinates;
// only a candidate whose FP32 r^2 lies inside [band_lo, band_hi] (a band wider than the
// proven FP32 error, computed on the host) is decided by the exact FP64 test, so the list is
// the exact FP64 set.  Neighbours are written column-major (nbr[k*n + i]) for coalescing.
__global__ void __launch_bounds__(kThreads) k_build_list(Atoms A, Cells C, double rl2, float band_lo,
                                                         float band_hi) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool active = i < A.n && rebuild_requested(A.flags);
    int cnt = 0;
    if (active) {
        const Box B = *A.box;
        const double4_32a pi = A.pos[i];
        const float4 fi = A.posf[i];
        const int nx = C.nc[0], ny = C.nc[1], nz = C.nc[2];
        const int cx = cell_coord(pi.x, B.invL[0], nx);
        const int cy = cell_coord(pi.y, B.invL[1], ny);
        const int cz = cell_coord(pi.z, B.invL[2], nz);
        const float Lx = B.Lf[0], Ly = B.Lf[1], Lz = B.Lf[2];
        const float ix = B.invLf[0], iy = B.invLf[1], iz = B.invLf[2];
        int32_t *row = A.nbr + (size_t)i * A.k_max;
        for (int dz = -1; dz <= 1; dz++) {
            int z = cz + dz;
            z += (z < 0) ? nz : 0;
            z -= (z >= nz) ? nz : 0;
            for (int dy = -1; dy <= 1; dy++) {
                int y = cy + dy;
                y += (y < 0) ? ny : 0;
                y -= (y >= ny) ? ny : 0;
                for (int dx = -1; dx <= 1; dx++) {
                    int x = cx + dx;
                    x += (x < 0) ? nx : 0;
                    x -= (x >= nx) ? nx : 0;
                    int c = (z * ny + y) * nx + x;
                    int s = C.cell_start[c], e = C.cell_start[c + 1];
                    for (int j = s; j < e; j++) {
                        if (j == i) continue;
                        float4 fj = A.posf[j];
                        float ddx = fj.x - fi.x, ddy = fj.y - fi.y, ddz = fj.z - fi.z;
                        ddx = fmaf(-Lx, rintf(ddx * ix), ddx);
                        ddy = fmaf(-Ly, rintf(ddy * iy), ddy);
                        ddz = fmaf(-Lz, rintf(ddz * iz), ddz);
                        float r2 = fmaf(ddx, ddx, fmaf(ddy, ddy, ddz * ddz));
                        bool in = r2 < band_lo;
                        if (!in && r2 <= band_hi) in = within_exact(pi, A.pos[j], B, rl2);
                        if (in) {
                            if (cnt < A.k_max) row[cnt] = j;
                            cnt++;
                        }
                    }
                }
            }
        }
        A.count[i] = cnt;
        if (cnt > A.k_max) atomicOr(&A.flags->error, FLAG_OVERFLOW);
    }
    int m = __reduce_max_sync(0xffffffffu, cnt);
    if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(&A.flags->max_count, m);
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

cudaError_t launch_rebuild(const Atoms &A, const Cells &C, double rl2, float band_lo, float band_hi,
                           cudaStream_t s) {
    const int nb = blocks_for(A.n, kThreads);
    if (A.n > 0) k_bin<<<nb, kThreads, 0, s>>>(A, C);
    k_scan_tiles<<<C.ntiles, kScanThreads, 0, s>>>(C, A.flags);
    k_scan_top<<<1, kScanThreads, 0, s>>>(C, A.flags);
    k_scan_apply<<<C.ntiles, kScanThreads, 0, s>>>(C, A.flags);
    if (A.n > 0) {
        k_scatter<<<nb, kThreads, 0, s>>>(A, C);
        k_cell_sort<<<blocks_for(C.ncell, kThreads), kThreads, 0, s>>>(A, C);
        k_gather<<<nb, kThreads, 0, s>>>(A);
        k_copyback<<<nb, kThreads, 0, s>>>(A);
        k_build_list<<<nb, kThreads, 0, s>>>(A, C, rl2, band_lo, band_hi);
    }
    return cudaGetLastError();
}

}  // namespace mdk
