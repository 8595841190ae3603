// Per-item device functions of the hot path, shared by the stand-alone kernels and the
// persistent step kernel.  Each function does the work of one item (an atom, a cell or a
// scan tile); the callers supply the loop.
//
// Systems: one or several independent replicas (batched systems).  Atoms of replica r
// occupy a contiguous range of the per-atom arrays; rep[i] (NULL for a single system) gives
// the replica of slot i, boxes[r] its box, rc[r] its link-cell grid, whose cells occupy the
// global cell range [rc[r].base, rc[r].base + ncell_r).
#pragma once

#include <cuda_runtime.h>

#include "md_internal.cuh"

namespace mdk {
namespace ph {

__device__ __forceinline__ bool rebuild_requested(const Flags *f) {
    return *reinterpret_cast<const volatile int32_t *>(&f->need_rebuild) != 0;
}

__device__ __forceinline__ int replica_of(const Atoms &A, int i) { return A.rep ? A.rep[i] : 0; }

// Cell index along one edge from the wrapped fractional coordinate.
__device__ __forceinline__ int cell_coord(double x, double invL, int nc) {
    double s = x * invL;
    s = s - floor(s);
    int c = (int)(s * (double)nc);
    return min(max(c, 0), nc - 1);
}

__device__ __forceinline__ float wrap1(double x, double L, double invL) {
    return (float)(x - L * floor(x * invL));
}

__device__ __forceinline__ float4 wrapped(const double4_32a &p, const Box &B, int species) {
    return make_float4(wrap1(p.x, B.L[0], B.invL[0]), wrap1(p.y, B.L[1], B.invL[1]),
                       wrap1(p.z, B.L[2], B.invL[2]), __int_as_float(species));
}

__device__ __forceinline__ int global_cell(const double4_32a &p, const Box &B, const RepCells &g) {
    const int cx = cell_coord(p.x, B.invL[0], g.nc[0]);
    const int cy = cell_coord(p.y, B.invL[1], g.nc[1]);
    const int cz = cell_coord(p.z, B.invL[2], g.nc[2]);
    return g.base + (cz * g.nc[1] + cy) * g.nc[0] + cx;
}

// Block-wide exclusive scan of one int per thread; returns the block total in `total`.
__device__ __forceinline__ int block_exclusive_scan(int v, int *warp_sums, int &total) {
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

// ---------------------------------------------------------------- integration (§2.3, §2.2)
// v += (dt/2) F/m;  r += dt v;  [z *= s];  skin check against the positions of the last build.
// Separately rounded FP64 operations, as in the definition.
__device__ __forceinline__ void kick_drift(const Atoms &A, const Box *boxes, int i, double half_dt, double dt,
                                           double s, bool strain, double lim2) {
    double4_32a v = A.vel[i];
    const double4_32a f = A.force[i];
    double4_32a p = A.pos[i];
    v.x = __dadd_rn(v.x, __dmul_rn(__dmul_rn(half_dt, f.x), v.w));
    v.y = __dadd_rn(v.y, __dmul_rn(__dmul_rn(half_dt, f.y), v.w));
    v.z = __dadd_rn(v.z, __dmul_rn(__dmul_rn(half_dt, f.z), v.w));
    p.x = __dadd_rn(p.x, __dmul_rn(dt, v.x));
    p.y = __dadd_rn(p.y, __dmul_rn(dt, v.y));
    p.z = __dadd_rn(p.z, __dmul_rn(dt, v.z));
    if (strain) p.z = __dmul_rn(p.z, s);
    A.vel[i] = v;
    A.pos[i] = p;
    const double4_32a r = A.ref[i];
    const double ex = __dsub_rn(p.x, r.x), ey = __dsub_rn(p.y, r.y), ez = __dsub_rn(p.z, r.z);
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
    if (d2 > lim2 || !(d2 == d2)) {
        A.flags->need_rebuild = 1;
        A.flags->skin_exceeded = 1;
    }
    A.posf[i] = wrapped(p, boxes[replica_of(A, i)], A.spec[i]);
}

__device__ __forceinline__ void check_displacement(const Atoms &A, int i, double lim2) {
    const double4_32a p = A.pos[i], r = A.ref[i];
    const double ex = __dsub_rn(p.x, r.x), ey = __dsub_rn(p.y, r.y), ez = __dsub_rn(p.z, r.z);
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
    if (d2 > lim2 || !(d2 == d2)) {
        A.flags->need_rebuild = 1;
        A.flags->skin_exceeded = 1;
    }
}

// ---------------------------------------------------------------- rebuild (§3.2.1, §3.2.2)
__device__ __forceinline__ void bin_atom(const Atoms &A, const Cells &C, const Box *boxes, int i) {
    const int r = replica_of(A, i);
    const int c = global_cell(A.pos[i], boxes[r], C.rc[r]);
    A.cell_of[i] = c;
    A.slot[i] = atomicAdd(&C.cell_count[c], 1);
}

// The scan works on tiles of blockDim.x * kScanItems cells.
constexpr int kScanItems = 4;

__device__ __forceinline__ int scan_tiles(const Cells &C) {
    const int tile = blockDim.x * kScanItems;
    return (C.ncell + tile - 1) / tile;
}

// Scan phase 1: tile sums.
__device__ __forceinline__ void scan_tile_sum(const Cells &C, int tile, int *ws) {
    const int base = tile * blockDim.x * kScanItems + threadIdx.x * kScanItems;
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++)
        if (base + k < C.ncell) s += C.cell_count[base + k];
    int total;
    block_exclusive_scan(s, ws, total);
    if (threadIdx.x == 0) C.tile_sums[tile] = total;
}

// Scan phase 2 (one block): exclusive scan of the tile sums in place.
__device__ __forceinline__ void scan_top(const Cells &C, int *ws) {
    const int ntiles = scan_tiles(C);
    int carry = 0;
    for (int base = 0; base < ntiles; base += blockDim.x * kScanItems) {
        const int idx = base + threadIdx.x * kScanItems;
        int v[kScanItems], s = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            v[k] = (idx + k < ntiles) ? C.tile_sums[idx + k] : 0;
            s += v[k];
        }
        int total;
        int pre = block_exclusive_scan(s, ws, total) + carry;
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            if (idx + k < ntiles) C.tile_sums[idx + k] = pre;
            pre += v[k];
        }
        carry += total;
    }
}

// Scan phase 3: cell_start of each cell of the tile (cell_start[ncell] = total by the last tile).
__device__ __forceinline__ void scan_apply(const Cells &C, int tile, int *ws) {
    const int idx = tile * blockDim.x * kScanItems + threadIdx.x * kScanItems;
    int v[kScanItems], s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        v[k] = (idx + k < C.ncell) ? C.cell_count[idx + k] : 0;
        s += v[k];
    }
    int total;
    int pre = block_exclusive_scan(s, ws, total) + C.tile_sums[tile];
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        if (idx + k < C.ncell) C.cell_start[idx + k] = pre;
        pre += v[k];
    }
    if (tile == scan_tiles(C) - 1 && threadIdx.x == blockDim.x - 1) C.cell_start[C.ncell] = pre;
}

__device__ __forceinline__ void scatter_atom(const Atoms &A, const Cells &C, int i) {
    A.order[C.cell_start[A.cell_of[i]] + A.slot[i]] = i;
}

// Inside each cell, order the atoms by caller id (deterministic renumbering), one warp per
// cell: the element with key rank q (the number of smaller keys in the cell) goes to slot
// s + q.  Keys are unique, so the ranks are a permutation.  The sorted slots are written to
// A.sorted (A.order is read while ranking); the cell count is reset for the next build.
__device__ __forceinline__ void sort_cell_warp(const Atoms &A, const Cells &C, int c, int lane) {
    const int s = C.cell_start[c], e = C.cell_start[c + 1];
    for (int a = s + lane; a < e; a += 32) {
        const int v = A.order[a];
        const int key = A.id[v];
        int rank = 0;
        for (int b = s; b < e; b++) rank += A.id[A.order[b]] < key ? 1 : 0;
        A.sorted[s + rank] = v;
    }
    if (lane == 0) C.cell_count[c] = 0;
}

__device__ __forceinline__ void gather_atom(const Atoms &A, int k) {
    const int o = A.sorted[k];
    A.pos_tmp[k] = A.pos[o];
    A.vel_tmp[k] = A.vel[o];
    A.force_tmp[k] = A.force[o];
    A.id_tmp[k] = A.id[o];
    A.spec_tmp[k] = A.spec[o];
}

__device__ __forceinline__ void copyback_atom(const Atoms &A, const Box *boxes, int k) {
    const double4_32a p = A.pos_tmp[k];
    A.pos[k] = p;
    A.ref[k] = p;
    A.vel[k] = A.vel_tmp[k];
    A.force[k] = A.force_tmp[k];
    const int id = A.id_tmp[k], sp = A.spec_tmp[k];
    A.id[k] = id;
    A.spec[k] = sp;
    A.rank[id] = k;
    A.posf[k] = wrapped(p, boxes[replica_of(A, k)], sp);
}

// The exact neighbour test: the IEEE operations, order and absence of contraction of the
// definition d = r_j - r_i; d -= L*rint(d*(1/L)); r2 = (dx dx + dy dy) + dz dz.
__device__ __forceinline__ double mi_exact(double d, double L, double invL) {
    return __dsub_rn(d, __dmul_rn(L, rint(__dmul_rn(d, invL))));
}

__device__ __forceinline__ bool within_exact(const double4_32a &pi, const double4_32a &pj, const Box &B,
                                             double rl2) {
    const double dx = mi_exact(__dsub_rn(pj.x, pi.x), B.L[0], B.invL[0]);
    const double dy = mi_exact(__dsub_rn(pj.y, pi.y), B.L[1], B.invL[1]);
    const double dz = mi_exact(__dsub_rn(pj.z, pi.z), B.L[2], B.invL[2]);
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return r2 < rl2;
}

// Full list row of atom i (cell order) from the 27 cells around its cell, one thread per
// atom: the threads of a warp, whose atoms share a link cell, read the same candidate at the
// same time (one broadcast load each).  Candidates are screened with FP32 wrapped
// coordinates, shifted by whole box edges for neighbour cells across the periodic boundary
// (no rounding to the nearest image per candidate); a neighbour cell whose nearest face is
// beyond r_list (plus the band) is skipped.  Only a candidate whose FP32 r^2 lies in
// [band_lo, band_hi] (a band wider than the proven FP32 error) is decided by the exact FP64
// test, so the row is the exact FP64 set, listed by cell in (dz, dy, dx) order and by
// ascending slot inside a cell.  Returns the neighbour count (rows are cut at k_max).
__device__ __forceinline__ int build_row(const Atoms &A, const Cells &C, const Box *boxes, int i, double rl2,
                                         float band_lo, float band_hi) {
    const int r = replica_of(A, i);
    const Box &B = boxes[r];
    const RepCells g = C.rc[r];
    const double4_32a pi = A.pos[i];
    const float4 fi = A.posf[i];
    const int nx = g.nc[0], ny = g.nc[1], nz = g.nc[2];
    const int cx = cell_coord(pi.x, B.invL[0], nx);
    const int cy = cell_coord(pi.y, B.invL[1], ny);
    const int cz = cell_coord(pi.z, B.invL[2], nz);
    const float Lx = B.Lf[0], Ly = B.Lf[1], Lz = B.Lf[2];
    const float ex = Lx / nx, ey = Ly / ny, ez = Lz / nz;     // cell edges
    // distance from the atom to the lower / upper face of its own cell, per axis
    const float lox = fmaxf(fi.x - cx * ex, 0.f), hix = fmaxf((cx + 1) * ex - fi.x, 0.f);
    const float loy = fmaxf(fi.y - cy * ey, 0.f), hiy = fmaxf((cy + 1) * ey - fi.y, 0.f);
    const float loz = fmaxf(fi.z - cz * ez, 0.f), hiz = fmaxf((cz + 1) * ez - fi.z, 0.f);
    int32_t *row = A.nbr + (size_t)i * A.k_max;
    int cnt = 0;
    for (int dz = -1; dz <= 1; dz++) {
        int z = cz + dz;
        float sz = 0.f;
        if (z < 0) { z += nz; sz = -Lz; }
        if (z >= nz) { z -= nz; sz = Lz; }
        const float mz = dz < 0 ? loz : (dz > 0 ? hiz : 0.f);
        for (int dy = -1; dy <= 1; dy++) {
            int y = cy + dy;
            float sy = 0.f;
            if (y < 0) { y += ny; sy = -Ly; }
            if (y >= ny) { y -= ny; sy = Ly; }
            const float my = dy < 0 ? loy : (dy > 0 ? hiy : 0.f);
            for (int dx = -1; dx <= 1; dx++) {
                int x = cx + dx;
                float sx = 0.f;
                if (x < 0) { x += nx; sx = -Lx; }
                if (x >= nx) { x -= nx; sx = Lx; }
                const float mx = dx < 0 ? lox : (dx > 0 ? hix : 0.f);
                if (fmaf(mx, mx, fmaf(my, my, mz * mz)) > band_hi) continue;  // cell out of range
                const int c = g.base + (z * ny + y) * nx + x;
                const int s = C.cell_start[c], e = C.cell_start[c + 1];
                const float ox = sx - fi.x, oy = sy - fi.y, oz = sz - fi.z;
                for (int j = s; j < e; j++) {
                    if (j == i) continue;
                    const float4 fj = A.posf[j];
                    const float ddx = fj.x + ox, ddy = fj.y + oy, ddz = fj.z + oz;
                    const float r2 = fmaf(ddx, ddx, fmaf(ddy, ddy, ddz * ddz));
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
    return cnt;
}

}  // namespace ph
}  // namespace mdk
