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

// FP64 positions wrapped into the box, and in the image of the last build (as below).
__device__ __forceinline__ double4_32a wrapped64(const double4_32a &p, const Box &B) {
    return make_double4_32a(p.x - B.L[0] * floor(p.x * B.invL[0]), p.y - B.L[1] * floor(p.y * B.invL[1]),
                            p.z - B.L[2] * floor(p.z * B.invL[2]), p.w);
}
__device__ __forceinline__ double4_32a build_image64(const double4_32a &p, const double4_32a &ref, const Box &B) {
    return make_double4_32a(p.x - B.L[0] * floor(ref.x * B.invL[0]), p.y - B.L[1] * floor(ref.y * B.invL[1]),
                            p.z - B.L[2] * floor(ref.z * B.invL[2]), p.w);
}

// FP32 position in the periodic image its atom was wrapped into at the last list build (the
// image of ref, the position at that build): the wrapped position until the atom crosses a box
// face, continuous after it, so that it stays within skin/2 of its link cell (the group walks
// add each cell's image shift to these coordinates; the list passes take the minimum image).
__device__ __forceinline__ float4 build_image(const double4_32a &p, const double4_32a &ref, const Box &B,
                                              int species) {
    return make_float4((float)(p.x - B.L[0] * floor(ref.x * B.invL[0])),
                       (float)(p.y - B.L[1] * floor(ref.y * B.invL[1])),
                       (float)(p.z - B.L[2] * floor(ref.z * B.invL[2])), __int_as_float(species));
}

// Double-float copy of an FP64 image coordinate q (MD_PREC_DF): q + xoff split into an FP32 high
// part and the FP32 rounding of the remainder.
__device__ __forceinline__ void store_dfpos(const Atoms &A, int i, const double4_32a &q, const Box &B) {
    const double x = q.x + B.xoff[0], y = q.y + B.xoff[1], z = q.z + B.xoff[2];
    const float xh = (float)x, yh = (float)y, zh = (float)z;
    A.posx[2 * (size_t)i] = make_float4(xh, yh, zh, 0.f);
    A.posx[2 * (size_t)i + 1] = make_float4((float)(x - (double)xh), (float)(y - (double)yh), (float)(z - (double)zh), 0.f);
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
                                           double s, bool strain, double lim2, const Thermo *th = nullptr) {
    double4_32a v = A.vel[i];
    if (th) {  // the thermostat half steps before this kick: v *= s_b, then v *= s_a
        const Thermo &t = th[replica_of(A, i)];
        v.x = __dmul_rn(__dmul_rn(v.x, t.s_b), t.s_a);
        v.y = __dmul_rn(__dmul_rn(v.y, t.s_b), t.s_a);
        v.z = __dmul_rn(__dmul_rn(v.z, t.s_b), t.s_a);
    }
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
    A.posf[i] = build_image(p, r, boxes[replica_of(A, i)], A.spec[i]);
    if (A.posd) {
        const Box &B = boxes[replica_of(A, i)];
        const double4_32a q = build_image64(p, r, B);
        A.posd[i] = q;
        if (A.posx) store_dfpos(A, i, q, B);
    }
}

// The predictor of the third-order predictor-corrector (md.h MD_INTEGRATOR_PC3): from the force f
// of the last evaluation (acceleration term q2 = (dt^2/2) f/m) and the third-derivative term q3,
//   r += dt v + q2 + q3,  v += (2 q2 + 3 q3) / dt,  g2 = q2 + 3 q3 (the predicted acceleration
// term, for the corrector), then the skin check and the pass copies, as after a drift.
__device__ __forceinline__ void predict_pc3(const Atoms &A, const Box *boxes, int i, double dt, double lim2) {
    double4_32a v = A.vel[i], p = A.pos[i];
    const double4_32a f = A.force[i], q3 = A.g3[i];
    const double h2 = 0.5 * dt * dt;
    const double ax = __dmul_rn(__dmul_rn(h2, f.x), v.w), ay = __dmul_rn(__dmul_rn(h2, f.y), v.w),
                 az = __dmul_rn(__dmul_rn(h2, f.z), v.w);
    p.x = __dadd_rn(p.x, __dadd_rn(__dadd_rn(__dmul_rn(dt, v.x), ax), q3.x));
    p.y = __dadd_rn(p.y, __dadd_rn(__dadd_rn(__dmul_rn(dt, v.y), ay), q3.y));
    p.z = __dadd_rn(p.z, __dadd_rn(__dadd_rn(__dmul_rn(dt, v.z), az), q3.z));
    const double bx = __dmul_rn(3.0, q3.x), by = __dmul_rn(3.0, q3.y), bz = __dmul_rn(3.0, q3.z);
    v.x = __dadd_rn(v.x, __ddiv_rn(__dadd_rn(__dmul_rn(2.0, ax), bx), dt));
    v.y = __dadd_rn(v.y, __ddiv_rn(__dadd_rn(__dmul_rn(2.0, ay), by), dt));
    v.z = __dadd_rn(v.z, __ddiv_rn(__dadd_rn(__dmul_rn(2.0, az), bz), dt));
    A.g2[i] = make_double4_32a(__dadd_rn(ax, bx), __dadd_rn(ay, by), __dadd_rn(az, bz), 0.0);
    A.vel[i] = v;
    A.pos[i] = p;
    const double4_32a r = A.ref[i];
    const double ex = __dsub_rn(p.x, r.x), ey = __dsub_rn(p.y, r.y), ez = __dsub_rn(p.z, r.z);
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
    if (d2 > lim2 || !(d2 == d2)) {
        A.flags->need_rebuild = 1;
        A.flags->skin_exceeded = 1;
    }
    A.posf[i] = build_image(p, r, boxes[replica_of(A, i)], A.spec[i]);
    if (A.posd) {
        const Box &B = boxes[replica_of(A, i)];
        const double4_32a q = build_image64(p, r, B);
        A.posd[i] = q;
        if (A.posx) store_dfpos(A, i, q, B);
    }
}

// What opens a step: the half kick and drift of velocity Verlet, or the predictor.
__device__ __forceinline__ void open_step(const Atoms &A, const Box *boxes, int i, int motion, double half_dt,
                                          double dt, double s, bool strain, double lim2, const Thermo *th = nullptr) {
    if (motion == kMotionPC3) predict_pc3(A, boxes, i, dt, lim2);
    else kick_drift(A, boxes, i, half_dt, dt, s, strain, lim2, th);
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

// Stencil table of cell group g (one system): the staged slot of the first atom of each of its
// 9 (gx + 2) stencil cells and the total; a group whose neighbourhood exceeds the staging capacity
// sets tile_bad (the passes then take the list path until the next build).
__device__ __forceinline__ void group_table(const Cells &C, int g, Flags *f) {
    const RepCells rg = C.rc[0];
    const int nx = rg.nc[0], ny = rg.nc[1], nz = rg.nc[2];
    const int gxi = g % C.ngx, row = g / C.ngx, y = row % ny, z = row / ny;
    const int x0 = gxi * C.gx, len = min(C.gx, nx - x0);
    int32_t *loc = C.grp_loc + (size_t)g * (C.st_cells + 1);
    int acc = 0, q = 0;
    for (int dz = -1; dz <= 1; dz++) {
        const int zz = (z + dz + nz) % nz;
        for (int dy = -1; dy <= 1; dy++) {
            const int yy = (y + dy + ny) % ny;
            for (int dx = 0; dx < C.gx + 2; dx++, q++) {
                loc[q] = acc;
                if (dx > len + 1) continue;   // a shorter last group: empty slots
                const int xx = (x0 - 1 + dx + nx) % nx;
                const int c = rg.base + (zz * ny + yy) * nx + xx;
                acc += C.cell_start[c + 1] - C.cell_start[c];
            }
        }
    }
    loc[C.st_cells] = acc;
    atomicMax(&f->tile_max, acc);
    if (acc > C.cap) f->tile_bad = 1;
}

__device__ __forceinline__ void gather_atom(const Atoms &A, int k) {
    const int o = A.sorted[k];
    A.pos_tmp[k] = A.pos[o];
    A.vel_tmp[k] = A.vel[o];
    A.force_tmp[k] = A.force[o];
    A.id_tmp[k] = A.id[o];
    A.spec_tmp[k] = A.spec[o];
    if (A.g3) {
        A.g2_tmp[k] = A.g2[o];
        A.g3_tmp[k] = A.g3[o];
    }
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
    if (A.g3) {
        A.g2[k] = A.g2_tmp[k];
        A.g3[k] = A.g3_tmp[k];
    }
    A.posf[k] = wrapped(p, boxes[replica_of(A, k)], sp);
    if (A.posd) {
        const Box &B = boxes[replica_of(A, k)];
        const double4_32a q = wrapped64(p, B);
        A.posd[k] = q;
        if (A.posx) store_dfpos(A, k, q, B);
    }
}

// The FP64 pair walk's row order (one warp per atom): the entries j > i first, those inside
// r_cut at this build's FP32 positions (cin[i] of them) ahead of the others, then the entries
// j < i, each group in its order; cup[i] = the number of entries j > i.  The order only steers
// the walk (its flattened rows take the inside entries first, so that lanes rarely idle on a
// pair beyond r_cut); which entries count is still decided by every pass's own FP64 test.  The
// whole row (k_max <= kPairsKMax) is read into registers before any entry is written back.
__device__ __forceinline__ void partition_row_warp(const Atoms &A, const Box *boxes, int i, int lane) {
    const int cnt = min(A.count[i], A.k_max);
    const NbrRow row = nbr_row(A, i);
    const Box &B = boxes[replica_of(A, i)];
    const float4 pi = A.posf[i];
    int v[kPairsKMax / 32];
    unsigned in = 0;   // bit c: entry 32 c + lane lies inside r_cut
#pragma unroll
    for (int c = 0; c < kPairsKMax / 32; c++) {
        const int k = 32 * c + lane;
        v[c] = k < cnt ? *row.ptr(k) : -1;
        if (v[c] > i) {
            const float4 pj = A.posf[v[c]];
            float dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
            dx = fmaf(-B.Lf[0], rintf(dx * B.invLf[0]), dx);
            dy = fmaf(-B.Lf[1], rintf(dy * B.invLf[1]), dy);
            dz = fmaf(-B.Lf[2], rintf(dz * B.invLf[2]), dz);
            if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < A.pair_rc2f) in |= 1u << c;
        }
    }
    __syncwarp();
    const unsigned below = (1u << lane) - 1u;
    int nup = 0, nin = 0;
#pragma unroll
    for (int pass = 0; pass < 2; pass++) {
#pragma unroll
        for (int c = 0; c < kPairsKMax / 32; c++) {
            const bool up = v[c] > i && ((in >> c & 1u) != 0) == (pass == 0);
            const unsigned m = __ballot_sync(0xffffffffu, up);
            if (up) *row.ptr(nup + __popc(m & below)) = v[c];
            nup += __popc(m);
        }
        if (pass == 0) nin = nup;
    }
    int pos = nup;
#pragma unroll
    for (int c = 0; c < kPairsKMax / 32; c++) {
        const bool lo = v[c] >= 0 && v[c] < i;
        const unsigned m = __ballot_sync(0xffffffffu, lo);
        if (lo) *row.ptr(pos + __popc(m & below)) = v[c];
        pos += __popc(m);
    }
    if (lane == 0) {
        A.cup[i] = nup;
        A.cin[i] = nin;
    }
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

// The exact test of a candidate in the FP32 band, kept out of line: it is rare, and inlined it
// would be predicated into every iteration of the candidate loop.
static __device__ __noinline__ bool within_exact_band(const double4_32a *pos, int i, int j, const Box &B,
                                                      double rl2) {
    return within_exact(pos[i], pos[j], B, rl2);
}

// Candidates per iteration of the list build's inner loop (their loads are issued together):
// 4 or 2.  On GB300 4 built the fcc Cu list 10 % faster than 2, and 8 30 % slower than 4.
#ifndef MD_BUILD_UNROLL
#define MD_BUILD_UNROLL 4
#endif
// Smallest lane group whose last atoms take several lanes each: a warp-wide group only.  In the
// 4-lane groups of bcc Fe cells (eight cells per warp, about five atoms each) it built the lists
// 20 % slower on GB300 (0.78 against 0.63 ms per rebuild at 1.02M atoms).
#ifndef MD_BUILD_SLICE_MIN_G
#define MD_BUILD_SLICE_MIN_G 32
#endif

// Full list rows of the atoms of link cell c (§3.2.1: candidates from the cells around it, 27 for
// cells r_list wide, 125 for cells r_list / 2 wide) by a group of G lanes (G = 4, 8, 16 or 32;
// 32 / G cells per warp): lane a of the group takes atoms s + a, s + a + G, ... of the cell.  All
// lanes of the group walk the same neighbour cells and the same candidates in the same order,
// so a candidate is one broadcast load for the group and
// the control flow is uniform inside it.  Candidates are screened with FP32 wrapped coordinates,
// shifted by whole box edges for neighbour cells across the periodic boundary (no rounding to the
// nearest image per candidate).  Only a candidate whose FP32 r^2 lies in [band_lo, band_hi] (a band
// wider than the proven FP32 error) is decided by the exact FP64 test, so each row is the exact
// FP64 set, listed by cell in (dz, dy, dx) order and by ascending slot inside a cell.  Rows are cut
// at k_max (the count is kept).  Returns the longest row of this lane's atoms.  The stencil of
// +-reach cells along each edge needs >= 2 reach + 1 cells per edge (no cell visited twice).
// LOCAL (group walks, one system, reach 1): 1, every entry is also written to the 16-bit local
// list as the slot of the candidate in its cell group's stage (grp_loc of the stencil cell plus
// the candidate's rank inside its cell); 2, only the entries j > i are, as the half row of the
// half walk (lcount of them).
// The cells of the stencil of link cell (cx, cy, cz) of a replica (+-R cells along each edge), in
// (dz, dy, dx) order: fn(js, je, sx, sy, sz, dz, dy, dx) with the cell's slot range and the shift
// by whole box edges that puts a cell across the periodic boundary next to the home cell.
template <typename Fn>
__device__ __forceinline__ void for_stencil(const Cells &C, const RepCells &g, int R, int cx, int cy, int cz,
                                            float Lx, float Ly, float Lz, Fn &&fn) {
    const int nx = g.nc[0], ny = g.nc[1], nz = g.nc[2];
    for (int dz = -R; dz <= R; dz++) {
        int z = cz + dz;
        float sz = 0.f;
        if (z < 0) { z += nz; sz = -Lz; }
        if (z >= nz) { z -= nz; sz = Lz; }
        for (int dy = -R; dy <= R; dy++) {
            int y = cy + dy;
            float sy = 0.f;
            if (y < 0) { y += ny; sy = -Ly; }
            if (y >= ny) { y -= ny; sy = Ly; }
            const int rowc = g.base + (z * ny + y) * nx;
            for (int dx = -R; dx <= R; dx++) {
                int x = cx + dx;
                float sx = 0.f;
                if (x < 0) { x += nx; sx = -Lx; }
                if (x >= nx) { x -= nx; sx = Lx; }
                const int cc = rowc + x;
                fn(C.cell_start[cc], C.cell_start[cc + 1], sx, sy, sz, dz, dy, dx);
            }
        }
    }
}

// Full list rows of the atoms of link cell c (§3.2.1: candidates from the cells around it, 27 for
// cells r_list wide, 125 for cells r_list / 2 wide) by a group of G lanes (G = 4, 8, 16 or 32;
// 32 / G cells per warp): lane a of the group takes atoms s + a, s + a + G, ... of the cell.  All
// lanes of the group walk the same neighbour cells and the same candidates in the same order,
// so a candidate is one broadcast load for the group and
// the control flow is uniform inside it.  Candidates are screened with FP32 wrapped coordinates,
// shifted by whole box edges for neighbour cells across the periodic boundary (no rounding to the
// nearest image per candidate).  Only a candidate whose FP32 r^2 lies in [band_lo, band_hi] (a band
// wider than the proven FP32 error) is decided by the exact FP64 test, so each row is the exact
// FP64 set, listed by cell in (dz, dy, dx) order and by ascending slot inside a cell.  Rows are cut
// at k_max (the count is kept).  Returns the longest row of this lane's atoms.  The stencil of
// +-reach cells along each edge needs >= 2 reach + 1 cells per edge (no cell visited twice).
// In a warp-wide group (G = 32), the last atoms of a cell, when they fill at most half the warp (the
// 4 atoms after the first 32 of a 36-atom fcc Cu cell), take L = 2, 4, ... lanes each:
// lane l of an atom tests candidates js + l, js + l + L, ... of every stencil cell, and a ballot
// over the atom's L lanes places the accepted ones in slot order, so the rows are the same.
// LOCAL (group walks, one system, reach 1): 1, every entry is also written to the 16-bit local
// list as the slot of the candidate in its cell group's stage (grp_loc of the stencil cell plus
// the candidate's rank inside its cell); 2, only the entries j > i are, as the half row of the
// half walk (lcount of them).  Those builds keep one lane per atom, and write the global rows
// (A.nbr) only when `rows` is set (the counts always): the step kernel's group walks read the
// local rows alone while every group fits its stage.
template <int G, int LOCAL>
__device__ __forceinline__ int build_cell_group(const Atoms &A, const Cells &C, const Box *boxes, int c, int gl,
                                                double rl2, float band_lo, float band_hi, bool rows = true) {
    const int s = C.cell_start[c], e = C.cell_start[c + 1];
    if (s == e) return 0;
    const int r = replica_of(A, s);
    const Box &B = boxes[r];
    const RepCells g = C.rc[r];
    const int nx = g.nc[0], ny = g.nc[1], nz = g.nc[2];
    const int local = c - g.base;
    const int cx = local % nx, cy = (local / nx) % ny, cz = local / (nx * ny);
    const float Lx = B.Lf[0], Ly = B.Lf[1], Lz = B.Lf[2];
    const int R = C.reach;
    const int kmax = A.k_max;
    const long long plane = 4LL * A.n;
    const bool edge = cx < R || cx >= nx - R || cy < R || cy >= ny - R || cz < R || cz >= nz - R;
    int longest = 0;
    for (int a0 = s; a0 < e; a0 += G) {
        if constexpr (LOCAL == 0 && G >= MD_BUILD_SLICE_MIN_G) {
            if (2 * (e - a0) <= G) {   // the last atoms of the cell: L lanes each
                const int rem = e - a0;
                int lg = 1;
                while ((rem << (lg + 1)) <= G) lg++;
                const int L = 1 << lg;
                const int a = gl >> lg, sl = gl & (L - 1);
                const bool act = a < rem;
                const int i = a0 + a, ii = act ? i : s;
                const float4 fi = A.posf[ii];
                const int gbase = (int)(threadIdx.x & 31) & ~(G - 1);
                const unsigned gmask = G == 32 ? 0xffffffffu : ((1u << G) - 1u) << gbase;
                const unsigned lmask = L == 32 ? 0xffffffffu : (1u << L) - 1u;
                const int sh = gbase + (a << lg);
                int32_t *const row = A.nbr + 4 * (size_t)ii;
                int cnt = 0;
                for_stencil(C, g, R, cx, cy, cz, Lx, Ly, Lz,
                            [&](int js, int je, float sx, float sy, float sz, int, int, int) {
                    const float ox = sx - fi.x, oy = sy - fi.y, oz = sz - fi.z;
                    for (int j0 = js; j0 < je; j0 += L) {   // the same trip count on every lane of the group
                        const int j = j0 + sl;
                        bool in = false;
                        if (j < je) {
                            const float4 f = A.posf[j];
                            const float dx = f.x + ox, dy = f.y + oy, dz = f.z + oz;
                            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                            if (r2 <= band_hi)
                                in = (r2 < band_lo || within_exact_band(A.pos, ii, j, B, rl2)) && act && j != i;
                        }
                        const unsigned sub = (__ballot_sync(gmask, in) >> sh) & lmask;
                        if (in) {
                            const int k = cnt + __popc(sub & ((1u << sl) - 1u));
                            if (k < kmax) row[(long long)(k >> 2) * plane + (k & 3)] = j;
                        }
                        cnt += __popc(sub);
                    }
                });
                if (act) {
                    if (sl == 0) {
                        A.count[i] = cnt;
                        A.wrap[i] = edge ? 1 : 0;
                        if (cnt > kmax) atomicOr(&A.flags->error, FLAG_OVERFLOW);
                    }
                    longest = max(longest, cnt);
                }
                break;
            }
        }
        const int i = a0 + gl;
        const bool act = i < e;
        const int ii = act ? i : s;
        const float4 fi = A.posf[ii];
        int32_t *wp = A.nbr + 4 * (size_t)ii;   // entry cnt of the row (planes of 4 entries)
        uint16_t *lwp = LOCAL ? A.lnbr + 4 * (size_t)ii : nullptr;   // the same entry of the local list
        int cnt = 0, lcnt = 0;
        int lbase = 0;   // staged slot of the first atom of the current candidate cell (local list)
        // one candidate: append j to the row if it is a neighbour
        auto visit = [&](int j, int js, float r2) {
            if (r2 <= band_hi) {
                const bool in = r2 < band_lo || within_exact_band(A.pos, ii, j, B, rl2);
                if (in && act && j != i) {
                    if (cnt < kmax) {
                        if (LOCAL == 0 || rows) *wp = j;
                        if constexpr (LOCAL == 1) *lwp = (uint16_t)(lbase + (j - js));
                        if constexpr (LOCAL == 2) {
                            if (j > i) {
                                *lwp = (uint16_t)(lbase + (j - js));
                                lcnt++;
                                lwp += (lcnt & 3) ? 1 : plane - 3;
                            }
                        }
                    }
                    cnt++;
                    const long long adv = (cnt & 3) ? 1 : plane - 3;
                    wp += adv;
                    if constexpr (LOCAL == 1) lwp += adv;
                }
            }
        };
        // cell group of the home cell (group walks): stencil slots of this cell's neighbours
        const int32_t *gloc = nullptr;
        int gx0 = 0;
        if constexpr (LOCAL) {
            const int gxi = cx / C.gx;
            gx0 = gxi * C.gx;
            gloc = C.grp_loc + (size_t)((cz * ny + cy) * C.ngx + gxi) * (C.st_cells + 1);
        }
        for_stencil(C, g, R, cx, cy, cz, Lx, Ly, Lz,
                    [&](int js, int je, float sx, float sy, float sz, int dz, int dy, int dx) {
            if constexpr (LOCAL) lbase = gloc[((dz + 1) * 3 + (dy + 1)) * (C.gx + 2) + (cx - gx0 + dx + 1)];
            const float ox = sx - fi.x, oy = sy - fi.y, oz = sz - fi.z;
            int j = js;
#if MD_BUILD_UNROLL >= 4
            for (; j + 3 < je; j += 4) {
                const float4 f0 = A.posf[j], f1 = A.posf[j + 1], f2 = A.posf[j + 2], f3 = A.posf[j + 3];
                const float ax = f0.x + ox, ay = f0.y + oy, az = f0.z + oz;
                const float bx = f1.x + ox, by = f1.y + oy, bz = f1.z + oz;
                const float cx2 = f2.x + ox, cy2 = f2.y + oy, cz2 = f2.z + oz;
                const float dx2 = f3.x + ox, dy2 = f3.y + oy, dz2 = f3.z + oz;
                const float r0 = fmaf(ax, ax, fmaf(ay, ay, az * az));
                const float r1 = fmaf(bx, bx, fmaf(by, by, bz * bz));
                const float rr2 = fmaf(cx2, cx2, fmaf(cy2, cy2, cz2 * cz2));
                const float rr3 = fmaf(dx2, dx2, fmaf(dy2, dy2, dz2 * dz2));
                visit(j, js, r0);
                visit(j + 1, js, r1);
                visit(j + 2, js, rr2);
                visit(j + 3, js, rr3);
            }
#endif
            for (; j + 1 < je; j += 2) {
                const float4 f0 = A.posf[j], f1 = A.posf[j + 1];
                const float ax = f0.x + ox, ay = f0.y + oy, az = f0.z + oz;
                const float bx = f1.x + ox, by = f1.y + oy, bz = f1.z + oz;
                const float r0 = fmaf(ax, ax, fmaf(ay, ay, az * az));
                const float r1 = fmaf(bx, bx, fmaf(by, by, bz * bz));
                visit(j, js, r0);
                visit(j + 1, js, r1);
            }
            if (j < je) {
                const float4 f0 = A.posf[j];
                const float ax = f0.x + ox, ay = f0.y + oy, az = f0.z + oz;
                visit(j, js, fmaf(ax, ax, fmaf(ay, ay, az * az)));
            }
        });
        if (act) {
            A.count[i] = cnt;
            A.wrap[i] = edge ? 1 : 0;
            if constexpr (LOCAL == 2) A.lcount[i] = lcnt;
            if (cnt > kmax) atomicOr(&A.flags->error, FLAG_OVERFLOW);
            longest = max(longest, cnt);
        }
    }
    return longest;
}

// The list phase over all cells: warp w of nwarps takes cell groups w, w + nwarps, ...; every
// lane returns the longest row it built (all 32 lanes of a warp take part in every iteration).
template <int G, int LOCAL>
__device__ __forceinline__ int build_cells(const Atoms &A, const Cells &C, const Box *boxes, long long warp,
                                           long long nwarps, int lane, double rl2, float band_lo, float band_hi,
                                           bool rows = true) {
    constexpr int CPW = 32 / G;   // cells per warp
    int m = 0;
    for (long long c0 = warp * CPW; c0 < C.ncell; c0 += nwarps * CPW) {
        const long long c = c0 + lane / G;
        if (c < C.ncell)
            m = max(m, build_cell_group<G, LOCAL>(A, C, boxes, (int)c, lane & (G - 1), rl2, band_lo, band_hi, rows));
    }
    return m;
}

template <int LOCAL>
__device__ __forceinline__ int build_cells_any(int G, const Atoms &A, const Cells &C, const Box *boxes, long long warp,
                                               long long nwarps, int lane, double rl2, float band_lo, float band_hi,
                                               bool rows = true) {
    if (G == 4) return build_cells<4, LOCAL>(A, C, boxes, warp, nwarps, lane, rl2, band_lo, band_hi, rows);
    if (G == 8) return build_cells<8, LOCAL>(A, C, boxes, warp, nwarps, lane, rl2, band_lo, band_hi, rows);
    if (G == 16) return build_cells<16, LOCAL>(A, C, boxes, warp, nwarps, lane, rl2, band_lo, band_hi, rows);
    return build_cells<32, LOCAL>(A, C, boxes, warp, nwarps, lane, rl2, band_lo, band_hi, rows);
}

}  // namespace ph
}  // namespace mdk
