// Staged passes of the mixed-precision step kernel: the two EAM passes of Eq. (1) over cell
// groups instead of single atoms.  A group is gx consecutive link cells along x (the home cells);
// its neighbourhood, the 3 x 3 x (gx + 2) stencil of cells around them, is copied into shared
// memory with each periodic image's shift already added (§3.2.1's link cells, here as a unit of
// data reuse).  Two neighbour walks read the stage.  In the staged walk every home atom reads its
// neighbours through its 16-bit local list (the same entries as the global list, as staged
// slots), so a pair costs a shared-memory load instead of a scattered global one and needs no
// minimum image.
//
// The half walk computes each pair once (a half list and Newton's third law, §3.2.2): the other
// atom's share is summed in shared memory per stage slot and added to global FP64 accumulators
// once per group.
//
// The cell walk is the link-cell method without a Verlet list (the limit of §3.2.1's hybrid with
// no list): a warp takes one home atom at a time, its 32 lanes test 32 staged candidates of the
// 27 cells around the atom's cell at a time, and the hits (r < r_cut) are queued per warp and
// evaluated 32 at a time, so that the pair terms run with all lanes busy.
//
// Pipeline.  The last warp of the block is the producer: it stages the block's groups, one after
// the other, into C.nbuf stage buffers (two where they fit), while the other warps (the consumers)
// compute the group in the other buffer.  Every stencil row is at most three runs of cells that
// are consecutive both in the global cell order and in the stage (the image left of x = 0, the
// cells inside the box, the image right of it); each run moves with one bulk copy (cp.async.bulk,
// global to this block's shared memory, completion counted in bytes on the buffer's "full"
// mbarrier), issued by its own producer lane.  Once the copies have landed the producer adds the
// periodic shifts of the runs that need one and arrives on the buffer's "ready" mbarrier.
// Consumers wait on "ready", claim the group's work a warp at a time from a shared counter (so
// that warps flow from one group into the next without a block-wide barrier) and arrive on the
// buffer's "empty" mbarrier when they find no work left; the producer waits on "empty" before it
// refills the buffer (and, in the half walk, first adds the buffer's shares to the FP64
// accumulators).  Every wait is bounded: past the launch's poll limit, or once another wait has
// given up, a wait fails, marks the launch aborted (FLAG_TIMEOUT) and the block leaves the pass;
// the producer then waits (bounded again) for its own copies in flight.
//
// Slot layout of a stage: stencil cell s = ((dz + 1) 3 + (dy + 1)) (gx + 2) + (x - x0 + 1) holds its
// atoms in cell order from slot grp_loc[g][s]; the home atoms of the group are contiguous in the
// global cell order (cells x0 .. x0 + len - 1 of one row).
#pragma once

#include <cuda_runtime.h>

#include "md_passes.cuh"

namespace mdk {
namespace tl {

// Stencil cells of a group of at most kTileMaxGx cells, and the slot table (with the total).
constexpr int kTileMaxGx = kGroupMaxGx;
constexpr int kTileMaxSt = 9 * (kTileMaxGx + 2);
constexpr int kStageBufs = MD_STAGE_BUFS;

struct Group {
    int h0, h1;   // home atoms [h0, h1) (global slots)
    int len;      // home cells
};

// ---- mbarrier and bulk-copy primitives (this block's shared memory only) ----
__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(unsigned long long *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive(unsigned long long *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}
// Bytes the current phase waits for besides the arrivals (no arrival of its own).
__device__ __forceinline__ void bar_expect_tx(unsigned long long *b, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_test(unsigned long long *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(saddr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned) from global memory to
// this block's shared memory, its completion counted on barrier b.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, unsigned long long *b) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     saddr(dst)),
                 "l"(src), "r"(bytes), "r"(saddr(b))
                 : "memory");
}
// Orders this thread's earlier generic-proxy accesses (and those it has observed) before its
// later async-proxy ones: the bulk copies read what plain stores wrote and overwrite what plain
// loads and stores used.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }

// Shared-memory state of the pipeline.
struct Pipe {
    unsigned long long full[kStageBufs];    // buffer b's copies landed: the producer's 32 lanes + the bytes
    unsigned long long ready[kStageBufs];   // buffer b shifted and released to the consumers (32 lanes)
    unsigned long long empty[kStageBufs];   // every consumer thread done with buffer b
    int next[kStageBufs];                   // first unclaimed work unit of buffer b's group
    int hdr[kStageBufs][4];                 // group, first and end home atom, home cells
    int loc[kStageBufs][kTileMaxSt + 1];    // slot table of buffer b's group
};

// Once per launch, by one thread (the block synchronises after).
template <int NT>
__device__ __forceinline__ void pipe_init(Pipe &p) {
    for (int b = 0; b < kStageBufs; b++) {
        bar_init(&p.full[b], 32);
        bar_init(&p.ready[b], 32);
        bar_init(&p.empty[b], NT - 32);
        p.next[b] = 0;
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Bounded wait for the completion of the phase of barrier b with parity `parity`.  False after
// `limit` polls (the launch is then marked aborted) or once the launch is aborted.
__device__ __forceinline__ bool bar_wait(unsigned long long *b, uint32_t parity, unsigned long long limit,
                                         int *abort, Flags *f) {
    for (unsigned long long k = 0;; ++k) {
        if (bar_test(b, parity)) return true;
        if ((k & 63) == 63) {   // the abort word is a global load: read it every 64 polls
            if (*reinterpret_cast<volatile int *>(abort)) return false;
            if (k >= limit) {
                atomicExch(abort, 1);
                atomicOr(&f->error, FLAG_TIMEOUT);
                return false;
            }
        }
        __nanosleep(32);
    }
}

// Launch-wide pieces of a group pass.
struct PassCtl {
    unsigned long long limit;   // polls of a bounded wait
    int *abort;                 // the grid barrier's abort word
    Flags *flags;
    bool withhold;              // self-test of the bounded waits: this block's producer stages nothing
};

// Group g's geometry.
__device__ __forceinline__ Group group_of(const Cells &C, int g) {
    const RepCells rg = C.rc[0];
    const int nx = rg.nc[0], ny = rg.nc[1];
    const int gxi = g % C.ngx, row = g / C.ngx, y = row % ny, z = row / ny;
    const int x0 = gxi * C.gx, len = min(C.gx, nx - x0);
    const int c0 = rg.base + (z * ny + y) * nx + x0;
    return Group{C.cell_start[c0], C.cell_start[c0 + len], len};
}

// The runs of group g's stage (slot table loc): per stencil row (dz, dy) up to three ranges of
// consecutive cells, each contiguous in the global cell order and in the stage: the image of
// x = nx - 1 left of the box (first group of a row), the cells inside the box, the image of x = 0
// right of it (last group).  Run l = 3 r + k (row r, part k) for l < 27: stage slots
// [slot, slot + n) take atoms [atom, atom + n) plus the periodic shift (sx, sy, sz); n = 0 for a
// run that does not exist or holds no atom.
struct Run {
    int slot, atom, n;
    bool shifted;   // some component of the shift is nonzero
    float sx, sy, sz;
};

__device__ __forceinline__ Run run_of(const Cells &C, const Box &B, int g, const int *loc, int l) {
    Run R{0, 0, 0, false, 0.f, 0.f, 0.f};
    if (l >= 27) return R;
    const RepCells rg = C.rc[0];
    const int nx = rg.nc[0], ny = rg.nc[1], nz = rg.nc[2];
    const int gxi = g % C.ngx, row = g / C.ngx, y = row % ny, z = row / ny;
    const int x0 = gxi * C.gx, len = min(C.gx, nx - x0), W = C.gx + 2;
    const int dmax = len + 1;              // stencil columns 0 .. len + 1 hold atoms (x = x0 - 1 + column)
    const int mid0 = x0 == 0 ? 1 : 0;      // first column inside the box
    const int mid1 = min(dmax, nx - x0);   // last column inside the box
    const int r = l / 3, k = l - 3 * r;
    int yy = y + r % 3 - 1, zz = z + r / 3 - 1;
    if (yy < 0) { yy += ny; R.sy = -B.Lf[1]; } else if (yy >= ny) { yy -= ny; R.sy = B.Lf[1]; }
    if (zz < 0) { zz += nz; R.sz = -B.Lf[2]; } else if (zz >= nz) { zz -= nz; R.sz = B.Lf[2]; }
    const int crow = rg.base + (zz * ny + yy) * nx;   // the row's cell at x = 0
    const int *lr = loc + r * W;
    int c0, c1, cell;
    if (k == 0) {
        if (mid0 != 1) return R;
        c0 = 0; c1 = 0; cell = crow + nx - 1; R.sx = -B.Lf[0];
    } else if (k == 1) {
        if (mid1 < mid0) return R;
        c0 = mid0; c1 = mid1; cell = crow + x0 - 1 + mid0;
    } else {
        if (dmax <= mid1) return R;
        c0 = mid1 + 1; c1 = dmax; cell = crow; R.sx = B.Lf[0];
    }
    R.slot = lr[c0];
    R.n = lr[c1 + 1] - lr[c0];
    R.shifted = R.sx != 0.f || R.sy != 0.f || R.sz != 0.f;
    if (R.n > 0) R.atom = C.cell_start[cell];
    return R;
}

// The runs with atoms, one at a time, in every lane (each lane set up run `lane` in R).
template <typename F>
__device__ __forceinline__ void for_each_run(const Run &R, unsigned mask, F &&f) {
    while (mask) {
        const int l = __ffs(mask) - 1;
        mask &= mask - 1;
        Run q;
        q.slot = __shfl_sync(0xffffffffu, R.slot, l);
        q.atom = __shfl_sync(0xffffffffu, R.atom, l);
        q.n = __shfl_sync(0xffffffffu, R.n, l);
        q.sx = __shfl_sync(0xffffffffu, R.sx, l);
        q.sy = __shfl_sync(0xffffffffu, R.sy, l);
        q.sz = __shfl_sync(0xffffffffu, R.sz, l);
        f(q);
    }
}

// Producer (one warp): stage group g into buffer b (use u of the buffer; st: its slots, acc: its
// half-walk sums or NULL) and release it to the consumers.  Lane l sets up run l and moves it
// with one bulk copy; once the copies have landed the warp adds the periodic shifts of the runs
// that need one in shared memory.  False if the wait for the copies gave up.
__device__ __forceinline__ bool stage_issue(const Cells &C, const Box &B, const float4 *src, int g, Pipe &p, int b,
                                            unsigned u, float4 *st, float4 *acc, const PassCtl &ctl) {
    const int lane = threadIdx.x & 31;
    int *loc = p.loc[b];
    const int32_t *gl = C.grp_loc + (size_t)g * (C.st_cells + 1);
    fence_proxy_async();
    for (int q = lane; q <= C.st_cells; q += 32) loc[q] = gl[q];
    __syncwarp();
    if (lane == 0) {
        const Group G = group_of(C, g);
        p.hdr[b][0] = g;
        p.hdr[b][1] = G.h0;
        p.hdr[b][2] = G.h1;
        p.hdr[b][3] = G.len;
        p.next[b] = 0;
    }
    const Run R = run_of(C, B, g, loc, lane);
    const uint32_t bytes = __reduce_add_sync(0xffffffffu, 16u * (uint32_t)R.n);
    if (lane == 0) bar_expect_tx(&p.full[b], bytes);
    __syncwarp();
    if (R.n > 0) bulk_g2s(st + R.slot, src + R.atom, 16u * (uint32_t)R.n, &p.full[b]);
    bar_arrive(&p.full[b]);
    if (acc)
        for (int t = lane; t < loc[C.st_cells]; t += 32) acc[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!bar_wait(&p.full[b], u & 1u, ctl.limit, ctl.abort, ctl.flags)) return false;
    for_each_run(R, __ballot_sync(0xffffffffu, R.n > 0 && R.shifted), [&](const Run &q) {
        for (int t = lane; t < q.n; t += 32) {
            float4 &v = st[q.slot + t];
            v.x += q.sx;
            v.y += q.sy;
            v.z += q.sz;
        }
    });
    bar_arrive(&p.ready[b]);   // every lane: its own stores released with its arrival
    return true;
}

// Producer, half walk: add buffer b's per-slot sums to the FP64 accumulators (the density (x)
// when !FORCE, else the force (x, y, z) and pair energy (w)).
template <bool FORCE>
__device__ __forceinline__ void flush_buffer(const Atoms &A, const Cells &C, const Box &B, const Pipe &p, int b,
                                             const float4 *acc) {
    const int lane = threadIdx.x & 31;
    const Run R = run_of(C, B, p.hdr[b][0], p.loc[b], lane);
    for_each_run(R, __ballot_sync(0xffffffffu, R.n > 0), [&](const Run &q) {
        for (int t = lane; t < q.n; t += 32) {
            const float4 a = acc[q.slot + t];
            if (FORCE) {
                if (a.x != 0.f || a.y != 0.f || a.z != 0.f || a.w != 0.f) {
                    double4_32a *f = A.f_acc + q.atom + t;
                    atomicAdd(&f->x, (double)a.x);
                    atomicAdd(&f->y, (double)a.y);
                    atomicAdd(&f->z, (double)a.z);
                    if (a.w != 0.f) atomicAdd(&f->w, (double)a.w);
                }
            } else if (a.x != 0.f) {
                atomicAdd(&A.rho_acc[q.atom + t], (double)a.x);
            }
        }
    });
}

// Groups of this block in one pass: g = blockIdx.x, + gridDim.x, ...
__device__ __forceinline__ unsigned block_groups(const Cells &C) {
    const int nb = (int)gridDim.x, g0 = (int)blockIdx.x;
    return g0 < C.n_groups ? (unsigned)((C.n_groups - g0 + nb - 1) / nb) : 0u;
}

template <int NT>
__device__ __forceinline__ bool is_producer() {
    return (threadIdx.x >> 5) == NT / 32 - 1;
}

// Producer of one pass: stages the block's groups, s = seq, seq + 1, ... (seq: the block's
// running group count in this launch) into buffer s mod nbuf, src the positions (float4 per
// atom); for the half walk (HALF_FORCE: 0 density, 1 force; -1 no half walk) it first adds the
// sums of the group the buffer held before to the FP64 accumulators.
template <int HALF_FORCE>
__device__ __noinline__ void produce(const Atoms &A, const Cells &C, const Box &B, const float4 *src, Pipe &p,
                                     float4 *stage, float4 *accs, unsigned seq, const PassCtl &ctl) {
    if (ctl.withhold) return;   // the consumers' waits run out; nothing is in flight
    const unsigned nbuf = (unsigned)C.nbuf, count = block_groups(C);
    unsigned held = 0, u_last[kStageBufs];
    bool ok = true;
    int g = blockIdx.x;
    for (unsigned s = seq; s < seq + count; s++, g += gridDim.x) {
        const int b = (int)(s % nbuf);
        const unsigned u = s / nbuf;
        if (held >> b & 1u) {
            if (!bar_wait(&p.empty[b], (u - 1u) & 1u, ctl.limit, ctl.abort, ctl.flags)) {
                ok = false;
                break;
            }
            if constexpr (HALF_FORCE >= 0) flush_buffer<HALF_FORCE == 1>(A, C, B, p, b, accs + (size_t)b * C.cap);
        }
        held |= 1u << b;
        u_last[b] = u;
        if (!stage_issue(C, B, src, g, p, b, u, stage + (size_t)b * C.cap,
                         HALF_FORCE >= 0 ? accs + (size_t)b * C.cap : nullptr, ctl)) {
            ok = false;
            break;
        }
    }
    for (int b = 0; b < (int)nbuf; b++) {
        if (!(held >> b & 1u)) continue;
        const unsigned u = u_last[b];
        if (ok && bar_wait(&p.empty[b], u & 1u, ctl.limit, ctl.abort, ctl.flags)) {
            if constexpr (HALF_FORCE >= 0) flush_buffer<HALF_FORCE == 1>(A, C, B, p, b, accs + (size_t)b * C.cap);
        } else {
            // given up: wait (bounded, whatever the abort word says) for this buffer's copies
            ok = false;
            for (unsigned long long k = 0; k < ctl.limit && !bar_test(&p.full[b], u & 1u); ++k) __nanosleep(100);
        }
    }
}

// Consumer: wait until the block's group number s is staged; its buffer (s mod nbuf) in b.
__device__ __forceinline__ bool acquire(const Cells &C, Pipe &p, unsigned s, const PassCtl &ctl, int &b) {
    const unsigned nbuf = (unsigned)C.nbuf;
    b = (int)(s % nbuf);
    return bar_wait(&p.ready[b], (s / nbuf) & 1u, ctl.limit, ctl.abort, ctl.flags);
}

// Consumer: this warp is done with buffer b (called by all 32 lanes).
__device__ __forceinline__ void release(Pipe &p, int b) {
    __syncwarp();
    bar_arrive(&p.empty[b]);
}

// Consumer: the next `unit` work items of buffer b's group (the same value in every lane).
__device__ __forceinline__ int claim(Pipe &p, int b, int unit) {
    int c = 0;
    if ((threadIdx.x & 31) == 0) c = atomicAdd(&p.next[b], unit);
    return __shfl_sync(0xffffffffu, c, 0);
}

// Density pass, one lane of home atom i (i >= h1: a padding lane of the last warp).
template <int T, int KIND, bool SMT>
__device__ __forceinline__ void density_item(const Atoms &A, const Pot &P, const float4 *st, int h1, int i, int lane) {
    const bool live = i < h1;
    float hi = 0.f, lo = 0.f;
    float4 pi = make_float4(0.f, 0.f, 0.f, 0.f);
    if (live) {
        pi = A.posf[i];
        const int cnt = min(A.count[i], A.k_max);
        const NbrRow16 row = lnbr_row(A, i);
        unsigned viol = 0;
        auto term = [&](const float4 &pj) -> float {
            return ps::rho_term32<KIND, false, SMT>(P, 0, 0, pj.x - pi.x, pj.y - pi.y, pj.z - pi.z, viol);
        };
        // two neighbours per iteration; the local list entries of the next iteration are loaded
        // before this iteration's terms are computed
        auto entry = [&](int q) { return q < cnt ? (int)ld_phase(row.ptr(q)) : 0; };
        int k = lane;
        int n0 = entry(k), n1 = entry(k + T);
        for (; k + T < cnt; k += 2 * T) {
            const float4 p0 = st[n0], p1 = st[n1];
            n0 = entry(k + 2 * T);
            n1 = entry(k + 3 * T);
            const float a0 = term(p0), a1 = term(p1);
            ps::two_sum_add(hi, lo, a0);
            ps::two_sum_add(hi, lo, a1);
        }
        if (k < cnt) ps::two_sum_add(hi, lo, term(st[n0]));
        if (viol) atomicAdd(&A.flags->range_violations, (unsigned long long)viol);
    }
    ps::lane_sum_df<T>(hi, lo);
    if (live && lane == 0) ps::density32_finish(A, P, i, 0, pi, hi, lo);
}

// Force pass, one lane of home atom i; returns i for the lane that finished it, else -1.
template <int T, int KIND, bool ENERGY, bool SMT>
__device__ __forceinline__ int force_item(const Atoms &A, const Pot &P, const float4 *st, int h1, int i, int lane,
                                          double half_dt, bool kick, double (&part)[kPartials]) {
    const bool live = i < h1;
    ps::Acc32 a;
    if (live) {
        const float4 pi = A.p2f[i];
        const int cnt = min(A.count[i], A.k_max);
        const NbrRow16 row = lnbr_row(A, i);
        unsigned viol = 0;
        auto pair = [&](const float4 &pj) {
            ps::pair32<KIND, false, ENERGY, SMT>(P, 0, 0, pi.w, pj.w, pj.x - pi.x, pj.y - pi.y, pj.z - pi.z, a, viol);
        };
        auto entry = [&](int q) { return q < cnt ? (int)ld_phase(row.ptr(q)) : 0; };
        int k = lane;
        int n0 = entry(k), n1 = entry(k + T);
        for (; k + T < cnt; k += 2 * T) {
            const float4 p0 = st[n0], p1 = st[n1];
            n0 = entry(k + 2 * T);
            n1 = entry(k + 3 * T);
            pair(p0);
            pair(p1);
        }
        if (k < cnt) pair(st[n0]);
        if (viol) atomicAdd(&A.flags->range_violations, (unsigned long long)viol);
    }
    ps::lane_sum_acc<T, ENERGY>(a);
    if (!(live && lane == 0)) return -1;
    ps::force32_finish<ENERGY>(A, i, a, half_dt, kick, part);
    return i;
}

// ---- cell walk ----
// Candidates of the home atom at stage slot si in home cell xl of the group (stencil row width W):
// the 9 slot ranges [loc[r W + xl], loc[r W + xl + 3]), r = 0..8.  Every hit (r^2 < r_cut^2, not
// the atom itself) is passed to hit(pj) once, with all 32 lanes for each full batch of 32 and
// the remaining lanes < n for the last; hit must not use warp collectives.
template <typename F>
__device__ __forceinline__ void cells_scan(const float4 *st, const int *loc, int W, int xl, int si,
                                           const float4 &pi, float rc2f, uint16_t *q, F &&hit) {
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    int nq = 0;
    for (int r = 0; r < 9; r++) {
        const int lo = loc[r * W + xl], hi = loc[r * W + xl + 3];
        for (int b = lo; b < hi; b += 32) {
            const int sj = b + lane;
            bool h = false;
            if (sj < hi && sj != si) {
                const float4 pj = st[sj];
                const float dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
                h = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < rc2f;
            }
            const unsigned m = __ballot_sync(0xffffffffu, h);
            if (h) q[nq + __popc(m & below)] = (uint16_t)sj;
            nq += __popc(m);
            if (nq >= 32) {   // a full batch: every lane evaluates one queued pair
                __syncwarp();
                hit(st[q[lane]]);
                const int rest = nq - 32;
                const uint16_t v = lane < rest ? q[32 + lane] : (uint16_t)0;
                __syncwarp();
                if (lane < rest) q[lane] = v;
                nq = rest;
                __syncwarp();
            }
        }
    }
    __syncwarp();
    if (lane < nq) hit(st[q[lane]]);
    __syncwarp();
}

// Home cell (0 .. len-1) of the home atom at stage slot si.
__device__ __forceinline__ int home_cell(const int *loc, int W, int len, int si) {
    int xl = 0;
    while (xl + 1 < len && si >= loc[4 * W + 2 + xl]) xl++;
    return xl;
}

// Density pass of the cell walk, home atom i of group G (one warp).
template <int KIND, bool SMT>
__device__ __forceinline__ void density_cell_atom(const Atoms &A, const Pot &P, const float4 *st, const int *loc, int W,
                                                  const Group &G, int i, uint16_t *q) {
    const int lane = threadIdx.x & 31;
    const int si = loc[4 * W + 1] + (i - G.h0);   // home atoms follow the first home cell's slot
    const float4 pi = st[si];                     // a home cell is never shifted: the atom's own coordinates
    float hi = 0.f, lo = 0.f;
    unsigned viol = 0;
    cells_scan(st, loc, W, home_cell(loc, W, G.len, si), si, pi, P.rc2f, q, [&](const float4 &pj) {
        ps::two_sum_add(hi, lo, ps::rho_term32<KIND, false, SMT>(P, 0, 0, pj.x - pi.x, pj.y - pi.y, pj.z - pi.z, viol));
    });
    if (viol) atomicAdd(&A.flags->range_violations, (unsigned long long)viol);
    ps::lane_sum_df<32>(hi, lo);
    if (lane == 0) ps::density32_finish(A, P, i, 0, pi, hi, lo);
}

// Force pass of the cell walk, home atom i of group G (one warp), + the second half kick, and
// with fuse the next step's first half kick and drift, as in the list walk.
template <int KIND, bool ENERGY, bool SMT>
__device__ __forceinline__ void force_cell_atom(const Atoms &A, const Pot &P, const Box *boxes, const float4 *st,
                                                const int *loc, int W, const Group &G, int i, uint16_t *q,
                                                double half_dt, double dt, double lim2, bool fuse,
                                                double (&part)[kPartials]) {
    const int lane = threadIdx.x & 31;
    const int si = loc[4 * W + 1] + (i - G.h0);
    const float4 pi = st[si];
    ps::Acc32 a;
    unsigned viol = 0;
    cells_scan(st, loc, W, home_cell(loc, W, G.len, si), si, pi, P.rc2f, q, [&](const float4 &pj) {
        ps::pair32<KIND, false, ENERGY, SMT>(P, 0, 0, pi.w, pj.w, pj.x - pi.x, pj.y - pi.y, pj.z - pi.z, a, viol);
    });
    if (viol) atomicAdd(&A.flags->range_violations, (unsigned long long)viol);
    ps::lane_sum_acc<32, ENERGY>(a);
    if (lane == 0) {
        ps::force32_finish<ENERGY>(A, i, a, half_dt, true, part);
        if (fuse) ph::kick_drift(A, boxes, i, half_dt, dt, 1.0, false, lim2);
    }
}

// ---- half walk (Newton's third law) ----
// Home atom i takes the pairs of its half row (the neighbours j > i in cell order, as stage
// slots): its own sums stay in registers and go to the FP64 accumulators once; the neighbour's
// share goes to its stage slot's FP32 accumulator in shared memory (a shared atomic add), which
// the producer adds to the FP64 accumulators once per group (flush_buffer).

template <int T, int KIND, bool SMT>
__device__ __forceinline__ void density_half_item(const Atoms &A, const Pot &P, const float4 *st, float4 *acc, int h1,
                                                  int i, int lane) {
    const bool live = i < h1;
    float hi = 0.f, lo = 0.f;
    if (live) {
        const float4 pi = A.posf[i];
        const int cnt = A.lcount[i];
        const NbrRow16 row = lnbr_row(A, i);
        unsigned viol = 0;
        auto pair = [&](int lj) {
            const float4 pj = st[lj];
            const float phi = ps::rho_term32<KIND, false, SMT>(P, 0, 0, pj.x - pi.x, pj.y - pi.y, pj.z - pi.z, viol);
            ps::two_sum_add(hi, lo, phi);
            if (phi != 0.f) atomicAdd(&acc[lj].x, phi);
        };
        auto entry = [&](int q) { return q < cnt ? (int)ld_phase(row.ptr(q)) : 0; };
        int k = lane;
        int n0 = entry(k), n1 = entry(k + T);
        for (; k + T < cnt; k += 2 * T) {
            const int a0 = n0, a1 = n1;
            n0 = entry(k + 2 * T);
            n1 = entry(k + 3 * T);
            pair(a0);
            pair(a1);
        }
        if (k < cnt) pair(n0);
        if (viol) atomicAdd(&A.flags->range_violations, (unsigned long long)viol);
    }
    ps::lane_sum_df<T>(hi, lo);
    if (live && lane == 0) atomicAdd(&A.rho_acc[i], (double)hi + (double)lo);
}

// Force pass of the half walk; on the energy step every lane adds its pairs' virial (each pair
// once, full weight) to its partial sums.
template <int T, int KIND, bool ENERGY, bool SMT>
__device__ __forceinline__ void force_half_item(const Atoms &A, const Pot &P, const float4 *st, float4 *acc, int h1,
                                                int i, int lane, double (&part)[kPartials]) {
    const bool live = i < h1;
    float fx = 0.f, fy = 0.f, fz = 0.f, ep = 0.f;
    if (live) {
        const float4 pi = A.p2f[i];
        const int cnt = A.lcount[i];
        const NbrRow16 row = lnbr_row(A, i);
        unsigned viol = 0;
        float wxx = 0.f, wyy = 0.f, wzz = 0.f, wyz = 0.f, wxz = 0.f, wxy = 0.f;
        auto pair = [&](int lj) {
            const float4 pj = st[lj];
            const float dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
            float V;
            const float gr =
                ps::pair_g32<KIND, false, SMT, ENERGY>(P, 0, 0, pi.w, pj.w, fmaf(dx, dx, fmaf(dy, dy, dz * dz)), V, viol);
            const float ax = gr * dx, ay = gr * dy, az = gr * dz;
            fx += ax;
            fy += ay;
            fz += az;
            if (gr != 0.f) {
                atomicAdd(&acc[lj].x, -ax);
                atomicAdd(&acc[lj].y, -ay);
                atomicAdd(&acc[lj].z, -az);
            }
            if (ENERGY) {
                ep = fmaf(0.5f, V, ep);
                if (V != 0.f) atomicAdd(&acc[lj].w, 0.5f * V);
                wxx = fmaf(-ax, dx, wxx);
                wyy = fmaf(-ay, dy, wyy);
                wzz = fmaf(-az, dz, wzz);
                wyz = fmaf(-ay, dz, wyz);
                wxz = fmaf(-ax, dz, wxz);
                wxy = fmaf(-ax, dy, wxy);
            }
        };
        auto entry = [&](int q) { return q < cnt ? (int)ld_phase(row.ptr(q)) : 0; };
        int k = lane;
        int n0 = entry(k), n1 = entry(k + T);
        for (; k + T < cnt; k += 2 * T) {
            const int a0 = n0, a1 = n1;
            n0 = entry(k + 2 * T);
            n1 = entry(k + 3 * T);
            pair(a0);
            pair(a1);
        }
        if (k < cnt) pair(n0);
        if (viol) atomicAdd(&A.flags->range_violations, (unsigned long long)viol);
        if (ENERGY) {
            part[2] += wxx; part[3] += wyy; part[4] += wzz;
            part[5] += wyz; part[6] += wxz; part[7] += wxy;
        }
    }
    fx = ps::lane_sum<T>(fx);
    fy = ps::lane_sum<T>(fy);
    fz = ps::lane_sum<T>(fz);
    if (ENERGY) ep = ps::lane_sum<T>(ep);
    if (live && lane == 0) {
        double4_32a *f = A.f_acc + i;
        atomicAdd(&f->x, (double)fx);
        atomicAdd(&f->y, (double)fy);
        atomicAdd(&f->z, (double)fz);
        if (ENERGY) atomicAdd(&f->w, (double)ep);
    }
}

// Between the half walk's passes, per atom: F(rho), F'(rho) and the pass-2 copy from the summed
// density; the force accumulators cleared for the force pass.
__device__ __forceinline__ void half_embed(const Atoms &A, const Pot &P, int i) {
    const double rho = A.rho_acc[i];
    double dF;
    const double F = eam::embed64(P, 0, rho, dF, A.flags);
    A.rho[i] = rho;
    A.dF[i] = dF;
    A.e_atom[i] = F;
    const float4 p = A.posf[i];
    A.p2f[i] = make_float4(p.x, p.y, p.z, (float)dF);
    A.f_acc[i] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
}

// After the half walk's force pass, per atom: the summed force, the second half kick, on the
// energy step the atom's energy and partial sums; the density accumulator cleared for the next
// step (the caller fuses the next step's first half kick and drift after it).
template <bool ENERGY>
__device__ __forceinline__ void half_kick(const Atoms &A, int i, double half_dt, double (&part)[kPartials]) {
    const double4_32a f = A.f_acc[i];
    A.force[i] = make_double4_32a(f.x, f.y, f.z, 0.0);
    if (!isfinite(f.x + f.y + f.z)) atomicOr(&A.flags->error, FLAG_NONFINITE);
    double4_32a v = A.vel[i];
    eam::kick_and_partials(v, f.x, f.y, f.z, half_dt, true);
    A.vel[i] = v;
    if (ENERGY) {
        const double e = A.e_atom[i] + f.w;
        A.e_atom[i] = e;
        const double m = 1.0 / (kMvv2e * v.w);
        part[0] += e;
        part[1] += m * fma(v.x, v.x, fma(v.y, v.y, v.z * v.z));
        part[8] += m * v.x; part[9] += m * v.y; part[10] += m * v.z;
    }
    A.rho_acc[i] = 0.0;
}

}  // namespace tl
}  // namespace mdk
