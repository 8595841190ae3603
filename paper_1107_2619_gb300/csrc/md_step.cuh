// The persistent step kernel: n time steps (§2.3: velocity Verlet, or the third-order
// predictor-corrector, sp.motion) of one system or of a batch of replicas in ONE cooperative
// launch.  Under the predictor-corrector "half kick + drift" below reads "predictor" and "half
// kick" after the force reads "corrector".  Phases are separated by a grid barrier:
//
//   [box update (strain)] -> half kick + drift + skin check              (first step only)
//   per step:  [rebuild: bin | scan x3 | scatter | cell sort | gather | copyback | list]
//              -> density pass -> force pass + half kick [+ next step's half kick + drift]
//
// The next step's first half kick and drift are fused into the force pass (each atom does
// them right after its own force): the force pass gathers only the pass-2 copies (p2f/p2d),
// never the positions the drift writes.  Under a strain ramp the box changes every step, so
// the fused form is replaced by a separate box update + kick phase.
//
// The grid barrier waits at most `spin_limit` polls; a block that gives up marks the launch
// aborted (FLAG_TIMEOUT) and every block returns at its next barrier.
//
// Segments (StepParams::stop_at_rebuild, resume): a launch may instead end at the top of a step
// that needs a rebuild (the step already opened), recording the step in Flags::seg_done; the
// rebuild kernel k_rebuild (the same rebuild phases, as a cooperative launch of its own) then
// rebuilds, and a resuming launch continues at that step without the first-step prologue.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>

#include "md_passes.cuh"
#include "md_tile.cuh"

namespace mdk {
namespace st {

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Generation barrier over all blocks of a cooperative launch (all co-resident).
__device__ __forceinline__ bool grid_sync(GridBarrier *b, unsigned nblocks, unsigned long long limit, Flags *f) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = &b->gen;
        const unsigned gen = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(&b->count, 1u) + 1u;
        if (arrived == nblocks) {
            atomicExch(&b->count, 0u);
            __threadfence();
            atomicAdd(&b->gen, 1u);
        } else {
            unsigned long long polls = 0;
            while (*vgen == gen) {
                if (*reinterpret_cast<volatile int *>(&b->abort)) break;
                if (++polls > limit) {
                    atomicExch(&b->abort, 1);
                    atomicOr(&f->error, FLAG_TIMEOUT);
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *reinterpret_cast<volatile int *>(&b->abort) == 0;
}

// Box matrix times the strain matrix diag(1, 1, s) (§2.2), every replica.
__device__ __forceinline__ void strain_boxes(Box *boxes, int n_rep, double s) {
    for (int r = 0; r < n_rep; r++) {
        Box b = boxes[r];
        b.L[2] = __dmul_rn(b.L[2], s);
        b.invL[2] = 1.0 / b.L[2];
        b.Lf[2] = (float)b.L[2];
        b.invLf[2] = (float)b.invL[2];
        b.Lh[2] = (float)b.L[2];
        b.Ll[2] = (float)(b.L[2] - (double)b.Lh[2]);
        boxes[r] = b;
    }
}

// ---- Nose-Hoover thermostat (§2.1.2), one per replica ----
// Kinetic energy of every replica into its fixed-point accumulator: one warp per chunk of at most
// kKeChunk atoms of one replica, one integer atomic per chunk (the sum does not depend on order).
__device__ __forceinline__ void ke_sums(const Atoms &A, const StepParams &sp, long long tid, long long stride) {
    const int lane = threadIdx.x & 31;
    for (long long c = tid >> 5; c < sp.n_ke_chunks; c += stride >> 5) {
        const int2 ch = sp.ke_chunks[c];
        const int end = min(ch.y + kKeChunk, sp.rep_off[ch.x + 1]);
        unsigned long long acc = 0;
        for (int i = ch.y + lane; i < end; i += 32) {
            const double4_32a v = A.vel[i];   // v.w = 1 / (m mvv2e): KE_i = |v|^2 / (2 v.w)
            const double ke = 0.5 * fma(v.x, v.x, fma(v.y, v.y, v.z * v.z)) / v.w;
            acc += (unsigned long long)llrint(ke * kKeFix);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) atomicAdd(&sp.thermo[ch.x].ke_fix, acc);
    }
}

// One thermostat half step of length h from kinetic energy ke: pi += (h/2)(2 KE - g kT)/Q;
// scale = exp(-pi h); xi += pi h; pi += (h/2)(2 KE scale^2 - g kT)/Q.  Returns KE scale^2.
__device__ __forceinline__ double thermo_half(Thermo &t, double ke, double h, double &scale) {
    t.pi += 0.5 * h * (2.0 * ke - t.gkt) / t.q;
    scale = exp(-t.pi * h);
    t.xi += t.pi * h;
    const double ke2 = ke * scale * scale;
    t.pi += 0.5 * h * (2.0 * ke2 - t.gkt) / t.q;
    return ke2;
}

// The half step that closes a velocity-Verlet step (after) and / or the one that opens the next
// (before), from the accumulated kinetic energy; every thread takes a share of the replicas.
__device__ __forceinline__ void thermo_update(const StepParams &sp, int n_rep, long long tid, long long stride,
                                              bool after, bool before) {
    for (long long r = tid; r < n_rep; r += stride) {
        Thermo &t = sp.thermo[r];
        double ke = (double)t.ke_fix / kKeFix;
        t.ke_fix = 0;
        double sb = 1.0, sa = 1.0;
        if (after) ke = thermo_half(t, ke, sp.half_dt, sb);
        if (before) ke = thermo_half(t, ke, sp.half_dt, sa);
        t.s_b = sb;
        t.s_a = sa;
    }
}

// Minimum resident blocks per SM requested from the compiler (caps registers per thread).
// Threads per block of the list walk with the table in shared memory (one block per SM).
#ifndef MD_SMT_THREADS
#define MD_SMT_THREADS 1024
#endif

#ifndef MD_STEP_MIN_BLOCKS_DF   // the double-float passes hold more live values per lane
#define MD_STEP_MIN_BLOCKS_DF 8
#endif
#ifndef MD_STEP_MIN_BLOCKS
#define MD_STEP_MIN_BLOCKS 8
#endif
// Blocks of 128 threads per SM the FP64 step kernel is built for: 4 (128 registers) measured 2-3 %
// faster than 8 (64 registers, with spills) and 6 on fcc Cu 500k with the full list; the pair
// walk over the half list is built for 5 (96 registers): 2.80 -> 2.74 ms per step against 4, 2.86
// at 6 (the full list at 5: 4.79 -> 4.89).
#ifndef MD_STEP_MIN_BLOCKS_FP64
#define MD_STEP_MIN_BLOCKS_FP64 4
#endif
#ifndef MD_STEP_MIN_BLOCKS_PAIRS
#define MD_STEP_MIN_BLOCKS_PAIRS 5
#endif

// The walks over cell groups staged in shared memory (md_tile.cuh).
template <int WALK>
constexpr bool kGroupWalk = WALK == kWalkStaged || WALK == kWalkCells || WALK == kWalkHalf;

// The list rebuild (§3.2.1: bin, counting sort, Verlet list; and for the walks that need them the
// group tables, local rows or the half-list row order), every block of a cooperative launch
// taking part, with grid barriers between the phases.  srow: the step's profiling stamps (1..9)
// or NULL.  False once the launch is aborted (a barrier gave up).  G: the lanes per link cell of
// the list build as a compile-time constant (one build variant in the kernel: fewer registers),
// or 0 for sp.list_group at run time.
template <int WALK, int G = 0>
__device__ __forceinline__ bool rebuild_phases(const Atoms &A, const Cells &C, Box *boxes, const StepParams &sp,
                                               GridBarrier *bar, int *ws, unsigned long long *srow) {
    const unsigned nb = gridDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)nb * blockDim.x;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
#define RB_SYNC()                                                   \
    do {                                                            \
        if (!grid_sync(bar, nb, sp.spin_limit, A.flags)) return false; \
    } while (0)
#define MD_STAMP(q) \
    if (srow) srow[q] = globaltimer()

    for (long long i = tid; i < A.n; i += stride) ph::bin_atom(A, C, boxes, (int)i);
    RB_SYNC();
    MD_STAMP(1);
    const int ntiles = ph::scan_tiles(C);
    for (int t = blockIdx.x; t < ntiles; t += nb) ph::scan_tile_sum(C, t, ws);
    RB_SYNC();
    MD_STAMP(2);
    if (blockIdx.x == 0) {
        if (threadIdx.x == 0) {
            A.flags->max_count = 0;
            A.flags->tile_bad = 0;
            A.flags->tile_max = 0;
        }
        ph::scan_top(C, ws);
    }
    RB_SYNC();
    MD_STAMP(3);
    for (int t = blockIdx.x; t < ntiles; t += nb) ph::scan_apply(C, t, ws);
    RB_SYNC();
    MD_STAMP(4);
    for (long long i = tid; i < A.n; i += stride) ph::scatter_atom(A, C, (int)i);
    if constexpr (kGroupWalk<WALK>) {
        for (long long g = tid; g < C.n_groups; g += stride) ph::group_table(C, (int)g, A.flags);
    } else {
        if (C.tile && lead) A.flags->tile_bad = 1;   // this build writes no local lists
    }
    RB_SYNC();
    MD_STAMP(5);
    for (long long c = tid >> 5; c < C.ncell; c += stride >> 5) ph::sort_cell_warp(A, C, (int)c, threadIdx.x & 31);
    RB_SYNC();
    MD_STAMP(6);
    for (long long k = tid; k < A.n; k += stride) ph::gather_atom(A, (int)k);
    RB_SYNC();
    MD_STAMP(7);
    for (long long k = tid; k < A.n; k += stride) ph::copyback_atom(A, boxes, (int)k);
    RB_SYNC();
    MD_STAMP(8);
    // the group walks need the global rows only when some group does not fit its stage
    const bool rows = !kGroupWalk<WALK> || *reinterpret_cast<volatile int32_t *>(&A.flags->tile_bad);
    if (WALK != kWalkCells || rows) {
        constexpr int LOCAL = WALK == kWalkStaged ? 1 : (WALK == kWalkHalf ? 2 : 0);
        int m;
        if constexpr (G > 0)
            m = ph::build_cells<G, LOCAL>(A, C, boxes, tid >> 5, stride >> 5, threadIdx.x & 31, sp.rl2, sp.band_lo,
                                          sp.band_hi, rows);
        else
            m = ph::build_cells_any<LOCAL>(sp.list_group, A, C, boxes, tid >> 5, stride >> 5, threadIdx.x & 31, sp.rl2,
                                           sp.band_lo, sp.band_hi, rows);
        m = __reduce_max_sync(0xffffffffu, m);
        if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(&A.flags->max_count, m);
    }
    if constexpr (WALK == kWalkPairs) {   // each row's entries j > i first
        RB_SYNC();
        for (long long i = tid >> 5; i < A.n; i += stride >> 5) ph::partition_row_warp(A, boxes, (int)i, threadIdx.x & 31);
    }
    RB_SYNC();
    MD_STAMP(9);
    return true;
#undef MD_STAMP
#undef RB_SYNC
}

// NT threads per block.  SMT: the knot table of species pair (0, 0) (of the only species, or of
// the host species of an alloy) is copied into dynamic shared memory at the start of the launch
// and the passes read it there (one 1024-thread block per SM); other pairs read the global table.
// WALK (kWalkStaged, kWalkCells, kWalkHalf): the passes run over cell groups staged in shared
// memory (md_tile.cuh) whenever every group's neighbourhood fitted the stage at the last build,
// else over atoms through the list.  The cell walk builds no list at a rebuild unless a group
// did not fit (the list walk then needs one).  The half walk adds two phases: F(rho) after the
// density pass and the kicks after the force pass (each waits for every group's shares).

template <int PREC, int T, int KIND, bool MULTI, int NT, bool SMT, int WALK>
__global__ void __launch_bounds__(NT, NT == kThreads ? (PREC == MD_PREC_DF       ? MD_STEP_MIN_BLOCKS_DF
                                                        : WALK == kWalkPairs     ? MD_STEP_MIN_BLOCKS_PAIRS
                                                        : PREC == MD_PREC_FP64   ? MD_STEP_MIN_BLOCKS_FP64
                                                                                 : MD_STEP_MIN_BLOCKS)
                                                      : 1)
    k_step(Atoms A, Cells C, Pot P, StepParams sp, GridBarrier *bar, unsigned long long *stamps) {
    __shared__ int ws[32];
    __shared__ std::conditional_t<kGroupWalk<WALK>, tl::Pipe, int> pipe;   // the group walks' pipeline
    __shared__ uint16_t cells_q[WALK == kWalkCells ? NT / 32 : 1][kCellsQueue];
    // the FP64 pair walk's per-warp sums (flattened rows, T >= kFlatLanes)
    constexpr int kPairSlotsW = WALK == kWalkPairs && T >= ps::kFlatLanes ? ps::kPairSlots(32 / T) : 0;
    __shared__ double pair_sums[kPairSlotsW > 0 ? NT / 32 * kPairSlotsW : 1];
    double *const psum = pair_sums + (threadIdx.x >> 5) * kPairSlotsW;
    extern __shared__ float4 sm_table_f4[];   // [SMT table][stage]
    // The group walks' stage needs the room: their shared copy holds only the rows of the pass
    // under way (the phi rows in the density pass, the derivative rows in the force pass), loaded
    // at the start of each pass (Pot::smt_phi = 0).
    constexpr bool kSplitTable = SMT && kGroupWalk<WALK> && !MULTI && MD_DTABLE;
    float4 *const stage = sm_table_f4 + (SMT ? (kSplitTable ? 1 : 2) * P.nk : 0);
    float4 *const half_acc = stage + (WALK == kWalkHalf ? (size_t)C.nbuf * C.cap : 0);   // half walk: per-slot sums
    const unsigned nb = gridDim.x;
    const long long tid = (long long)blockIdx.x * NT + threadIdx.x;
    const long long stride = (long long)nb * NT;
    if (SMT && !kSplitTable) {
        const float4 *src = reinterpret_cast<const float4 *>(P.VP32);
        if constexpr (!MULTI && MD_DTABLE) {   // derivative rows, then the phi rows
            for (int q = threadIdx.x; q < P.nk; q += NT) {
                sm_table_f4[q] = __ldg(P.D32 + q);
                sm_table_f4[P.nk + q] = __ldg(src + 2 * q + 1);
            }
        } else {
            for (int q = threadIdx.x; q < 2 * P.nk; q += NT) sm_table_f4[(q & 1) * P.nk + (q >> 1)] = __ldg(src + q);
        }
        __syncthreads();
    }
    if constexpr (kGroupWalk<WALK>) {
        if (threadIdx.x == 0) tl::pipe_init<NT>(pipe);
        __syncthreads();
    }
    unsigned seq = 0;   // groups this block has taken in this launch: the pipeline's phase count
    // (withhold_arrival 2: block 0's staging producer releases no group, so that its consumers'
    // bounded waits run out; the self-test of those waits)
    const tl::PassCtl ctl{sp.spin_limit, &bar->abort, A.flags, sp.withhold_arrival == 2 && blockIdx.x == 0};
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    const bool strain = sp.strain_scale != 1.0;
    Box *boxes = A.boxes;
    const long long items = ((long long)A.n * T + 31) / 32 * 32;  // whole warps (lane sums)
    long long step = 0;
    if (lead) step = A.flags->step;
#define MD_SYNC()                                                   \
    do {                                                            \
        if (!grid_sync(bar, nb, sp.spin_limit, A.flags)) return;   \
    } while (0)

    const bool thermo = sp.thermo != nullptr;
    int s0 = 0;
    if (sp.resume) {   // the step was opened by the launch that stopped at its rebuild request
        s0 = *reinterpret_cast<volatile int32_t *>(&A.flags->seg_done);
        if (s0 >= sp.n_steps || (*reinterpret_cast<volatile int32_t *>(&A.flags->error) & FLAG_TIMEOUT)) return;
    } else {
        if (stamps && lead) stamps[0] = globaltimer();
        // first half kick + drift of the first step
        if (strain) {
            if (lead) strain_boxes(boxes, A.n_rep, sp.strain_scale);
            MD_SYNC();
        }
        if (lead && sp.rebuild_every > 0 && (step + 1) % sp.rebuild_every == 0) A.flags->need_rebuild = 1;
        if (thermo) {  // the thermostat half step that opens the first step
            ke_sums(A, sp, tid, stride);
            MD_SYNC();
            thermo_update(sp, A.n_rep, tid, stride, false, true);
            MD_SYNC();
        }
        for (long long i = tid; i < A.n; i += stride) {
            ph::open_step(A, boxes, (int)i, sp.motion, sp.half_dt, sp.dt, sp.strain_scale, strain, sp.lim2,
                          thermo ? sp.thermo : nullptr);
            if constexpr (WALK == kWalkHalf) A.rho_acc[i] = 0.0;
        }
        if (sp.withhold_arrival == 1 && blockIdx.x == 0) {
            // self-test of the bounded wait: this block never arrives; it waits (bounded) until
            // the others have given up and marked the launch aborted, then leaves.
            if (threadIdx.x == 0) {
                unsigned long long polls = 0;
                while (!*reinterpret_cast<volatile int *>(&bar->abort) && ++polls < 4 * sp.spin_limit) __nanosleep(100);
                if (gridDim.x == 1) atomicOr(&A.flags->error, FLAG_TIMEOUT);  // nobody else to give up
            }
            __syncthreads();
            return;
        }
        MD_SYNC();
    }

    unsigned long long *srow = nullptr;
    for (int s = s0; s < sp.n_steps; s++) {
        // (a resumed step keeps the stamps of the launch that stopped and of the rebuild kernel)
        const bool resumed = sp.resume && s == s0;
        if (stamps && lead) {
            srow = stamps + kStampsPerStep * (s + 1);
            if (!resumed) srow[0] = globaltimer();
        }
#define MD_STAMP(q) \
    if (srow) srow[q] = globaltimer()
        // ------------------------------------------------ list rebuild when flagged
        if (ph::rebuild_requested(A.flags)) {
            if (sp.stop_at_rebuild) {   // the rebuild kernel takes it, then a resuming launch
                if (lead) A.flags->seg_done = s;
                return;
            }
            if (!rebuild_phases<WALK>(A, C, boxes, sp, bar, ws, srow)) return;
        } else if (srow && !resumed) {
            const unsigned long long t0 = srow[0];
            for (int q = 1; q <= 9; q++) srow[q] = t0;
        }
        // ------------------------------------------------ density pass
        if constexpr (kSplitTable) {
            const float4 *src = reinterpret_cast<const float4 *>(P.VP32);
            for (int q = threadIdx.x; q < P.nk; q += NT) sm_table_f4[q] = __ldg(src + 2 * q + 1);
            __syncthreads();
        }
        if (lead && A.flags->need_rebuild) {  // every block has passed the rebuild decision
            A.flags->n_rebuilds++;
            A.flags->need_rebuild = 0;
        }
        bool tiled = false;
        if constexpr (kGroupWalk<WALK>) tiled = *reinterpret_cast<volatile int32_t *>(&A.flags->tile_bad) == 0;
        if constexpr (kGroupWalk<WALK>) {
            if (tiled) {
                if (tl::is_producer<NT>()) {
                    tl::produce<WALK == kWalkHalf ? 0 : -1>(A, C, boxes[0], A.posf, pipe, stage, half_acc, seq, ctl);
                } else {
                    for (unsigned q = seq, qe = seq + tl::block_groups(C); q < qe; q++) {
                        int b;
                        if (!tl::acquire(C, pipe, q, ctl, b)) break;
                        const tl::Group G{pipe.hdr[b][1], pipe.hdr[b][2], pipe.hdr[b][3]};
                        const float4 *st = stage + (size_t)b * C.cap;
                        if constexpr (WALK == kWalkCells) {
                            for (int c = tl::claim(pipe, b, 1); c < G.h1 - G.h0; c = tl::claim(pipe, b, 1))
                                tl::density_cell_atom<KIND, SMT>(A, P, st, pipe.loc[b], C.gx + 2, G, G.h0 + c,
                                                                 cells_q[threadIdx.x >> 5]);
                        } else {
                            const int gi = ((G.h1 - G.h0) * T + 31) & ~31;
                            for (int c = tl::claim(pipe, b, 32); c < gi; c = tl::claim(pipe, b, 32)) {
                                const int it = c + (threadIdx.x & 31);
                                if constexpr (WALK == kWalkStaged)
                                    tl::density_item<T, KIND, SMT>(A, P, st, G.h1, G.h0 + it / T, it & (T - 1));
                                else
                                    tl::density_half_item<T, KIND, SMT>(A, P, st, half_acc + (size_t)b * C.cap, G.h1,
                                                                        G.h0 + it / T, it & (T - 1));
                            }
                        }
                        tl::release(pipe, b);
                    }
                }
                seq += tl::block_groups(C);
                if constexpr (WALK == kWalkHalf) {   // F(rho) once every group has added its share
                    MD_SYNC();
                    for (long long i = tid; i < A.n; i += stride) tl::half_embed(A, P, (int)i);
                }
            }
        }
        const bool energy_step = s == sp.n_steps - 1 && sp.energy_last;
        if constexpr (WALK == kWalkPairs) {   // each pair once, then F(rho) once every share is in
            for (long long g = tid; g < items; g += stride)
                ps::density64_pairs<T, KIND>(A, P, boxes, g, energy_step, psum);
            MD_SYNC();
            for (long long i = tid; i < A.n; i += stride) ps::pairs_embed64(A, P, (int)i);
        } else if (!tiled) {
            for (long long g = tid; g < items; g += stride)
                ps::density_item<PREC, T, KIND, MULTI, SMT>(A, P, boxes, g, energy_step);
        }
        MD_SYNC();
        MD_STAMP(10);
        if constexpr (kSplitTable) {   // every warp of the block has left the density pass (barrier above)
            for (int q = threadIdx.x; q < P.nk; q += NT) sm_table_f4[q] = __ldg(P.D32 + q);
            __syncthreads();
        }
        // ------------------------------------------------ force pass (+ kicks)
        const bool last = s == sp.n_steps - 1;
        const bool fuse = !last && !strain && !thermo;
        if (fuse && lead && sp.rebuild_every > 0 && (step + s + 2) % sp.rebuild_every == 0)
            A.flags->need_rebuild = 1;
        double part[kPartials];
#pragma unroll
        for (int q = 0; q < kPartials; q++) part[q] = 0.0;
        if (last && sp.energy_last) {
            if constexpr (kGroupWalk<WALK>) {
                if (tiled) {
                    if (tl::is_producer<NT>()) {
                        tl::produce<WALK == kWalkHalf ? 1 : -1>(A, C, boxes[0], A.p2f, pipe, stage, half_acc, seq, ctl);
                    } else {
                        for (unsigned q = seq, qe = seq + tl::block_groups(C); q < qe; q++) {
                            int b;
                            if (!tl::acquire(C, pipe, q, ctl, b)) break;
                            const tl::Group G{pipe.hdr[b][1], pipe.hdr[b][2], pipe.hdr[b][3]};
                            const float4 *st = stage + (size_t)b * C.cap;
                            if constexpr (WALK == kWalkCells) {
                                for (int c = tl::claim(pipe, b, 1); c < G.h1 - G.h0; c = tl::claim(pipe, b, 1))
                                    tl::force_cell_atom<KIND, true, SMT>(A, P, boxes, st, pipe.loc[b], C.gx + 2, G,
                                                                         G.h0 + c, cells_q[threadIdx.x >> 5], sp.half_dt,
                                                                         sp.dt, sp.lim2, false, part);
                            } else {
                                const int gi = ((G.h1 - G.h0) * T + 31) & ~31;
                                for (int c = tl::claim(pipe, b, 32); c < gi; c = tl::claim(pipe, b, 32)) {
                                    const int it = c + (threadIdx.x & 31);
                                    if constexpr (WALK == kWalkStaged)
                                        tl::force_item<T, KIND, true, SMT>(A, P, st, G.h1, G.h0 + it / T, it & (T - 1),
                                                                           sp.half_dt, true, part);
                                    else
                                        tl::force_half_item<T, KIND, true, SMT>(A, P, st, half_acc + (size_t)b * C.cap,
                                                                                G.h1, G.h0 + it / T, it & (T - 1), part);
                                }
                            }
                            tl::release(pipe, b);
                        }
                    }
                    seq += tl::block_groups(C);
                    if constexpr (WALK == kWalkHalf) {   // the kick once every group has added its share
                        MD_SYNC();
                        for (long long i = tid; i < A.n; i += stride) tl::half_kick<true>(A, (int)i, sp.half_dt, part);
                    }
                }
            }
            if constexpr (WALK == kWalkPairs) {   // each pair once, then the kicks once every share is in
                for (long long g = tid; g < items; g += stride)
                    ps::force64_pairs<T, KIND, true>(A, P, boxes, g, part, psum);
                MD_SYNC();
                for (long long i = tid; i < A.n; i += stride) ps::pairs_kick64<true>(A, (int)i, sp.half_dt, sp.motion, part);
            } else if (!tiled) {
                for (long long g = tid; g < items; g += stride)
                    ps::force_item<PREC, T, KIND, MULTI, true, SMT>(A, P, boxes, g, sp.half_dt, sp.motion, part);
            }
            eam::block_partials<NT>(part, A.partials, A.part_stride);
        } else {
            if constexpr (kGroupWalk<WALK>) {
                if (tiled) {
                    if (tl::is_producer<NT>()) {
                        tl::produce<WALK == kWalkHalf ? 1 : -1>(A, C, boxes[0], A.p2f, pipe, stage, half_acc, seq, ctl);
                    } else {
                        for (unsigned q = seq, qe = seq + tl::block_groups(C); q < qe; q++) {
                            int b;
                            if (!tl::acquire(C, pipe, q, ctl, b)) break;
                            const tl::Group G{pipe.hdr[b][1], pipe.hdr[b][2], pipe.hdr[b][3]};
                            const float4 *st = stage + (size_t)b * C.cap;
                            if constexpr (WALK == kWalkCells) {
                                for (int c = tl::claim(pipe, b, 1); c < G.h1 - G.h0; c = tl::claim(pipe, b, 1))
                                    tl::force_cell_atom<KIND, false, SMT>(A, P, boxes, st, pipe.loc[b], C.gx + 2, G,
                                                                         G.h0 + c, cells_q[threadIdx.x >> 5], sp.half_dt,
                                                                         sp.dt, sp.lim2, fuse, part);
                            } else {
                                const int gi = ((G.h1 - G.h0) * T + 31) & ~31;
                                for (int c = tl::claim(pipe, b, 32); c < gi; c = tl::claim(pipe, b, 32)) {
                                    const int it = c + (threadIdx.x & 31);
                                    if constexpr (WALK == kWalkStaged) {
                                        const int i = tl::force_item<T, KIND, false, SMT>(
                                            A, P, st, G.h1, G.h0 + it / T, it & (T - 1), sp.half_dt, true, part);
                                        if (fuse && i >= 0)
                                            ph::kick_drift(A, boxes, i, sp.half_dt, sp.dt, sp.strain_scale, false,
                                                           sp.lim2);
                                    } else {
                                        tl::force_half_item<T, KIND, false, SMT>(A, P, st, half_acc + (size_t)b * C.cap,
                                                                                 G.h1, G.h0 + it / T, it & (T - 1), part);
                                    }
                                }
                            }
                            tl::release(pipe, b);
                        }
                    }
                    seq += tl::block_groups(C);
                    if constexpr (WALK == kWalkHalf) {   // the kicks once every group has added its share
                        MD_SYNC();
                        for (long long i = tid; i < A.n; i += stride) {
                            tl::half_kick<false>(A, (int)i, sp.half_dt, part);
                            if (fuse) ph::kick_drift(A, boxes, (int)i, sp.half_dt, sp.dt, sp.strain_scale, false, sp.lim2);
                        }
                    }
                }
            }
            if constexpr (WALK == kWalkPairs) {
                for (long long g = tid; g < items; g += stride)
                    ps::force64_pairs<T, KIND, false>(A, P, boxes, g, part, psum);
                MD_SYNC();
                for (long long i = tid; i < A.n; i += stride) {
                    ps::pairs_kick64<false>(A, (int)i, sp.half_dt, sp.motion, part);
                    if (fuse) ph::open_step(A, boxes, (int)i, sp.motion, sp.half_dt, sp.dt, sp.strain_scale, false, sp.lim2);
                }
            } else if (!tiled) {
                for (long long g = tid; g < items; g += stride) {
                    const int i = ps::force_item<PREC, T, KIND, MULTI, false, SMT>(A, P, boxes, g, sp.half_dt,
                                                                                   sp.motion, part);
                    if (fuse && i >= 0)
                        ph::open_step(A, boxes, i, sp.motion, sp.half_dt, sp.dt, sp.strain_scale, false, sp.lim2);
                }
            }
        }
        MD_SYNC();
        MD_STAMP(11);
        if (thermo) {
            // close this step and open the next with thermostat half steps
            ke_sums(A, sp, tid, stride);
            MD_SYNC();
            thermo_update(sp, A.n_rep, tid, stride, true, !last);
            if (!last && lead) {
                if (strain) strain_boxes(boxes, A.n_rep, sp.strain_scale);
                if (sp.rebuild_every > 0 && (step + s + 2) % sp.rebuild_every == 0) A.flags->need_rebuild = 1;
            }
            MD_SYNC();
            if (!last) {
                for (long long i = tid; i < A.n; i += stride)
                    ph::kick_drift(A, boxes, (int)i, sp.half_dt, sp.dt, sp.strain_scale, strain, sp.lim2, sp.thermo);
                MD_SYNC();
            } else {
                for (long long i = tid; i < A.n; i += stride) {
                    const double sb = sp.thermo[ph::replica_of(A, (int)i)].s_b;
                    double4_32a v = A.vel[i];
                    v.x = __dmul_rn(v.x, sb);
                    v.y = __dmul_rn(v.y, sb);
                    v.z = __dmul_rn(v.z, sb);
                    A.vel[i] = v;
                }
            }
        } else if (!last && strain) {
            if (lead) {
                strain_boxes(boxes, A.n_rep, sp.strain_scale);
                if (sp.rebuild_every > 0 && (step + s + 2) % sp.rebuild_every == 0) A.flags->need_rebuild = 1;
            }
            MD_SYNC();
            for (long long i = tid; i < A.n; i += stride)
                ph::kick_drift(A, boxes, (int)i, sp.half_dt, sp.dt, sp.strain_scale, true, sp.lim2);
            MD_SYNC();
        }
    }
    if (lead) {
        A.flags->step = step + sp.n_steps;
        A.flags->seg_done = sp.n_steps;
    }
#undef MD_STAMP
#undef MD_SYNC
}


template <int PREC, int T, int KIND, bool MULTI, int NT = kThreads, bool SMT = false, int WALK = kWalkList>
cudaError_t launch_t(const Atoms &A, const Cells &C, const Pot &P, const StepParams &sp, GridBarrier *bar,
                     unsigned long long *stamps, int *grid_out, cudaStream_t s) {
    static int per_sm = -1;
    static int n_sm = 0;
    static size_t per_sm_dyn = 0;
    static bool attr = false;
    const size_t dyn_max = WALK == kWalkCells ? kSmemDynMaxCells : kSmemDynMax;
    constexpr bool kSplitTable = SMT && kGroupWalk<WALK> && !MULTI && MD_DTABLE;
    const size_t dyn = (SMT ? (size_t)P.nk * (kSplitTable ? 16 : 32) : 0) +
                       (kGroupWalk<WALK> ? (size_t)C.nbuf * C.cap * sizeof(float4) * (WALK == kWalkHalf ? 2 : 1) : 0);
    if (dyn > dyn_max) return cudaErrorInvalidConfiguration;
    if ((SMT || kGroupWalk<WALK>) && !attr) {  // opt in to a large dynamic shared-memory carve-out (once)
        cudaError_t e = cudaFuncSetAttribute(k_step<PREC, T, KIND, MULTI, NT, SMT, WALK>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_max);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    if (per_sm < 0 || dyn != per_sm_dyn) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step<PREC, T, KIND, MULTI, NT, SMT, WALK>, NT,
                                                              dyn);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        per_sm_dyn = dyn;
    }
    const long long work = std::max<long long>((long long)A.n * T, (long long)C.ncell);
    const int need = (int)std::max<long long>(1, (work + NT - 1) / NT);
    const int grid = std::max(1, std::min(per_sm * n_sm, need));
    if (grid_out) *grid_out = grid;
    if (sp.n_steps <= 0) return cudaSuccess;  // preparation only (attributes, occupancy): no launch
    cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(GridBarrier), s);
    if (e != cudaSuccess) return e;
    Atoms a = A;
    Cells c = C;
    Pot p = P;
    if (kSplitTable) p.smt_phi = 0;
    StepParams q = sp;
    void *args[] = {&a, &c, &p, &q, &bar, &stamps};
    return cudaLaunchCooperativeKernel((const void *)k_step<PREC, T, KIND, MULTI, NT, SMT, WALK>, dim3(grid), dim3(NT),
                                       args, dyn, s);
}

// The rebuild between two launches of the step kernel (md_internal.cuh launch_rebuild_step).
constexpr int kRebuildThreads = 256;
#ifndef MD_REBUILD_MIN_BLOCKS   // blocks of kRebuildThreads per SM the rebuild kernel is built for
#define MD_REBUILD_MIN_BLOCKS 4
#endif

template <int WALK, int G>
__global__ void __launch_bounds__(kRebuildThreads, MD_REBUILD_MIN_BLOCKS)
    k_rebuild(Atoms A, Cells C, StepParams sp, GridBarrier *bar, unsigned long long *stamps) {
    __shared__ int ws[32];
    // every block reads the same words, written before this launch: all take part or none
    const int s = *reinterpret_cast<volatile int32_t *>(&A.flags->seg_done);
    if (s >= sp.n_steps || !ph::rebuild_requested(A.flags) ||
        (*reinterpret_cast<volatile int32_t *>(&A.flags->error) & FLAG_TIMEOUT))
        return;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    unsigned long long *srow = stamps && lead ? stamps + kStampsPerStep * (s + 1) : nullptr;
    if (!rebuild_phases<WALK, G>(A, C, A.boxes, sp, bar, ws, srow)) return;
    if (lead) {   // every block has passed the rebuild decision (the barriers above)
        A.flags->n_rebuilds++;
        A.flags->need_rebuild = 0;
    }
}

template <int WALK, int G>
cudaError_t launch_rebuild_g(const Atoms &A, const Cells &C, const StepParams &sp, GridBarrier *bar,
                             unsigned long long *stamps, cudaStream_t s) {
    static int grid = 0;
    if (grid == 0) {
        int dev = 0, n_sm = 0, per_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rebuild<WALK, G>, kRebuildThreads, 0);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        grid = per_sm * n_sm;
    }
    cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(GridBarrier), s);
    if (e != cudaSuccess) return e;
    Atoms a = A;
    Cells c = C;
    StepParams q = sp;
    void *args[] = {&a, &c, &q, &bar, &stamps};
    return cudaLaunchCooperativeKernel((const void *)k_rebuild<WALK, G>, dim3(grid), dim3(kRebuildThreads), args, 0,
                                       s);
}

template <int WALK>
cudaError_t launch_rebuild_t(const Atoms &A, const Cells &C, const StepParams &sp, GridBarrier *bar,
                             unsigned long long *stamps, cudaStream_t s) {
    switch (sp.list_group) {
        case 4: return launch_rebuild_g<WALK, 4>(A, C, sp, bar, stamps, s);
        case 8: return launch_rebuild_g<WALK, 8>(A, C, sp, bar, stamps, s);
        case 16: return launch_rebuild_g<WALK, 16>(A, C, sp, bar, stamps, s);
        default: return launch_rebuild_g<WALK, 32>(A, C, sp, bar, stamps, s);
    }
}

template <int PREC, int T>
cudaError_t launch_kind(const Atoms &A, const Cells &C, const Pot &P, const StepParams &sp, GridBarrier *bar,
                        unsigned long long *stamps, int *grid_out, cudaStream_t s) {
    if constexpr (PREC == MD_PREC_DF) {   // one species, knot tables
        if (P.kind != MD_POT_TABLES || P.ns != 1) return cudaErrorInvalidValue;
        return launch_t<PREC, T, MD_POT_TABLES, false>(A, C, P, sp, bar, stamps, grid_out, s);
    } else {
        if constexpr (PREC == MD_PREC_FP64) {   // each pair once: one species, FS or tables
            if (A.pairs) {
                if (P.kind == MD_POT_FS_ANALYTIC)
                    return launch_t<PREC, T, MD_POT_FS_ANALYTIC, false, kThreads, false, kWalkPairs>(A, C, P, sp, bar,
                                                                                                    stamps, grid_out, s);
                if (P.kind == MD_POT_TABLES && P.ns == 1)
                    return launch_t<PREC, T, MD_POT_TABLES, false, kThreads, false, kWalkPairs>(A, C, P, sp, bar, stamps,
                                                                                               grid_out, s);
                return cudaErrorInvalidValue;
            }
        }
        if (P.kind == MD_POT_FS_ANALYTIC)
            return launch_t<PREC, T, MD_POT_FS_ANALYTIC, false>(A, C, P, sp, bar, stamps, grid_out, s);
        if (P.kind == MD_POT_KNOTS)
            return P.ns == 1 ? launch_t<PREC, T, MD_POT_KNOTS, false>(A, C, P, sp, bar, stamps, grid_out, s)
                             : launch_t<PREC, T, MD_POT_KNOTS, true>(A, C, P, sp, bar, stamps, grid_out, s);
        if (P.ns == 1) {
            if (smem_table_bytes(P.kind, P.ns, PREC, P.nk) > 0) {
                if constexpr (PREC == MD_PREC_MIXED && T <= 8) {
                    if (C.tile == kWalkStaged)
                        return launch_t<PREC, T, MD_POT_TABLES, false, 1024, true, kWalkStaged>(A, C, P, sp, bar, stamps,
                                                                                               grid_out, s);
                    if (C.tile == kWalkCells)
                        return launch_t<PREC, T, MD_POT_TABLES, false, 1024, true, kWalkCells>(A, C, P, sp, bar, stamps,
                                                                                              grid_out, s);
                    if (C.tile == kWalkHalf)
                        return launch_t<PREC, T, MD_POT_TABLES, false, 1024, true, kWalkHalf>(A, C, P, sp, bar, stamps,
                                                                                             grid_out, s);
                }
                return launch_t<PREC, T, MD_POT_TABLES, false, MD_SMT_THREADS, true>(A, C, P, sp, bar, stamps, grid_out,
                                                                                    s);
            }
            return launch_t<PREC, T, MD_POT_TABLES, false>(A, C, P, sp, bar, stamps, grid_out, s);
        }
        // several species: the table of pair (0, 0), the host species, in shared memory
        if (MD_SMEM_TABLE && PREC == MD_PREC_MIXED && (size_t)P.nk * 32 <= kSmemTableMax)
            return launch_t<PREC, T, MD_POT_TABLES, true, MD_SMT_THREADS, true>(A, C, P, sp, bar, stamps, grid_out, s);
        return launch_t<PREC, T, MD_POT_TABLES, true>(A, C, P, sp, bar, stamps, grid_out, s);
    }
}

}  // namespace st

// One launcher per (precision, lanes per atom), each defined in its own translation unit
// (md_step_{m,d,e}_{a,b,c}.cu: the instantiations compile in parallel); md_step_dispatch.cu picks.
#define MD_STEP_FN(P, T) launch_step_##P##_l##T
#define MD_STEP_DECL(P, T)                                                                                  \
    cudaError_t MD_STEP_FN(P, T)(const Atoms &A, const Cells &C, const Pot &Pt, const StepParams &sp,     \
                                 GridBarrier *bar, unsigned long long *stamps, int *grid_out, cudaStream_t s)
#define MD_STEP_DEFINE(P, PREC, T)                                                                          \
    MD_STEP_DECL(P, T) { return st::launch_kind<PREC, T>(A, C, Pt, sp, bar, stamps, grid_out, s); }
MD_STEP_DECL(m, 1); MD_STEP_DECL(m, 2); MD_STEP_DECL(m, 4); MD_STEP_DECL(m, 8); MD_STEP_DECL(m, 16); MD_STEP_DECL(m, 32);
MD_STEP_DECL(d, 1); MD_STEP_DECL(d, 2); MD_STEP_DECL(d, 4); MD_STEP_DECL(d, 8); MD_STEP_DECL(d, 16); MD_STEP_DECL(d, 32);
MD_STEP_DECL(e, 1); MD_STEP_DECL(e, 2); MD_STEP_DECL(e, 4); MD_STEP_DECL(e, 8); MD_STEP_DECL(e, 16); MD_STEP_DECL(e, 32);

}  // namespace mdk
