// Staged passes of the mixed-precision step kernel: the two EAM passes of Eq. (1) over cell
// groups instead of single atoms.  One block takes one group at a time: gx consecutive link
// cells along x (the home cells) whose neighbourhood, the 3 x 3 x (gx + 2) stencil of cells
// around them, the block copies into shared memory with each periodic image's shift already
// added (§3.2.1's link cells, here as a unit of data reuse).  Two neighbour walks read the
// stage.  In the staged walk every home atom reads its neighbours through its 16-bit local list
// (the same entries as the global list, as staged slots), so a pair costs a shared-memory load
// instead of a scattered global one and needs no minimum image.
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
// Slot layout of a stage: stencil cell s = ((dz + 1) 3 + (dy + 1)) (gx + 2) + (x - x0 + 1) holds its
// atoms in cell order from slot grp_loc[g][s]; the home atoms of the group are contiguous in the
// global cell order (cells x0 .. x0 + len - 1 of one row).
#pragma once

#include <cuda_runtime.h>

#include "md_passes.cuh"

namespace mdk {
namespace tl {

// Stencil cells of a group of at most kTileMaxGx cells, and the slot table (with the total).
constexpr int kTileMaxGx = 8;
constexpr int kTileMaxSt = 9 * (kTileMaxGx + 2);

struct Group {
    int h0, h1;   // home atoms [h0, h1) (global slots)
    int len;      // home cells
};

// Stencil cell q of group g: the link cell it stages and the periodic shift of its image.
struct StencilCell {
    int c;
    float sx, sy, sz;
};

__device__ __forceinline__ StencilCell stencil_cell(const Cells &C, const RepCells &rg, const Box &B, int g, int q) {
    const int nx = rg.nc[0], ny = rg.nc[1], nz = rg.nc[2];
    const int gxi = g % C.ngx, row = g / C.ngx, y = row % ny, z = row / ny;
    const int W = C.gx + 2, xs = q % W, rr = q / W;
    int xx = gxi * C.gx - 1 + xs, yy = y + rr % 3 - 1, zz = z + rr / 3 - 1;
    StencilCell s{0, 0.f, 0.f, 0.f};
    if (xx < 0) { xx += nx; s.sx = -B.Lf[0]; } else if (xx >= nx) { xx -= nx; s.sx = B.Lf[0]; }
    if (yy < 0) { yy += ny; s.sy = -B.Lf[1]; } else if (yy >= ny) { yy -= ny; s.sy = B.Lf[1]; }
    if (zz < 0) { zz += nz; s.sz = -B.Lf[2]; } else if (zz >= nz) { zz -= nz; s.sz = B.Lf[2]; }
    s.c = rg.base + (zz * ny + yy) * nx + xx;
    return s;
}

// Copy group g's stencil from src (float4 per atom, x y z in Å, w kept) into st, shifting each
// periodic image by its box edge, and clear acc (the half walk's accumulators; NULL: none).
// loc receives the group's slot table.  Returns the home range.
template <int NT>
__device__ __forceinline__ Group stage_group(const Cells &C, const Box &B, const float4 *src, int g, float4 *st,
                                             int *loc, float4 *acc = nullptr) {
    const RepCells rg = C.rc[0];
    const int nx = rg.nc[0], ny = rg.nc[1];
    const int gxi = g % C.ngx, row = g / C.ngx, y = row % ny, z = row / ny;
    const int x0 = gxi * C.gx, len = min(C.gx, nx - x0);
    const int32_t *gl = C.grp_loc + (size_t)g * (C.st_cells + 1);
    __syncthreads();   // the previous group's stage, accumulators and table are no longer read
    for (int q = threadIdx.x; q <= C.st_cells; q += NT) loc[q] = gl[q];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int q = warp; q < C.st_cells; q += NT / 32) {
        const int n = loc[q + 1] - loc[q];
        if (n == 0) continue;   // an empty cell, or a slot past the end of a shorter last group
        const StencilCell sc = stencil_cell(C, rg, B, g, q);
        const int js = C.cell_start[sc.c];
        float4 *dst = st + loc[q];
        for (int t = lane; t < n; t += 32) {
            float4 v = src[js + t];
            v.x += sc.sx;
            v.y += sc.sy;
            v.z += sc.sz;
            dst[t] = v;
            if (acc) acc[loc[q] + t] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    const int c0 = rg.base + (z * ny + y) * nx + x0;
    Group G{C.cell_start[c0], C.cell_start[c0 + len], len};
    __syncthreads();
    return G;
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

// Density pass of group G by the cell walk: warp w of the block takes home atoms w, w + NT/32, ...
template <int NT, int KIND, bool SMT>
__device__ __forceinline__ void density_cells(const Atoms &A, const Pot &P, const float4 *st, const int *loc, int W,
                                              const Group &G, uint16_t *q) {
    const int lane = threadIdx.x & 31;
    const int home0 = loc[4 * W + 1];   // stage slot of the first home atom
    for (int i = G.h0 + (threadIdx.x >> 5); i < G.h1; i += NT / 32) {
        const int si = home0 + (i - G.h0);
        const float4 pi = st[si];       // a home cell is never shifted: the atom's own coordinates
        float hi = 0.f, lo = 0.f;
        unsigned viol = 0;
        cells_scan(st, loc, W, home_cell(loc, W, G.len, si), si, pi, P.rc2f, q, [&](const float4 &pj) {
            ps::two_sum_add(hi, lo, ps::rho_term32<KIND, false, SMT>(P, 0, 0, pj.x - pi.x, pj.y - pi.y, pj.z - pi.z,
                                                                      viol));
        });
        if (viol) atomicAdd(&A.flags->range_violations, (unsigned long long)viol);
        ps::lane_sum_df<32>(hi, lo);
        if (lane == 0) ps::density32_finish(A, P, i, 0, pi, hi, lo);
    }
}

// Force pass of group G by the cell walk (+ the second half kick, and with fuse the next step's
// first half kick and drift, as in the list walk).
template <int NT, int KIND, bool ENERGY, bool SMT>
__device__ __forceinline__ void force_cells(const Atoms &A, const Pot &P, const Box *boxes, const float4 *st,
                                            const int *loc, int W, const Group &G, uint16_t *q, double half_dt,
                                            double dt, double lim2, bool fuse, double (&part)[kPartials]) {
    const int lane = threadIdx.x & 31;
    const int home0 = loc[4 * W + 1];
    for (int i = G.h0 + (threadIdx.x >> 5); i < G.h1; i += NT / 32) {
        const int si = home0 + (i - G.h0);
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
}

// ---- half walk (Newton's third law) ----
// Home atom i takes the pairs of its half row (the neighbours j > i in cell order, as stage
// slots): its own sums stay in registers and go to the FP64 accumulators once; the neighbour's
// share goes to its stage slot's FP32 accumulator in shared memory (a shared atomic add), which
// flush_group adds to the FP64 accumulators once per group.

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

// Add the stage accumulators of group g (all its pair terms done) to the FP64 accumulators:
// the density (x) when !FORCE, else the force (x, y, z) and pair energy (w).
template <int NT, bool FORCE>
__device__ __forceinline__ void flush_group(const Atoms &A, const Cells &C, const Box &B, int g, const float4 *acc,
                                            const int *loc) {
    __syncthreads();
    const RepCells rg = C.rc[0];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int q = warp; q < C.st_cells; q += NT / 32) {
        const int n = loc[q + 1] - loc[q];
        if (n == 0) continue;
        const int js = C.cell_start[stencil_cell(C, rg, B, g, q).c];
        for (int t = lane; t < n; t += 32) {
            const float4 a = acc[loc[q] + t];
            if (FORCE) {
                if (a.x != 0.f || a.y != 0.f || a.z != 0.f || a.w != 0.f) {
                    double4_32a *f = A.f_acc + js + t;
                    atomicAdd(&f->x, (double)a.x);
                    atomicAdd(&f->y, (double)a.y);
                    atomicAdd(&f->z, (double)a.z);
                    if (a.w != 0.f) atomicAdd(&f->w, (double)a.w);
                }
            } else if (a.x != 0.f) {
                atomicAdd(&A.rho_acc[js + t], (double)a.x);
            }
        }
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
