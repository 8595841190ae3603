// Neighbour gathers of the learned per-atom surrogate: descriptors, forces, and the
// descriptor tangent used by the force term of the training loss.  One warp per atom, lane k
// = radial-basis channel k (32 channels = 32 lanes).  The lanes first evaluate the geometry of
// 32 list entries at once (lane q: entry q), stage it in shared memory, and then all lanes walk
// the entries inside the descriptor cutoff, each adding its own channel.  The per-channel
// quantities of neighbour j (its gradient row g_j) are then one coalesced 128-byte row read.
//
//   descriptors  G_ik = sum_j b_k(r_ij)
//   forces       F_i  = sum_j [ sum_k (g_ik + g_jk) b_k'(r_ij) ] (r_j - r_i) / r_ij
//   tangent      u_ik = sum_j b_k'(r_ij) (r_j - r_i) / r_ij . (phi_j - phi_i),  phi = dL/dF
// with g = dE/dG.  The pair coefficient is symmetric in (i, j), so the forces are central pair
// forces and the virial has the pair form.  FP32 arithmetic; FP64 kick and partial sums.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "md_eam_common.cuh"
#include "md_phases.cuh"

namespace mdk {

namespace {

constexpr int kWarps = kThreads / 32;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float mi(float d, float L, float iL) { return d - L * rintf(d * iL); }

// Per-pair constants of one chunk of list entries, compacted: the pairs inside rd occupy
// slots 0 .. n-1 in list order.  P0 = (r, fc, fc', j bits), P1 = (unit vector, fc / w^2).
struct Stage {
    float4 P0[kWarps][32];
    float4 P1[kWarps][32];
};

// Geometry of list entries [base, base + 32) of atom i into the compacted slots; returns the
// number of pairs inside rd.
__device__ __forceinline__ int stage_chunk(const Atoms &A, const SurNet &S, const float4 &pi, const Box &B,
                                           const NbrRow &row, int cnt, int base, int lane, float4 *P0,
                                           float4 *P1) {
    const int q = base + lane;
    const bool valid = q < cnt;
    const int j = valid ? __ldg(row.ptr(q)) : 0;
    const float4 pj = __ldg(A.posf + j);
    const float dx = mi(pj.x - pi.x, B.Lf[0], B.invLf[0]);
    const float dy = mi(pj.y - pi.y, B.Lf[1], B.invLf[1]);
    const float dz = mi(pj.z - pi.z, B.Lf[2], B.invLf[2]);
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const bool inside = valid && r2 < S.rd2 && r2 > 0.f;
    const unsigned m = __ballot_sync(kFull, inside);
    if (inside) {
        const float rinv = rsqrtf(r2);
        const float r = r2 * rinv;
        float sn, cs;
        __sincosf(S.pi_rd * r, &sn, &cs);
        const float fc = 0.5f * (cs + 1.f);
        const int slot = __popc(m & ((1u << lane) - 1u));
        P0[slot] = make_float4(r, fc, -0.5f * S.pi_rd * sn, __int_as_float(j));
        P1[slot] = make_float4(dx * rinv, dy * rinv, dz * rinv, fc * S.invw2);
    }
    __syncwarp();
    return __popc(m);
}

// 2^x (PTX ex2.approx.ftz: relative error < 2^-22).
__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

constexpr float kLog2e = 1.4426950408889634f;

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

// ---------------------------------------------------------------- descriptors
// FP32 rows G[i][k] (S.G), or, for the tensor-core network, the standardised input
// x = (G - gmu) ginv rounded to bf16 in the 128-atom tile layout the MMA reads (S.Gt):
// tile t = i / 128, row r = i % 128, column k at byte t*8192 + (r/8)*512 + (k/8)*128 + (r%8)*16 + (k%8)*2.
__global__ void __launch_bounds__(kThreads) k_sur_desc(Atoms A, SurNet S, int a0, int a1, int bf16) {
    __shared__ Stage st;
    __shared__ __align__(16) __nv_bfloat16 out[kWarps][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const float mu = S.mu0 + S.dmu * (float)lane;
    const float kx = -S.inv2w2 * kLog2e;   // b = 2^(kx a^2) fc
    const float gm = S.gmu[lane], gi = S.ginv[lane];
    for (long long i0 = a0 + (long long)blockIdx.x * kWarps + w; i0 < a1; i0 += (long long)gridDim.x * kWarps) {
        const int i = (int)i0;
        const Box &B = A.boxes[ph::replica_of(A, i)];
        const float4 pi = A.posf[i];
        const int cnt = min(A.count[i], A.k_max);
        const NbrRow row = nbr_row(A, i);
        float G = 0.f, G2 = 0.f;
        for (int base = 0; base < cnt; base += 32) {
            const int np = stage_chunk(A, S, pi, B, row, cnt, base, lane, st.P0[w], st.P1[w]);
            int q = 0;
            for (; q + 1 < np; q += 2) {
                const float2 p0 = *reinterpret_cast<const float2 *>(&st.P0[w][q]);
                const float2 p1 = *reinterpret_cast<const float2 *>(&st.P0[w][q + 1]);
                const float a0_ = p0.x - mu, a1_ = p1.x - mu;
                G = fmaf(ex2(kx * a0_ * a0_), p0.y, G);
                G2 = fmaf(ex2(kx * a1_ * a1_), p1.y, G2);
            }
            if (q < np) {
                const float2 p0 = *reinterpret_cast<const float2 *>(&st.P0[w][q]);
                const float a0_ = p0.x - mu;
                G = fmaf(ex2(kx * a0_ * a0_), p0.y, G);
            }
            __syncwarp();
        }
        G += G2;
        if (bf16) {
            out[w][lane] = __float2bfloat16_rn((G - gm) * gi);
            __syncwarp();
            if (lane < 4) {
                const int r = i & (kSurTile - 1);
                const size_t off = (size_t)(i / kSurTile) * kSurTileBytes + (r >> 3) * 512 + lane * 128 + (r & 7) * 16;
                *reinterpret_cast<uint4 *>(S.Gt + off) = reinterpret_cast<const uint4 *>(out[w])[lane];
            }
            __syncwarp();
        } else {
            S.G[(size_t)i * kSurNb + lane] = G;
        }
    }
}

// ---------------------------------------------------------------- forces (+ kick, partials)
// phi_scale > 0 (training): also phi_i = phi_scale (F_i - Fref_i) and part[0] = sum |F_i - Fref_i|^2.
template <bool ENERGY, bool TRAIN>
__global__ void __launch_bounds__(kThreads) k_sur_force(Atoms A, SurNet S, int a0, int a1, int kick, double half_dt,
                                                        float phi_scale) {
    __shared__ Stage st;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const float mu = S.mu0 + S.dmu * (float)lane;
    const float kx = -S.inv2w2 * kLog2e;
    double part[kPartials];
#pragma unroll
    for (int q = 0; q < kPartials; q++) part[q] = 0.0;
    for (long long i0 = a0 + (long long)blockIdx.x * kWarps + w; i0 < a1; i0 += (long long)gridDim.x * kWarps) {
        const int i = (int)i0;
        const Box &B = A.boxes[ph::replica_of(A, i)];
        const float4 pi = A.posf[i];
        const int cnt = min(A.count[i], A.k_max);
        const NbrRow row = nbr_row(A, i);
        const float gi = S.g[(size_t)i * kSurNb + lane];
        float fx = 0.f, fy = 0.f, fz = 0.f;
        float wxx = 0.f, wyy = 0.f, wzz = 0.f, wyz = 0.f, wxz = 0.f, wxy = 0.f;
        // one pair: c = (g_ik + g_jk) b_k'(r) (this lane's channel), f += c * unit vector;
        // on the energy step the virial -1/2 c r u (x) u
        auto pair = [&](const float4 &p0, const float4 &p1, float gj) {
            const float a = p0.x - mu;
            const float bp = ex2(kx * a * a) * fmaf(-a, p1.w, p0.z);   // b_k'(r)
            const float c = (gi + gj) * bp;
            fx = fmaf(c, p1.x, fx);
            fy = fmaf(c, p1.y, fy);
            fz = fmaf(c, p1.z, fz);
            if (ENERGY && !TRAIN) {
                const float h = -0.5f * c * p0.x;
                wxx = fmaf(h * p1.x, p1.x, wxx);
                wyy = fmaf(h * p1.y, p1.y, wyy);
                wzz = fmaf(h * p1.z, p1.z, wzz);
                wyz = fmaf(h * p1.y, p1.z, wyz);
                wxz = fmaf(h * p1.x, p1.z, wxz);
                wxy = fmaf(h * p1.x, p1.y, wxy);
            }
        };
        // the g_j rows of 8 pairs are loaded before any of them is used (8 independent loads in
        // flight per lane), then the 8 pairs are added
        constexpr int kBatch = 8;
        for (int base = 0; base < cnt; base += 32) {
            const int np = stage_chunk(A, S, pi, B, row, cnt, base, lane, st.P0[w], st.P1[w]);
            for (int q0 = 0; q0 < np; q0 += kBatch) {
                float gj[kBatch];
#pragma unroll
                for (int u = 0; u < kBatch; u++) {
                    const int q = min(q0 + u, np - 1);
                    gj[u] = __ldg(S.g + (size_t)__float_as_int(st.P0[w][q].w) * kSurNb + lane);
                }
#pragma unroll
                for (int u = 0; u < kBatch; u++)
                    if (q0 + u < np) pair(st.P0[w][q0 + u], st.P1[w][q0 + u], gj[u]);
            }
            __syncwarp();
        }
        fx = warp_sum(fx);
        fy = warp_sum(fy);
        fz = warp_sum(fz);
        if (ENERGY && !TRAIN) {
            wxx = warp_sum(wxx); wyy = warp_sum(wyy); wzz = warp_sum(wzz);
            wyz = warp_sum(wyz); wxz = warp_sum(wxz); wxy = warp_sum(wxy);
        }
        if (lane == 0) {
            A.force[i] = make_double4_32a(fx, fy, fz, 0.0);
            if (!isfinite(fx + fy + fz)) atomicOr(&A.flags->error, FLAG_NONFINITE);
            if (TRAIN) {
                const double4_32a fr = S.fref[i];
                const float ex = fx - (float)fr.x, ey = fy - (float)fr.y, ez = fz - (float)fr.z;
                S.phi[i] = make_float4(phi_scale * ex, phi_scale * ey, phi_scale * ez, 0.f);
                part[0] += (double)ex * ex + (double)ey * ey + (double)ez * ez;
            } else {
                double4_32a v = A.vel[i];
                eam::kick_and_partials(v, fx, fy, fz, half_dt, kick != 0);
                if (kick) A.vel[i] = v;
                if (ENERGY) {
                    const double m = 1.0 / (kMvv2e * v.w);
                    part[0] += A.e_atom[i];
                    part[1] += m * fma(v.x, v.x, fma(v.y, v.y, v.z * v.z));
                    part[2] += wxx; part[3] += wyy; part[4] += wzz;
                    part[5] += wyz; part[6] += wxz; part[7] += wxy;
                    part[8] += m * v.x; part[9] += m * v.y; part[10] += m * v.z;
                }
            }
        }
    }
    if (ENERGY || TRAIN) eam::block_partials(part, A.partials, A.part_stride);
}

// ---------------------------------------------------------------- tangent of the descriptors
// u_ik (standardised: times ginv_k) for the force term of the loss gradient.
__global__ void __launch_bounds__(kThreads) k_sur_u(Atoms A, SurNet S, int a0, int a1) {
    __shared__ Stage st;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const float mu = S.mu0 + S.dmu * (float)lane;
    const float kx = -S.inv2w2 * kLog2e;
    const float gi = S.ginv[lane];
    for (long long i0 = a0 + (long long)blockIdx.x * kWarps + w; i0 < a1; i0 += (long long)gridDim.x * kWarps) {
        const int i = (int)i0;
        const Box &B = A.boxes[ph::replica_of(A, i)];
        const float4 pi = A.posf[i];
        const float4 fi = S.phi[i];
        const int cnt = min(A.count[i], A.k_max);
        const NbrRow row = nbr_row(A, i);
        float u = 0.f;
        for (int base = 0; base < cnt; base += 32) {
            const int np = stage_chunk(A, S, pi, B, row, cnt, base, lane, st.P0[w], st.P1[w]);
            for (int q = 0; q < np; q++) {
                const float4 p0 = st.P0[w][q], p1 = st.P1[w][q];
                const float4 fj = __ldg(S.phi + __float_as_int(p0.w));
                const float t = p1.x * (fj.x - fi.x) + p1.y * (fj.y - fi.y) + p1.z * (fj.z - fi.z);
                const float a = p0.x - mu;
                u = fmaf(ex2(kx * a * a) * fmaf(-a, p1.w, p0.z), t, u);
            }
            __syncwarp();
        }
        S.u[(size_t)i * kSurNb + lane] = u * gi;
    }
}

// ---------------------------------------------------------------- per-replica energy terms
// One block per replica r of [r0, r1): E_r = sum of its per-atom energies (fixed order);
// ce[2r] = 2 w_e (E_r - Eref_r) / (S N_r^2), ce[2r+1] = w_e/S ((E_r - Eref_r)/N_r)^2, S = r1 - r0.
__global__ void k_sur_frames(Atoms A, SurNet S, const int32_t *rep_off, int r0, int r1, double w_e) {
    __shared__ double sh[kThreads / 32];
    const int r = r0 + blockIdx.x;
    const int b = rep_off[r], e = rep_off[r + 1];
    double x = 0.0;
    for (int i = b + threadIdx.x; i < e; i += blockDim.x) x += A.e_atom[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(kFull, x, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        double E = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) E += sh[k];
        const double nr = (double)(e - b), ns = (double)(r1 - r0);
        const double d = E - S.eref[r];
        S.ce[2 * r] = nr > 0 ? 2.0 * w_e * d / (ns * nr * nr) : 0.0;
        S.ce[2 * r + 1] = nr > 0 ? w_e / ns * (d / nr) * (d / nr) : 0.0;
    }
}

// ---------------------------------------------------------------- descriptor statistics
// Per-block sums of G_k and G_k^2 over all atoms: part[b][k], part[b][32 + k].
__global__ void k_sur_stats(Atoms A, SurNet S, double *part) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __shared__ double sh[kWarps][2 * kSurNb];
    double s1 = 0.0, s2 = 0.0;
    for (long long i = (long long)blockIdx.x * kWarps + w; i < A.n; i += (long long)gridDim.x * kWarps) {
        const double g = S.G[i * kSurNb + lane];
        s1 += g;
        s2 += g * g;
    }
    sh[w][lane] = s1;
    sh[w][kSurNb + lane] = s2;
    __syncthreads();
    if (threadIdx.x < 2 * kSurNb) {
        double t = 0.0;
        for (int k = 0; k < kWarps; k++) t += sh[k][threadIdx.x];
        part[(size_t)blockIdx.x * 2 * kSurNb + threadIdx.x] = t;
    }
}

__global__ void k_sur_kick_drift(Atoms A, double half_dt, double dt, double lim2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    ph::kick_drift(A, A.boxes, i, half_dt, dt, 1.0, false, lim2);
}

// Rows of 32 floats from cell order back to the caller's order.
__global__ void k_sur_unsort_rows(Atoms A, const float *src, float *dst) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)A.n * kSurNb) return;
    const int i = (int)(t / kSurNb), k = (int)(t % kSurNb);
    dst[(size_t)A.id[i] * kSurNb + k] = src[t];
}

int gather_blocks(int n_atoms) { return std::max(1, std::min(blocks_for(n_atoms, kWarps), 8192)); }

}  // namespace

int sur_force_blocks(int n_atoms) { return gather_blocks(n_atoms); }

cudaError_t launch_sur_kick_drift(const Atoms &A, double half_dt, double dt, double lim2, cudaStream_t s) {
    if (A.n == 0) return cudaSuccess;
    k_sur_kick_drift<<<blocks_for(A.n, kThreads), kThreads, 0, s>>>(A, half_dt, dt, lim2);
    return cudaGetLastError();
}

cudaError_t launch_sur_descriptors(const Atoms &A, const SurNet &S, int a0, int a1, cudaStream_t s) {
    if (a1 <= a0) return cudaSuccess;
    k_sur_desc<<<gather_blocks(a1 - a0), kThreads, 0, s>>>(A, S, a0, a1, S.bf16);
    return cudaGetLastError();
}

cudaError_t launch_sur_force(const Atoms &A, const SurNet &S, int a0, int a1, bool kick, bool energy,
                             double half_dt, double phi_scale, int *rows_out, cudaStream_t s) {
    const int nb = gather_blocks(a1 - a0);
    if (rows_out) *rows_out = nb;
    if (a1 <= a0) return cudaSuccess;
    if (phi_scale > 0.0)
        k_sur_force<true, true><<<nb, kThreads, 0, s>>>(A, S, a0, a1, 0, 0.0, (float)phi_scale);
    else if (energy)
        k_sur_force<true, false><<<nb, kThreads, 0, s>>>(A, S, a0, a1, kick, half_dt, 0.f);
    else
        k_sur_force<false, false><<<nb, kThreads, 0, s>>>(A, S, a0, a1, kick, half_dt, 0.f);
    return cudaGetLastError();
}

cudaError_t launch_sur_u(const Atoms &A, const SurNet &S, int a0, int a1, cudaStream_t s) {
    if (a1 <= a0) return cudaSuccess;
    k_sur_u<<<gather_blocks(a1 - a0), kThreads, 0, s>>>(A, S, a0, a1);
    return cudaGetLastError();
}

cudaError_t launch_sur_frame_terms(const Atoms &A, const SurNet &S, const int32_t *rep_off, int r0, int r1,
                                   double w_e, cudaStream_t s) {
    if (r1 <= r0) return cudaSuccess;
    k_sur_frames<<<r1 - r0, 256, 0, s>>>(A, S, rep_off, r0, r1, w_e);
    return cudaGetLastError();
}

cudaError_t launch_sur_stats(const Atoms &A, const SurNet &S, double *part, int blocks, cudaStream_t s) {
    k_sur_stats<<<blocks, kThreads, 0, s>>>(A, S, part);
    return cudaGetLastError();
}

cudaError_t launch_sur_unsort_rows(const Atoms &A, const float *src, float *dst, cudaStream_t s) {
    if (A.n == 0) return cudaSuccess;
    k_sur_unsort_rows<<<blocks_for((long long)A.n * kSurNb, 256), 256, 0, s>>>(A, src, dst);
    return cudaGetLastError();
}

}  // namespace mdk
