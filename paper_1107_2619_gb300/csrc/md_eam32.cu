// Mixed-precision EAM passes (the two sums of Eq. (1), per-atom gathers over the full list).
//
// Pair and density terms in FP32 from FP32 wrapped coordinates; the density sum is carried
// error-free in an FP32 (hi, lo) pair and rounded to FP64 before F(rho); F, F', the second
// half kick of velocity Verlet and the energy/virial partial sums are FP64.
//   pass 1  rho_i = sum_j phi_{s_i s_j}(r_ij);  F_i, F'_i;  p2f[i] = (x, y, z, F'_i)
//   pass 2  f_i = sum_j [V'(r) + F'_i phi'_{s_i s_j}(r) + F'_j phi'_{s_j s_i}(r)] d / r
#include <cuda_runtime.h>

#include "md_eam_common.cuh"

namespace mdk {

using namespace eam;

namespace {

__device__ __forceinline__ float mi32(float d, float L, float invL) { return fmaf(-L, rintf(d * invL), d); }

// Knot-table row of a species pair: (V c0..c3, phi c0..c3) as 8 floats in one 32-byte load.
__device__ __forceinline__ void row32(const double4_32a *tab, size_t idx, float (&v)[4], float (&p)[4]) {
    const double4_32a d = tab[idx];
    unpack2(d.x, v[0], v[1]);
    unpack2(d.y, v[2], v[3]);
    unpack2(d.z, p[0], p[1]);
    unpack2(d.w, p[2], p[3]);
}

__device__ __forceinline__ float4 phi_half32(const double4_32a *tab, size_t idx) {
    return __ldg(reinterpret_cast<const float4 *>(tab + idx) + 1);
}

template <int T, int KIND, bool MULTI>
__global__ void __launch_bounds__(kThreads) k_density32(Atoms A, Pot P) {
    clear_rebuild_once(A.flags);
    const long long g = (long long)blockIdx.x * kThreads + threadIdx.x;
    const int i = (int)(g / T), lane = (int)(g & (T - 1));
    const bool live = i < A.n;
    float hi = 0.f, lo = 0.f;
    float4 pi = make_float4(0.f, 0.f, 0.f, 0.f);
    int si = 0;
    if (live) {
        const Box B = *A.box;
        const float Lx = B.Lf[0], Ly = B.Lf[1], Lz = B.Lf[2];
        const float ix = B.invLf[0], iy = B.invLf[1], iz = B.invLf[2];
        pi = A.posf[i];
        si = MULTI ? __float_as_int(pi.w) : 0;
        const int cnt = min(A.count[i], A.k_max);
        const int *__restrict__ row = A.nbr + (size_t)i * A.k_max;
        for (int k = lane; k < cnt; k += T) {
            const int j = __ldg(row + k);
            const float4 pj = __ldg(A.posf + j);
            const float dx = mi32(pj.x - pi.x, Lx, ix);
            const float dy = mi32(pj.y - pi.y, Ly, iy);
            const float dz = mi32(pj.z - pi.z, Lz, iz);
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            if (!(r2 < P.rc2f)) continue;
            const float r = r2 * rsqrtf(r2);
            float phi;
            if (KIND == MD_POT_FS_ANALYTIC) {
                phi = fs_phi<float>(P.fsf, P.bdf, r);
            } else {
                const int sj = MULTI ? __float_as_int(pj.w) : 0;
                float t, d;
                bool below;
                const int kr = knot_row((r - P.r_minf) * P.inv_drf, P.nk, t, below);
                if (below) atomicAdd(&A.flags->range_violations, 1ull);
                const float4 c = phi_half32(P.VP32, (size_t)(si * P.ns + sj) * P.nk + kr);
                phi = cubic(t, c.x, c.y, c.z, c.w, below, d);
            }
            two_sum_add(hi, lo, phi);
        }
    }
    lane_sum_df<T>(hi, lo);
    if (live && lane == 0) {
        const double rho = (double)hi + (double)lo;
        double dF;
        const double F = embed64(P, si, rho, dF, A.flags);
        A.rho[i] = rho;
        A.dF[i] = dF;
        A.e_atom[i] = F;
        A.p2f[i] = make_float4(pi.x, pi.y, pi.z, (float)dF);
    }
}

template <int T, int KIND, bool MULTI, bool ENERGY>
__global__ void __launch_bounds__(kThreads) k_force32(Atoms A, Pot P, double half_dt, int kick) {
    const long long g = (long long)blockIdx.x * kThreads + threadIdx.x;
    const int i = (int)(g / T), lane = (int)(g & (T - 1));
    const bool live = i < A.n;
    float fx = 0.f, fy = 0.f, fz = 0.f, ep = 0.f;
    float wxx = 0.f, wyy = 0.f, wzz = 0.f, wyz = 0.f, wxz = 0.f, wxy = 0.f;
    if (live) {
        const Box B = *A.box;
        const float Lx = B.Lf[0], Ly = B.Lf[1], Lz = B.Lf[2];
        const float ix = B.invLf[0], iy = B.invLf[1], iz = B.invLf[2];
        const float4 pi = A.p2f[i];
        const float Fpi = pi.w;
        const int si = MULTI ? A.spec[i] : 0;
        const int cnt = min(A.count[i], A.k_max);
        const int *__restrict__ row = A.nbr + (size_t)i * A.k_max;
        for (int k = lane; k < cnt; k += T) {
            const int j = __ldg(row + k);
            const float4 pj = __ldg(A.p2f + j);
            const float dx = mi32(pj.x - pi.x, Lx, ix);
            const float dy = mi32(pj.y - pi.y, Ly, iy);
            const float dz = mi32(pj.z - pi.z, Lz, iz);
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            if (!(r2 < P.rc2f)) continue;
            const float rinv = rsqrtf(r2);
            const float r = r2 * rinv;
            const float Fpj = pj.w;
            float V, g;
            if (KIND == MD_POT_FS_ANALYTIC) {
                float dV;
                V = fs_V<float>(P.fsf, r, dV);
                g = fmaf(Fpi + Fpj, fs_dphi<float>(P.fsf, P.bdf, r), dV);
            } else {
                const int sj = MULTI ? __ldg(A.spec + j) : 0;
                float t;
                bool below;
                const int kr = knot_row((r - P.r_minf) * P.inv_drf, P.nk, t, below);
                if (below) atomicAdd(&A.flags->range_violations, 1ull);
                float cv[4], cp[4], dVk, dab;
                row32(P.VP32, (size_t)(si * P.ns + sj) * P.nk + kr, cv, cp);
                V = cubic(t, cv[0], cv[1], cv[2], cv[3], below, dVk);
                cubic(t, cp[0], cp[1], cp[2], cp[3], below, dab);
                float gk;
                if (MULTI) {
                    const float4 c = phi_half32(P.VP32, (size_t)(sj * P.ns + si) * P.nk + kr);
                    float dba;
                    cubic(t, c.x, c.y, c.z, c.w, below, dba);
                    gk = fmaf(Fpi, dab, fmaf(Fpj, dba, dVk));
                } else {
                    gk = fmaf(Fpi + Fpj, dab, dVk);
                }
                g = gk * P.inv_drf;
            }
            const float gr = g * rinv;
            fx = fmaf(gr, dx, fx);
            fy = fmaf(gr, dy, fy);
            fz = fmaf(gr, dz, fz);
            if (ENERGY) {
                ep = fmaf(0.5f, V, ep);
                const float hg = -0.5f * gr;
                wxx = fmaf(hg * dx, dx, wxx);
                wyy = fmaf(hg * dy, dy, wyy);
                wzz = fmaf(hg * dz, dz, wzz);
                wyz = fmaf(hg * dy, dz, wyz);
                wxz = fmaf(hg * dx, dz, wxz);
                wxy = fmaf(hg * dx, dy, wxy);
            }
        }
    }
    fx = lane_sum<T>(fx);
    fy = lane_sum<T>(fy);
    fz = lane_sum<T>(fz);
    if (ENERGY) {
        ep = lane_sum<T>(ep);
        wxx = lane_sum<T>(wxx); wyy = lane_sum<T>(wyy); wzz = lane_sum<T>(wzz);
        wyz = lane_sum<T>(wyz); wxz = lane_sum<T>(wxz); wxy = lane_sum<T>(wxy);
    }
    double part[kPartials];
#pragma unroll
    for (int q = 0; q < kPartials; q++) part[q] = 0.0;
    if (live && lane == 0) {
        A.force[i] = make_double4_32a(fx, fy, fz, 0.0);
        if (!isfinite(fx + fy + fz)) atomicOr(&A.flags->error, FLAG_NONFINITE);
        double4_32a v = A.vel[i];
        kick_and_partials(v, fx, fy, fz, half_dt, kick != 0);
        if (kick) A.vel[i] = v;
        if (ENERGY) {
            const double e = A.e_atom[i] + (double)ep;
            A.e_atom[i] = e;
            const double m = 1.0 / (kMvv2e * v.w);
            part[0] = e;
            part[1] = m * fma(v.x, v.x, fma(v.y, v.y, v.z * v.z));
            part[2] = wxx; part[3] = wyy; part[4] = wzz;
            part[5] = wyz; part[6] = wxz; part[7] = wxy;
            part[8] = m * v.x; part[9] = m * v.y; part[10] = m * v.z;
        }
    }
    if (ENERGY) block_partials(part, A.partials);
}

template <int T>
void density_t(const Atoms &A, const Pot &P, cudaStream_t s) {
    const int nb = A.n > 0 ? blocks_for_lanes<T>(A.n) : 1;
    if (P.kind == MD_POT_FS_ANALYTIC) k_density32<T, MD_POT_FS_ANALYTIC, false><<<nb, kThreads, 0, s>>>(A, P);
    else if (P.ns == 1) k_density32<T, MD_POT_TABLES, false><<<nb, kThreads, 0, s>>>(A, P);
    else k_density32<T, MD_POT_TABLES, true><<<nb, kThreads, 0, s>>>(A, P);
}

template <int T, bool ENERGY>
void force_te(const Atoms &A, const Pot &P, double half_dt, int kick, cudaStream_t s) {
    const int nb = blocks_for_lanes<T>(A.n);
    if (P.kind == MD_POT_FS_ANALYTIC)
        k_force32<T, MD_POT_FS_ANALYTIC, false, ENERGY><<<nb, kThreads, 0, s>>>(A, P, half_dt, kick);
    else if (P.ns == 1)
        k_force32<T, MD_POT_TABLES, false, ENERGY><<<nb, kThreads, 0, s>>>(A, P, half_dt, kick);
    else
        k_force32<T, MD_POT_TABLES, true, ENERGY><<<nb, kThreads, 0, s>>>(A, P, half_dt, kick);
}

template <int T>
void force_t(const Atoms &A, const Pot &P, bool kick, bool energy, double half_dt, cudaStream_t s) {
    if (energy) force_te<T, true>(A, P, half_dt, kick, s);
    else force_te<T, false>(A, P, half_dt, kick, s);
}

}  // namespace

cudaError_t launch_density32(const Atoms &A, const Pot &P, int lanes, cudaStream_t s) {
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

cudaError_t launch_force32(const Atoms &A, const Pot &P, int lanes, bool kick, bool energy, double half_dt,
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

}  // namespace mdk
