// FP64 EAM passes (the two sums of Eq. (1), per-atom gathers over the full list), the
// deterministic energy reduction, and the precision dispatch.
//   pass 1  rho_i = sum_j phi_{s_i s_j}(r_ij);  F_i, F'_i;  p2d[i] = (x, y, z, F'_i)
//   pass 2  f_i = sum_j [V'(r) + F'_i phi'_{s_i s_j}(r) + F'_j phi'_{s_j s_i}(r)] d / r,
//           then the second half kick and the FP64 partial sums.
#include <cuda_runtime.h>

#include "md_eam_common.cuh"

namespace mdk {

using namespace eam;

cudaError_t launch_density32(const Atoms &A, const Pot &P, int lanes, cudaStream_t s);
cudaError_t launch_force32(const Atoms &A, const Pot &P, int lanes, bool kick, bool energy, double half_dt,
                           cudaStream_t s);

namespace {

__device__ __forceinline__ double mi64(double d, double L, double invL) { return fma(-L, rint(d * invL), d); }

template <int T, int KIND, bool MULTI>
__global__ void __launch_bounds__(kThreads) k_density64(Atoms A, Pot P) {
    clear_rebuild_once(A.flags);
    const long long g = (long long)blockIdx.x * kThreads + threadIdx.x;
    const int i = (int)(g / T), lane = (int)(g & (T - 1));
    const bool live = i < A.n;
    double rho = 0.0;
    double4_32a pi = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    int si = 0;
    if (live) {
        const Box B = *A.box;
        pi = A.pos[i];
        si = MULTI ? A.spec[i] : 0;
        const int cnt = min(A.count[i], A.k_max);
        const int *__restrict__ row = A.nbr + (size_t)i * A.k_max;
        for (int k = lane; k < cnt; k += T) {
            const int j = __ldg(row + k);
            const double4_32a pj = A.pos[j];
            const double dx = mi64(pj.x - pi.x, B.L[0], B.invL[0]);
            const double dy = mi64(pj.y - pi.y, B.L[1], B.invL[1]);
            const double dz = mi64(pj.z - pi.z, B.L[2], B.invL[2]);
            const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
            if (!(r2 < P.rc2)) continue;
            const double r = r2 * rsqrt64(r2);
            if (KIND == MD_POT_FS_ANALYTIC) {
                rho += fs_phi<double>(P.fs, P.bd, r);
            } else {
                const int sj = MULTI ? (int)pj.w : 0;
                double t, d;
                bool below;
                const int kr = knot_row((r - P.r_min) * P.inv_dr, P.nk, t, below);
                if (below) atomicAdd(&A.flags->range_violations, 1ull);
                const double4_32a c = P.VP64[((size_t)(si * P.ns + sj) * P.nk + kr) * 2 + 1];
                rho += cubic(t, c.x, c.y, c.z, c.w, below, d);
            }
        }
    }
    rho = lane_sum<T>(rho);
    if (live && lane == 0) {
        double dF;
        const double F = embed64(P, si, rho, dF, A.flags);
        A.rho[i] = rho;
        A.dF[i] = dF;
        A.e_atom[i] = F;
        A.p2d[i] = make_double4_32a(pi.x, pi.y, pi.z, dF);
    }
}

template <int T, int KIND, bool MULTI, bool ENERGY>
__global__ void __launch_bounds__(kThreads) k_force64(Atoms A, Pot P, double half_dt, int kick) {
    const long long g = (long long)blockIdx.x * kThreads + threadIdx.x;
    const int i = (int)(g / T), lane = (int)(g & (T - 1));
    const bool live = i < A.n;
    double fx = 0.0, fy = 0.0, fz = 0.0, ep = 0.0;
    double wxx = 0.0, wyy = 0.0, wzz = 0.0, wyz = 0.0, wxz = 0.0, wxy = 0.0;
    if (live) {
        const Box B = *A.box;
        const double4_32a pi = A.p2d[i];
        const double Fpi = pi.w;
        const int si = MULTI ? A.spec[i] : 0;
        const int cnt = min(A.count[i], A.k_max);
        const int *__restrict__ row = A.nbr + (size_t)i * A.k_max;
        for (int k = lane; k < cnt; k += T) {
            const int j = __ldg(row + k);
            const double4_32a pj = A.p2d[j];
            const double dx = mi64(pj.x - pi.x, B.L[0], B.invL[0]);
            const double dy = mi64(pj.y - pi.y, B.L[1], B.invL[1]);
            const double dz = mi64(pj.z - pi.z, B.L[2], B.invL[2]);
            const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
            if (!(r2 < P.rc2)) continue;
            const double rinv = rsqrt64(r2);
            const double r = r2 * rinv;
            const double Fpj = pj.w;
            double V, g;
            if (KIND == MD_POT_FS_ANALYTIC) {
                double dV;
                V = fs_V<double>(P.fs, r, dV);
                g = fma(Fpi + Fpj, fs_dphi<double>(P.fs, P.bd, r), dV);
            } else {
                const int sj = MULTI ? __ldg(A.spec + j) : 0;
                double t;
                bool below;
                const int kr = knot_row((r - P.r_min) * P.inv_dr, P.nk, t, below);
                if (below) atomicAdd(&A.flags->range_violations, 1ull);
                const size_t ab = ((size_t)(si * P.ns + sj) * P.nk + kr) * 2;
                const double4_32a cv = P.VP64[ab], cp = P.VP64[ab + 1];
                double dVk, dab;
                V = cubic(t, cv.x, cv.y, cv.z, cv.w, below, dVk);
                cubic(t, cp.x, cp.y, cp.z, cp.w, below, dab);
                double gk;
                if (MULTI) {
                    const double4_32a cb = P.VP64[((size_t)(sj * P.ns + si) * P.nk + kr) * 2 + 1];
                    double dba;
                    cubic(t, cb.x, cb.y, cb.z, cb.w, below, dba);
                    gk = fma(Fpi, dab, fma(Fpj, dba, dVk));
                } else {
                    gk = fma(Fpi + Fpj, dab, dVk);
                }
                g = gk * P.inv_dr;
            }
            const double gr = g * rinv;
            fx = fma(gr, dx, fx);
            fy = fma(gr, dy, fy);
            fz = fma(gr, dz, fz);
            if (ENERGY) {
                ep = fma(0.5, V, ep);
                const double hg = -0.5 * gr;
                wxx = fma(hg * dx, dx, wxx);
                wyy = fma(hg * dy, dy, wyy);
                wzz = fma(hg * dz, dz, wzz);
                wyz = fma(hg * dy, dz, wyz);
                wxz = fma(hg * dx, dz, wxz);
                wxy = fma(hg * dx, dy, wxy);
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
            const double e = A.e_atom[i] + ep;
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

// Deterministic final reduction of the per-block partials: fixed thread-to-block mapping and
// a fixed tree, so repeated runs give bitwise identical totals.
__global__ void k_reduce(const double *__restrict__ partials, int nblocks, double *out) {
    __shared__ double sh[256];
    for (int q = 0; q < kPartials; q++) {
        double s = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += 256) s += partials[(size_t)b * kPartials + q];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[q] = sh[0];
        __syncthreads();
    }
}

template <int T>
void density_t(const Atoms &A, const Pot &P, cudaStream_t s) {
    const int nb = A.n > 0 ? blocks_for_lanes<T>(A.n) : 1;
    if (P.kind == MD_POT_FS_ANALYTIC) k_density64<T, MD_POT_FS_ANALYTIC, false><<<nb, kThreads, 0, s>>>(A, P);
    else if (P.ns == 1) k_density64<T, MD_POT_TABLES, false><<<nb, kThreads, 0, s>>>(A, P);
    else k_density64<T, MD_POT_TABLES, true><<<nb, kThreads, 0, s>>>(A, P);
}

template <int T, bool ENERGY>
void force_te(const Atoms &A, const Pot &P, double half_dt, int kick, cudaStream_t s) {
    const int nb = blocks_for_lanes<T>(A.n);
    if (P.kind == MD_POT_FS_ANALYTIC)
        k_force64<T, MD_POT_FS_ANALYTIC, false, ENERGY><<<nb, kThreads, 0, s>>>(A, P, half_dt, kick);
    else if (P.ns == 1)
        k_force64<T, MD_POT_TABLES, false, ENERGY><<<nb, kThreads, 0, s>>>(A, P, half_dt, kick);
    else
        k_force64<T, MD_POT_TABLES, true, ENERGY><<<nb, kThreads, 0, s>>>(A, P, half_dt, kick);
}

template <int T>
void force_t(const Atoms &A, const Pot &P, bool kick, bool energy, double half_dt, cudaStream_t s) {
    if (energy) force_te<T, true>(A, P, half_dt, kick, s);
    else force_te<T, false>(A, P, half_dt, kick, s);
}

cudaError_t density64(const Atoms &A, const Pot &P, int lanes, cudaStream_t s) {
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

cudaError_t force64(const Atoms &A, const Pot &P, int lanes, bool kick, bool energy, double half_dt,
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

}  // namespace

int partial_blocks(int n, int lanes) {
    return n > 0 ? (int)(((long long)n * lanes + kThreads - 1) / kThreads) : 0;
}

cudaError_t launch_density(const Atoms &A, const Pot &P, int precision, int lanes, cudaStream_t s) {
    return precision == MD_PREC_FP64 ? density64(A, P, lanes, s) : launch_density32(A, P, lanes, s);
}

cudaError_t launch_force(const Atoms &A, const Pot &P, int precision, int lanes, bool kick, bool energy,
                         double half_dt, cudaStream_t s) {
    return precision == MD_PREC_FP64 ? force64(A, P, lanes, kick, energy, half_dt, s)
                                     : launch_force32(A, P, lanes, kick, energy, half_dt, s);
}

cudaError_t launch_reduce(const Atoms &A, int nblocks, double *out, cudaStream_t s) {
    k_reduce<<<1, 256, 0, s>>>(A.partials, nblocks, out);
    return cudaGetLastError();
}

}  // namespace mdk
