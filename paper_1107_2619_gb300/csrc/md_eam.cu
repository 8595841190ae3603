// The two sums of Eq. (1) of the MOLDY paper, as per-atom gathers over the full list.
//
// Pass 1 (k_density):  rho_i = sum_j phi_{s_i s_j}(r_ij),  F_i = F(rho_i),  F'_i.
// Pass 2 (k_force):    f_i = sum_j [V'(r) + F'_i phi'_{s_i s_j}(r) + F'_j phi'_{s_j s_i}(r)] d/r,
//                      d = r_j - r_i (minimum image), optionally followed by the second half
//                      kick of velocity Verlet (§2.3) and the per-block FP64 partial sums of
//                      the energy, kinetic energy, virial and momentum.
// Each thread owns one atom and writes only that atom (the symmetric list of §3.2.2: every
// pair term is computed twice, once by each atom, so no locks or atomics are needed).
//
// Precision:  FP64 path - every operation in double.
//             Mixed path - pair and density terms in FP32 from FP32 wrapped coordinates;
//             the density sum is carried error-free in a (hi, lo) FP32 pair and rounded to
//             FP64 before F(rho); F, F', the integration and all reductions are FP64.
#include <cuda_runtime.h>

#include "md_internal.cuh"

namespace mdk {

namespace {

// 1/sqrt(x): FP32 hardware estimate refined by two Newton-Raphson steps in FP64
// (y <- y + y (1 - x y^2) / 2); relative error ~1e-16.
__device__ __forceinline__ double rsqrt64(double x) {
    double y = (double)rsqrtf((float)x);
    double e = fma(-x * y, y, 1.0);
    y = fma(0.5 * y, e, y);
    e = fma(-x * y, y, 1.0);
    return fma(0.5 * y, e, y);
}

// Error-free FP32 accumulation (Knuth's TwoSum): hi + lo carries the exact running sum of
// the FP32 terms to ~2^-48 relative.
__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float x) {
    float s = hi + x;
    float bp = s - hi;
    float err = (hi - (s - bp)) + (x - bp);
    hi = s;
    lo += err;
}

// ---- knot tables: x in units of the knot spacing; rows (c0, c1, c2, c3), row nk-1 linear ----
template <typename R, typename R4>
__device__ __forceinline__ R tab_eval(const R4 *__restrict__ tab, int nk, R x, R &dydx_knots,
                                      Flags *flags) {
    if (x >= R(0)) {
        int k = (x < (R)(nk - 1)) ? (int)x : nk - 1;
        R t = x - (R)k;
        R4 c = tab[k];
        dydx_knots = fma(t, fma(R(3) * c.w, t, R(2) * c.z), c.y);
        return fma(t, fma(t, fma(t, c.w, c.z), c.y), c.x);
    }
    R4 c = tab[0];
    atomicAdd(&flags->range_violations, 1ull);
    dydx_knots = c.y;
    return fma(x, c.y, c.x);
}

template <typename R, typename R4>
__device__ __forceinline__ R tab_deriv(const R4 *__restrict__ tab, int nk, R x, Flags *flags) {
    R d;
    tab_eval<R, R4>(tab, nk, x, d, flags);
    return d;
}

// ---- analytic Finnis-Sinclair pair functions (fs = d, c, A, beta, c0, c1, c2) ----
// bd = beta / d
template <typename R>
__device__ __forceinline__ R fs_phi(const R *fs, R bd, R r) {
    R t = r - fs[0];
    if (t >= R(0)) return R(0);
    return t * t * fma(bd, t, R(1));
}

template <typename R>
__device__ __forceinline__ R fs_dphi(const R *fs, R bd, R r) {
    R t = r - fs[0];
    if (t >= R(0)) return R(0);
    return t * fma(R(3) * bd, t, R(2));
}

template <typename R>
__device__ __forceinline__ R fs_V(const R *fs, R r, R &dV) {
    R u = r - fs[1];
    if (u >= R(0)) {
        dV = R(0);
        return R(0);
    }
    R q = fma(fma(fs[6], r, fs[5]), r, fs[4]);
    R dq = fma(R(2) * fs[6], r, fs[5]);
    dV = u * fma(u, dq, R(2) * q);
    return u * u * q;
}

// F and F' in FP64 for both precisions (one evaluation per atom).
__device__ __forceinline__ double embed64(const Pot &P, int a, double rho, double &dF, Flags *flags) {
    if (P.kind == MD_POT_FS_ANALYTIC) {
        if (!(rho > 0.0)) {
            dF = 0.0;
            return 0.0;
        }
        double s = sqrt(rho);
        dF = -0.5 * P.fs[2] / s;
        return -P.fs[2] * s;
    }
    double x = (rho - P.rho_min) * P.inv_drho;
    double d;
    double F = tab_eval<double, double4_32a>(P.F64 + (size_t)a * P.nk, P.nk, x, d, flags);
    if (x > (double)(P.nk - 1)) atomicAdd(&flags->range_violations, 1ull);
    dF = d * P.inv_drho;
    return F;
}

__device__ __forceinline__ void block_partials(double (&v)[kPartials], double *out) {
    __shared__ double sh[kThreads / 32][kPartials];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kPartials; q++) {
        double x = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[w][q] = x;
    }
    __syncthreads();
    if (threadIdx.x < kPartials) {
        double s = 0.0;
        for (int k = 0; k < kThreads / 32; k++) s += sh[k][threadIdx.x];
        out[(size_t)blockIdx.x * kPartials + threadIdx.x] = s;
    }
}

__device__ __forceinline__ void clear_rebuild_once(Flags *f) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (f->need_rebuild) f->n_rebuilds++;
        f->need_rebuild = 0;
    }
}

// =============================== FP64 path ===============================
template <int KIND, bool MULTI>
__global__ void __launch_bounds__(kThreads) k_density64(Atoms A, Pot P) {
    clear_rebuild_once(A.flags);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    const Box B = *A.box;
    const double4_32a pi = A.pos[i];
    const int si = MULTI ? A.spec[i] : 0;
    const int cnt = min(A.count[i], A.k_max);
    const size_t n = (size_t)A.n;
    double rho = 0.0;
    for (int k = 0; k < cnt; k++) {
        const int j = __ldg(A.nbr + (size_t)k * n + i);
        const double4_32a pj = A.pos[j];
        double dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
        dx = fma(-B.L[0], rint(dx * B.invL[0]), dx);
        dy = fma(-B.L[1], rint(dy * B.invL[1]), dy);
        dz = fma(-B.L[2], rint(dz * B.invL[2]), dz);
        const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
        if (r2 < P.rc2) {
            const double r = r2 * rsqrt64(r2);
            if (KIND == MD_POT_FS_ANALYTIC) {
                rho += fs_phi<double>(P.fs, P.bd, r);
            } else {
                const int sj = MULTI ? (int)pj.w : 0;
                double d;
                rho += tab_eval<double, double4_32a>(P.P64 + (size_t)(si * P.ns + sj) * P.nk, P.nk,
                                                 (r - P.r_min) * P.inv_dr, d, A.flags);
            }
        }
    }
    double dF;
    const double F = embed64(P, si, rho, dF, A.flags);
    A.rho[i] = rho;
    A.dF[i] = dF;
    A.e_atom[i] = F;
}

template <int KIND, bool MULTI, bool KICK, bool ENERGY>
__global__ void __launch_bounds__(kThreads) k_force64(Atoms A, Pot P, double half_dt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < A.n;
    double part[kPartials];
#pragma unroll
    for (int q = 0; q < kPartials; q++) part[q] = 0.0;
    if (live) {
        const Box B = *A.box;
        const double4_32a pi = A.pos[i];
        const int si = MULTI ? A.spec[i] : 0;
        const double Fpi = A.dF[i];
        const int cnt = min(A.count[i], A.k_max);
        const size_t n = (size_t)A.n;
        double fx = 0.0, fy = 0.0, fz = 0.0, ep = 0.0;
        double wxx = 0.0, wyy = 0.0, wzz = 0.0, wyz = 0.0, wxz = 0.0, wxy = 0.0;
        for (int k = 0; k < cnt; k++) {
            const int j = __ldg(A.nbr + (size_t)k * n + i);
            const double4_32a pj = A.pos[j];
            double dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
            dx = fma(-B.L[0], rint(dx * B.invL[0]), dx);
            dy = fma(-B.L[1], rint(dy * B.invL[1]), dy);
            dz = fma(-B.L[2], rint(dz * B.invL[2]), dz);
            const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
            if (!(r2 < P.rc2)) continue;
            const double rinv = rsqrt64(r2);
            const double r = r2 * rinv;
            const double Fpj = A.dF[j];
            double V, dV, g;
            if (KIND == MD_POT_FS_ANALYTIC) {
                V = fs_V<double>(P.fs, r, dV);
                g = fma(Fpi + Fpj, fs_dphi<double>(P.fs, P.bd, r), dV);
            } else {
                const int sj = MULTI ? (int)pj.w : 0;
                const double x = (r - P.r_min) * P.inv_dr;
                double dVk;
                V = tab_eval<double, double4_32a>(P.V64 + (size_t)(si * P.ns + sj) * P.nk, P.nk, x, dVk,
                                              A.flags);
                const double dab = tab_deriv<double, double4_32a>(P.P64 + (size_t)(si * P.ns + sj) * P.nk,
                                                              P.nk, x, A.flags);
                double gk;
                if (MULTI) {
                    const double dba = tab_deriv<double, double4_32a>(
                        P.P64 + (size_t)(sj * P.ns + si) * P.nk, P.nk, x, A.flags);
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
        double4_32a fo = A.force[i];
        fo.x = fx;
        fo.y = fy;
        fo.z = fz;
        A.force[i] = fo;
        if (!isfinite(fx + fy + fz)) atomicOr(&A.flags->error, FLAG_NONFINITE);
        double4_32a v = A.vel[i];
        if (KICK) {  // second half kick, the same IEEE operations as v += (dt/2 * f) * (acc/m)
            v.x = __dadd_rn(v.x, __dmul_rn(__dmul_rn(half_dt, fx), v.w));
            v.y = __dadd_rn(v.y, __dmul_rn(__dmul_rn(half_dt, fy), v.w));
            v.z = __dadd_rn(v.z, __dmul_rn(__dmul_rn(half_dt, fz), v.w));
            A.vel[i] = v;
        }
        if (ENERGY) {
            const double e = A.e_atom[i] + ep;
            A.e_atom[i] = e;
            const double m = fo.w;
            part[0] = e;
            part[1] = m * fma(v.x, v.x, fma(v.y, v.y, v.z * v.z));
            part[2] = wxx; part[3] = wyy; part[4] = wzz;
            part[5] = wyz; part[6] = wxz; part[7] = wxy;
            part[8] = m * v.x; part[9] = m * v.y; part[10] = m * v.z;
        }
    }
    if (ENERGY) block_partials(part, A.partials);
}

// =============================== mixed path ===============================
__device__ __forceinline__ float mi32(float d, float L, float invL) { return fmaf(-L, rintf(d * invL), d); }

template <int KIND, bool MULTI>
__global__ void __launch_bounds__(kThreads) k_density32(Atoms A, Pot P) {
    clear_rebuild_once(A.flags);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    const Box B = *A.box;
    const float Lx = B.Lf[0], Ly = B.Lf[1], Lz = B.Lf[2];
    const float ix = B.invLf[0], iy = B.invLf[1], iz = B.invLf[2];
    const float4 pi = A.posf[i];
    const int si = MULTI ? __float_as_int(pi.w) : 0;
    const int cnt = min(A.count[i], A.k_max);
    const size_t n = (size_t)A.n;
    float hi = 0.f, lo = 0.f;
    for (int k = 0; k < cnt; k++) {
        const int j = __ldg(A.nbr + (size_t)k * n + i);
        const float4 pj = A.posf[j];
        const float dx = mi32(pj.x - pi.x, Lx, ix);
        const float dy = mi32(pj.y - pi.y, Ly, iy);
        const float dz = mi32(pj.z - pi.z, Lz, iz);
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        if (r2 < P.rc2f) {
            const float r = r2 * rsqrtf(r2);
            float phi;
            if (KIND == MD_POT_FS_ANALYTIC) {
                phi = fs_phi<float>(P.fsf, P.bdf, r);
            } else {
                const int sj = MULTI ? __float_as_int(pj.w) : 0;
                float d;
                phi = tab_eval<float, float4>(P.P32 + (size_t)(si * P.ns + sj) * P.nk, P.nk,
                                              (r - P.r_minf) * P.inv_drf, d, A.flags);
            }
            two_sum_add(hi, lo, phi);
        }
    }
    const double rho = (double)hi + (double)lo;
    double dF;
    const double F = embed64(P, si, rho, dF, A.flags);
    A.rho[i] = rho;
    A.dF[i] = dF;
    A.e_atom[i] = F;
    A.p2f[i] = make_float4(pi.x, pi.y, pi.z, (float)dF);
}

template <int KIND, bool MULTI, bool KICK, bool ENERGY>
__global__ void __launch_bounds__(kThreads) k_force32(Atoms A, Pot P, double half_dt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < A.n;
    double part[kPartials];
#pragma unroll
    for (int q = 0; q < kPartials; q++) part[q] = 0.0;
    if (live) {
        const Box B = *A.box;
        const float Lx = B.Lf[0], Ly = B.Lf[1], Lz = B.Lf[2];
        const float ix = B.invLf[0], iy = B.invLf[1], iz = B.invLf[2];
        const float4 pi = A.p2f[i];
        const float Fpi = pi.w;
        const int si = MULTI ? A.spec[i] : 0;
        const int cnt = min(A.count[i], A.k_max);
        const size_t n = (size_t)A.n;
        float fx = 0.f, fy = 0.f, fz = 0.f, ep = 0.f;
        float wxx = 0.f, wyy = 0.f, wzz = 0.f, wyz = 0.f, wxz = 0.f, wxy = 0.f;
        for (int k = 0; k < cnt; k++) {
            const int j = __ldg(A.nbr + (size_t)k * n + i);
            const float4 pj = A.p2f[j];
            const float dx = mi32(pj.x - pi.x, Lx, ix);
            const float dy = mi32(pj.y - pi.y, Ly, iy);
            const float dz = mi32(pj.z - pi.z, Lz, iz);
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            if (!(r2 < P.rc2f)) continue;
            const float rinv = rsqrtf(r2);
            const float r = r2 * rinv;
            const float Fpj = pj.w;
            float V, dV, g;
            if (KIND == MD_POT_FS_ANALYTIC) {
                V = fs_V<float>(P.fsf, r, dV);
                g = fmaf(Fpi + Fpj, fs_dphi<float>(P.fsf, P.bdf, r), dV);
            } else {
                const int sj = MULTI ? __ldg(A.spec + j) : 0;
                const float x = (r - P.r_minf) * P.inv_drf;
                float dVk;
                V = tab_eval<float, float4>(P.V32 + (size_t)(si * P.ns + sj) * P.nk, P.nk, x, dVk,
                                            A.flags);
                const float dab = tab_deriv<float, float4>(P.P32 + (size_t)(si * P.ns + sj) * P.nk,
                                                           P.nk, x, A.flags);
                float gk;
                if (MULTI) {
                    const float dba = tab_deriv<float, float4>(P.P32 + (size_t)(sj * P.ns + si) * P.nk,
                                                               P.nk, x, A.flags);
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
        double4_32a fo = A.force[i];
        fo.x = fx;
        fo.y = fy;
        fo.z = fz;
        A.force[i] = fo;
        if (!isfinite(fx + fy + fz)) atomicOr(&A.flags->error, FLAG_NONFINITE);
        double4_32a v = A.vel[i];
        if (KICK) {
            v.x = __dadd_rn(v.x, __dmul_rn(__dmul_rn(half_dt, fo.x), v.w));
            v.y = __dadd_rn(v.y, __dmul_rn(__dmul_rn(half_dt, fo.y), v.w));
            v.z = __dadd_rn(v.z, __dmul_rn(__dmul_rn(half_dt, fo.z), v.w));
            A.vel[i] = v;
        }
        if (ENERGY) {
            const double e = A.e_atom[i] + (double)ep;
            A.e_atom[i] = e;
            const double m = fo.w;
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

template <int KIND, bool MULTI>
void density_dispatch(const Atoms &A, const Pot &P, int prec, int nb, cudaStream_t s) {
    if (prec == MD_PREC_FP64)
        k_density64<KIND, MULTI><<<nb, kThreads, 0, s>>>(A, P);
    else
        k_density32<KIND, MULTI><<<nb, kThreads, 0, s>>>(A, P);
}

template <int KIND, bool MULTI, bool KICK, bool ENERGY>
void force_dispatch3(const Atoms &A, const Pot &P, int prec, double half_dt, int nb, cudaStream_t s) {
    if (prec == MD_PREC_FP64)
        k_force64<KIND, MULTI, KICK, ENERGY><<<nb, kThreads, 0, s>>>(A, P, half_dt);
    else
        k_force32<KIND, MULTI, KICK, ENERGY><<<nb, kThreads, 0, s>>>(A, P, half_dt);
}

template <int KIND, bool MULTI>
void force_dispatch(const Atoms &A, const Pot &P, int prec, bool kick, bool energy, double half_dt,
                    int nb, cudaStream_t s) {
    if (kick) {
        if (energy) force_dispatch3<KIND, MULTI, true, true>(A, P, prec, half_dt, nb, s);
        else force_dispatch3<KIND, MULTI, true, false>(A, P, prec, half_dt, nb, s);
    } else {
        if (energy) force_dispatch3<KIND, MULTI, false, true>(A, P, prec, half_dt, nb, s);
        else force_dispatch3<KIND, MULTI, false, false>(A, P, prec, half_dt, nb, s);
    }
}

}  // namespace

cudaError_t launch_density(const Atoms &A, const Pot &P, int precision, cudaStream_t s) {
    const int nb = A.n > 0 ? blocks_for(A.n, kThreads) : 1;
    if (P.kind == MD_POT_FS_ANALYTIC) density_dispatch<MD_POT_FS_ANALYTIC, false>(A, P, precision, nb, s);
    else if (P.ns == 1) density_dispatch<MD_POT_TABLES, false>(A, P, precision, nb, s);
    else density_dispatch<MD_POT_TABLES, true>(A, P, precision, nb, s);
    return cudaGetLastError();
}

cudaError_t launch_force(const Atoms &A, const Pot &P, int precision, bool kick, bool energy,
                         double half_dt, cudaStream_t s) {
    if (A.n == 0) return cudaSuccess;
    const int nb = blocks_for(A.n, kThreads);
    if (P.kind == MD_POT_FS_ANALYTIC)
        force_dispatch<MD_POT_FS_ANALYTIC, false>(A, P, precision, kick, energy, half_dt, nb, s);
    else if (P.ns == 1)
        force_dispatch<MD_POT_TABLES, false>(A, P, precision, kick, energy, half_dt, nb, s);
    else
        force_dispatch<MD_POT_TABLES, true>(A, P, precision, kick, energy, half_dt, nb, s);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const Atoms &A, double *out, cudaStream_t s) {
    k_reduce<<<1, 256, 0, s>>>(A.partials, A.n > 0 ? blocks_for(A.n, kThreads) : 0, out);
    return cudaGetLastError();
}

}  // namespace mdk
