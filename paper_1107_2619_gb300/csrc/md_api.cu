// C ABI of libmd.so (declarations and contracts in include/md.h).
//
// Host-side orchestration of the hot path of the MOLDY method: argument checks (the paper
// halts before the run on an unsupported species, §3.1), the potential tables, the device
// buffers, and the order of the kernels in a velocity-Verlet step (§2.3):
//   [box *= strain] -> half kick + drift + skin check -> [rebuild: bin, sort, list]
//   -> density pass -> force pass + half kick (+ FP64 partial sums on the last step)
// The host never waits inside a multi-step call; device conditions are collected in a
// flags block and read once at the end.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "md_internal.cuh"

using namespace mdk;

struct md_ctx {
    md_config cfg{};
    cudaStream_t stream = nullptr;
    int64_t n = 0;
    int precision = MD_PREC_FP64;
    int ns = 1;
    double r_cut = 0, skin = 0, r_list = 0, rl2 = 0, lim2 = 0;
    double dt = 0, half_dt = 0, strain_scale = 1.0;
    double L[3] = {0, 0, 0};  // host mirror of the device box
    Atoms A{};
    Cells C{};
    Pot P{};
    Box *d_box = nullptr;
    Flags *d_flags = nullptr;
    double *d_reduce = nullptr;
    void *d_stage = nullptr;
    size_t stage_bytes = 0;
    Flags *h_flags = nullptr;   // pinned
    double *h_reduce = nullptr; // pinned [kPartials]
    std::vector<void *> allocs;
    int64_t step = 0;
    int lanes = 1;              // lanes per atom of the force passes
    bool list_valid = false, forces_valid = false, energy_valid = false;
    std::string err;
    // tracing
    int64_t launches = 0;
    bool profiling = false;
    md_profile prof{};
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
};

namespace {

// Kernels enqueued by one launch_rebuild (kept in step with md_neighbour.cu).
constexpr int kRebuildLaunches = 9;

md_status fail(md_ctx *c, md_status s, const std::string &what, cudaError_t e = cudaSuccess) {
    if (c) {
        c->err = what;
        if (e != cudaSuccess) {
            c->err += ": ";
            c->err += cudaGetErrorString(e);
        }
    }
    return s;
}

#define MD_CK(call)                                                          \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) return fail(ctx, MD_ERR_CUDA, #call, e_);     \
    } while (0)

template <typename T>
cudaError_t dalloc(md_ctx *ctx, T **p, size_t count) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, (count > 0 ? count : 1) * sizeof(T));
    if (e == cudaSuccess) {
        ctx->allocs.push_back(q);
        *p = static_cast<T *>(q);
    }
    return e;
}

float ulp32(double x) {
    int e;
    std::frexp(x, &e);  // x = m 2^e, m in [0.5, 1)
    return (float)std::ldexp(1.0, e - 24);
}

// FP32 screening band of the list build (see k_build_list).  Each wrapped FP32 coordinate is
// within u/2 of its FP64 value (u = ulp32 of the largest box edge); the FP32 difference and
// the minimum-image shift add at most 1.5u + ulp32(r_list)/2 more, so each component of d is
// within delta = 2u + ulp32(r_list)/2 of the FP64 one.  Then |r2_32 - r2_64| <= 2 sqrt(3) r_list
// delta + 3 delta^2 plus the FP32 rounding of r^2 (< 6e-7 r_list^2).  The band is 4x that.
void list_band(const md_ctx *c, float &lo, float &hi) {
    double Lmax = std::fmax(c->L[0], std::fmax(c->L[1], c->L[2]));
    double u = ulp32(Lmax);
    double delta = 2.0 * u + 0.5 * ulp32(c->r_list);
    double bound = 2.0 * std::sqrt(3.0) * c->r_list * delta + 3.0 * delta * delta + 6e-7 * c->rl2;
    double band = 4.0 * bound;
    lo = std::nextafter((float)(c->rl2 - band), -INFINITY);
    hi = std::nextafter((float)(c->rl2 + band), INFINITY);
}

int cells_along(double L, double r_list) {
    int nc = (int)std::floor(L / r_list);
    while (nc > 0 && L / nc < r_list * (1.0 + 1e-12)) nc--;
    return nc;
}

Box make_box(const double L[3]) {
    Box b;
    for (int k = 0; k < 3; k++) {
        b.L[k] = L[k];
        b.invL[k] = 1.0 / L[k];
        b.Lf[k] = (float)L[k];
        b.invLf[k] = (float)b.invL[k];
    }
    return b;
}

// Monomial coefficients of the cubic Hermite interpolant on each interval of a uniform knot
// grid, in t = (x - x_k)/h: c0 = y_k, c1 = h y'_k, c2 = 3(y_k+1 - y_k) - 2 h y'_k - h y'_k+1,
// c3 = 2(y_k - y_k+1) + h y'_k + h y'_k+1.  Row nk-1 continues linearly past the last knot.
void cubic_rows(const double *tab, int nk, double h, double4_32a *out64) {
    const double *y = tab, *yp = tab + nk;
    for (int k = 0; k < nk; k++) {
        double4_32a c;
        if (k < nk - 1) {
            double s0 = h * yp[k], s1 = h * yp[k + 1];
            c = make_double4_32a(y[k], s0, 3.0 * (y[k + 1] - y[k]) - 2.0 * s0 - s1,
                             2.0 * (y[k] - y[k + 1]) + s0 + s1);
        } else {
            c = make_double4_32a(y[k], h * yp[k], 0.0, 0.0);
        }
        out64[k] = c;
    }
}

md_status sync_and_check(md_ctx *ctx, bool strict_skin) {
    MD_CK(cudaMemcpyAsync(ctx->h_flags, ctx->d_flags, sizeof(Flags), cudaMemcpyDeviceToHost, ctx->stream));
    MD_CK(cudaStreamSynchronize(ctx->stream));
    const Flags &f = *ctx->h_flags;
    if (f.error & FLAG_OVERFLOW) {
        ctx->list_valid = false;
        return fail(ctx, MD_ERR_NBR_OVERFLOW,
                    "neighbour list overflow: " + std::to_string(f.max_count) + " > k_max " +
                        std::to_string(ctx->A.k_max));
    }
    if (f.error & FLAG_NONFINITE) return fail(ctx, MD_ERR_NONFINITE, "non-finite force");
    if (strict_skin && f.skin_exceeded)
        return fail(ctx, MD_ERR_SKIN, "an atom moved more than skin/2 between scheduled rebuilds");
    return MD_OK;
}

// Clear the sticky device error bits (called at the start of every compute call).
cudaError_t reset_errors(md_ctx *ctx) {
    cudaError_t e = cudaMemsetAsync(&ctx->d_flags->error, 0, sizeof(int32_t), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(&ctx->d_flags->skin_exceeded, 0, sizeof(int32_t), ctx->stream);
    return e;
}

cudaError_t enqueue_rebuild(md_ctx *ctx) {
    float lo, hi;
    list_band(ctx, lo, hi);
    return launch_rebuild(ctx->A, ctx->C, ctx->rl2, lo, hi, ctx->stream);
}

// Pass 1 + pass 2 at the current positions (rebuilding first if needed), with the FP64
// partial sums; enqueue only.
cudaError_t enqueue_forces(md_ctx *ctx) {
    ctx->launches += 4 + kRebuildLaunches + (ctx->list_valid ? 0 : 1);
    cudaError_t e = launch_check_displacement(ctx->A, ctx->lim2, ctx->stream);
    if (e == cudaSuccess && !ctx->list_valid) e = launch_set_rebuild(ctx->d_flags, ctx->stream);
    if (e == cudaSuccess) e = enqueue_rebuild(ctx);
    if (e == cudaSuccess) e = launch_density(ctx->A, ctx->P, ctx->precision, ctx->lanes, ctx->stream);
    if (e == cudaSuccess)
        e = launch_force(ctx->A, ctx->P, ctx->precision, ctx->lanes, false, true, 0.0, ctx->stream);
    if (e == cudaSuccess)
        e = launch_reduce(ctx->A, partial_blocks(ctx->A.n, ctx->lanes), ctx->d_reduce, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->h_reduce, ctx->d_reduce, sizeof(double) * kPartials,
                            cudaMemcpyDeviceToHost, ctx->stream);
    return e;
}

md_status compute_forces(md_ctx *ctx) {
    MD_CK(reset_errors(ctx));
    MD_CK(enqueue_forces(ctx));
    md_status s = sync_and_check(ctx, false);
    if (s != MD_OK) return s;
    ctx->list_valid = ctx->forces_valid = ctx->energy_valid = true;
    return MD_OK;
}

cudaEvent_t next_event(md_ctx *ctx) {
    if (ctx->ev_used == ctx->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        ctx->ev_pool.push_back(e);
    }
    return ctx->ev_pool[ctx->ev_used++];
}

// Record a profiling mark on the stream (no-op when profiling is off).
cudaError_t mark(md_ctx *ctx) {
    if (!ctx->profiling) return cudaSuccess;
    cudaEvent_t e = next_event(ctx);
    if (!e) return cudaErrorMemoryAllocation;
    return cudaEventRecord(e, ctx->stream);
}

// After a synchronisation: fold the marks of a step sequence (5 per step:
// start, after kick, after rebuild, after density, after force) into the sums.
void collect_marks(md_ctx *ctx) {
    if (!ctx->profiling) {
        ctx->ev_used = 0;
        return;
    }
    for (size_t b = 0; b + 4 < ctx->ev_used; b += 5) {
        float t[4];
        for (int k = 0; k < 4; k++) cudaEventElapsedTime(&t[k], ctx->ev_pool[b + k], ctx->ev_pool[b + k + 1]);
        ctx->prof.ms_kick += t[0];
        ctx->prof.ms_rebuild += t[1];
        ctx->prof.ms_density += t[2];
        ctx->prof.ms_force += t[3];
        ctx->prof.n_kick++;
        ctx->prof.n_rebuild++;
        ctx->prof.n_density++;
        ctx->prof.n_force++;
    }
    ctx->ev_used = 0;
}

md_status ensure_stage(md_ctx *ctx, size_t bytes) {
    if (ctx->stage_bytes >= bytes) return MD_OK;
    if (ctx->d_stage) {
        for (auto &p : ctx->allocs)
            if (p == ctx->d_stage) p = nullptr;
        cudaFree(ctx->d_stage);
        ctx->d_stage = nullptr;
        ctx->stage_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&ctx->d_stage, bytes);
    if (e != cudaSuccess) return fail(ctx, MD_ERR_OOM, "staging buffer", e);
    ctx->stage_bytes = bytes;
    return MD_OK;
}

md_status copy_out(md_ctx *ctx, const void *src, void *dst, size_t bytes, int on_device) {
    MD_CK(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          ctx->stream));
    MD_CK(cudaStreamSynchronize(ctx->stream));
    return MD_OK;
}

}  // namespace

extern "C" {

int32_t md_abi_version(void) { return MD_ABI_VERSION; }

const char *md_status_string(md_status s) {
    switch (s) {
        case MD_OK: return "ok";
        case MD_ERR_ARG: return "invalid argument";
        case MD_ERR_SPECIES: return "unsupported species";
        case MD_ERR_BOX: return "invalid box";
        case MD_ERR_NBR_OVERFLOW: return "neighbour list overflow";
        case MD_ERR_SKIN: return "skin exceeded";
        case MD_ERR_NONFINITE: return "non-finite value";
        case MD_ERR_TABLE_RANGE: return "table range";
        case MD_ERR_TIMEOUT: return "device wait timed out";
        case MD_ERR_CUDA: return "CUDA error";
        case MD_ERR_OOM: return "out of device memory";
        case MD_ERR_STATE: return "invalid state";
        case MD_ERR_CAPACITY: return "input exceeds a fixed capacity";
    }
    return "unknown status";
}

const char *md_last_error(const md_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void md_destroy(md_ctx *ctx) {
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    for (void *p : ctx->allocs)
        if (p) cudaFree(p);
    if (ctx->d_stage) cudaFree(ctx->d_stage);
    if (ctx->h_flags) cudaFreeHost(ctx->h_flags);
    if (ctx->h_reduce) cudaFreeHost(ctx->h_reduce);
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    delete ctx;
}

md_status md_create(const md_config *cfg, const md_potential *pot, const double *pos, const double *vel,
                    const int32_t *species, int32_t on_device, md_ctx **out) {
    if (!out) return MD_ERR_ARG;
    *out = nullptr;
    if (!cfg || !pot || (!pos && cfg->n_atoms > 0)) return MD_ERR_ARG;
    md_ctx *ctx = new (std::nothrow) md_ctx();
    if (!ctx) return MD_ERR_OOM;
    auto bail = [&](md_status s) {
        std::string keep = ctx->err;
        md_destroy(ctx);
        (void)keep;
        return s;
    };
    ctx->cfg = *cfg;
    ctx->stream = static_cast<cudaStream_t>(cfg->stream);
    const int64_t n = cfg->n_atoms;
    if (n < 0 || n > INT32_MAX / 2) return bail(MD_ERR_ARG);
    if (cfg->k_max < 1 || cfg->skin < 0.0 || !(cfg->dt_fs >= 0.0) || cfg->rebuild_every < 0)
        return bail(MD_ERR_ARG);
    if (cfg->precision != MD_PREC_FP64 && cfg->precision != MD_PREC_MIXED) return bail(MD_ERR_ARG);
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
            if (a != b && cfg->h[3 * a + b] != 0.0) return bail(MD_ERR_BOX);
    for (int k = 0; k < 3; k++) {
        ctx->L[k] = cfg->h[4 * k];
        if (!(ctx->L[k] > 0.0)) return bail(MD_ERR_BOX);
    }
    // potential (§3.1)
    int ns = pot->n_species;
    if (pot->kind == MD_POT_FS_ANALYTIC) {
        if (ns != 1 || !(pot->r_cut > 0.0) || pot->fs[0] <= 0.0) return bail(MD_ERR_ARG);
    } else if (pot->kind == MD_POT_TABLES) {
        if (ns < 1 || ns > 8 || pot->n_knots < 2 || !pot->tables || !(pot->r_cut > pot->r_min) ||
            !(pot->rho_max > pot->rho_min))
            return bail(MD_ERR_ARG);
    } else {
        return bail(MD_ERR_ARG);
    }
    if (!pot->masses_amu) return bail(MD_ERR_ARG);
    std::vector<double> mass(ns);
    for (int a = 0; a < ns; a++) {
        mass[a] = pot->masses_amu[a];
        if (!(mass[a] > 0.0)) return bail(MD_ERR_ARG);
    }
    ctx->ns = ns;
    ctx->n = n;
    ctx->precision = cfg->precision;
    ctx->r_cut = pot->r_cut;
    ctx->skin = cfg->skin;
    ctx->r_list = pot->r_cut + cfg->skin;
    ctx->rl2 = ctx->r_list * ctx->r_list;
    ctx->lim2 = 0.25 * cfg->skin * cfg->skin;
    ctx->dt = cfg->dt_fs;
    ctx->half_dt = 0.5 * cfg->dt_fs;
    ctx->strain_scale = 1.0 + cfg->strain_rate_zz * cfg->dt_fs * 1.0e-15;
    for (int k = 0; k < 3; k++) {
        ctx->C.nc[k] = cells_along(ctx->L[k], ctx->r_list);
        if (ctx->C.nc[k] < 3) {
            ctx->err = "box edge holds fewer than 3 link cells of width r_cut + skin";
            return bail(MD_ERR_BOX);
        }
    }
    // lanes per atom: given, or from the expected neighbour count (4/3 pi r_list^3 x density)
    {
        const int want = cfg->lanes_per_atom;
        if (want != 0 && (want < 1 || want > 32 || (want & (want - 1)) != 0)) return bail(MD_ERR_ARG);
        if (want) {
            ctx->lanes = want;
        } else {
            const double vol = ctx->L[0] * ctx->L[1] * ctx->L[2];
            const double k_est = 4.18879020478639 * ctx->r_list * ctx->r_list * ctx->r_list * (double)n / vol;
            int t = 1;
            while (t < 32 && t * 12 < k_est) t *= 2;
            ctx->lanes = t;
        }
    }
    // host copies of the inputs
    std::vector<double> hpos(3 * n), hvel(3 * n, 0.0);
    std::vector<int32_t> hspec(n, 0);
    if (n > 0) {
        auto fetch = [&](void *dst, const void *src, size_t bytes) {
            if (!on_device) {
                std::memcpy(dst, src, bytes);
                return true;
            }
            return cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost) == cudaSuccess;
        };
        if (!fetch(hpos.data(), pos, sizeof(double) * 3 * n)) return bail(MD_ERR_CUDA);
        if (vel && !fetch(hvel.data(), vel, sizeof(double) * 3 * n)) return bail(MD_ERR_CUDA);
        if (species && !fetch(hspec.data(), species, sizeof(int32_t) * n)) return bail(MD_ERR_CUDA);
    }
    for (int64_t i = 0; i < n; i++) {
        if (hspec[i] < 0 || hspec[i] >= ns) {
            ctx->err = "atom " + std::to_string(i) + " has species " + std::to_string(hspec[i]) +
                       " not supported by the potential";
            return bail(MD_ERR_SPECIES);
        }
        for (int c = 0; c < 3; c++)
            if (!std::isfinite(hpos[3 * i + c]) || !std::isfinite(hvel[3 * i + c])) return bail(MD_ERR_NONFINITE);
    }
    const double acc = 1.0 / kMvv2e;  // (eV/Å)/amu -> Å/fs^2
    std::vector<double4_32a> p4(n), v4(n), f4(n);
    std::vector<int32_t> iota(n);
    for (int64_t i = 0; i < n; i++) {
        double m = mass[hspec[i]];
        p4[i] = make_double4_32a(hpos[3 * i], hpos[3 * i + 1], hpos[3 * i + 2], (double)hspec[i]);
        v4[i] = make_double4_32a(hvel[3 * i], hvel[3 * i + 1], hvel[3 * i + 2], acc / m);
        f4[i] = make_double4_32a(0.0, 0.0, 0.0, m);
        iota[i] = (int32_t)i;
    }
    // device buffers
    Atoms &A = ctx->A;
    A.n = (int)n;
    A.k_max = cfg->k_max;
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t r) { if (r != cudaSuccess && e == cudaSuccess) e = r; };
    chk(dalloc(ctx, &A.pos, n)); chk(dalloc(ctx, &A.vel, n)); chk(dalloc(ctx, &A.force, n));
    chk(dalloc(ctx, &A.ref, n)); chk(dalloc(ctx, &A.pos_tmp, n)); chk(dalloc(ctx, &A.vel_tmp, n));
    chk(dalloc(ctx, &A.force_tmp, n)); chk(dalloc(ctx, &A.posf, n)); chk(dalloc(ctx, &A.p2f, n));
    chk(dalloc(ctx, &A.p2d, n));
    chk(dalloc(ctx, &A.rho, n)); chk(dalloc(ctx, &A.dF, n)); chk(dalloc(ctx, &A.e_atom, n));
    chk(dalloc(ctx, &A.id, n)); chk(dalloc(ctx, &A.id_tmp, n)); chk(dalloc(ctx, &A.rank, n));
    chk(dalloc(ctx, &A.spec, n)); chk(dalloc(ctx, &A.spec_tmp, n)); chk(dalloc(ctx, &A.cell_of, n));
    chk(dalloc(ctx, &A.slot, n)); chk(dalloc(ctx, &A.order, n)); chk(dalloc(ctx, &A.count, n));
    chk(dalloc(ctx, &A.nbr, (size_t)n * cfg->k_max));
    const int nblocks = n > 0 ? partial_blocks((int)n, 32) : 1;  // enough rows for any lane count
    chk(dalloc(ctx, &A.partials, (size_t)nblocks * kPartials));
    chk(dalloc(ctx, &ctx->d_box, 1));
    chk(dalloc(ctx, &ctx->d_flags, 1));
    chk(dalloc(ctx, &ctx->d_reduce, kPartials));
    Cells &C = ctx->C;
    C.ncell = C.nc[0] * C.nc[1] * C.nc[2];
    C.ntiles = (C.ncell + 4095) / 4096;
    chk(dalloc(ctx, &C.cell_count, C.ncell));
    chk(dalloc(ctx, &C.cell_start, C.ncell + 1));
    chk(dalloc(ctx, &C.tile_sums, C.ntiles));
    if (e != cudaSuccess) return bail(fail(ctx, MD_ERR_OOM, "device allocation", e));
    A.box = ctx->d_box;
    A.flags = ctx->d_flags;
    if (cudaMallocHost(&ctx->h_flags, sizeof(Flags)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_reduce, sizeof(double) * kPartials) != cudaSuccess)
        return bail(MD_ERR_OOM);
    std::memset(ctx->h_flags, 0, sizeof(Flags));
    std::memset(ctx->h_reduce, 0, sizeof(double) * kPartials);
    // potential tables
    Pot &P = ctx->P;
    P.kind = pot->kind;
    P.ns = ns;
    P.rc2 = pot->r_cut * pot->r_cut;
    P.rc2f = (float)P.rc2;
    for (int k = 0; k < 7; k++) {
        P.fs[k] = pot->fs[k];
        P.fsf[k] = (float)pot->fs[k];
    }
    if (pot->kind == MD_POT_FS_ANALYTIC) {
        P.bd = pot->fs[3] / pot->fs[0];
        P.bdf = (float)P.bd;
    }
    if (pot->kind == MD_POT_TABLES) {
        const int nk = pot->n_knots;
        P.nk = nk;
        P.r_min = pot->r_min;
        P.inv_dr = (nk - 1) / (pot->r_cut - pot->r_min);
        P.rho_min = pot->rho_min;
        P.inv_drho = (nk - 1) / (pot->rho_max - pot->rho_min);
        P.r_minf = (float)P.r_min;
        P.inv_drf = (float)P.inv_dr;
        const double hr = (pot->r_cut - pot->r_min) / (nk - 1);
        const double hrho = (pot->rho_max - pot->rho_min) / (nk - 1);
        const size_t npair = (size_t)ns * ns;
        std::vector<double4_32a> VP64(npair * nk * 2), F64((size_t)ns * nk), rv(nk), rp(nk);
        std::vector<float> VP32(npair * nk * 8);
        const size_t tl = 2 * (size_t)nk;
        for (int a = 0; a < ns; a++)
            for (int b = 0; b < ns; b++) {
                const double *tv = pot->tables + (size_t)(a * ns + b) * tl;
                const double *tvt = pot->tables + (size_t)(b * ns + a) * tl;
                for (size_t q = 0; q < tl; q++)
                    if (tv[q] != tvt[q]) {
                        ctx->err = "V table must be symmetric in its two species";
                        return bail(MD_ERR_ARG);
                    }
                cubic_rows(tv, nk, hr, rv.data());
                cubic_rows(pot->tables + (npair + a * ns + b) * tl, nk, hr, rp.data());
                const size_t base = (size_t)(a * ns + b) * nk;
                for (int k = 0; k < nk; k++) {
                    VP64[(base + k) * 2] = rv[k];
                    VP64[(base + k) * 2 + 1] = rp[k];
                    float *f = &VP32[(base + k) * 8];
                    const double c[8] = {rv[k].x, rv[k].y, rv[k].z, rv[k].w, rp[k].x, rp[k].y, rp[k].z, rp[k].w};
                    for (int q = 0; q < 8; q++) f[q] = (float)c[q];
                }
            }
        for (int a = 0; a < ns; a++)
            cubic_rows(pot->tables + (2 * npair + a) * tl, nk, hrho, &F64[(size_t)a * nk]);
        double4_32a *dVP64, *dVP32, *dF64;
        chk(dalloc(ctx, &dVP64, VP64.size()));
        chk(dalloc(ctx, &dVP32, VP32.size() / 8));
        chk(dalloc(ctx, &dF64, F64.size()));
        if (e != cudaSuccess) return bail(fail(ctx, MD_ERR_OOM, "table allocation", e));
        chk(cudaMemcpy(dVP64, VP64.data(), VP64.size() * sizeof(double4_32a), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(dVP32, VP32.data(), VP32.size() * sizeof(float), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(dF64, F64.data(), F64.size() * sizeof(double4_32a), cudaMemcpyHostToDevice));
        P.VP64 = dVP64;
        P.VP32 = dVP32;
        P.F64 = dF64;
    }
    // initial state (caller order = cell order until the first build)
    Box box = make_box(ctx->L);
    Flags flags{};
    flags.need_rebuild = 1;
    if (n > 0) {
        chk(cudaMemcpy(A.pos, p4.data(), n * sizeof(double4_32a), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(A.ref, p4.data(), n * sizeof(double4_32a), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(A.vel, v4.data(), n * sizeof(double4_32a), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(A.force, f4.data(), n * sizeof(double4_32a), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(A.id, iota.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(A.rank, iota.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(A.spec, hspec.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
    chk(cudaMemcpy(ctx->d_box, &box, sizeof(Box), cudaMemcpyHostToDevice));
    chk(cudaMemcpy(ctx->d_flags, &flags, sizeof(Flags), cudaMemcpyHostToDevice));
    chk(cudaMemset(C.cell_count, 0, sizeof(int32_t) * C.ncell));
    chk(cudaMemset(A.partials, 0, sizeof(double) * nblocks * kPartials));
    chk(cudaDeviceSynchronize());
    chk(launch_wrap(A, ctx->stream));
    chk(cudaStreamSynchronize(ctx->stream));
    if (e != cudaSuccess) return bail(fail(ctx, MD_ERR_CUDA, "initial upload", e));
    *out = ctx;
    return MD_OK;
}

md_status md_build_neighbours(md_ctx *ctx) {
    if (!ctx) return MD_ERR_ARG;
    MD_CK(reset_errors(ctx));
    MD_CK(launch_set_rebuild(ctx->d_flags, ctx->stream));
    MD_CK(enqueue_rebuild(ctx));
    MD_CK(launch_clear_rebuild(ctx->d_flags, ctx->stream));
    ctx->launches += 2 + kRebuildLaunches;
    md_status s = sync_and_check(ctx, false);
    if (s != MD_OK) return s;
    ctx->list_valid = true;
    ctx->energy_valid = false;  // per-atom rho/F'/energies are not renumbered
    return MD_OK;
}

md_status md_eam_forces(md_ctx *ctx, double *pe_out) {
    if (!ctx) return MD_ERR_ARG;
    md_status s = compute_forces(ctx);
    if (s != MD_OK) return s;
    if (pe_out) *pe_out = ctx->h_reduce[0];
    return MD_OK;
}

md_status md_step(md_ctx *ctx, int32_t n_steps) {
    if (!ctx || n_steps < 0) return MD_ERR_ARG;
    if (n_steps == 0) return MD_OK;
    // link cells are fixed in fractional coordinates; under compression keep them >= r_list wide
    if (ctx->strain_scale != 1.0) {
        double Lz = ctx->L[2];
        for (int32_t s = 0; s < n_steps; s++) Lz *= ctx->strain_scale;
        int nc = cells_along(std::fmin(Lz, ctx->L[2]), ctx->r_list);
        if (nc < 3) return fail(ctx, MD_ERR_BOX, "strain made the box thinner than 3 link cells");
        if (nc < ctx->C.nc[2]) {
            ctx->C.nc[2] = nc;
            ctx->C.ncell = ctx->C.nc[0] * ctx->C.nc[1] * nc;
            ctx->C.ntiles = (ctx->C.ncell + 4095) / 4096;
        }
    }
    MD_CK(reset_errors(ctx));
    if (!ctx->forces_valid) {
        MD_CK(enqueue_forces(ctx));
    }
    const int every = ctx->cfg.rebuild_every;
    for (int32_t s = 0; s < n_steps; s++) {
        MD_CK(mark(ctx));
        if (ctx->strain_scale != 1.0) {
            MD_CK(launch_box_update(ctx->d_box, ctx->strain_scale, ctx->stream));
            ctx->L[2] *= ctx->strain_scale;
            ctx->launches++;
        }
        MD_CK(launch_kick_drift(ctx->A, ctx->half_dt, ctx->dt, ctx->strain_scale, ctx->lim2, ctx->stream));
        MD_CK(mark(ctx));
        if (every > 0 && (ctx->step + 1) % every == 0) {
            MD_CK(launch_set_rebuild(ctx->d_flags, ctx->stream));
            ctx->launches++;
        }
        MD_CK(enqueue_rebuild(ctx));
        MD_CK(mark(ctx));
        MD_CK(launch_density(ctx->A, ctx->P, ctx->precision, ctx->lanes, ctx->stream));
        MD_CK(mark(ctx));
        MD_CK(launch_force(ctx->A, ctx->P, ctx->precision, ctx->lanes, true, s == n_steps - 1, ctx->half_dt,
                           ctx->stream));
        MD_CK(mark(ctx));
        ctx->launches += 3 + kRebuildLaunches;
        ctx->step++;
    }
    MD_CK(launch_reduce(ctx->A, partial_blocks(ctx->A.n, ctx->lanes), ctx->d_reduce, ctx->stream));
    ctx->launches++;
    MD_CK(cudaMemcpyAsync(ctx->h_reduce, ctx->d_reduce, sizeof(double) * kPartials, cudaMemcpyDeviceToHost,
                          ctx->stream));
    md_status st = sync_and_check(ctx, ctx->cfg.strict_skin != 0);
    collect_marks(ctx);
    if (st != MD_OK) {
        ctx->forces_valid = ctx->energy_valid = false;
        return st;
    }
    ctx->list_valid = ctx->forces_valid = ctx->energy_valid = true;
    return MD_OK;
}

md_status md_energy(md_ctx *ctx, md_energies *out) {
    if (!ctx || !out) return MD_ERR_ARG;
    if (!ctx->energy_valid) {
        md_status s = compute_forces(ctx);
        if (s != MD_OK) return s;
    }
    const double *r = ctx->h_reduce;
    std::memset(out, 0, sizeof(*out));
    out->pe = r[0];
    out->ke = 0.5 * r[1] * kMvv2e;
    out->te = out->pe + out->ke;
    out->temperature = ctx->n > 1 ? 2.0 * out->ke / ((double)(3 * ctx->n - 3) * kKb) : 0.0;
    const double W[9] = {r[2], r[7], r[6], r[7], r[3], r[5], r[6], r[5], r[4]};
    std::memcpy(out->virial, W, sizeof(W));
    out->volume = ctx->L[0] * ctx->L[1] * ctx->L[2];
    out->pressure_gpa = (2.0 * out->ke + r[2] + r[3] + r[4]) / (3.0 * out->volume) * kEva3ToGpa;
    for (int k = 0; k < 3; k++) {
        out->momentum[k] = r[8 + k];
        out->box[k] = ctx->L[k];
    }
    out->step = ctx->step;
    out->n_rebuilds = (int64_t)ctx->h_flags->n_rebuilds;
    out->max_neighbours = ctx->h_flags->max_count;
    out->range_violations = (int64_t)ctx->h_flags->range_violations;
    return MD_OK;
}

md_status md_get(md_ctx *ctx, int32_t what, void *dst, int32_t on_device) {
    if (!ctx || (!dst && ctx->n > 0)) return MD_ERR_ARG;
    const int64_t n = ctx->n;
    if (n == 0) return MD_OK;
    Atoms &A = ctx->A;
    md_status s;
    switch (what) {
        case MD_GET_POS:
        case MD_GET_VEL:
        case MD_GET_FORCE: {
            if (what == MD_GET_FORCE && !ctx->forces_valid && (s = compute_forces(ctx)) != MD_OK) return s;
            if ((s = ensure_stage(ctx, sizeof(double) * 3 * n)) != MD_OK) return s;
            const double4_32a *src = what == MD_GET_POS ? A.pos : (what == MD_GET_VEL ? A.vel : A.force);
            MD_CK(launch_unsort_vec(A, src, static_cast<double *>(ctx->d_stage), ctx->stream));
            return copy_out(ctx, ctx->d_stage, dst, sizeof(double) * 3 * n, on_device);
        }
        case MD_GET_RHO:
        case MD_GET_EATOM:
        case MD_GET_DF: {
            if (!ctx->energy_valid && (s = compute_forces(ctx)) != MD_OK) return s;
            if ((s = ensure_stage(ctx, sizeof(double) * n)) != MD_OK) return s;
            const double *src = what == MD_GET_RHO ? A.rho : (what == MD_GET_EATOM ? A.e_atom : A.dF);
            MD_CK(launch_unsort_scalar(A, src, static_cast<double *>(ctx->d_stage), ctx->stream));
            return copy_out(ctx, ctx->d_stage, dst, sizeof(double) * n, on_device);
        }
        case MD_GET_NBR_COUNT:
        case MD_GET_SPECIES: {
            if (what == MD_GET_NBR_COUNT && !ctx->list_valid && (s = md_build_neighbours(ctx)) != MD_OK) return s;
            if ((s = ensure_stage(ctx, sizeof(int32_t) * n)) != MD_OK) return s;
            MD_CK(launch_unsort_int(A, what == MD_GET_NBR_COUNT ? A.count : A.spec,
                                    static_cast<int32_t *>(ctx->d_stage), ctx->stream));
            return copy_out(ctx, ctx->d_stage, dst, sizeof(int32_t) * n, on_device);
        }
        case MD_GET_NBR_LIST: {
            if (!ctx->list_valid && (s = md_build_neighbours(ctx)) != MD_OK) return s;
            const size_t bytes = sizeof(int32_t) * (size_t)n * A.k_max;
            if ((s = ensure_stage(ctx, bytes)) != MD_OK) return s;
            MD_CK(launch_unsort_list(A, static_cast<int32_t *>(ctx->d_stage), ctx->stream));
            return copy_out(ctx, ctx->d_stage, dst, bytes, on_device);
        }
        default:
            return fail(ctx, MD_ERR_ARG, "unknown md_get selector");
    }
}

md_status md_tune(md_ctx *ctx, int32_t *lanes_out) {
    if (!ctx) return MD_ERR_ARG;
    md_status st = ctx->list_valid ? MD_OK : md_build_neighbours(ctx);
    if (st != MD_OK) return st;
    if (ctx->n > 0) {
        cudaEvent_t e0, e1;
        MD_CK(cudaEventCreate(&e0));
        MD_CK(cudaEventCreate(&e1));
        float best = 1e30f;
        int best_t = ctx->lanes;
        const int keep = ctx->lanes;
        for (int t = 1; t <= 32; t *= 2) {
            ctx->lanes = t;
            for (int rep = 0; rep < 4; rep++) {  // first round is a warm-up
                MD_CK(cudaEventRecord(e0, ctx->stream));
                MD_CK(launch_density(ctx->A, ctx->P, ctx->precision, t, ctx->stream));
                MD_CK(launch_force(ctx->A, ctx->P, ctx->precision, t, false, false, 0.0, ctx->stream));
                MD_CK(cudaEventRecord(e1, ctx->stream));
                MD_CK(cudaEventSynchronize(e1));
                float ms = 0.f;
                MD_CK(cudaEventElapsedTime(&ms, e0, e1));
                if (rep > 0 && ms < best) {
                    best = ms;
                    best_t = t;
                }
                ctx->launches += 2;
            }
        }
        (void)keep;
        ctx->lanes = best_t;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        ctx->energy_valid = false;  // partial-sum rows depend on the lane count
        st = sync_and_check(ctx, false);
        if (st != MD_OK) return st;
    }
    if (lanes_out) *lanes_out = ctx->lanes;
    return MD_OK;
}

md_status md_set_profiling(md_ctx *ctx, int32_t on) {
    if (!ctx) return MD_ERR_ARG;
    ctx->profiling = on != 0;
    const int64_t launches = ctx->prof.launches;
    ctx->prof = md_profile{};
    ctx->prof.launches = launches;
    ctx->ev_used = 0;
    return MD_OK;
}

md_status md_get_profile(const md_ctx *ctx, md_profile *out) {
    if (!ctx || !out) return MD_ERR_ARG;
    *out = ctx->prof;
    out->launches = ctx->launches;
    return MD_OK;
}

md_status md_set_state(md_ctx *ctx, const double *pos, const double *vel, const double *force,
                       int32_t on_device) {
    if (!ctx) return MD_ERR_ARG;
    const int64_t n = ctx->n;
    if (n == 0) return MD_OK;
    md_status s;
    if ((s = ensure_stage(ctx, sizeof(double) * 3 * n)) != MD_OK) return s;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const double *src[3] = {pos, vel, force};
    double4_32a *dst[3] = {ctx->A.pos, ctx->A.vel, ctx->A.force};
    for (int q = 0; q < 3; q++) {
        if (!src[q]) continue;
        MD_CK(cudaMemcpyAsync(ctx->d_stage, src[q], sizeof(double) * 3 * n, kind, ctx->stream));
        MD_CK(launch_sort_in_vec(ctx->A, static_cast<const double *>(ctx->d_stage), dst[q], ctx->stream));
    }
    if (pos) MD_CK(launch_wrap(ctx->A, ctx->stream));
    MD_CK(cudaStreamSynchronize(ctx->stream));
    if (pos || force) ctx->forces_valid = (force != nullptr);
    ctx->energy_valid = false;
    return MD_OK;
}

}  // extern "C"
