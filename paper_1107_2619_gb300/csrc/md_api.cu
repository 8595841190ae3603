// C ABI of libmd.so (declarations and contracts in include/md.h).
//
// Host-side orchestration of the hot path of the MOLDY method: argument checks (the paper
// halts before the run on an unsupported species, §3.1), the potential tables, the device
// buffers, and the launches.  A step sequence md_step(n) is ONE cooperative launch of the
// persistent step kernel (md_step.cuh): half kick + drift + skin check, [list rebuild],
// density pass, force pass + half kick, for n steps (§2.3), followed by the FP64 reduction
// of the last step's energies.  The host never waits inside it; device conditions are
// collected in a flags block and read once at the end.
//
// A context holds one system or a batch of independent replicas (md_create_batch): the
// replicas' atoms are stored back to back, each replica with its own box and link cells,
// and one launch advances all of them.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "md_df.cuh"
#include "md_internal.cuh"

using namespace mdk;

struct md_ctx {
    md_config cfg{};
    cudaStream_t stream = nullptr;
    int64_t n = 0;
    int precision = MD_PREC_FP64;
    int ns = 1;
    int n_rep = 1;
    std::vector<int64_t> rep_off;        // [n_rep + 1] first atom of each replica
    std::vector<double> L;               // [3 n_rep] host mirror of the device boxes
    double r_cut = 0, skin = 0, r_list = 0, rl2 = 0, lim2 = 0;
    double dt = 0, half_dt = 0, strain_scale = 1.0;
    Atoms A{};
    Cells C{};
    Pot P{};
    std::vector<RepCells> rc;            // host copy of the per-replica cell grids
    Box *d_boxes = nullptr;
    RepCells *d_rc = nullptr;
    int32_t *d_rep_off = nullptr;
    Flags *d_flags = nullptr;
    GridBarrier *d_bar = nullptr;
    double *d_reduce = nullptr;
    double *d_rep_sums = nullptr;
    unsigned long long *d_stamps = nullptr;
    size_t stamps_cap = 0;
    void *d_stage = nullptr;
    size_t stage_bytes = 0;
    Flags *h_flags = nullptr;            // pinned
    double *h_reduce = nullptr;          // pinned [kPartials]
    unsigned long long *h_stamps = nullptr;  // pinned
    std::vector<void *> allocs;
    int64_t step = 0;
    int lanes = 1;
    int part_rows = 0;                   // rows of partial sums written by the last energy pass
    bool list_valid = false, forces_valid = false, energy_valid = false;
    std::string err;
    // tracing
    int64_t launches = 0;
    bool profiling = false;
    md_profile prof{};
    // CUDA graphs of step sequences, keyed by the number of steps
    bool use_graph = false;
    cudaStream_t cap_stream = nullptr;   // private stream the graphs are recorded on
    std::map<int, cudaGraphExec_t> graphs;
    std::map<int, int> graph_rows;
    std::map<int, int> graph_launches;
    // Nose-Hoover thermostat (md_set_thermostat)
    bool thermo_on = false;
    Thermo *d_thermo = nullptr;
    int2 *d_ke_chunks = nullptr;
    int n_ke_chunks = 0;
    std::vector<double> h_rep;           // [5 n_rep] replica sums after the last thermostatted md_step
    // learned surrogate (kind MD_POT_SURROGATE)
    bool sur = false;          // context kind
    bool sur_set = false;      // network given
    bool sur_img_stale = true; // bf16 operand image older than theta
    bool sur_ref = false;      // training references valid for the current positions
    md_surrogate sur_spec{};
    SurNet S{};
    float *d_theta = nullptr, *d_adam_m = nullptr, *d_adam_v = nullptr, *d_gmu = nullptr, *d_ginv = nullptr;
    float *d_grad = nullptr;
    unsigned char *d_img = nullptr;
    double4_32a *d_fref = nullptr;
    int adam_t = 0;
    int sur_part_blocks = 0;
};

namespace {

constexpr int kRebuildLaunches = 9;                     // kernels of one stand-alone launch_rebuild
constexpr unsigned long long kSpinLimit = 20000000ull;  // barrier polls (~2 s) before giving up

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

// FP32 screening band of the list build (ph::build_cell_group).  Each wrapped FP32 coordinate is
// within u/2 of its FP64 value (u = ulp32 of the largest box edge); adding the FP32 box edge
// for a periodic neighbour cell (itself within u/2 of the FP64 edge) rounds once more (< u)
// and the difference once more (< ulp32(r_list)/2 near the cutoff), so each component of d is
// within delta = 3u + ulp32(r_list)/2 of the FP64 one.  Then |r2_32 - r2_64| <= 2 sqrt(3)
// r_list delta + 3 delta^2 plus the FP32 rounding of r^2 (< 6e-7 r_list^2).  The band is 4x.
// The same bound for r_cut: an FP32 r^2 above rc2 + 4 bound is beyond r_cut in FP64 too.
float cut_skin_bound(const md_ctx *c, double r_cut) {
    double Lmax = 0.0;
    for (double l : c->L) Lmax = std::fmax(Lmax, l);
    const double u = ulp32(Lmax), rc2 = r_cut * r_cut;
    const double delta = 3.0 * u + 0.5 * ulp32(r_cut);
    const double bound = 2.0 * std::sqrt(3.0) * r_cut * delta + 3.0 * delta * delta + 6e-7 * rc2;
    return std::nextafter((float)(rc2 + 4.0 * bound), INFINITY);
}

void list_band(const md_ctx *c, float &lo, float &hi) {
    double Lmax = 0.0;
    for (double l : c->L) Lmax = std::fmax(Lmax, l);
    double u = ulp32(Lmax);
    double delta = 3.0 * u + 0.5 * ulp32(c->r_list);
    double bound = 2.0 * std::sqrt(3.0) * c->r_list * delta + 3.0 * delta * delta + 6e-7 * c->rl2;
    double band = 4.0 * bound;
    lo = std::nextafter((float)(c->rl2 - band), -INFINITY);
    hi = std::nextafter((float)(c->rl2 + band), INFINITY);
}

// Lanes per link cell of the list build, from the mean cell occupancy (a whole warp per cell
// above 12 atoms: on GB300 the single broadcast candidate stream of a warp-wide group built the
// fcc Cu list faster than 8-lane groups with fewer idle lanes, 1.29 against about 1.8 ms per build;
// 4 lanes up to 6 atoms: the bcc Fe lists about 4 % faster than with 8).
#ifndef MD_LIST_GROUP_MAX
#define MD_LIST_GROUP_MAX 32
#endif
int ph_list_group(const md_ctx *c) {
    const double m = c->C.ncell > 0 ? (double)c->n / (double)c->C.ncell : 0.0;
    return std::min(MD_LIST_GROUP_MAX, m <= 6.0 ? 4 : (m <= 12.0 ? 16 : 32));
}

// Link cells of width >= r_list along an edge of length L.  The count is capped at 2^20 before
// the integer conversion (a grid that large fails the total-cell check of md_create anyway).
int cells_along(double L, double r_list) {
    const double q = std::floor(L / r_list);
    int nc = q < 1048576.0 ? (int)q : 1048576;
    while (nc > 0 && L / nc < r_list * (1.0 + 1e-12)) nc--;
    return nc;
}

// skin: the double-float offset xoff = 2 (L + skin) + 1 keeps every image coordinate plus xoff
// within a factor of two of every other (image coordinates lie in [-skin/2, L + skin/2)), also
// while a strain ramp shrinks the box, so that differences of their FP32 high parts are exact.
Box make_box(const double *L, double skin) {
    Box b;
    for (int k = 0; k < 3; k++) {
        b.L[k] = L[k];
        b.invL[k] = 1.0 / L[k];
        b.Lf[k] = (float)L[k];
        b.invLf[k] = (float)b.invL[k];
        b.Lh[k] = (float)L[k];
        b.Ll[k] = (float)(L[k] - (double)b.Lh[k]);
        b.xoff[k] = 2.0 * (L[k] + skin) + 1.0;
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
    if (f.error & FLAG_TIMEOUT) {
        ctx->forces_valid = ctx->energy_valid = false;
        return fail(ctx, MD_ERR_TIMEOUT, "a grid barrier of the step kernel gave up waiting");
    }
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
    return launch_rebuild(ctx->A, ctx->C, ctx->rl2, lo, hi, ph_list_group(ctx), ctx->stream);
}

// Surrogate network at the current positions (list valid): descriptors, then energies and
// dE/dG of every atom.
cudaError_t enqueue_sur_net(md_ctx *ctx, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    if (ctx->S.bf16 && ctx->sur_img_stale) {
        e = launch_sur_pack(ctx->d_theta, ctx->d_img, s);
        ctx->sur_img_stale = false;
        ctx->launches++;
    }
    if (e == cudaSuccess) e = launch_sur_descriptors(ctx->A, ctx->S, 0, (int)ctx->n, s);
    if (e == cudaSuccess)
        e = ctx->S.bf16 ? launch_sur_net_tc(ctx->A, ctx->S, s) : launch_sur_net32(ctx->A, ctx->S, 0, (int)ctx->n, s);
    ctx->launches += 2;
    return e;
}

// One velocity-Verlet step of the surrogate: half kick + drift (+ skin check), list rebuild
// when flagged (the rebuild kernels return at once otherwise), network, force + half kick.
cudaError_t enqueue_sur_step(md_ctx *ctx, bool energy, bool scheduled_rebuild, int *rows, cudaStream_t s) {
    cudaError_t e = launch_sur_kick_drift(ctx->A, ctx->half_dt, ctx->dt, ctx->lim2, s);
    if (e == cudaSuccess && scheduled_rebuild) e = launch_set_rebuild(ctx->d_flags, s);
    float lo, hi;
    list_band(ctx, lo, hi);
    if (e == cudaSuccess) e = launch_rebuild(ctx->A, ctx->C, ctx->rl2, lo, hi, ph_list_group(ctx), s);
    if (e == cudaSuccess) e = launch_clear_rebuild(ctx->d_flags, s);
    if (e == cudaSuccess) e = enqueue_sur_net(ctx, s);
    if (e == cudaSuccess)
        e = launch_sur_force(ctx->A, ctx->S, 0, (int)ctx->n, true, energy, ctx->half_dt, 0.0, rows, s);
    ctx->launches += 3 + kRebuildLaunches + (scheduled_rebuild ? 1 : 0);
    return e;
}

// Pass 1 + pass 2 at the current positions with stand-alone kernels (rebuilding first if
// needed), with the FP64 partial sums; enqueue only.
cudaError_t enqueue_forces(md_ctx *ctx) {
    if (ctx->sur) {
        ctx->launches += 4 + kRebuildLaunches + (ctx->list_valid ? 0 : 1);
        cudaError_t e = launch_check_displacement(ctx->A, ctx->lim2, ctx->stream);
        if (e == cudaSuccess && !ctx->list_valid) e = launch_set_rebuild(ctx->d_flags, ctx->stream);
        if (e == cudaSuccess) e = enqueue_rebuild(ctx);
        if (e == cudaSuccess) e = launch_clear_rebuild(ctx->d_flags, ctx->stream);
        if (e == cudaSuccess) e = enqueue_sur_net(ctx, ctx->stream);
        int rows = 0;
        if (e == cudaSuccess)
            e = launch_sur_force(ctx->A, ctx->S, 0, (int)ctx->n, false, true, 0.0, 0.0, &rows, ctx->stream);
        ctx->part_rows = rows;
        if (e == cudaSuccess) e = launch_reduce(ctx->A, rows, ctx->d_reduce, ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ctx->h_reduce, ctx->d_reduce, sizeof(double) * kPartials, cudaMemcpyDeviceToHost,
                                ctx->stream);
        return e;
    }
    ctx->launches += 4 + kRebuildLaunches + (ctx->list_valid ? 0 : 1);
    cudaError_t e = launch_check_displacement(ctx->A, ctx->lim2, ctx->stream);
    if (e == cudaSuccess && !ctx->list_valid) e = launch_set_rebuild(ctx->d_flags, ctx->stream);
    if (e == cudaSuccess) e = enqueue_rebuild(ctx);
    if (e == cudaSuccess) e = launch_density(ctx->A, ctx->P, ctx->precision, ctx->lanes, ctx->stream);
    if (e == cudaSuccess)
        e = launch_force(ctx->A, ctx->P, ctx->precision, ctx->lanes, false, true, 0.0, ctx->stream);
    ctx->part_rows = partial_blocks((int)ctx->n, ctx->lanes) + (ctx->A.pairs ? partial_blocks((int)ctx->n, 1) : 0);
    if (e == cudaSuccess) e = launch_reduce(ctx->A, ctx->part_rows, ctx->d_reduce, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->h_reduce, ctx->d_reduce, sizeof(double) * kPartials, cudaMemcpyDeviceToHost,
                            ctx->stream);
    return e;
}

md_status compute_forces(md_ctx *ctx) {
    if (ctx->sur && !ctx->sur_set) return fail(ctx, MD_ERR_STATE, "surrogate network not set (md_set_surrogate)");
    ctx->h_rep.clear();   // the partial sums below are of the current velocities
    MD_CK(reset_errors(ctx));
    MD_CK(enqueue_forces(ctx));
    md_status s = sync_and_check(ctx, false);
    if (s != MD_OK) return s;
    ctx->list_valid = ctx->forces_valid = ctx->energy_valid = true;
    return MD_OK;
}

md_status ensure_stage(md_ctx *ctx, size_t bytes) {
    if (ctx->stage_bytes >= bytes) return MD_OK;
    if (ctx->d_stage) {
        cudaFree(ctx->d_stage);
        ctx->d_stage = nullptr;
        ctx->stage_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&ctx->d_stage, bytes);
    if (e != cudaSuccess) return fail(ctx, MD_ERR_OOM, "staging buffer", e);
    ctx->stage_bytes = bytes;
    return MD_OK;
}

md_status ensure_stamps(md_ctx *ctx, size_t count) {
    if (ctx->stamps_cap >= count) return MD_OK;
    if (ctx->d_stamps) cudaFree(ctx->d_stamps);
    if (ctx->h_stamps) cudaFreeHost(ctx->h_stamps);
    ctx->d_stamps = nullptr;
    ctx->h_stamps = nullptr;
    ctx->stamps_cap = 0;
    MD_CK(cudaMalloc(&ctx->d_stamps, count * sizeof(unsigned long long)));
    MD_CK(cudaMallocHost(&ctx->h_stamps, count * sizeof(unsigned long long)));
    ctx->stamps_cap = count;
    return MD_OK;
}

md_status copy_out(md_ctx *ctx, const void *src, void *dst, size_t bytes, int on_device) {
    MD_CK(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          ctx->stream));
    MD_CK(cudaStreamSynchronize(ctx->stream));
    return MD_OK;
}

StepParams step_params(md_ctx *ctx, int n_steps) {
    StepParams sp{};
    sp.n_steps = n_steps;
    sp.energy_last = 1;
    sp.half_dt = ctx->half_dt;
    sp.dt = ctx->dt;
    sp.strain_scale = ctx->strain_scale;
    sp.lim2 = ctx->lim2;
    sp.rebuild_every = ctx->cfg.rebuild_every;
    sp.rl2 = ctx->rl2;
    list_band(ctx, sp.band_lo, sp.band_hi);
    sp.list_group = ph_list_group(ctx);
    if (ctx->thermo_on) {
        sp.thermo = ctx->d_thermo;
        sp.ke_chunks = ctx->d_ke_chunks;
        sp.n_ke_chunks = ctx->n_ke_chunks;
        sp.rep_off = ctx->d_rep_off;
    }
    sp.spin_limit = kSpinLimit;
    sp.motion = ctx->cfg.integrator == MD_INTEGRATOR_PC3 ? kMotionPC3 : kMotionVerlet;
    return sp;
}

// The work of md_step(n) after any initial force evaluation: the persistent launch, the
// energy reduction and the copies back.  `rows` receives the partial-sum rows written.
// Rebuild segments of an md_step(n) call (0: one launch, rebuilds inside it): for the FP64 step
// kernel (4 blocks of 128 threads per SM: its in-kernel list build runs at a quarter of the
// rebuild kernel's occupancy) on systems large enough that a rebuild costs more than two extra
// launches; about 1.5 per rebuild expected from the rebuild interval seen so far.  (The mixed and
// double-float step kernels keep 32 warps per SM, and measured no faster with segments.)
constexpr int64_t kSegmentMinAtoms = 32768;
constexpr int kSegmentsMax = 64;
int step_segments(md_ctx *ctx, int n_steps) {
    if (ctx->precision != MD_PREC_FP64 || ctx->n < kSegmentMinAtoms || n_steps < 1) return 0;
    const unsigned long long nr = ctx->h_flags ? ctx->h_flags->n_rebuilds : 0;
    const int64_t every = ctx->step > 0 && nr > 0 ? std::max<int64_t>(1, ctx->step / (int64_t)nr) : 8;
    return (int)std::min<int64_t>(kSegmentsMax, (3 * (int64_t)n_steps) / (2 * every) + 2);
}

cudaError_t enqueue_steps(md_ctx *ctx, int n_steps, unsigned long long *stamps, int *rows, cudaStream_t stream,
                          int *launches = nullptr) {
    if (launches) *launches = 2;
    if (ctx->sur) {
        cudaError_t e = cudaSuccess;
        const int every = ctx->cfg.rebuild_every;
        for (int q = 0; q < n_steps && e == cudaSuccess; q++) {
            const bool sched = every > 0 && (ctx->step + q + 1) % every == 0;
            e = enqueue_sur_step(ctx, q == n_steps - 1, sched, rows, stream);
        }
        if (e == cudaSuccess) e = launch_reduce(ctx->A, *rows, ctx->d_reduce, stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ctx->h_reduce, ctx->d_reduce, sizeof(double) * kPartials, cudaMemcpyDeviceToHost,
                                stream);
        return e;
    }
    const StepParams sp = step_params(ctx, n_steps);
    int grid = 0;
    // Segments: the step kernel stops at a rebuild request, the rebuild kernel (more warps per
    // SM than the step kernel keeps) builds the list, a launch resumes the steps; R such pairs,
    // the last launch rebuilding in-kernel should more rebuilds fall due than R covers.
    const int R = step_segments(ctx, n_steps);
    StepParams sp1 = sp;
    sp1.stop_at_rebuild = R > 0;
    cudaError_t e = launch_step(ctx->A, ctx->C, ctx->P, ctx->precision, ctx->lanes, sp1, ctx->d_bar, stamps, &grid,
                                stream);
    for (int r = 0; r < R && e == cudaSuccess; r++) {
        e = launch_rebuild_step(ctx->A, ctx->C, ctx->P, ctx->precision, ctx->lanes, sp, ctx->d_bar, stamps, stream);
        StepParams sp2 = sp;
        sp2.resume = 1;
        sp2.stop_at_rebuild = r + 1 < R;
        if (e == cudaSuccess)
            e = launch_step(ctx->A, ctx->C, ctx->P, ctx->precision, ctx->lanes, sp2, ctx->d_bar, stamps, &grid,
                            stream);
    }
    if (launches) *launches = 2 + 2 * R;
    if (e == cudaSuccess) e = launch_reduce(ctx->A, grid, ctx->d_reduce, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->h_reduce, ctx->d_reduce, sizeof(double) * kPartials, cudaMemcpyDeviceToHost,
                            stream);
    *rows = grid;
    return e;
}

// Fold the %globaltimer stamps of one launch into the profile.  Row s+1 of kStampsPerStep
// stamps belongs to step s: [0] start, [1..9] after each rebuild sub-phase (bin, tile sums,
// top scan, apply, scatter, cell sort, gather, copyback, list; all equal to [0] when no
// rebuild ran), [10] after the density pass, [11] after the force pass.  Row 0 holds the
// launch start; the first half kick ends where step 0 starts.
void collect_stamps(md_ctx *ctx, int n_steps) {
    const unsigned long long *t = ctx->h_stamps;
    ctx->prof.ms_kick += (t[kStampsPerStep] - t[0]) * 1e-6;
    ctx->prof.n_kick += 1;
    for (int s = 1; s <= n_steps; s++) {
        const unsigned long long *r = t + kStampsPerStep * s;
        ctx->prof.ms_rebuild += (r[9] - r[0]) * 1e-6;
        for (int q = 0; q < 9; q++) ctx->prof.ms_rebuild_part[q] += (r[q + 1] - r[q]) * 1e-6;
        ctx->prof.ms_density += (r[10] - r[9]) * 1e-6;
        ctx->prof.ms_force += (r[11] - r[10]) * 1e-6;
    }
    ctx->prof.n_rebuild += n_steps;
    ctx->prof.n_density += n_steps;
    ctx->prof.n_force += n_steps;
}

void drop_graphs(md_ctx *ctx) {
    for (auto &g : ctx->graphs) cudaGraphExecDestroy(g.second);
    ctx->graphs.clear();
    ctx->graph_rows.clear();
    ctx->graph_launches.clear();
}

// --------------------------------------------------------------------------- creation
struct Inputs {
    std::vector<double> pos, vel;
    std::vector<int32_t> spec;
};

md_status create_common(md_ctx *ctx, const md_config *cfg, const md_potential *pot, const Inputs &in,
                        const std::vector<int64_t> &rep_n, const std::vector<double> &L) {
    const int n_rep = (int)rep_n.size();
    int64_t n = 0;
    ctx->rep_off.assign(n_rep + 1, 0);
    for (int r = 0; r < n_rep; r++) {
        ctx->rep_off[r + 1] = ctx->rep_off[r] + rep_n[r];
        n += rep_n[r];
    }
    ctx->cfg = *cfg;
    ctx->stream = static_cast<cudaStream_t>(cfg->stream);
    ctx->n_rep = n_rep;
    ctx->L = L;
    if (n < 0 || n > INT32_MAX / 8) return MD_ERR_ARG;
    if (cfg->k_max < 1 || cfg->skin < 0.0 || !(cfg->dt_fs >= 0.0) || cfg->rebuild_every < 0) return MD_ERR_ARG;
    if (cfg->precision != MD_PREC_FP64 && cfg->precision != MD_PREC_MIXED && cfg->precision != MD_PREC_DF)
        return MD_ERR_ARG;
    if (cfg->precision == MD_PREC_DF && (pot->kind != MD_POT_TABLES || pot->n_species != 1)) {
        ctx->err = "double-float precision takes one species with knot tables";
        return MD_ERR_ARG;
    }
    if (cfg->integrator != MD_INTEGRATOR_VERLET && cfg->integrator != MD_INTEGRATOR_PC3) return MD_ERR_ARG;
    if (cfg->integrator == MD_INTEGRATOR_PC3 &&
        (cfg->strain_rate_zz != 0.0 || pot->kind == MD_POT_SURROGATE ||
         (cfg->passes != MD_PASSES_AUTO && cfg->passes != MD_PASSES_LIST &&
          !(cfg->passes == MD_PASSES_HALF && cfg->precision == MD_PREC_FP64)))) {
        ctx->err = "the predictor-corrector takes the list walks (full, or the FP64 half list), no strain ramp and "
                   "no surrogate";
        return MD_ERR_ARG;
    }
    for (double l : L)
        if (!(l > 0.0)) return MD_ERR_BOX;
    // potential (§3.1)
    const int ns = pot->n_species;
    if (pot->kind == MD_POT_FS_ANALYTIC) {
        if (ns != 1 || !(pot->r_cut > 0.0) || pot->fs[0] <= 0.0) return MD_ERR_ARG;
    } else if (pot->kind == MD_POT_TABLES) {
        if (ns < 1 || ns > 8 || pot->n_knots < 2 || !pot->tables || !(pot->r_cut > pot->r_min) ||
            !(pot->rho_max > pot->rho_min))
            return MD_ERR_ARG;
    } else if (pot->kind == MD_POT_KNOTS) {
        if (ns < 1 || ns > 8 || pot->n_knots < 1 || pot->n_knots > 32 || !pot->tables || !(pot->r_cut > 0.0))
            return MD_ERR_ARG;
        const int K = pot->n_knots;
        for (int t = 0; t < 2 * ns * ns; t++)
            for (int q = 0; q < K; q++) {
                const double c = pot->tables[(size_t)t * 2 * K + q], rk = pot->tables[(size_t)t * 2 * K + K + q];
                if (!std::isfinite(c) || !(rk <= pot->r_cut) || !std::isfinite(rk)) return MD_ERR_ARG;
            }
        for (int a = 0; a < ns; a++)
            for (int b = 0; b < ns; b++)
                for (int q = 0; q < 2 * K; q++)
                    if (pot->tables[(size_t)(a * ns + b) * 2 * K + q] != pot->tables[(size_t)(b * ns + a) * 2 * K + q]) {
                        ctx->err = "V knot sums must be symmetric in their two species";
                        return MD_ERR_ARG;
                    }
    } else if (pot->kind == MD_POT_SURROGATE) {
        if (ns != 1 || !(pot->r_cut > 0.0)) return MD_ERR_ARG;
        if (cfg->strain_rate_zz != 0.0) return MD_ERR_ARG;
        ctx->sur = true;
    } else {
        return MD_ERR_ARG;
    }
    if (!pot->masses_amu) return MD_ERR_ARG;
    std::vector<double> mass(ns);
    for (int a = 0; a < ns; a++) {
        mass[a] = pot->masses_amu[a];
        if (!(mass[a] > 0.0)) return MD_ERR_ARG;
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
    // link cells of each replica (fixed in fractional coordinates, >= 3 per edge), r_list wide.
    // Built with MD_CELL_REACH_MAX=2, cells are r_list / 2 wide (a 5 x 5 x 5 stencil: 15.6 r_list^3
    // of list candidates instead of 27 r_list^3) when every edge holds >= 5 of them and they hold
    // >= 3 atoms on average: a faster list build, but on GB300 slightly slower passes (the coarser
    // cell order keeps more of a warp's neighbours in the same lines), so it is off by default.
    ctx->rc.resize(n_rep);
    for (int k = 0; k < n_rep * 3; k++)
        if (cells_along(L[k], ctx->r_list) < 3) {
            ctx->err = "a box edge holds fewer than 3 link cells of width r_cut + skin";
            return MD_ERR_BOX;
        }
#ifndef MD_CELL_REACH_MAX
#define MD_CELL_REACH_MAX 1
#endif
    int reach = MD_CELL_REACH_MAX >= 2 ? 2 : 1;
    if (reach == 2) {
        long long half_cells = 0;
        for (int r = 0; r < n_rep; r++) {
            long long c = 1;
            for (int k = 0; k < 3; k++) {
                const int nc = cells_along(L[3 * r + k], 0.5 * ctx->r_list);
                if (nc < 5) reach = 1;
                c *= nc;
            }
            half_cells += c;
        }
        if (half_cells <= 0 || (double)n < 3.0 * (double)half_cells) reach = 1;
    }
    ctx->C.reach = reach;
    long long ncell = 0;
    for (int r = 0; r < n_rep; r++) {
        for (int k = 0; k < 3; k++) ctx->rc[r].nc[k] = cells_along(L[3 * r + k], ctx->r_list / reach);
        ctx->rc[r].base = (int)ncell;
        ncell += (long long)ctx->rc[r].nc[0] * ctx->rc[r].nc[1] * ctx->rc[r].nc[2];
        if (ncell > INT32_MAX / 2) return MD_ERR_BOX;
    }
    // lanes per atom: given, or from the expected neighbour count (4/3 pi r_list^3 x density)
    {
        const int want = cfg->lanes_per_atom;
        if (want != 0 && want != 1 && want != 2 && want != 4 && want != 8 && want != 16 && want != 32)
            return MD_ERR_ARG;
        if (want) {
            ctx->lanes = want;
        } else {
            double vol = 0.0;
            for (int r = 0; r < n_rep; r++) vol += L[3 * r] * L[3 * r + 1] * L[3 * r + 2];
            const double k_est = 4.18879020478639 * ctx->r_list * ctx->r_list * ctx->r_list * (double)n / vol;
            int t = 1;
            while (t < 8 && t * 12 < k_est) t *= 2;
            ctx->lanes = t;
        }
    }
    for (int64_t i = 0; i < n; i++) {
        if (in.spec[i] < 0 || in.spec[i] >= ns) {
            ctx->err = "atom " + std::to_string(i) + " has species " + std::to_string(in.spec[i]) +
                       " not supported by the potential";
            return MD_ERR_SPECIES;
        }
        for (int c = 0; c < 3; c++)
            if (!std::isfinite(in.pos[3 * i + c]) || !std::isfinite(in.vel[3 * i + c])) return MD_ERR_NONFINITE;
    }
    const double acc = 1.0 / kMvv2e;  // (eV/Å)/amu -> Å/fs^2
    std::vector<double4_32a> p4(n), v4(n), f4(n);
    std::vector<int32_t> iota(n), rep(n_rep > 1 ? n : 0);
    if (n_rep > 1)
        for (int r = 0; r < n_rep; r++)
            for (int64_t i = ctx->rep_off[r]; i < ctx->rep_off[r + 1]; i++) rep[i] = r;
    for (int64_t i = 0; i < n; i++) {
        const double m = mass[in.spec[i]];
        p4[i] = make_double4_32a(in.pos[3 * i], in.pos[3 * i + 1], in.pos[3 * i + 2], (double)in.spec[i]);
        v4[i] = make_double4_32a(in.vel[3 * i], in.vel[3 * i + 1], in.vel[3 * i + 2], acc / m);
        f4[i] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
        iota[i] = (int32_t)i;
    }
    // device buffers
    Atoms &A = ctx->A;
    A.n = (int)n;
    A.k_max = cfg->k_max;
    A.n_rep = n_rep;
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
    chk(dalloc(ctx, &A.wrap, n));
    if (cfg->precision != MD_PREC_MIXED && pot->kind != MD_POT_SURROGATE) chk(dalloc(ctx, &A.posd, n));
    if (cfg->precision == MD_PREC_DF) {   // double-float coordinates: high and low parts per atom
        chk(dalloc(ctx, &A.posx, 2 * (size_t)n));
        chk(dalloc(ctx, &A.p2x, 2 * (size_t)n));
    }
#ifndef MD_IMAGE_SHORTCUT
#define MD_IMAGE_SHORTCUT 1
#endif
    A.image_fixed = (MD_IMAGE_SHORTCUT && cfg->strain_rate_zz == 0.0) ? 1 : 0;
    chk(dalloc(ctx, &A.nbr, nbr_entries(n, cfg->k_max)));
#ifndef MD_FP64_DCACHE
#define MD_FP64_DCACHE 1
#endif
    // FP64, one species: the per-entry derivative cache of the force pass (16 B per list entry)
    if ((cfg->precision == MD_PREC_DF || (MD_FP64_DCACHE && cfg->precision == MD_PREC_FP64)) &&
        pot->kind != MD_POT_SURROGATE && ns == 1)
        chk(dalloc(ctx, &A.dcache, nbr_entries(n, cfg->k_max)));
    if (cfg->integrator == MD_INTEGRATOR_PC3) {
        chk(dalloc(ctx, &A.g2, n)); chk(dalloc(ctx, &A.g3, n));
        chk(dalloc(ctx, &A.g2_tmp, n)); chk(dalloc(ctx, &A.g3_tmp, n));
        if (e == cudaSuccess) e = cudaMemset(A.g2, 0, sizeof(double4_32a) * (size_t)(n > 0 ? n : 1));
        if (e == cudaSuccess) e = cudaMemset(A.g3, 0, sizeof(double4_32a) * (size_t)(n > 0 ? n : 1));
    }
    if (n_rep > 1) chk(dalloc(ctx, &A.rep, n));
    A.sorted = A.cell_of;  // cell_of is consumed by the scatter before the in-cell sort writes
    // partial-sum rows: a stand-alone force launch at up to 32 lanes per atom (and, for the FP64
    // pair walk, the per-atom phase after it), or a persistent grid
    const int rows = std::max(partial_blocks((int)n, 32) + partial_blocks((int)n, 1), 8192);
    A.part_stride = rows;
    chk(dalloc(ctx, &A.partials, (size_t)rows * kPartials));
    chk(dalloc(ctx, &ctx->d_boxes, n_rep));
    chk(dalloc(ctx, &ctx->d_rc, n_rep));
    chk(dalloc(ctx, &ctx->d_rep_off, n_rep + 1));
    chk(dalloc(ctx, &ctx->d_rep_sums, (size_t)n_rep * 5));
    chk(dalloc(ctx, &ctx->d_flags, 1));
    chk(dalloc(ctx, &ctx->d_bar, 1));
    chk(dalloc(ctx, &ctx->d_reduce, kPartials));
    Cells &C = ctx->C;
    C.ncell = (int)ncell;
    C.ntiles = (C.ncell + 511) / 512;   // tiles of the persistent kernel's scan (128 x 4 cells)
    C.rc = ctx->d_rc;
    chk(dalloc(ctx, &C.cell_count, C.ncell));
    chk(dalloc(ctx, &C.cell_start, C.ncell + 1));
    chk(dalloc(ctx, &C.tile_sums, C.ntiles + 1));
    // group walks (MD_PASSES_STAGED, _CELLS, _HALF): groups of gx cells along x whose
    // 3 x 3 x (gx + 2) neighbourhood fits the stage 15 % above the mean occupancy.  Staged and
    // half walks: gx such that a group's home atoms fill whole rounds of a 1024-thread block at
    // the context's lanes per atom (with a 10 % margin for the spread of cell occupancy), of
    // nearly equal choices the larger; cell walk (a warp per atom): the largest gx (fewest
    // stencil copies).
    {
        const size_t tbytes = pot->kind == MD_POT_TABLES ? smem_table_bytes(pot->kind, ns, cfg->precision, pot->n_knots)
                                                         : 0;
        const bool eligible = tbytes > 0 && n_rep == 1 && reach == 1 && !ctx->sur && cfg->strain_rate_zz == 0.0 &&
                              ctx->lanes <= 8 && n > 0;
        // FP64 and the half list: the pair walk over the full list's entries j > i (kWalkPairs)
        const bool pairs = cfg->precision == MD_PREC_FP64 && cfg->passes == MD_PASSES_HALF;
        if (pairs) {
            if (ns != 1 || ctx->sur || (pot->kind != MD_POT_TABLES && pot->kind != MD_POT_FS_ANALYTIC) ||
                cfg->k_max > kPairsKMax) {
                ctx->err = "the FP64 half list takes one species (FS or tables) and k_max <= 256";
                return MD_ERR_ARG;
            }
            A.pairs = 1;
            A.pair_rc2f = (float)(pot->r_cut * pot->r_cut);
            chk(dalloc(ctx, &A.cup, n));
            chk(dalloc(ctx, &A.cin, n));
            chk(dalloc(ctx, &A.rho_acc, n));
            chk(dalloc(ctx, &A.f_acc, n));
            chk(dalloc(ctx, &A.e_acc, n));
            if (e == cudaSuccess) e = cudaMemset(A.rho_acc, 0, sizeof(double) * (size_t)(n > 0 ? n : 1));
            if (e == cudaSuccess) e = cudaMemset(A.e_acc, 0, sizeof(double) * (size_t)(n > 0 ? n : 1));
            if (e == cudaSuccess) e = cudaMemset(A.f_acc, 0, sizeof(double4_32a) * (size_t)(n > 0 ? n : 1));
        }
        const bool grouped = !pairs && (cfg->passes == MD_PASSES_STAGED || cfg->passes == MD_PASSES_CELLS ||
                                        cfg->passes == MD_PASSES_HALF);
        if (cfg->passes != MD_PASSES_AUTO && cfg->passes != MD_PASSES_LIST && !grouped && !pairs) return MD_ERR_ARG;
        if (grouped && !eligible) {
            ctx->err = "group walks need mixed precision, one system, one species with a knot table that fits "
                       "in shared memory, no strain ramp and at most 8 lanes per atom";
            return MD_ERR_ARG;
        }
        C.tile = kWalkList;
        if (eligible && grouped) {
            const int walk = cfg->passes == MD_PASSES_STAGED ? kWalkStaged
                                                              : (cfg->passes == MD_PASSES_CELLS ? kWalkCells : kWalkHalf);
            const int nx = ctx->rc[0].nc[0];
            const double m = (double)n / (double)ncell;
            const size_t dyn_max = walk == kWalkCells ? kSmemDynMaxCells : kSmemDynMax;
            // a stage slot holds a float4 position, and for the half walk a float4 of sums; as many
            // stage buffers (up to MD_STAGE_BUFS, 2 for the half walk) as hold a group of at least
            // one cell
            const size_t slot = sizeof(float4) * (walk == kWalkHalf ? 2 : 1);
            int best = 0, cap = 0, nbuf = 0;
            for (int nb = walk == kWalkHalf ? std::min(2, MD_STAGE_BUFS) : MD_STAGE_BUFS; nb >= 1 && best == 0; nb--) {
                // the group walks hold one of the table's two row sets at a time
                cap = (int)std::min<size_t>((dyn_max - (MD_DTABLE ? tbytes / 2 : tbytes)) / (slot * nb), 65535);
                nbuf = nb;
                // the widest group whose neighbourhood fits with 15 % to spare
                for (int g = 1; g <= std::min(kGroupMaxGx, nx); g++)
                    if (9.0 * (g + 2) * m * 1.15 <= cap) best = g;
            }
            if (best > 0) {
                C.tile = walk;
                C.gx = best;
                C.ngx = (nx + best - 1) / best;
                C.n_groups = C.ngx * ctx->rc[0].nc[1] * ctx->rc[0].nc[2];
                C.st_cells = 9 * (best + 2);
                C.cap = cap;
                C.nbuf = nbuf;
                chk(dalloc(ctx, &C.grp_loc, (size_t)C.n_groups * (C.st_cells + 1)));
                if (walk == kWalkStaged || walk == kWalkHalf) chk(dalloc(ctx, &A.lnbr, nbr_entries(n, cfg->k_max)));
                if (walk == kWalkHalf) {
                    chk(dalloc(ctx, &A.lcount, n));
                    chk(dalloc(ctx, &A.rho_acc, n));
                    chk(dalloc(ctx, &A.f_acc, n));
                }
            } else {
                ctx->err = "group walks: the link-cell occupancy is too high for the stage";
                return MD_ERR_ARG;
            }
        }
    }
    if (e != cudaSuccess) return fail(ctx, MD_ERR_OOM, "device allocation", e);
    A.boxes = ctx->d_boxes;
    A.flags = ctx->d_flags;
    if (cudaMallocHost(&ctx->h_flags, sizeof(Flags)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_reduce, sizeof(double) * kPartials) != cudaSuccess)
        return MD_ERR_OOM;
    std::memset(ctx->h_flags, 0, sizeof(Flags));
    std::memset(ctx->h_reduce, 0, sizeof(double) * kPartials);
    // potential tables
    Pot &P = ctx->P;
    P.kind = pot->kind;
    P.ns = ns;
    P.rc2 = pot->r_cut * pot->r_cut;
    P.rc2f = (float)P.rc2;
    P.rc2f_skin = cut_skin_bound(ctx, pot->r_cut);
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
        P.smt_phi = nk;
        P.r_min = pot->r_min;
        P.inv_dr = (nk - 1) / (pot->r_cut - pot->r_min);
        P.xneg = -(pot->r_min * P.inv_dr);
        P.rho_min = pot->rho_min;
        P.inv_drho = (nk - 1) / (pot->rho_max - pot->rho_min);
        P.r_minf = (float)P.r_min;
        P.inv_drf = (float)P.inv_dr;
        const double hr = (pot->r_cut - pot->r_min) / (nk - 1);
        const double hrho = (pot->rho_max - pot->rho_min) / (nk - 1);
        const size_t npair = (size_t)ns * ns;
        std::vector<double4_32a> VP64(npair * nk * 2), F64((size_t)ns * nk), rv(nk), rp(nk);
        std::vector<float> VP32(npair * nk * 8);
        std::vector<float4> D32;
        std::vector<float> V0;
        std::vector<double4_32a> D64;
        std::vector<float4> TX, TVx;
        const size_t tl = 2 * (size_t)nk;
        for (int a = 0; a < ns; a++)
            for (int b = 0; b < ns; b++) {
                const double *tv = pot->tables + (size_t)(a * ns + b) * tl;
                const double *tvt = pot->tables + (size_t)(b * ns + a) * tl;
                for (size_t q = 0; q < tl; q++)
                    if (tv[q] != tvt[q]) {
                        ctx->err = "V table must be symmetric in its two species";
                        return MD_ERR_ARG;
                    }
                cubic_rows(tv, nk, hr, rv.data());
                cubic_rows(pot->tables + (npair + a * ns + b) * tl, nk, hr, rp.data());
                const size_t base = (size_t)(a * ns + b) * nk;
                if (ns == 1) {   // the force pass's derivative rows (see Pot::D32)
                    auto scale = [&](const std::vector<double4_32a> &rw) {   // max |2 c2|, |3 c3| -> [2^14, 2^15)
                        double m = 0.0;
                        for (int k = 0; k < nk; k++) m = std::max(m, std::max(std::fabs(2.0 * rw[k].z), std::fabs(3.0 * rw[k].w)));
                        return m > 0.0 ? std::ldexp(1.0, (int)std::floor(std::log2(m)) - 14) : 1.0;
                    };
                    auto pack = [](double a2, double a3) {   // (a2, a3) as binary16 in one 32-bit word
                        const uint32_t u = (uint32_t)__half_as_ushort(__float2half_rn((float)a2)) |
                                           ((uint32_t)__half_as_ushort(__float2half_rn((float)a3)) << 16);
                        float f;
                        std::memcpy(&f, &u, sizeof f);
                        return f;
                    };
                    const double sv = scale(rv), sp = scale(rp);
                    D32.resize(nk);
                    V0.resize(nk);
                    for (int k = 0; k < nk; k++) V0[k] = (float)rv[k].x;
                    for (int k = 0; k < nk; k++)
                        D32[k] = make_float4((float)rv[k].y, (float)rp[k].y, pack(2.0 * rv[k].z / sv, 3.0 * rv[k].w / sv),
                                             pack(2.0 * rp[k].z / sp, 3.0 * rp[k].w / sp));
                    P.dsv = (float)sv;
                    P.dsp = (float)sp;
                    D64.resize(2 * (size_t)nk);
                    const double s = P.inv_dr;
                    for (int k = 0; k < nk; k++) {
                        D64[2 * k] = make_double4_32a(rv[k].y * s, 2.0 * rv[k].z * s, 3.0 * rv[k].w * s, 0.0);
                        D64[2 * k + 1] = make_double4_32a(rp[k].y * s, 2.0 * rp[k].z * s, 3.0 * rp[k].w * s, 0.0);
                    }
                    // double-float rows (see Pot::TX, Pot::TVx)
                    TX.resize(4 * (size_t)nk);
                    TVx.resize(2 * (size_t)nk);
                    auto hl = [](double x) { return df::from_double(x); };
                    for (int k = 0; k < nk; k++) {
                        const df::F2 p0 = hl(rp[k].x), p1 = hl(rp[k].y), v0 = hl(rv[k].x), v1 = hl(rv[k].y);
                        const df::F2 pd1 = hl(rp[k].y * s), pd2 = hl(2.0 * rp[k].z * s);
                        const df::F2 vd1 = hl(rv[k].y * s), vd2 = hl(2.0 * rv[k].z * s);
                        TX[4 * k] = make_float4(p0.h, p0.l, p1.h, p1.l);
                        TX[4 * k + 1] = make_float4((float)rp[k].z, (float)rp[k].w, (float)(3.0 * rp[k].w * s),
                                                    (float)(3.0 * rv[k].w * s));
                        TX[4 * k + 2] = make_float4(pd1.h, pd1.l, pd2.h, pd2.l);
                        TX[4 * k + 3] = make_float4(vd1.h, vd1.l, vd2.h, vd2.l);
                        TVx[2 * k] = make_float4(v0.h, v0.l, v1.h, v1.l);
                        TVx[2 * k + 1] = make_float4((float)rv[k].z, (float)rv[k].w, 0.f, 0.f);
                    }
                    const df::F2 idr = hl(P.inv_dr), x0 = hl(P.r_min * P.inv_dr);
                    P.idr_h = idr.h;
                    P.idr_l = idr.l;
                    P.x0_h = x0.h;
                    P.x0_l = x0.l;
                }
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
        if (e != cudaSuccess) return fail(ctx, MD_ERR_OOM, "table allocation", e);
        chk(cudaMemcpy(dVP64, VP64.data(), VP64.size() * sizeof(double4_32a), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(dVP32, VP32.data(), VP32.size() * sizeof(float), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(dF64, F64.data(), F64.size() * sizeof(double4_32a), cudaMemcpyHostToDevice));
        P.VP64 = dVP64;
        P.VP32 = dVP32;
        P.F64 = dF64;
        if (!D64.empty()) {
            double4_32a *dD64;
            float4 *dTX, *dTV;
            chk(dalloc(ctx, &dD64, D64.size()));
            chk(dalloc(ctx, &dTX, TX.size()));
            chk(dalloc(ctx, &dTV, TVx.size()));
            if (e != cudaSuccess) return fail(ctx, MD_ERR_OOM, "table allocation", e);
            chk(cudaMemcpy(dD64, D64.data(), D64.size() * sizeof(double4_32a), cudaMemcpyHostToDevice));
            chk(cudaMemcpy(dTX, TX.data(), TX.size() * sizeof(float4), cudaMemcpyHostToDevice));
            chk(cudaMemcpy(dTV, TVx.data(), TVx.size() * sizeof(float4), cudaMemcpyHostToDevice));
            P.D64 = dD64;
            P.TX = dTX;
            P.TVx = dTV;
        }
        if (!D32.empty()) {
            float4 *dD32;
            chk(dalloc(ctx, &dD32, D32.size()));
            if (e != cudaSuccess) return fail(ctx, MD_ERR_OOM, "table allocation", e);
            float *dV0;
            chk(dalloc(ctx, &dV0, V0.size()));
            if (e != cudaSuccess) return fail(ctx, MD_ERR_OOM, "table allocation", e);
            chk(cudaMemcpy(dD32, D32.data(), D32.size() * sizeof(float4), cudaMemcpyHostToDevice));
            chk(cudaMemcpy(dV0, V0.data(), V0.size() * sizeof(float), cudaMemcpyHostToDevice));
            P.D32 = dD32;
            P.V0 = dV0;
        }
    }
    if (pot->kind == MD_POT_KNOTS) {
        const int K = pot->n_knots, nf = 2 * ns * ns;
        P.nkt = K;
        std::vector<double2> k64((size_t)nf * K);
        std::vector<float2> k32((size_t)nf * K);
        for (int t = 0; t < nf; t++)
            for (int q = 0; q < K; q++) {
                const double c = pot->tables[(size_t)t * 2 * K + q], rk = pot->tables[(size_t)t * 2 * K + K + q];
                k64[(size_t)t * K + q] = make_double2(c, rk);
                k32[(size_t)t * K + q] = make_float2((float)c, (float)rk);
            }
        for (int a = 0; a < ns; a++) P.A64[a] = pot->tables[(size_t)nf * 2 * K + a];
        double2 *d64;
        float2 *d32;
        chk(dalloc(ctx, &d64, k64.size()));
        chk(dalloc(ctx, &d32, k32.size()));
        if (e != cudaSuccess) return fail(ctx, MD_ERR_OOM, "knot allocation", e);
        chk(cudaMemcpy(d64, k64.data(), k64.size() * sizeof(double2), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(d32, k32.data(), k32.size() * sizeof(float2), cudaMemcpyHostToDevice));
        P.K64 = d64;
        P.K32 = d32;
    }
    // initial state (caller order = cell order until the first build)
    std::vector<Box> boxes(n_rep);
    for (int r = 0; r < n_rep; r++) boxes[r] = make_box(&L[3 * r], cfg->skin);
    std::vector<int32_t> off32(n_rep + 1);
    for (int r = 0; r <= n_rep; r++) off32[r] = (int32_t)ctx->rep_off[r];
    Flags flags{};
    flags.need_rebuild = 1;
    if (n > 0) {
        chk(cudaMemcpy(A.pos, p4.data(), n * sizeof(double4_32a), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(A.ref, p4.data(), n * sizeof(double4_32a), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(A.vel, v4.data(), n * sizeof(double4_32a), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(A.force, f4.data(), n * sizeof(double4_32a), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(A.id, iota.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(A.rank, iota.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(A.spec, in.spec.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice));
        if (n_rep > 1) chk(cudaMemcpy(A.rep, rep.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
    chk(cudaMemcpy(ctx->d_boxes, boxes.data(), n_rep * sizeof(Box), cudaMemcpyHostToDevice));
    chk(cudaMemcpy(ctx->d_rc, ctx->rc.data(), n_rep * sizeof(RepCells), cudaMemcpyHostToDevice));
    chk(cudaMemcpy(ctx->d_rep_off, off32.data(), (n_rep + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
    chk(cudaMemcpy(ctx->d_flags, &flags, sizeof(Flags), cudaMemcpyHostToDevice));
    chk(cudaMemset(C.cell_count, 0, sizeof(int32_t) * C.ncell));
    chk(cudaMemset(A.wrap, 1, n));   // every atom takes the minimum image until the first build
    chk(cudaMemset(A.partials, 0, sizeof(double) * rows * kPartials));
    chk(cudaDeviceSynchronize());
    chk(launch_wrap(A, ctx->stream));
    chk(cudaStreamSynchronize(ctx->stream));
    if (e != cudaSuccess) return fail(ctx, MD_ERR_CUDA, "initial upload", e);
    return MD_OK;
}

bool fetch(void *dst, const void *src, size_t bytes, int on_device) {
    if (bytes == 0) return true;
    if (!on_device) {
        std::memcpy(dst, src, bytes);
        return true;
    }
    return cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost) == cudaSuccess;
}


// --------------------------------------------------------------------------- surrogate
md_status sur_alloc(md_ctx *ctx) {
    if (ctx->d_theta) return MD_OK;
    const int64_t n = std::max<int64_t>(ctx->n, 1);
    const int64_t ntiles = (n + kSurTile - 1) / kSurTile;
    SurNet &S = ctx->S;
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t r) { if (r != cudaSuccess && e == cudaSuccess) e = r; };
    unsigned char *Gt = nullptr;
    float *G = nullptr, *g = nullptr, *u = nullptr, *gpart = nullptr;
    float4 *phi = nullptr;
    double *eref = nullptr, *ce = nullptr;
    chk(dalloc(ctx, &ctx->d_theta, kSurParams));
    chk(dalloc(ctx, &ctx->d_adam_m, kSurParams));
    chk(dalloc(ctx, &ctx->d_adam_v, kSurParams));
    chk(dalloc(ctx, &ctx->d_grad, kSurParams));
    chk(dalloc(ctx, &ctx->d_gmu, kSurNb));
    chk(dalloc(ctx, &ctx->d_ginv, kSurNb));
    chk(dalloc(ctx, &ctx->d_img, kSurImgBytes));
    chk(dalloc(ctx, &Gt, (size_t)ntiles * kSurTileBytes));
    chk(dalloc(ctx, &G, (size_t)n * kSurNb));
    chk(dalloc(ctx, &g, (size_t)n * kSurNb));
    chk(dalloc(ctx, &u, (size_t)n * kSurNb));
    chk(dalloc(ctx, &phi, n));
    chk(dalloc(ctx, &ctx->d_fref, n));
    chk(dalloc(ctx, &eref, ctx->n_rep));
    chk(dalloc(ctx, &ce, 2 * (size_t)ctx->n_rep));
    ctx->sur_part_blocks = sur_net32_blocks((int)n);
    chk(dalloc(ctx, &gpart, (size_t)ctx->sur_part_blocks * kSurParams));
    if (e != cudaSuccess) return fail(ctx, MD_ERR_OOM, "surrogate buffers", e);
    chk(cudaMemset(Gt, 0, (size_t)ntiles * kSurTileBytes));
    chk(cudaMemset(g, 0, sizeof(float) * (size_t)n * kSurNb));
    chk(cudaMemset(phi, 0, sizeof(float4) * (size_t)n));
    chk(cudaMemset(ce, 0, sizeof(double) * 2 * (size_t)ctx->n_rep));
    if (e != cudaSuccess) return fail(ctx, MD_ERR_CUDA, "surrogate buffers", e);
    S.theta = ctx->d_theta;
    S.gmu = ctx->d_gmu;
    S.ginv = ctx->d_ginv;
    S.img = ctx->d_img;
    S.Gt = Gt;
    S.G = G;
    S.g = g;
    S.u = u;
    S.phi = phi;
    S.fref = ctx->d_fref;
    S.eref = eref;
    S.ce = ce;
    S.gpart = gpart;
    return MD_OK;
}

// Neighbour list valid for the current positions (rebuilt when any atom moved > skin/2).
md_status sur_ensure_list(md_ctx *ctx) {
    MD_CK(reset_errors(ctx));
    MD_CK(launch_check_displacement(ctx->A, ctx->lim2, ctx->stream));
    if (!ctx->list_valid) MD_CK(launch_set_rebuild(ctx->d_flags, ctx->stream));
    MD_CK(enqueue_rebuild(ctx));
    MD_CK(launch_clear_rebuild(ctx->d_flags, ctx->stream));
    ctx->launches += 3 + kRebuildLaunches;
    md_status s = sync_and_check(ctx, false);
    if (s == MD_OK) ctx->list_valid = true;
    return s;
}

// FP32 descriptors of every atom into S.G.
cudaError_t sur_descriptors32(md_ctx *ctx) {
    SurNet S = ctx->S;
    S.bf16 = 0;
    ctx->launches++;
    return launch_sur_descriptors(ctx->A, S, 0, (int)ctx->n, ctx->stream);
}

// Steps 1-5 of a training pass over replicas [r0, r1): network (FP32) -> per-replica energy
// terms -> forces and phi = dL/dF -> descriptor tangents u -> per-block parameter gradients.
cudaError_t sur_train_pass(md_ctx *ctx, int r0, int r1, double w_e, double w_f, int *rows, int *blocks) {
    const int a0 = (int)ctx->rep_off[r0], a1 = (int)ctx->rep_off[r1];
    const double phi_scale = 2.0 * w_f / (3.0 * (double)std::max(a1 - a0, 1));
    cudaError_t e = launch_sur_net32(ctx->A, ctx->S, a0, a1, ctx->stream);
    if (e == cudaSuccess) e = launch_sur_frame_terms(ctx->A, ctx->S, ctx->d_rep_off, r0, r1, w_e, ctx->stream);
    if (e == cudaSuccess)
        e = launch_sur_force(ctx->A, ctx->S, a0, a1, false, false, 0.0, phi_scale, rows, ctx->stream);
    if (e == cudaSuccess) e = launch_sur_u(ctx->A, ctx->S, a0, a1, ctx->stream);
    if (e == cudaSuccess) e = launch_sur_train_tiles(ctx->A, ctx->S, a0, a1, blocks, ctx->stream);
    ctx->launches += 5;
    return e;
}

// Energy and force loss terms of the last training pass over [r0, r1) (after the stream is idle).
md_status sur_loss_terms(md_ctx *ctx, int r0, int r1, double w_f, double *loss) {
    std::vector<double> ce(2 * (size_t)(r1 - r0));
    MD_CK(cudaMemcpy(ce.data(), ctx->S.ce + 2 * (size_t)r0, ce.size() * sizeof(double), cudaMemcpyDeviceToHost));
    double le = 0.0;
    for (int r = 0; r < r1 - r0; r++) le += ce[2 * (size_t)r + 1];
    const double nb = (double)std::max<int64_t>(ctx->rep_off[r1] - ctx->rep_off[r0], 1);
    loss[0] = le;
    loss[1] = w_f / (3.0 * nb) * ctx->h_reduce[0];
    return MD_OK;
}

md_status sur_check_train(md_ctx *ctx, double w_e, double w_f) {
    if (!ctx->sur || !ctx->sur_set) return fail(ctx, MD_ERR_STATE, "no surrogate network in this context");
    if (!ctx->sur_ref) return fail(ctx, MD_ERR_STATE, "no training references for the current positions");
    if (!(w_e >= 0.0) || !(w_f > 0.0)) return fail(ctx, MD_ERR_ARG, "loss weights: w_e >= 0 and w_f > 0");
    return MD_OK;
}

uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
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
    drop_graphs(ctx);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    for (void *p : ctx->allocs)
        if (p) cudaFree(p);
    if (ctx->d_stage) cudaFree(ctx->d_stage);
    if (ctx->d_stamps) cudaFree(ctx->d_stamps);
    if (ctx->h_flags) cudaFreeHost(ctx->h_flags);
    if (ctx->h_reduce) cudaFreeHost(ctx->h_reduce);
    if (ctx->h_stamps) cudaFreeHost(ctx->h_stamps);
    delete ctx;
}

md_status md_create(const md_config *cfg, const md_potential *pot, const double *pos, const double *vel,
                    const int32_t *species, int32_t on_device, md_ctx **out) {
    if (!out) return MD_ERR_ARG;
    *out = nullptr;
    if (!cfg || !pot || (!pos && cfg->n_atoms > 0) || cfg->n_atoms < 0) return MD_ERR_ARG;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
            if (a != b && cfg->h[3 * a + b] != 0.0) return MD_ERR_BOX;
    const int64_t n = cfg->n_atoms;
    if (n > INT32_MAX / 8) return MD_ERR_ARG;
    Inputs in;
    in.pos.assign(3 * n, 0.0);
    in.vel.assign(3 * n, 0.0);
    in.spec.assign(n, 0);
    if (!fetch(in.pos.data(), pos, sizeof(double) * 3 * n, on_device) ||
        (vel && !fetch(in.vel.data(), vel, sizeof(double) * 3 * n, on_device)) ||
        (species && !fetch(in.spec.data(), species, sizeof(int32_t) * n, on_device)))
        return MD_ERR_CUDA;
    md_ctx *ctx = new (std::nothrow) md_ctx();
    if (!ctx) return MD_ERR_OOM;
    std::vector<double> L = {cfg->h[0], cfg->h[4], cfg->h[8]};
    md_status s = create_common(ctx, cfg, pot, in, {n}, L);
    if (s != MD_OK) {
        md_destroy(ctx);
        return s;
    }
    *out = ctx;
    return MD_OK;
}

md_status md_create_batch(int32_t n_replicas, const md_config *cfgs, const md_potential *pot,
                          const double *const *pos, const double *const *vel, const int32_t *const *species,
                          int32_t on_device, md_ctx **out) {
    if (!out) return MD_ERR_ARG;
    *out = nullptr;
    if (n_replicas < 1 || !cfgs || !pot || !pos) return MD_ERR_ARG;
    const md_config &c0 = cfgs[0];
    std::vector<int64_t> rep_n(n_replicas);
    std::vector<double> L(3 * (size_t)n_replicas);
    int64_t n = 0;
    for (int r = 0; r < n_replicas; r++) {
        const md_config &c = cfgs[r];
        if (c.n_atoms < 0 || (!pos[r] && c.n_atoms > 0)) return MD_ERR_ARG;
        if (c.skin != c0.skin || c.k_max != c0.k_max || c.dt_fs != c0.dt_fs || c.precision != c0.precision ||
            c.rebuild_every != c0.rebuild_every || c.strain_rate_zz != c0.strain_rate_zz ||
            c.integrator != c0.integrator)
            return MD_ERR_ARG;
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++)
                if (a != b && c.h[3 * a + b] != 0.0) return MD_ERR_BOX;
        for (int k = 0; k < 3; k++) L[3 * r + k] = c.h[4 * k];
        rep_n[r] = c.n_atoms;
        n += c.n_atoms;
    }
    if (n > INT32_MAX / 8) return MD_ERR_ARG;
    Inputs in;
    in.pos.assign(3 * n, 0.0);
    in.vel.assign(3 * n, 0.0);
    in.spec.assign(n, 0);
    int64_t off = 0;
    for (int r = 0; r < n_replicas; r++) {
        const int64_t m = rep_n[r];
        if (!fetch(&in.pos[3 * off], pos[r], sizeof(double) * 3 * m, on_device) ||
            (vel && vel[r] && !fetch(&in.vel[3 * off], vel[r], sizeof(double) * 3 * m, on_device)) ||
            (species && species[r] && !fetch(&in.spec[off], species[r], sizeof(int32_t) * m, on_device)))
            return MD_ERR_CUDA;
        off += m;
    }
    md_ctx *ctx = new (std::nothrow) md_ctx();
    if (!ctx) return MD_ERR_OOM;
    md_config cfg = c0;
    cfg.n_atoms = n;
    md_status s = create_common(ctx, &cfg, pot, in, rep_n, L);
    if (s != MD_OK) {
        md_destroy(ctx);
        return s;
    }
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

namespace {

// Caller-order state arrays to copy out after a stretch of steps (md_step_io).
struct StateOut {
    double *pos, *vel, *force;
    int on_device;
};

// The unsort kernels and copies of the requested arrays, enqueued only (three staging regions,
// so that the copies need no synchronisation in between).
// The device's address of a caller's host buffer in mapped pinned memory (which the device reads
// and writes directly over the host link), or NULL (pageable memory: copies through a stage).
void *mapped_host_ptr(const void *p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

md_status enqueue_state_out(md_ctx *ctx, const StateOut &o) {
    const size_t n3 = 3 * (size_t)ctx->n;
    md_status s = ensure_stage(ctx, 3 * n3 * sizeof(double));
    if (s != MD_OK) return s;
    const double4_32a *src[3] = {ctx->A.pos, ctx->A.vel, ctx->A.force};
    double *dst[3] = {o.pos, o.vel, o.force};
    for (int q = 0; q < 3; q++) {
        if (!dst[q]) continue;
        if (!o.on_device) {
            if (double *m = static_cast<double *>(mapped_host_ptr(dst[q]))) {
                MD_CK(launch_unsort_mapped(ctx->A, src[q], m, ctx->stream));
                ctx->launches++;
                continue;
            }
        }
        double *stage = static_cast<double *>(ctx->d_stage) + q * n3;
        MD_CK(launch_unsort_vec(ctx->A, src[q], stage, ctx->stream));
        MD_CK(cudaMemcpyAsync(dst[q], stage, n3 * sizeof(double),
                              o.on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
        ctx->launches++;
    }
    return MD_OK;
}

// The copies in and sort kernels of md_set_state, enqueued only.
md_status enqueue_state_in(md_ctx *ctx, const double *pos, const double *vel, const double *force, int on_device) {
    const size_t n3 = 3 * (size_t)ctx->n;
    md_status s = ensure_stage(ctx, 3 * n3 * sizeof(double));
    if (s != MD_OK) return s;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const double *src[3] = {pos, vel, force};
    double4_32a *dst[3] = {ctx->A.pos, ctx->A.vel, ctx->A.force};
    for (int q = 0; q < 3; q++) {
        if (!src[q]) continue;
        if (!on_device) {
            if (const double *m = static_cast<const double *>(mapped_host_ptr(src[q]))) {
                MD_CK(launch_sort_in_mapped(ctx->A, m, dst[q], ctx->stream));
                ctx->launches++;
                continue;
            }
        }
        double *stage = static_cast<double *>(ctx->d_stage) + q * n3;
        MD_CK(cudaMemcpyAsync(stage, src[q], n3 * sizeof(double), kind, ctx->stream));
        MD_CK(launch_sort_in_vec(ctx->A, stage, dst[q], ctx->stream));
        ctx->launches++;
    }
    if (pos) {
        MD_CK(launch_wrap(ctx->A, ctx->stream));
        ctx->launches++;
        ctx->sur_ref = false;
    }
    if (ctx->A.g3 && (pos || vel || force))   // the predictor-corrector restarts from this state
        MD_CK(cudaMemsetAsync(ctx->A.g3, 0, sizeof(double4_32a) * ctx->n, ctx->stream));
    if (pos || force) ctx->forces_valid = (force != nullptr);
    ctx->energy_valid = false;
    return MD_OK;
}

md_status step_impl(md_ctx *ctx, int32_t n_steps, const StateOut *out) {
    if (!ctx || n_steps < 0) return MD_ERR_ARG;
    if (n_steps == 0) {
        if (out && ctx->n > 0) {
            if (!ctx->forces_valid && out->force) {
                md_status s = compute_forces(ctx);
                if (s != MD_OK) return s;
            }
            md_status s = enqueue_state_out(ctx, *out);
            if (s != MD_OK) return s;
        }
        MD_CK(cudaStreamSynchronize(ctx->stream));
        return MD_OK;
    }
    // link cells are fixed in fractional coordinates; under compression keep them >= r_list wide
    if (ctx->strain_scale != 1.0) {
        bool changed = false;
        for (int r = 0; r < ctx->n_rep; r++) {
            double Lz = ctx->L[3 * r + 2];
            for (int32_t s = 0; s < n_steps; s++) Lz *= ctx->strain_scale;
            const int nc = cells_along(std::fmin(Lz, ctx->L[3 * r + 2]), ctx->r_list / ctx->C.reach);
            if (nc < 2 * ctx->C.reach + 1) return fail(ctx, MD_ERR_BOX, "strain made a box thinner than 3 link cells");
            if (nc < ctx->rc[r].nc[2]) {
                ctx->rc[r].nc[2] = nc;
                changed = true;
            }
        }
        if (changed) {  // fewer cells: the bases move down, the allocation still fits
            int base = 0;
            for (int r = 0; r < ctx->n_rep; r++) {
                ctx->rc[r].base = base;
                base += ctx->rc[r].nc[0] * ctx->rc[r].nc[1] * ctx->rc[r].nc[2];
            }
            ctx->C.ncell = base;
            MD_CK(cudaMemcpyAsync(ctx->d_rc, ctx->rc.data(), ctx->n_rep * sizeof(RepCells), cudaMemcpyHostToDevice,
                                  ctx->stream));
            MD_CK(cudaMemsetAsync(ctx->C.cell_count, 0, sizeof(int32_t) * ctx->C.ncell, ctx->stream));
            drop_graphs(ctx);
        }
    }
    if (ctx->sur) {
        if (!ctx->sur_set) return fail(ctx, MD_ERR_STATE, "surrogate network not set (md_set_surrogate)");
        ctx->sur_ref = false;
        if (ctx->S.bf16 && ctx->sur_img_stale) {
            MD_CK(launch_sur_pack(ctx->d_theta, ctx->d_img, ctx->stream));
            ctx->sur_img_stale = false;
        }
    }
    MD_CK(reset_errors(ctx));
    ctx->h_rep.clear();
    if (!ctx->forces_valid) MD_CK(enqueue_forces(ctx));
    unsigned long long *stamps = nullptr;
    if (ctx->profiling && !ctx->sur) {
        md_status st = ensure_stamps(ctx, kStampsPerStep * ((size_t)n_steps + 1));
        if (st != MD_OK) return st;
        stamps = ctx->d_stamps;
    }
    const bool graph = ctx->use_graph && !ctx->profiling && ctx->strain_scale == 1.0 &&
                       !(ctx->sur && ctx->cfg.rebuild_every > 0);
    int rows = 0;
    if (graph) {
        auto it = ctx->graphs.find(n_steps);
        if (it == ctx->graphs.end()) {
            if (!ctx->sur) {
                StepParams prep = step_params(ctx, 0);
                int pg = 0;
                MD_CK(launch_step(ctx->A, ctx->C, ctx->P, ctx->precision, ctx->lanes, prep, ctx->d_bar, nullptr, &pg,
                                  ctx->stream));
            }
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ge = nullptr;
            if (!ctx->cap_stream) MD_CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
            MD_CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
            int nl = 2;
            cudaError_t e = enqueue_steps(ctx, n_steps, nullptr, &rows, ctx->cap_stream, &nl);
            cudaError_t e2 = cudaStreamEndCapture(ctx->cap_stream, &g);
            if (e == cudaSuccess) e = e2;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess) return fail(ctx, MD_ERR_CUDA, "capturing the step graph", e);
            it = ctx->graphs.emplace(n_steps, ge).first;
            ctx->graph_rows[n_steps] = rows;
            ctx->graph_launches[n_steps] = nl;
        }
        MD_CK(cudaGraphLaunch(it->second, ctx->stream));
        rows = ctx->graph_rows[n_steps];
        ctx->launches += ctx->graph_launches[n_steps];
    } else {
        int nl = 2;
        MD_CK(enqueue_steps(ctx, n_steps, stamps, &rows, ctx->stream, &nl));
        ctx->launches += nl;
    }
    ctx->part_rows = rows;
    if (ctx->thermo_on) {  // the last half step rescaled the velocities after the energy sums
        MD_CK(launch_replica_sums(ctx->A, ctx->d_rep_off, ctx->n_rep, ctx->d_rep_sums, ctx->stream));
        ctx->h_rep.resize(5 * (size_t)ctx->n_rep);
        MD_CK(cudaMemcpyAsync(ctx->h_rep.data(), ctx->d_rep_sums, ctx->h_rep.size() * sizeof(double),
                              cudaMemcpyDeviceToHost, ctx->stream));
        ctx->launches++;
    }
    if (stamps)
        MD_CK(cudaMemcpyAsync(ctx->h_stamps, stamps, kStampsPerStep * ((size_t)n_steps + 1) * sizeof(unsigned long long),
                              cudaMemcpyDeviceToHost, ctx->stream));
    if (out && ctx->n > 0) {
        md_status so = enqueue_state_out(ctx, *out);
        if (so != MD_OK) return so;
    }
    md_status st = sync_and_check(ctx, ctx->cfg.strict_skin != 0);
    ctx->step += n_steps;
    for (int r = 0; r < ctx->n_rep; r++)
        for (int32_t s = 0; s < n_steps; s++) ctx->L[3 * r + 2] *= ctx->strain_scale;
    if (st != MD_OK) {
        ctx->forces_valid = ctx->energy_valid = false;
        return st;
    }
    if (stamps) collect_stamps(ctx, n_steps);
    ctx->forces_valid = ctx->energy_valid = true;
    // a rebuild inside a group walk's step kernel writes the local rows only (the cell walk no list)
    ctx->list_valid = ctx->C.tile == kWalkList;
    return MD_OK;
}

}  // namespace

md_status md_step(md_ctx *ctx, int32_t n_steps) { return step_impl(ctx, n_steps, nullptr); }

md_status md_step_io(md_ctx *ctx, int32_t n_steps, const double *pos_in, const double *vel_in,
                     const double *force_in, double *pos_out, double *vel_out, double *force_out,
                     md_energies *energies, int32_t on_device) {
    if (!ctx || n_steps < 0) return MD_ERR_ARG;
    if (ctx->n > 0 && (pos_in || vel_in || force_in)) {
        md_status s = enqueue_state_in(ctx, pos_in, vel_in, force_in, on_device);
        if (s != MD_OK) return s;
    }
    const StateOut out{pos_out, vel_out, force_out, on_device};
    md_status s = step_impl(ctx, n_steps, &out);
    if (s != MD_OK) return s;
    return energies ? md_energy(ctx, energies) : MD_OK;
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
    double mv2 = r[1], mom[3] = {r[8], r[9], r[10]};
    if (!ctx->h_rep.empty()) {  // velocities rescaled after the partial sums (thermostat)
        mv2 = 0.0;
        mom[0] = mom[1] = mom[2] = 0.0;
        for (int q = 0; q < ctx->n_rep; q++) {
            mv2 += ctx->h_rep[5 * (size_t)q + 1];
            for (int k = 0; k < 3; k++) mom[k] += ctx->h_rep[5 * (size_t)q + 2 + k];
        }
    }
    out->ke = 0.5 * mv2 * kMvv2e;
    out->te = out->pe + out->ke;
    const int64_t dof = 3 * ctx->n - 3 * (int64_t)ctx->n_rep;
    out->temperature = dof > 0 ? 2.0 * out->ke / ((double)dof * kKb) : 0.0;
    const double W[9] = {r[2], r[7], r[6], r[7], r[3], r[5], r[6], r[5], r[4]};
    std::memcpy(out->virial, W, sizeof(W));
    double vol = 0.0;
    for (int q = 0; q < ctx->n_rep; q++) vol += ctx->L[3 * q] * ctx->L[3 * q + 1] * ctx->L[3 * q + 2];
    out->volume = vol;
    out->pressure_gpa = (2.0 * out->ke + r[2] + r[3] + r[4]) / (3.0 * vol) * kEva3ToGpa;
    for (int k = 0; k < 3; k++) {
        out->momentum[k] = mom[k];
        out->box[k] = ctx->L[k];
    }
    out->step = ctx->step;
    out->n_rebuilds = (int64_t)ctx->h_flags->n_rebuilds;
    out->max_neighbours = ctx->h_flags->max_count;
    out->range_violations = (int64_t)ctx->h_flags->range_violations;
    return MD_OK;
}

md_status md_replica_energies(md_ctx *ctx, md_energies *out) {
    if (!ctx || !out) return MD_ERR_ARG;
    if (!ctx->energy_valid) {
        md_status s = compute_forces(ctx);
        if (s != MD_OK) return s;
    }
    const int nr = ctx->n_rep;
    MD_CK(launch_replica_sums(ctx->A, ctx->d_rep_off, nr, ctx->d_rep_sums, ctx->stream));
    ctx->launches++;
    std::vector<double> h(5 * (size_t)nr);
    MD_CK(cudaMemcpyAsync(h.data(), ctx->d_rep_sums, h.size() * sizeof(double), cudaMemcpyDeviceToHost,
                          ctx->stream));
    MD_CK(cudaStreamSynchronize(ctx->stream));
    for (int r = 0; r < nr; r++) {
        md_energies &o = out[r];
        std::memset(&o, 0, sizeof(o));
        const double *q = &h[5 * (size_t)r];
        const int64_t m = ctx->rep_off[r + 1] - ctx->rep_off[r];
        o.pe = q[0];
        o.ke = 0.5 * q[1] * kMvv2e;
        o.te = o.pe + o.ke;
        o.temperature = m > 1 ? 2.0 * o.ke / ((double)(3 * m - 3) * kKb) : 0.0;
        for (int k = 0; k < 3; k++) {
            o.momentum[k] = q[2 + k];
            o.box[k] = ctx->L[3 * r + k];
        }
        o.volume = o.box[0] * o.box[1] * o.box[2];
        o.pressure_gpa = NAN;  // the virial is reduced over the whole batch only
        o.step = ctx->step;
        o.n_rebuilds = (int64_t)ctx->h_flags->n_rebuilds;
        o.max_neighbours = ctx->h_flags->max_count;
        o.range_violations = (int64_t)ctx->h_flags->range_violations;
    }
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
            if (ctx->sur && what != MD_GET_EATOM)
                return fail(ctx, MD_ERR_STATE, "rho and F' are not defined for the surrogate");
            if (!ctx->energy_valid && (s = compute_forces(ctx)) != MD_OK) return s;
            if ((s = ensure_stage(ctx, sizeof(double) * n)) != MD_OK) return s;
            const double *src = what == MD_GET_RHO ? A.rho : (what == MD_GET_EATOM ? A.e_atom : A.dF);
            MD_CK(launch_unsort_scalar(A, src, static_cast<double *>(ctx->d_stage), ctx->stream));
            return copy_out(ctx, ctx->d_stage, dst, sizeof(double) * n, on_device);
        }
        case MD_GET_IMAGE: {
            if (!ctx->list_valid && (s = md_build_neighbours(ctx)) != MD_OK) return s;
            if ((s = ensure_stage(ctx, sizeof(double) * 3 * n)) != MD_OK) return s;
            MD_CK(launch_unsort_image(A, static_cast<double *>(ctx->d_stage), ctx->stream));
            return copy_out(ctx, ctx->d_stage, dst, sizeof(double) * 3 * n, on_device);
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
    if (ctx->sur) {  // the surrogate's gathers use one warp per atom
        if (lanes_out) *lanes_out = 32;
        return MD_OK;
    }
    if (ctx->n > 0) {
        md_status st = ctx->forces_valid ? MD_OK : compute_forces(ctx);
        if (st != MD_OK) return st;
        // Trials of the persistent step kernel itself: 3 steps from the current state at each
        // lane count, with no list rebuild (no skin trigger, no schedule, no strain), so that no
        // atom is renumbered; the state the steps change is saved first and put back after
        // every trial.
        const size_t n = (size_t)ctx->n;
        const size_t bytes = n * (4 * sizeof(double4_32a) + sizeof(float4)) + sizeof(Flags);
        unsigned char *snap = nullptr;
        MD_CK(cudaMalloc(&snap, bytes));
        double4_32a *s_pos = reinterpret_cast<double4_32a *>(snap), *s_vel = s_pos + n, *s_force = s_vel + n;
        double4_32a *s_posd = s_force + n;
        float4 *s_posf = reinterpret_cast<float4 *>(s_posd + n);
        Flags *s_flags = reinterpret_cast<Flags *>(s_posf + n);
        Atoms &A = ctx->A;
        auto copy = [&](bool save) {
            const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
            cudaError_t e = cudaMemcpyAsync(save ? s_pos : A.pos, save ? A.pos : s_pos, n * 32, k, ctx->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(save ? s_vel : A.vel, save ? A.vel : s_vel, n * 32, k, ctx->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(save ? s_force : A.force, save ? A.force : s_force, n * 32, k, ctx->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(save ? s_posf : A.posf, save ? A.posf : s_posf, n * 16, k, ctx->stream);
            if (e == cudaSuccess && A.posd)
                e = cudaMemcpyAsync(save ? s_posd : A.posd, save ? A.posd : s_posd, n * 32, k, ctx->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(save ? s_flags : ctx->d_flags, save ? ctx->d_flags : s_flags, sizeof(Flags), k,
                                    ctx->stream);
            return e;
        };
        StepParams sp = step_params(ctx, 3);
        sp.thermo = nullptr;   // trial steps leave the thermostat alone
        sp.motion = kMotionVerlet;   // and the predictor-corrector's Taylor terms (same passes)
        sp.lim2 = 1e300;
        sp.rebuild_every = 0;
        sp.strain_scale = 1.0;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaError_t e = copy(true);
        if (e == cudaSuccess) e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        float best = 1e30f;
        int best_t = ctx->lanes;
        for (int t = 1; t <= 32 && e == cudaSuccess; t *= 2) {
            for (int rep = 0; rep < 3 && e == cudaSuccess; rep++) {  // first round is a warm-up
                int grid = 0;
                StepParams prep = sp;
                prep.n_steps = 0;  // attributes and occupancy before the timed launch
                e = launch_step(A, ctx->C, ctx->P, ctx->precision, t, prep, ctx->d_bar, nullptr, &grid, ctx->stream);
                if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->stream);
                if (e == cudaSuccess)
                    e = launch_step(A, ctx->C, ctx->P, ctx->precision, t, sp, ctx->d_bar, nullptr, &grid, ctx->stream);
                if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
                if (e == cudaSuccess) e = copy(false);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e == cudaSuccess && rep > 0 && ms < best) {
                    best = ms;
                    best_t = t;
                }
                ctx->launches++;
            }
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaError_t e2 = cudaStreamSynchronize(ctx->stream);
        cudaFree(snap);
        if (e == cudaSuccess) e = e2;
        if (e != cudaSuccess) {
            ctx->forces_valid = ctx->energy_valid = false;
            return fail(ctx, MD_ERR_CUDA, "md_tune trial steps", e);
        }
        if (best_t != ctx->lanes) drop_graphs(ctx);
        ctx->lanes = best_t;
        ctx->energy_valid = false;  // the per-atom energies are those of a trial step
        st = sync_and_check(ctx, false);
        if (st != MD_OK) return st;
    }
    if (lanes_out) *lanes_out = ctx->lanes;
    return MD_OK;
}

md_status md_selftest_timeout(md_ctx *ctx) {
    if (!ctx || ctx->n == 0) return MD_ERR_ARG;
    if (ctx->sur) return fail(ctx, MD_ERR_STATE, "the bounded-barrier self-test runs the EAM step kernel");
    if (!ctx->forces_valid) {
        md_status st = compute_forces(ctx);
        if (st != MD_OK) return st;
    }
    StepParams sp = step_params(ctx, 1);
    sp.thermo = nullptr;
    sp.spin_limit = 20000;  // ~2-5 ms of polling
    // a step kernel that stages cell groups (and fits them: no fallback to the list walk) tests
    // its staging pipeline's waits instead of the grid barrier's
    const int walk = step_walk(ctx->A, ctx->C, ctx->P, ctx->precision, ctx->lanes);
    const bool staged = (walk == kWalkStaged || walk == kWalkCells || walk == kWalkHalf) && ctx->h_flags &&
                        ctx->h_flags->tile_bad == 0;
    sp.withhold_arrival = staged ? 2 : 1;
    MD_CK(reset_errors(ctx));
    int grid = 0;
    MD_CK(launch_step(ctx->A, ctx->C, ctx->P, ctx->precision, ctx->lanes, sp, ctx->d_bar, nullptr, &grid,
                      ctx->stream));
    ctx->launches++;
    md_status st = sync_and_check(ctx, false);
    // the state is no longer a clean step boundary: recompute before the next step
    ctx->forces_valid = ctx->energy_valid = false;
    return st;
}

md_status md_set_graph(md_ctx *ctx, int32_t on) {
    if (!ctx) return MD_ERR_ARG;
    if (!on) drop_graphs(ctx);
    ctx->use_graph = on != 0;
    return MD_OK;
}

md_status md_set_profiling(md_ctx *ctx, int32_t on) {
    if (!ctx) return MD_ERR_ARG;
    ctx->profiling = on != 0;
    ctx->prof = md_profile{};
    return MD_OK;
}

md_status md_get_profile(const md_ctx *ctx, md_profile *out) {
    if (!ctx || !out) return MD_ERR_ARG;
    *out = ctx->prof;
    out->launches = ctx->launches;
    return MD_OK;
}

md_status md_get_passes(md_ctx *ctx, md_passes *out) {
    if (!ctx || !out) return MD_ERR_ARG;
    MD_CK(cudaMemcpyAsync(ctx->h_flags, ctx->d_flags, sizeof(Flags), cudaMemcpyDeviceToHost, ctx->stream));
    MD_CK(cudaStreamSynchronize(ctx->stream));
    const Cells &C = ctx->C;
    out->walk = C.tile == kWalkStaged  ? MD_PASSES_STAGED
                : C.tile == kWalkCells ? MD_PASSES_CELLS
                : C.tile == kWalkHalf  ? MD_PASSES_HALF
                                       : MD_PASSES_LIST;
    out->cells_per_group = C.tile ? C.gx : 0;
    out->groups = C.tile ? C.n_groups : 0;
    out->capacity = C.tile ? C.cap : 0;
    out->last_max = C.tile ? ctx->h_flags->tile_max : 0;
    out->active = C.tile && ctx->lanes <= 8 && !ctx->h_flags->tile_bad;
    out->stage_buffers = C.tile ? C.nbuf : 0;
    if (ctx->A.pairs) {   // the FP64 half list over the full list's rows
        out->walk = MD_PASSES_HALF;
        out->active = 1;
    }
    return MD_OK;
}

md_status md_set_state(md_ctx *ctx, const double *pos, const double *vel, const double *force,
                       int32_t on_device) {
    if (!ctx) return MD_ERR_ARG;
    if (ctx->n == 0) return MD_OK;
    md_status s = enqueue_state_in(ctx, pos, vel, force, on_device);
    if (s != MD_OK) return s;
    MD_CK(cudaStreamSynchronize(ctx->stream));
    return MD_OK;
}

md_status md_set_surrogate(md_ctx *ctx, const md_surrogate *spec, const float *theta, const float *gmu,
                           const float *ginv) {
    if (!ctx || !spec || !theta) return MD_ERR_ARG;
    if (!ctx->sur) return fail(ctx, MD_ERR_STATE, "not a MD_POT_SURROGATE context");
    if (spec->nb != kSurNb || spec->h1 != kSurH1 || spec->h2 != kSurH2 ||
        (spec->net != MD_SUR_FP32 && spec->net != MD_SUR_BF16) || !(spec->width > 0.0) ||
        !std::isfinite(spec->mu0) || !std::isfinite(spec->dmu) || !(spec->rd > 0.0) ||
        std::fabs(spec->rd - ctx->r_cut) > 1e-12 * ctx->r_cut)
        return fail(ctx, MD_ERR_ARG, "surrogate spec: 32-64-64 network, width > 0, rd = the potential's r_cut");
    for (int p = 0; p < kSurParams; p++)
        if (!std::isfinite(theta[p])) return fail(ctx, MD_ERR_ARG, "non-finite network parameter");
    std::vector<float> mu(kSurNb, 0.f), iv(kSurNb, 1.f);
    for (int k = 0; k < kSurNb; k++) {
        if (gmu) mu[k] = gmu[k];
        if (ginv) iv[k] = ginv[k];
        if (!std::isfinite(mu[k]) || !std::isfinite(iv[k])) return fail(ctx, MD_ERR_ARG, "non-finite standardisation");
    }
    md_status st = sur_alloc(ctx);
    if (st != MD_OK) return st;
    MD_CK(cudaMemcpy(ctx->d_theta, theta, sizeof(float) * kSurParams, cudaMemcpyHostToDevice));
    MD_CK(cudaMemcpy(ctx->d_gmu, mu.data(), sizeof(float) * kSurNb, cudaMemcpyHostToDevice));
    MD_CK(cudaMemcpy(ctx->d_ginv, iv.data(), sizeof(float) * kSurNb, cudaMemcpyHostToDevice));
    MD_CK(cudaMemset(ctx->d_adam_m, 0, sizeof(float) * kSurParams));
    MD_CK(cudaMemset(ctx->d_adam_v, 0, sizeof(float) * kSurParams));
    ctx->adam_t = 0;
    SurNet &S = ctx->S;
    const double w = spec->width;
    S.mu0 = (float)spec->mu0;
    S.dmu = (float)spec->dmu;
    S.inv2w2 = (float)(1.0 / (2.0 * w * w));
    S.invw2 = (float)(1.0 / (w * w));
    S.rd = (float)spec->rd;
    S.rd2 = (float)(spec->rd * spec->rd);
    S.pi_rd = (float)(3.14159265358979323846 / spec->rd);
    S.bf16 = spec->net == MD_SUR_BF16;
    ctx->sur_spec = *spec;
    ctx->sur_set = true;
    ctx->sur_img_stale = true;
    ctx->forces_valid = ctx->energy_valid = false;
    drop_graphs(ctx);   // graphs hold the network view by value
    return MD_OK;
}

md_status md_sur_get_params(md_ctx *ctx, float *theta, float *gmu, float *ginv) {
    if (!ctx) return MD_ERR_ARG;
    if (!ctx->sur || !ctx->sur_set) return fail(ctx, MD_ERR_STATE, "no surrogate network in this context");
    MD_CK(cudaStreamSynchronize(ctx->stream));
    if (theta) MD_CK(cudaMemcpy(theta, ctx->d_theta, sizeof(float) * kSurParams, cudaMemcpyDeviceToHost));
    if (gmu) MD_CK(cudaMemcpy(gmu, ctx->d_gmu, sizeof(float) * kSurNb, cudaMemcpyDeviceToHost));
    if (ginv) MD_CK(cudaMemcpy(ginv, ctx->d_ginv, sizeof(float) * kSurNb, cudaMemcpyDeviceToHost));
    return MD_OK;
}

md_status md_sur_standardize(md_ctx *ctx) {
    if (!ctx) return MD_ERR_ARG;
    if (!ctx->sur || !ctx->sur_set) return fail(ctx, MD_ERR_STATE, "no surrogate network in this context");
    if (ctx->n == 0) return MD_OK;
    md_status st = sur_ensure_list(ctx);
    if (st != MD_OK) return st;
    MD_CK(sur_descriptors32(ctx));
    const int blocks = std::min(1024, blocks_for(ctx->n, kThreads / 32));
    const size_t bytes = sizeof(double) * 2 * kSurNb * blocks;
    if ((st = ensure_stage(ctx, bytes)) != MD_OK) return st;
    MD_CK(launch_sur_stats(ctx->A, ctx->S, static_cast<double *>(ctx->d_stage), blocks, ctx->stream));
    ctx->launches++;
    std::vector<double> part(2 * kSurNb * (size_t)blocks);
    MD_CK(cudaMemcpyAsync(part.data(), ctx->d_stage, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    MD_CK(cudaStreamSynchronize(ctx->stream));
    std::vector<float> th(kSurParams), mu0(kSurNb), iv0(kSurNb), mu1(kSurNb), iv1(kSurNb);
    MD_CK(cudaMemcpy(th.data(), ctx->d_theta, sizeof(float) * kSurParams, cudaMemcpyDeviceToHost));
    MD_CK(cudaMemcpy(mu0.data(), ctx->d_gmu, sizeof(float) * kSurNb, cudaMemcpyDeviceToHost));
    MD_CK(cudaMemcpy(iv0.data(), ctx->d_ginv, sizeof(float) * kSurNb, cudaMemcpyDeviceToHost));
    for (int k = 0; k < kSurNb; k++) {
        double s1 = 0.0, s2 = 0.0;
        for (int b = 0; b < blocks; b++) {
            s1 += part[(size_t)b * 2 * kSurNb + k];
            s2 += part[(size_t)b * 2 * kSurNb + kSurNb + k];
        }
        const double mean = s1 / (double)ctx->n;
        const double var = std::fmax(s2 / (double)ctx->n - mean * mean, 0.0);
        mu1[k] = (float)mean;
        iv1[k] = (float)(1.0 / std::fmax(std::sqrt(var), 1e-3));   // near-empty channels stay near 0
    }
    // same function of G: W1' = W1 ginv0 / ginv1,  b1' = b1 + W1 ginv0 (mu1 - mu0)
    for (int p = 0; p < kSurH1; p++) {
        double b = th[kSurH1 * kSurNb + p];
        for (int k = 0; k < kSurNb; k++) {
            const double w = th[p * kSurNb + k];
            b += w * iv0[k] * ((double)mu1[k] - (double)mu0[k]);
            th[p * kSurNb + k] = (float)(w * iv0[k] / iv1[k]);
        }
        th[kSurH1 * kSurNb + p] = (float)b;
    }
    MD_CK(cudaMemcpy(ctx->d_theta, th.data(), sizeof(float) * kSurParams, cudaMemcpyHostToDevice));
    MD_CK(cudaMemcpy(ctx->d_gmu, mu1.data(), sizeof(float) * kSurNb, cudaMemcpyHostToDevice));
    MD_CK(cudaMemcpy(ctx->d_ginv, iv1.data(), sizeof(float) * kSurNb, cudaMemcpyHostToDevice));
    MD_CK(cudaMemset(ctx->d_adam_m, 0, sizeof(float) * kSurParams));
    MD_CK(cudaMemset(ctx->d_adam_v, 0, sizeof(float) * kSurParams));
    ctx->adam_t = 0;
    ctx->sur_img_stale = true;
    ctx->forces_valid = ctx->energy_valid = false;
    return MD_OK;
}

md_status md_sur_get(md_ctx *ctx, int32_t what, float *dst, int32_t on_device) {
    if (!ctx || (!dst && ctx->n > 0)) return MD_ERR_ARG;
    if (!ctx->sur || !ctx->sur_set) return fail(ctx, MD_ERR_STATE, "no surrogate network in this context");
    if (what != MD_SUR_GET_G && what != MD_SUR_GET_DEDG) return fail(ctx, MD_ERR_ARG, "unknown md_sur_get selector");
    if (ctx->n == 0) return MD_OK;
    md_status st;
    if (what == MD_SUR_GET_G) {
        if ((st = sur_ensure_list(ctx)) != MD_OK) return st;
        MD_CK(sur_descriptors32(ctx));
    } else if (!ctx->forces_valid && (st = compute_forces(ctx)) != MD_OK) {
        return st;
    }
    const size_t bytes = sizeof(float) * (size_t)ctx->n * kSurNb;
    if ((st = ensure_stage(ctx, bytes)) != MD_OK) return st;
    MD_CK(launch_sur_unsort_rows(ctx->A, what == MD_SUR_GET_G ? ctx->S.G : ctx->S.g,
                                 static_cast<float *>(ctx->d_stage), ctx->stream));
    ctx->launches++;
    return copy_out(ctx, ctx->d_stage, dst, bytes, on_device);
}

md_status md_sur_set_reference(md_ctx *ctx, const double *e_ref, const double *f_ref, int32_t on_device) {
    if (!ctx || !e_ref || (!f_ref && ctx->n > 0)) return MD_ERR_ARG;
    if (!ctx->sur || !ctx->sur_set) return fail(ctx, MD_ERR_STATE, "no surrogate network in this context");
    md_status st = sur_ensure_list(ctx);
    if (st != MD_OK) return st;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    MD_CK(cudaMemcpyAsync(ctx->S.eref, e_ref, sizeof(double) * ctx->n_rep, kind, ctx->stream));
    if (ctx->n > 0) {
        if ((st = ensure_stage(ctx, sizeof(double) * 3 * ctx->n)) != MD_OK) return st;
        MD_CK(cudaMemcpyAsync(ctx->d_stage, f_ref, sizeof(double) * 3 * ctx->n, kind, ctx->stream));
        MD_CK(launch_sort_in_vec(ctx->A, static_cast<const double *>(ctx->d_stage), ctx->d_fref, ctx->stream));
        MD_CK(sur_descriptors32(ctx));
        ctx->launches++;
    }
    MD_CK(cudaStreamSynchronize(ctx->stream));
    ctx->sur_ref = true;
    return MD_OK;
}

md_status md_sur_loss_grad(md_ctx *ctx, int32_t rep_begin, int32_t rep_end, double w_e, double w_f,
                           double *loss, float *grad) {
    if (!ctx) return MD_ERR_ARG;
    md_status st = sur_check_train(ctx, w_e, w_f);
    if (st != MD_OK) return st;
    if (rep_begin < 0 || rep_end > ctx->n_rep || rep_begin >= rep_end) return fail(ctx, MD_ERR_ARG, "replica range");
    MD_CK(reset_errors(ctx));
    int rows = 0, blocks = 0;
    MD_CK(sur_train_pass(ctx, rep_begin, rep_end, w_e, w_f, &rows, &blocks));
    MD_CK(launch_sur_update(ctx->S, ctx->d_theta, ctx->d_adam_m, ctx->d_adam_v, ctx->d_grad, blocks, 1, 0.f,
                            ctx->stream));
    MD_CK(launch_reduce(ctx->A, rows, ctx->d_reduce, ctx->stream));
    MD_CK(cudaMemcpyAsync(ctx->h_reduce, ctx->d_reduce, sizeof(double) * kPartials, cudaMemcpyDeviceToHost,
                          ctx->stream));
    ctx->launches += 2;
    ctx->forces_valid = ctx->energy_valid = false;   // forces and energies of a sub-range only
    st = sync_and_check(ctx, false);
    if (st != MD_OK) return st;
    if (grad) MD_CK(cudaMemcpy(grad, ctx->d_grad, sizeof(float) * kSurParams, cudaMemcpyDeviceToHost));
    if (loss) return sur_loss_terms(ctx, rep_begin, rep_end, w_f, loss);
    return MD_OK;
}

md_status md_sur_train(md_ctx *ctx, int32_t n_iter, int32_t rep_begin, int32_t rep_end, int32_t batch_reps,
                       double lr, double w_e, double w_f, uint64_t seed, double *loss) {
    if (!ctx || n_iter < 0 || batch_reps < 1) return MD_ERR_ARG;
    md_status st = sur_check_train(ctx, w_e, w_f);
    if (st != MD_OK) return st;
    if (rep_begin < 0 || rep_end > ctx->n_rep || batch_reps > rep_end - rep_begin || !(lr > 0.0))
        return fail(ctx, MD_ERR_ARG, "replica range, batch size or learning rate");
    if (n_iter == 0) return MD_OK;
    const uint64_t nbatch = (uint64_t)((rep_end - rep_begin) / batch_reps);
    MD_CK(reset_errors(ctx));
    int rows = 0, blocks = 0, r0 = 0;
    for (int it = 0; it < n_iter; it++) {
        r0 = rep_begin + (int)(splitmix64(seed + (uint64_t)it) % nbatch) * batch_reps;
        MD_CK(sur_train_pass(ctx, r0, r0 + batch_reps, w_e, w_f, &rows, &blocks));
        if (it == n_iter - 1) {
            MD_CK(launch_reduce(ctx->A, rows, ctx->d_reduce, ctx->stream));
            MD_CK(cudaMemcpyAsync(ctx->h_reduce, ctx->d_reduce, sizeof(double) * kPartials, cudaMemcpyDeviceToHost,
                                  ctx->stream));
            ctx->launches++;
        }
        MD_CK(launch_sur_update(ctx->S, ctx->d_theta, ctx->d_adam_m, ctx->d_adam_v, nullptr, blocks, ++ctx->adam_t,
                                (float)lr, ctx->stream));
        ctx->launches++;
    }
    ctx->sur_img_stale = true;
    ctx->forces_valid = ctx->energy_valid = false;
    st = sync_and_check(ctx, false);
    if (st != MD_OK) return st;
    if (loss) return sur_loss_terms(ctx, r0, r0 + batch_reps, w_f, loss);
    return MD_OK;
}

md_status md_set_thermostat(md_ctx *ctx, int32_t on, const double *t_kelvin, const double *tau_fs) {
    if (!ctx) return MD_ERR_ARG;
    if (ctx->sur) return fail(ctx, MD_ERR_STATE, "the thermostat runs in the EAM step kernel");
    if (ctx->cfg.integrator == MD_INTEGRATOR_PC3 && on)
        return fail(ctx, MD_ERR_STATE, "the thermostat steps with velocity Verlet, not the predictor-corrector");
    if (!on) {
        if (ctx->thermo_on) drop_graphs(ctx);
        ctx->thermo_on = false;
        return MD_OK;
    }
    if (!t_kelvin || !tau_fs) return MD_ERR_ARG;
    const int nr = ctx->n_rep;
    for (int r = 0; r < nr; r++)
        if (!(t_kelvin[r] > 0.0) || !std::isfinite(t_kelvin[r]) || !(tau_fs[r] > 0.0) || !std::isfinite(tau_fs[r]))
            return fail(ctx, MD_ERR_ARG, "thermostat: T > 0 and tau > 0 for every replica");
    std::vector<int2> chunks;
    for (int r = 0; r < nr; r++)
        for (int64_t a = ctx->rep_off[r]; a < ctx->rep_off[r + 1]; a += kKeChunk) chunks.push_back(make_int2(r, (int)a));
    std::vector<Thermo> th(nr);
    for (int r = 0; r < nr; r++) {
        const int64_t m = ctx->rep_off[r + 1] - ctx->rep_off[r];
        th[r] = Thermo{};
        th[r].gkt = (double)(3 * m - 3) * kKb * t_kelvin[r];
        // thermal inertia from the relaxation time: Q = g k_B T tau^2 (eV fs^2)
        th[r].q = th[r].gkt * tau_fs[r] * tau_fs[r];
        if (!(th[r].q > 0.0) || !std::isfinite(th[r].q))
            return fail(ctx, MD_ERR_ARG, "thermostat: Q = g k_B T tau^2 is not a positive finite number");
        th[r].s_b = th[r].s_a = 1.0;
    }
    if (!ctx->d_thermo) MD_CK(dalloc(ctx, &ctx->d_thermo, nr));
    if (ctx->n_ke_chunks < (int)chunks.size()) MD_CK(dalloc(ctx, &ctx->d_ke_chunks, chunks.size()));
    ctx->n_ke_chunks = (int)chunks.size();
    MD_CK(cudaMemcpy(ctx->d_thermo, th.data(), nr * sizeof(Thermo), cudaMemcpyHostToDevice));
    if (!chunks.empty())
        MD_CK(cudaMemcpy(ctx->d_ke_chunks, chunks.data(), chunks.size() * sizeof(int2), cudaMemcpyHostToDevice));
    ctx->thermo_on = true;
    ctx->h_rep.clear();
    drop_graphs(ctx);   // graphs hold the step parameters by value
    return MD_OK;
}

md_status md_get_thermostat(md_ctx *ctx, double *out) {
    if (!ctx || !out) return MD_ERR_ARG;
    if (!ctx->d_thermo) return fail(ctx, MD_ERR_STATE, "no thermostat was set");
    if (!ctx->energy_valid) {
        md_status s = compute_forces(ctx);
        if (s != MD_OK) return s;
    }
    const int nr = ctx->n_rep;
    MD_CK(launch_replica_sums(ctx->A, ctx->d_rep_off, nr, ctx->d_rep_sums, ctx->stream));
    ctx->launches++;
    std::vector<double> h(5 * (size_t)nr);
    std::vector<Thermo> th(nr);
    MD_CK(cudaMemcpyAsync(h.data(), ctx->d_rep_sums, h.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    MD_CK(cudaMemcpyAsync(th.data(), ctx->d_thermo, nr * sizeof(Thermo), cudaMemcpyDeviceToHost, ctx->stream));
    MD_CK(cudaStreamSynchronize(ctx->stream));
    for (int r = 0; r < nr; r++) {
        const double pe = h[5 * (size_t)r], ke = 0.5 * h[5 * (size_t)r + 1] * kMvv2e;
        const Thermo &t = th[r];
        out[4 * r] = t.pi;
        out[4 * r + 1] = t.xi;
        out[4 * r + 2] = t.q;
        out[4 * r + 3] = ke + pe + 0.5 * t.q * t.pi * t.pi + t.gkt * t.xi;
    }
    return MD_OK;
}

}  // extern "C"
