// Internal declarations shared by the kernels and the C ABI layer of libmd.so.
// Per-atom state on the device is kept in link-cell order: every neighbour-list build
// renumbers the atoms so that the atoms of one link cell are adjacent and cells follow
// their index (the cache-friendly ordering of §3.2.1-3.2.2); id[] maps a slot to the
// caller's atom id.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "md.h"

namespace mdk {

// Units of §2.7 (CODATA 2018): amu (Å/fs)^2 in eV, Boltzmann constant, eV/Å^3 in GPa.
constexpr double kAmuKg = 1.66053906660e-27;
constexpr double kEvJ = 1.602176634e-19;
constexpr double kKb = 8.617333262e-5;
constexpr double kMvv2e = kAmuKg * 1.0e10 / kEvJ;
constexpr double kEva3ToGpa = kEvJ * 1.0e30 / 1.0e9;

enum : int32_t { FLAG_OVERFLOW = 1, FLAG_NONFINITE = 2, FLAG_TIMEOUT = 4 };

constexpr int kThreads = 128;     // threads per block of the per-atom kernels
// After an atom's force: nothing, the second half kick of velocity Verlet, or the corrector of the
// third-order predictor-corrector (md.h MD_INTEGRATOR_PC3).
enum : int { kMotionNone = 0, kMotionVerlet = 1, kMotionPC3 = 2 };
constexpr int kPartials = 11;     // per-block FP64 partial sums: pe, sum m v^2, W(6), p(3)
constexpr int kStampsPerStep = 12;  // %globaltimer stamps per step of the persistent kernel

// Current orthorhombic box of one system (changes under the strain ramp; kept in device
// memory so that a captured step reads the live value).
struct Box {
    double L[3];
    double invL[3];
    float Lf[3];
    float invLf[3];
    // double-float path (MD_PREC_DF): L as hi + lo, and the offset added to every image
    // coordinate before it is split into hi + lo, so that all high parts lie within a factor of
    // two of each other and their differences are exact
    float Lh[3], Ll[3];
    double xoff[3];
};

// Device-side status, read by the host after each synchronising call.
struct Flags {
    int32_t need_rebuild;   // set by the displacement check or the schedule; cleared by pass 1
    int32_t error;          // FLAG_* bits
    int32_t max_count;      // longest list at the last build
    int32_t skin_exceeded;  // an atom moved more than skin/2 since the last build
    unsigned long long n_rebuilds;
    unsigned long long range_violations;
    long long step;         // steps taken (the rebuild schedule counts from here)
    int32_t tile_bad;       // a cell group's neighbourhood exceeded the staging capacity at the last build
    int32_t tile_max;       // largest cell-group neighbourhood (atoms) at the last build
    int32_t seg_done;       // steps of the md_step call under way done when a launch of the step kernel
                            // stopped at a rebuild request (n_steps once the call's steps are all done)
};

// Device view of the potential.  Tables hold, per interval k of a uniform knot grid, the
// monomial coefficients (c0, c1, c2, c3) of the cubic in t = (x - x_k)/h; row n_knots-1 holds
// (y_end, h*y'_end, 0, 0) for the linear continuation past the last knot.  Pair tables fuse
// V and phi of a species pair per interval: VP32 row = 8 floats (V c0..c3, phi c0..c3) in
// one 32-byte load; VP64 = two double4 per interval (V, then phi).
struct Pot {
    int kind, ns, nk;
    int smt_phi;   // table copy in shared memory: first phi row (nk; 0 where a pass holds only its own rows)
    double rc2;
    float rc2f;
    float rc2f_skin;   // FP32 r^2 above which a pair is beyond r_cut whatever the FP32 rounding of its
                       // coordinates (the FP64 half list's skip of its skin entries)
    double fs[7];   // d, c, A, beta, c0, c1, c2
    float fsf[7];
    double bd;      // beta / d
    float bdf;
    double r_min, inv_dr, rho_min, inv_drho;
    double xneg;    // -r_min inv_dr: the knot coordinate of r is fma(r, inv_dr, xneg)
    float r_minf, inv_drf;
    const double4_32a *VP64;  // [((a*ns+b)*nk + k)*2 + {0: V, 1: phi_ab}]
    const double4_32a *VP32;  // [(a*ns+b)*nk + k], 8 floats
    const double4_32a *F64;   // [a*nk + k]
    // one species: [k] derivative rows of the force pass (mixed, table in shared memory): c1 of V,
    // c1 of phi, then (2 c2, 3 c3) of V and of phi as binary16 pairs scaled by 1/dsv and 1/dsp
    const float4 *D32;
    const float *V0;          // one species: [k] c0 of the V rows (V itself on the energy step)
    // one species, FP64 derivative cache: [2k + {0: V, 1: phi}] = (c1, 2 c2, 3 c3, 0) * inv_dr, the
    // r-derivative of the interval's cubic as a quadratic in t
    const double4_32a *D64;
    // one species, double-float path: [4k + q], q = 0: phi (c0 hi, lo, c1 hi, lo); 1: (phi c2, phi c3,
    // phi' e3, V' e3); 2: phi' (d1 hi, lo, d2 hi, lo); 3: V' (d1 hi, lo, d2 hi, lo) with d1 = c1 s,
    // d2 = 2 c2 s, e3 = 3 c3 s, s = inv_dr (the r-derivative); TVx [2k + q]: V (c0 hi, lo, c1 hi, lo),
    // (c2, c3, 0, 0) for the energy
    const float4 *TX;
    const float4 *TVx;
    float idr_h, idr_l;       // inv_dr as hi + lo
    float x0_h, x0_l;         // r_min inv_dr as hi + lo
    float dsv, dsp;
    // explicit knot sums (MD_POT_KNOTS): function t (V[a][b] = a*ns+b, phi[a][b] = ns*ns + a*ns+b)
    // has nkt terms (coefficient, radius) at K64/K32 + t*nkt; F_a = -A[a] sqrt(rho)
    int nkt;
    const double2 *K64;
    const float2 *K32;
    double A64[8];
};

// Link-cell grid of one replica: its cells are the global cells [base, base + nc0*nc1*nc2).
struct RepCells {
    int nc[3];
    int base;
};

// Grid barrier of the persistent step kernel (see md_step.cu).
struct GridBarrier {
    unsigned int count;
    unsigned int gen;
    int abort;
    int pad;
};

// Device view of the per-atom state (cell order).  A batch of replicas is stored as one
// system whose atoms of replica r are contiguous; rep[i] is NULL for a single system.
struct Atoms {
    int n, k_max;
    int n_rep;
    double4_32a *pos, *vel, *force, *ref;        // pos.w = species; vel.w = (1/mvv2e)/m
    double4_32a *posd;                           // FP64 path: pos in the periodic image of the last
                                                 // build (as posf; NULL on the mixed path)
    double4_32a *pos_tmp, *vel_tmp, *force_tmp;  // renumbering scratch
    float4 *posf;                            // FP32 wrapped position, w = species bits
    float4 *posx;                            // double-float path: [2 i] = high parts, [2 i + 1] = low parts
                                             // of the image coordinates plus Box::xoff
    float4 *p2x;                             // double-float pass 2: as posx, w = F'(rho) (hi, then lo)
    float4 *p2f;                             // mixed pass 2: wrapped position + F'(rho)
    double4_32a *p2d;                        // FP64 pass 2: position + F'(rho)
    double *rho, *dF, *e_atom;
    int32_t *id, *id_tmp, *rank, *spec, *spec_tmp;
    int32_t *cell_of, *slot, *order;
    int32_t *sorted;                         // order after the in-cell sort (aliases cell_of)
    int32_t *nbr, *count;                    // list entry k of atom i: see NbrRow; k < min(count, k_max)
    double2 *dcache;                         // FP64 path, one species: per list entry (same plane layout
                                             // as nbr) the radial factors of the pair force, (V'(r) / r,
                                             // phi'(r) / r), written by the density pass and read by
                                             // the force passes that need no energy (the pair walk:
                                             // both negated, read by every force pass); (0, 0)
                                             // beyond r_cut.  NULL: not kept
    uint8_t *wrap;                           // 1: the atom's link cell is on the box boundary at the
                                             // last build (some neighbour cell is a periodic image)
    int image_fixed;                         // 1: no strain ramp, so posf/p2f stay in the periodic
                                             // image of the last build (then wrap == 0 means no
                                             // minimum image is needed)
    uint16_t *lnbr;                          // staged walk: the same entries as slots of the atom's
                                             // cell-group stencil (same plane layout as nbr); half walk:
                                             // only the entries j > i, lcount of them
    int32_t *lcount;                         // half walk: entries of each half row
    int32_t *cup;                            // FP64 pair walk: entries j > i at the front of each row
    int32_t *cin;                            // FP64 pair walk: of those, the ones inside r_cut at the
                                             // build, at the very front
    int pairs;                               // 1: the FP64 pair walk (kWalkPairs)
    float pair_rc2f;                         // FP64 pair walk: r_cut^2 (the build's FP32 ordering)
    double *rho_acc;                         // half walk: density accumulators [n]
    double *e_acc;                           // FP64 pair walk: pair-energy accumulators [n]
    double4_32a *f_acc;                      // half walk: force (x, y, z) and pair-energy (w) accumulators
    double4_32a *g2, *g3;                    // predictor-corrector (md.h MD_INTEGRATOR_PC3): the predicted
                                             // acceleration term (dt^2/2) a and the third-derivative term
                                             // (dt^3/6) da/dt of each atom (NULL under velocity Verlet)
    double4_32a *g2_tmp, *g3_tmp;            // their renumbering scratch
    double *partials;                        // [kPartials][part_stride] per-block sums
    int part_stride;
    int32_t *rep;                            // replica of each slot (NULL: one system)
    Box *boxes;                              // [n_rep]
    Flags *flags;
};

// The neighbour list in planes of 4 entries: entry k of atom i is
// nbr[((k / 4) * n + i) * 4 + k % 4], so the 4 lanes of 8 consecutive atoms that read entries
// 4m..4m+3 read one 128-byte line, and a warp of 32 atoms writing entry k touches 4 lines.
// Allocated as ceil(k_max / 4) planes of 4 n entries.
struct NbrRow {
    int32_t *p;        // &nbr[4 i]
    long long plane;   // 4 n
    __host__ __device__ int32_t *ptr(int k) const { return p + (long long)(k >> 2) * plane + (k & 3); }
    __host__ __device__ int32_t &operator[](int k) const { return *ptr(k); }
};
__host__ __device__ inline NbrRow nbr_row(const Atoms &A, int i) {
    return NbrRow{A.nbr + 4 * (size_t)i, 4LL * A.n};
}
// The derivative cache of atom i in the list's plane layout (entry k at the offset of nbr[k]).
struct DRow {
    double2 *p;        // &dcache[4 i]
    long long plane;   // 4 n
    __host__ __device__ double2 *ptr(int k) const { return p + (long long)(k >> 2) * plane + (k & 3); }
};
__host__ __device__ inline DRow dcache_row(const Atoms &A, int i) {
    return DRow{A.dcache + 4 * (size_t)i, 4LL * A.n};
}
struct NbrRow16 {
    const uint16_t *p;
    long long plane;
    __host__ __device__ const uint16_t *ptr(int k) const { return p + (long long)(k >> 2) * plane + (k & 3); }
};
__host__ __device__ inline NbrRow16 lnbr_row(const Atoms &A, int i) {
    return NbrRow16{A.lnbr + 4 * (size_t)i, 4LL * A.n};
}
// Load of per-atom data that the persistent step kernel itself writes in an earlier phase
// (positions, pass-2 copies, list rows, species: written before a grid barrier, read after it).
// The read-only data path (ld.global.nc) is defined only for data no thread writes during the
// launch, so these are ordinary global loads; MD_LDG_PHASED=1 at build time takes the read-only
// path instead (for comparison).
#ifndef MD_LDG_PHASED
#define MD_LDG_PHASED 0
#endif
template <typename T>
__device__ __forceinline__ T ld_phase(const T *p) {
#if MD_LDG_PHASED
    return __ldg(p);
#else
    return *p;
#endif
}
inline size_t nbr_entries(int64_t n, int k_max) { return (size_t)((k_max + 3) / 4) * 4 * (size_t)n; }

struct Cells {
    int ncell;   // all replicas
    int reach;   // cells are r_list / reach wide; the list stencil is (2 reach + 1)^3 cells
    int ntiles;
    RepCells *rc;  // [n_rep], device
    int32_t *cell_count, *cell_start, *tile_sums;
    // Cell groups of the group walks (one system, cells r_list wide): groups of gx consecutive
    // cells along x.  The neighbourhood of a group is its 3 x 3 x (gx + 2) stencil of cells; stencil
    // cell s = ((dz + 1) 3 + (dy + 1)) (gx + 2) + (x - x0 + 1) for the group starting at x0.
    int tile;           // walk of the step kernel's passes: kWalkList (no groups), kWalkStaged (groups
                        // and 16-bit local lists), kWalkCells (groups, no list unless a group overflows),
                        // kWalkHalf (groups, 16-bit half lists, shared-memory accumulation)
    int gx, ngx, n_groups, st_cells;   // cells per group, groups per row, groups, 9 (gx + 2)
    int cap;            // atoms one stage buffer holds
    int nbuf;           // stage buffers per block (2: the next group is staged while one is computed)
    int32_t *grp_loc;   // [n_groups][st_cells + 1]: staged slot of the first atom of each stencil cell, total
};

constexpr int kGroupMaxGx = 8;   // cells per group at most (the stencil row is kGroupMaxGx + 2 cells)
// Stage buffers per block of the group walks at most (fewer where the neighbourhoods do not fit):
// the staged and cell walks take up to MD_STAGE_BUFS, the half walk (whose per-slot sums double a
// buffer) up to 2.  Measured on fcc Cu 500,000 atoms: staged 0.75 ms per step with 2 buffers of
// 8-cell groups, 0.68 ms with 3 of 6 cells, 0.67 ms with 4 of 4 cells; half 1.40 ms with 2 of 4
// cells, 1.91 ms with 3 of 2.
#ifndef MD_STAGE_BUFS
#define MD_STAGE_BUFS 4
#endif

// Neighbour walks of the step kernel's passes (md_config.passes).
enum : int { kWalkList = 0, kWalkStaged = 1, kWalkCells = 2, kWalkHalf = 3, kWalkPairs = 4 };
// kWalkPairs: FP64, one species, the list walk with each pair computed once (each row partitioned
// at every build so that its entries j > i come first, cup[i] of them), the neighbour's share
// added with FP64 atomics (md_config.passes = MD_PASSES_HALF on the FP64 path)
constexpr int kPairsKMax = 256;   // rows partitioned in registers: k_max <= 8 x 32

// Shared memory of the mixed-precision step kernel: a single-species knot table (2 float4 per
// knot) of at most kSmemTableMax bytes, and the stage of the group walks; together at most
// kSmemDynMax bytes (the static shared memory of a 1024-thread block comes on top).
constexpr size_t kSmemTableMax = 200 * 1024;
constexpr size_t kSmemDynMax = 222 * 1024;
constexpr int kCellsQueue = 64;   // cell walk: hit queue (16-bit stage slots) per warp, static shared
constexpr size_t kSmemDynMaxCells = kSmemDynMax - 32 * kCellsQueue * sizeof(uint16_t);
// 1: for one species the shared copy holds the force pass's derivative rows in place of the V
// rows, so the force pass reads one row per pair instead of two.
#ifndef MD_DTABLE
#define MD_DTABLE 1
#endif
#ifndef MD_SMEM_TABLE
#define MD_SMEM_TABLE 1
#endif
inline size_t smem_table_bytes(int kind, int ns, int precision, int nk) {
    const size_t b = (size_t)nk * 32;
    return (MD_SMEM_TABLE && kind == MD_POT_TABLES && ns == 1 && precision == MD_PREC_MIXED && b <= kSmemTableMax)
               ? b : 0;
}

// Launchers (stream-ordered, no synchronisation).
cudaError_t launch_set_rebuild(Flags *f, cudaStream_t s);
cudaError_t launch_clear_rebuild(Flags *f, cudaStream_t s);
cudaError_t launch_rebuild(const Atoms &A, const Cells &C, double rl2, float band_lo, float band_hi,
                           int list_group, cudaStream_t s);
cudaError_t launch_check_displacement(const Atoms &A, double lim2, cudaStream_t s);
cudaError_t launch_wrap(const Atoms &A, cudaStream_t s);
// lanes = T lanes per atom (1, 2, 4, 8, 16 or 32)
cudaError_t launch_density(const Atoms &A, const Pot &P, int precision, int lanes, cudaStream_t s);
cudaError_t launch_force(const Atoms &A, const Pot &P, int precision, int lanes, bool kick, bool energy,
                         double half_dt, cudaStream_t s);
int partial_blocks(int n, int lanes);  // blocks (and partial-sum rows) of a force launch
cudaError_t launch_reduce(const Atoms &A, int nblocks, double *out, cudaStream_t s);
cudaError_t launch_unsort_vec(const Atoms &A, const double4_32a *src, double *dst, cudaStream_t s);
cudaError_t launch_unsort_scalar(const Atoms &A, const double *src, double *dst, cudaStream_t s);
cudaError_t launch_unsort_image(const Atoms &A, double *dst, cudaStream_t s);
cudaError_t launch_unsort_int(const Atoms &A, const int32_t *src, int32_t *dst, cudaStream_t s);
cudaError_t launch_unsort_list(const Atoms &A, int32_t *dst, cudaStream_t s);
cudaError_t launch_sort_in_vec(const Atoms &A, const double *src, double4_32a *dst, cudaStream_t s);
// The same for caller buffers in mapped pinned host memory (device pointers of them), read or
// written in caller order by the device over the host link: no separate copy.
cudaError_t launch_sort_in_mapped(const Atoms &A, const double *src, double4_32a *dst, cudaStream_t s);
cudaError_t launch_unsort_mapped(const Atoms &A, const double4_32a *src, double *dst, cudaStream_t s);
cudaError_t launch_replica_sums(const Atoms &A, const int32_t *off, int n_rep, double *out, cudaStream_t s);

// Nose-Hoover thermostat of one replica (md_set_thermostat; §2.1.2).
struct Thermo {
    double pi, xi;          // friction (1/fs) and its time integral
    double q, gkt;          // thermal inertia Q (eV fs^2); g k_B T (eV), g = 3 N_r - 3
    double s_b, s_a;        // velocity scale factors of the half steps after / before a VV step
    unsigned long long ke_fix;  // kinetic energy accumulator in units of 2^-40 eV
    unsigned long long pad;
};
constexpr double kKeFix = 1099511627776.0;   // 2^40
constexpr int kKeChunk = 1024;               // atoms per chunk of the kinetic-energy sums

// Persistent step kernel (md_step.cu): n_steps velocity-Verlet steps in one cooperative
// launch; grid barriers between phases; per-phase %globaltimer stamps when stamps != NULL.
struct StepParams {
    int n_steps;
    int energy_last;      // FP64 partial sums on the last step
    double half_dt, dt, strain_scale, lim2;
    int rebuild_every;    // scheduled rebuild period (0: none)
    double rl2;
    float band_lo, band_hi;
    int list_group;       // lanes per link cell in the list build (4, 8, 16 or 32)
    Thermo *thermo;       // [n_rep] Nose-Hoover state, or NULL (NVE)
    const int2 *ke_chunks;  // (replica, first atom) of each chunk of <= kKeChunk atoms
    int n_ke_chunks;
    const int32_t *rep_off;  // [n_rep + 1]
    unsigned long long spin_limit;
    int withhold_arrival;  // self-test of the bounded waits: 1, block 0 skips its first grid-barrier
                           // arrival; 2 (group walks), block 0's staging producer releases no group
    int motion;            // kMotionVerlet or kMotionPC3: what the force pass does to each atom after
                           // its force (second half kick, or the corrector) and what opens a step
                           // (half kick + drift, or the predictor)
    int stop_at_rebuild;   // 1: at a step that needs a list rebuild, record the step in Flags::seg_done
                           // and end the launch (the rebuild kernel follows, then a resuming launch)
    int resume;            // 1: continue the md_step call at step Flags::seg_done (already opened: no
                           // prologue); nothing to do when that is n_steps
};
// With sp.n_steps == 0 it only prepares the launch (function attributes, occupancy query):
// done before a stream capture, so that a captured launch makes no other API call.
cudaError_t launch_step(const Atoms &A, const Cells &C, const Pot &P, int precision, int lanes,
                        const StepParams &sp, GridBarrier *bar, unsigned long long *stamps, int *grid_out,
                        cudaStream_t s);
int step_grid(const Pot &P, int precision, int lanes);   // blocks of the persistent launch
// The neighbour walk (kWalk*) of the step kernel launch_step runs for these arguments.
int step_walk(const Atoms &A, const Cells &C, const Pot &P, int precision, int lanes);
// The list rebuild of an md_step call between two launches of the step kernel: a cooperative
// kernel of its own (more warps per SM than the step kernel keeps), which does nothing unless
// the last launch stopped at a rebuild request (Flags::seg_done < sp.n_steps, need_rebuild set).
cudaError_t launch_rebuild_step(const Atoms &A, const Cells &C, const Pot &P, int precision, int lanes,
                                const StepParams &sp, GridBarrier *bar, unsigned long long *stamps, cudaStream_t s);

// ---------------------------------------------------------------- learned surrogate
// Per-atom energy E_i = f(x_i) of standardised radial-basis descriptors x_ik = (G_ik - gmu_k) ginv_k,
// G_ik = sum_j b_k(r_ij), b_k(r) = exp(-(r - mu_k)^2 / (2 w^2)) (cos(pi r / rd) + 1) / 2 for r < rd;
// f is a 32-64-64-1 SiLU network with parameters theta, packed W1 [64][32], b1, W2 [64][64], b2,
// w3 [64], b3.  The input gradient kept per atom is the one with respect to G (dE_i/dx_i * ginv).
constexpr int kSurNb = 32, kSurH1 = 64, kSurH2 = 64;
constexpr int kSurParams = kSurH1 * kSurNb + kSurH1 + kSurH2 * kSurH1 + kSurH2 + kSurH2 + 1;  // 6337
constexpr int kSurTile = 128;                      // atoms per tensor-core tile
constexpr int kSurTileBytes = kSurTile * kSurNb * 2;  // bf16 descriptor tile, core-matrix layout
// bf16 operand image of the tensor-core network, each matrix N x K in the no-swizzle
// K-major core-matrix layout: W1 (64 x 32), W2 (64 x 64), W2^T (64 x 64), W1^T (32 x 64)
constexpr int kSurImgW1 = 0, kSurImgW2 = 4096, kSurImgW2T = 12288, kSurImgW1T = 20480, kSurImgBytes = 24576;

struct SurNet {
    float mu0, dmu, inv2w2, invw2, rd, rd2, pi_rd;
    int bf16;                 // 1: tensor-core BF16 network, 0: FP32 network
    const float *theta;       // [kSurParams] parameters (FP32 master)
    const float *gmu, *ginv;  // [kSurNb] input standardisation
    const unsigned char *img; // [kSurImgBytes] bf16 operands (from theta)
    unsigned char *Gt;        // bf16 descriptor tiles [ceil(n/128)][kSurTileBytes]
    float *G;                 // FP32 descriptors [n][32] (FP32 network and training)
    float *g;                 // dE_i/dG_i [n][32]
    float4 *phi;              // training: dL/dF_i
    float *u;                 // training: [n][32]
    const double4_32a *fref;  // training: reference forces (cell order)
    double *eref;             // training: reference energies [n_rep]
    double *ce;               // training: per replica [2 r] = dL/dE_i, [2 r + 1] = its energy-loss term
    float *gpart;             // training: per-block parameter gradients [blocks][kSurParams]
};

// Surrogate launchers (md_sur_*.cu).  Atom ranges [a0, a1) are contiguous replicas.
cudaError_t launch_sur_kick_drift(const Atoms &A, double half_dt, double dt, double lim2, cudaStream_t s);
cudaError_t launch_sur_descriptors(const Atoms &A, const SurNet &S, int a0, int a1, cudaStream_t s);
cudaError_t launch_sur_net32(const Atoms &A, const SurNet &S, int a0, int a1, cudaStream_t s);
cudaError_t launch_sur_net_tc(const Atoms &A, const SurNet &S, cudaStream_t s);
cudaError_t launch_sur_force(const Atoms &A, const SurNet &S, int a0, int a1, bool kick, bool energy,
                             double half_dt, double phi_scale, int *rows_out, cudaStream_t s);
cudaError_t launch_sur_frame_terms(const Atoms &A, const SurNet &S, const int32_t *rep_off, int r0, int r1,
                                   double w_e, cudaStream_t s);
cudaError_t launch_sur_u(const Atoms &A, const SurNet &S, int a0, int a1, cudaStream_t s);
cudaError_t launch_sur_train_tiles(const Atoms &A, const SurNet &S, int a0, int a1, int *blocks_out,
                                   cudaStream_t s);
cudaError_t launch_sur_update(const SurNet &S, float *theta, float *adam_m, float *adam_v, float *grad_out,
                              int blocks, int t, float lr, cudaStream_t s);
cudaError_t launch_sur_pack(const float *theta, unsigned char *img, cudaStream_t s);
cudaError_t launch_sur_stats(const Atoms &A, const SurNet &S, double *part, int blocks, cudaStream_t s);
cudaError_t launch_sur_unsort_rows(const Atoms &A, const float *src, float *dst, cudaStream_t s);
int sur_net32_blocks(int n_atoms);
int sur_force_blocks(int n_atoms);

inline int blocks_for(long long n, int threads) { return (int)((n + threads - 1) / threads); }

}  // namespace mdk
