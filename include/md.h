/*
 * md.h - C ABI of the GB300 EAM hot-path library (libmd.so).
 *
 * The operation is the force calculation and time step of the MOLDY method
 * (Ackland et al., "The MOLDY short-range molecular dynamics package"):
 *   - link-cell binning and a Verlet neighbour list with padding (§3.2.1);
 *   - the two sums of Eq. (1): the host density rho_i = sum_j phi(r_ij) with
 *     F(rho_i), F'(rho_i), then the pair + embedding forces (§2, §3.1);
 *   - velocity-Verlet integration (§2.3) in the units of §2.7.
 * The force sums use the symmetric (full) neighbour list of §3.2.2, each atom
 * gathering its own sum, so no two threads write the same atom.
 *
 * Conventions shared by every entry point
 *   - Units (§2.7): lengths Å, masses amu, energies eV, time fs, velocities Å/fs,
 *     forces eV/Å, temperature K, pressure GPa.
 *   - Per-atom arrays are in the caller's atom order (index = atom id given at
 *     md_create), row-major [N][3] doubles for vectors.
 *   - `on_device` = 0: the pointer is host memory (pageable or pinned);
 *     1: it is CUDA device memory of the current device (e.g. a torch tensor).
 *   - Ownership: the caller owns every array it passes; the library copies what it
 *     needs before returning (inputs) or writes into the caller's array (outputs).
 *     The library owns its own device buffers (cells, lists, sorted state).
 *   - Work is issued on md_config.stream (a cudaStream_t; NULL = legacy default
 *     stream).  Every entry point that returns data synchronises that stream.
 *   - Errors: every call returns an md_status; no exception crosses the ABI.  The
 *     text of the last error of a context is kept until the next failing call and
 *     is read with md_last_error.  Conditions found on the device (list overflow,
 *     non-finite forces, table range) are reported by the next call that
 *     synchronises (md_step, md_eam_forces, md_build_neighbours, md_energy).
 *   - One context is used by one host thread at a time.
 */
#ifndef MD_H
#define MD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MD_ABI_VERSION 6

typedef struct md_ctx md_ctx; /* opaque, owned by the library */

typedef enum {
    MD_OK = 0,
    MD_ERR_ARG = 1,          /* bad argument (NULL pointer, size, unsupported option) */
    MD_ERR_SPECIES = 2,      /* species index out of range: the paper halts before the run
                                when the potential cannot handle a species (§3.1) */
    MD_ERR_BOX = 3,          /* box not orthorhombic, or an edge holds < 3 link cells */
    MD_ERR_NBR_OVERFLOW = 4, /* an atom has more than k_max neighbours (Table 1 `nnbrs`) */
    MD_ERR_SKIN = 5,         /* strict mode: an atom moved more than skin/2 since the build */
    MD_ERR_NONFINITE = 6,    /* NaN or Inf in positions or forces */
    MD_ERR_TABLE_RANGE = 7,  /* (reserved) strict table range mode */
    MD_ERR_TIMEOUT = 8,      /* a bounded device-side wait gave up */
    MD_ERR_CUDA = 9,         /* CUDA runtime error (text in md_last_error) */
    MD_ERR_OOM = 10,         /* device allocation failed */
    MD_ERR_STATE = 11,       /* call not valid in the context's state */
    MD_ERR_CAPACITY = 12     /* input larger than a fixed capacity (md_neighbours_noalloc) */
} md_status;

enum { MD_POT_FS_ANALYTIC = 1, MD_POT_TABLES = 2, MD_POT_SURROGATE = 3, MD_POT_KNOTS = 4 };
enum { MD_PREC_FP64 = 0, MD_PREC_MIXED = 1, MD_PREC_DF = 2 };

/*
 * The potential as data (the paper's potential interface, §3.1: V, phi, F and their
 * derivatives per species; the range from get_supported_potential_range).
 *   kind MD_POT_FS_ANALYTIC: one species, Finnis-Sinclair form with
 *     fs = {d, c, A, beta, c0, c1, c2}:
 *       phi(r) = (r-d)^2 + beta (r-d)^3 / d  (r < d),
 *       V(r)   = (r-c)^2 (c0 + c1 r + c2 r^2)  (r < c),   F(rho) = -A sqrt(rho);
 *     r_cut must be >= max(c, d).
 *   kind MD_POT_TABLES: n_species species, knot tables.  `tables` holds
 *     (2 ns^2 + ns) tables of 2*n_knots doubles each (n_knots values, then n_knots
 *     slopes at uniform knots): V[a][b] (a, b < ns; V[a][b] must equal V[b][a]),
 *     phi[a][b] = density at an atom of species a due to a neighbour of species b
 *     (EAM/FS asymmetric form, §2 and §3.1), F[a].  r-tables span [r_min, r_cut],
 *     F-tables span [rho_min, rho_max].  Each interval is the cubic Hermite
 *     polynomial through the end values and slopes; outside the span the table
 *     continues linearly from the end knot and the event is counted
 *     (md_energies.range_violations).
 *   kind MD_POT_KNOTS: n_species species, explicit cubic knot sums (the generic potential
 *     files of §3.1.1): V_ab and phi_ab = sum_k c_k (r_k - r)^3 for r < r_k, evaluated term by
 *     term (no table), F_a = -A_a sqrt(rho).  n_knots = K terms per function (pad with c = 0);
 *     `tables` holds the 2 ns^2 functions V[a][b] (V[a][b] must equal V[b][a]) then phi[a][b],
 *     each K coefficients then K radii r_k <= r_cut, then A[a] (ns values); ns <= 8, K <= 32.
 *   kind MD_POT_SURROGATE: the learned per-atom surrogate (md_set_surrogate); one
 *     species (n_species 1, species 0), r_cut = the descriptor cutoff rd; fs, n_knots,
 *     r_min, rho_min, rho_max and tables are ignored.
 * The library copies the tables at md_create.
 */
typedef struct {
    int32_t kind;
    int32_t n_species;
    const int32_t *atomic_numbers; /* [n_species], informational */
    const double *masses_amu;      /* [n_species] */
    double fs[7];
    int32_t n_knots;
    double r_min, r_cut; /* potential range (§3.1 get_supported_potential_range) */
    double rho_min, rho_max;
    const double *tables;
} md_potential;

/*
 * Run configuration (the fields of the paper's parameter file that the hot path
 * uses, Table 1).
 */
typedef struct {
    int64_t n_atoms;
    double h[9];           /* box matrix [a; b; c] rows in Å; must be diagonal (orthorhombic) */
    double skin;           /* `rpad`: list radius = r_cut + skin (§3.2.1) */
    int32_t k_max;         /* `nnbrs`: list capacity per atom */
    int32_t rebuild_every; /* `nbrupdate`: rebuild every n steps; 0 = only when needed */
    double dt_fs;          /* `deltat` */
    int32_t precision;     /* MD_PREC_FP64 (every sum, the integration and the reductions in
                              FP64; of the pair terms, 1/r and, in the half list's density
                              pass, r^2 are formed to FP64 accuracy from exact FP32 pieces,
                              relative error <= 4e-13, the rest is FP64 arithmetic), or
                              MD_PREC_MIXED (FP32 pair/density terms,
                              FP64 positions, velocities, density sum and reductions; with
                              one species and knot tables the force pass takes the quadratic
                              and cubic coefficients of each table cubic's derivative as
                              binary16, scaled per function by a power of two), or MD_PREC_DF
                              (one species, knot tables: the pair and density terms in
                              double-float arithmetic, each quantity the unevaluated sum of two
                              FP32 numbers, 48-bit significand, on the FP32 pipes; coordinates
                              offset so that their FP32 high parts subtract exactly; positions,
                              velocities, F(rho) and reductions FP64; results within 1e-11 of
                              the FP64 ones for boxes of a few hundred Å) */
    int32_t strict_skin;   /* 1: moving > skin/2 between scheduled rebuilds is MD_ERR_SKIN;
                              0: it triggers a rebuild */
    double strain_rate_zz; /* 1/s; each step the box z edge and all z coordinates are
                              multiplied by (1 + rate*dt) (§2.2 strain-rate loading) */
    void *stream;          /* cudaStream_t, or NULL */
    int32_t lanes_per_atom; /* threads sharing one atom's neighbour sums in the force passes:
                               1, 2, 4, 8, 16 or 32, or 0 = chosen from the expected neighbour
                               count (see md_tune).  Results depend on it only in rounding. */
    int32_t passes;         /* MD_PASSES_AUTO (0), MD_PASSES_LIST, MD_PASSES_STAGED, MD_PASSES_CELLS or
                               MD_PASSES_HALF: how the mixed-precision step kernel walks the neighbours */
    int32_t integrator;     /* MD_INTEGRATOR_VERLET (0) or MD_INTEGRATOR_PC3 (Table 1 `iverlet`: 1 and 0
                               respectively; see below) */
} md_config;

/*
 * Time integrator of md_step (§2.3: the paper offers two).
 *   VERLET: velocity Verlet (time reversible, bounded energy error in NVE).
 *   PC3: the third-order predictor-corrector (after Gear) for r'' = F/m on the scaled Taylor
 *     vector (r, dt v, (dt^2/2) a, (dt^3/6) b), b = da/dt: predict by the Taylor series to third
 *     order, evaluate the forces once at the predicted positions, then correct every term by
 *     c_k D with D = (dt^2/2) F/m - (the predicted acceleration term) and c = (1/6, 5/6, 1, 1/3).
 *     After md_step the forces (md_get) and the potential energy (md_energy) are those of the last
 *     predicted positions, the positions and velocities the corrected ones.  The third-derivative
 *     term is kept per atom between md_step calls; it starts at zero at md_create and is set to
 *     zero by md_set_state (and md_step_io, which calls it): the predictor restarts.  The
 *     acceleration term comes from the stored forces at each md_step, so an md_eam_forces call
 *     between steps restarts it from the forces at the current positions.  PC3 takes the list
 *     walk (or the FP64 half list) and no strain ramp, thermostat or surrogate (MD_ERR_ARG at
 *     md_create, MD_ERR_STATE at md_set_thermostat).
 */
enum { MD_INTEGRATOR_VERLET = 0, MD_INTEGRATOR_PC3 = 1 };

/*
 * Neighbour walk of the two EAM passes in the step kernel (md_step).  LIST: every atom reads
 * its neighbours' positions through the full Verlet list (§3.2.1) from global memory, and every
 * pair is computed twice (once for each atom: no write conflicts, the symmetric scheme of
 * §3.2.2).  The three group walks take the link cells in groups of consecutive cells along x;
 * a group's neighbourhood (the 3 x 3 x (gx + 2) stencil of cells around it, each periodic image
 * already shifted) is copied into shared memory and walked there.  In each 1024-thread block one
 * warp stages the block's next groups with bulk copies into 2 to 4 buffers while the other 31
 * warps compute the current ones, claiming work a warp at a time; the shared copy of the knot
 * table then holds only the rows of the pass under way:
 *  - STAGED: the group's atoms read their neighbours through a 16-bit copy of their list rows
 *    (the same entries, as stencil slots).  The list, the pair terms and their order are those
 *    of LIST; the separations are formed from the shifted FP32 positions instead of by the FP32
 *    minimum image, so results differ from LIST in rounding only.
 *  - CELLS: no Verlet list: each atom tests every staged atom of the 27 cells around its own
 *    (the link-cell method alone, §3.2.1), so a rebuild re-bins the atoms and builds no list;
 *    pairs closer than r_cut are the same set, summed in another order.  After md_step a CELLS
 *    context's list is rebuilt when it is next needed (md_eam_forces, md_get of the list).
 *  - HALF: a half list and Newton's third law (§3.2.2's half list): each pair is computed once,
 *    by the atom with the lower cell-order slot, through 16-bit half rows of stage slots.  The
 *    other atom's density, force and pair energy are summed in shared memory per stage slot,
 *    then added to FP64 accumulators with atomic adds, so that sums are exact to FP32 rounding
 *    per term but their order, and hence the last bits, varies from run to run.  Two light
 *    phases follow the passes: F(rho) after the density pass, the kicks after the force pass.
 * The group walks apply to mixed precision, one system (no batch), one species with a knot
 * table that fits in shared memory, no strain ramp, and 1-8 lanes per atom (more lanes walk
 * LIST); a build at which some group's neighbourhood exceeds the stage's capacity makes the
 * passes take the LIST walk until the next build (CELLS then builds the list).
 * On the FP64 path HALF is the half list over the full list instead (one species, FS analytic or
 * knot tables, k_max <= 256; batches, strain, thermostat and both integrators allowed): each build
 * reorders every row so that its entries j > i (cell order) come first, each pass computes every
 * pair once from those entries and adds the neighbour's share of rho, force and pair energy to
 * FP64 accumulators with atomic adds, and F(rho) and the kick follow in phases of their own.
 * Results agree with LIST's to about 1e-12 (relative; r^2 in its density pass comes from FP32
 * pieces, see `precision`); the order of the atomic adds, and so the last bits, varies from run
 * to run.  AUTO = LIST (on GB300, fcc Cu 500,000 atoms with its 5,000-knot
 * table: LIST 0.58 ms per step, STAGED 0.67, HALF 1.40, CELLS 2.75; STAGED's passes take about
 * as long as LIST's, its list build longer); a group walk where it does not apply is MD_ERR_ARG
 * at md_create.
 */
enum { MD_PASSES_AUTO = 0, MD_PASSES_LIST = 1, MD_PASSES_STAGED = 2, MD_PASSES_CELLS = 3, MD_PASSES_HALF = 4 };

typedef struct {
    int32_t walk;            /* the walk prepared: MD_PASSES_STAGED, MD_PASSES_CELLS or
                                MD_PASSES_HALF (cell groups at every build), else MD_PASSES_LIST */
    int32_t cells_per_group; /* gx */
    int32_t groups;          /* number of cell groups */
    int32_t capacity;        /* atoms one stage buffer holds */
    int32_t last_max;        /* largest group neighbourhood (atoms) at the last list build */
    int32_t active;          /* 1: the next md_step takes the prepared group walk (lanes <= 8, and
                                every group fitted at the last build) */
    int32_t stage_buffers;   /* stage buffers per block (2 to 4; 1 where a group fits only once):
                                the next groups are staged by bulk copies while one is computed */
} md_passes;

typedef struct {
    double pe, ke, te;    /* potential (Eq. 1), kinetic, total energy, eV */
    double temperature;   /* 2 KE / ((3N-3) k_B), K (§2.1.2) */
    double virial[9];     /* W = sum over pairs of r_ij (x) f_ij, eV, row-major */
    double pressure_gpa;  /* (2 KE + tr W) / (3 V) */
    double momentum[3];   /* total momentum, amu Å/fs */
    double volume;        /* Å^3 */
    double box[3];        /* current box edges, Å */
    int64_t step;         /* steps taken since md_create */
    int64_t n_rebuilds;   /* neighbour-list builds so far */
    int32_t max_neighbours;    /* longest list at the last build */
    int32_t pad;
    int64_t range_violations;  /* table lookups outside their span so far */
} md_energies;

/* md_get selectors */
enum {
    MD_GET_POS = 0,       /* double [N][3], unwrapped (§2.2) */
    MD_GET_VEL = 1,       /* double [N][3] */
    MD_GET_FORCE = 2,     /* double [N][3] at the current positions */
    MD_GET_RHO = 3,       /* double [N]: rho_i */
    MD_GET_EATOM = 4,     /* double [N]: F(rho_i) + 1/2 sum_j V(r_ij), the energy of an atom (§2) */
    MD_GET_DF = 5,        /* double [N]: F'(rho_i) */
    MD_GET_NBR_COUNT = 6, /* int32 [N]: neighbours of each atom (may exceed k_max on overflow) */
    MD_GET_NBR_LIST = 7,  /* int32 [N][k_max]: neighbour atom ids, unused slots -1, order unspecified */
    MD_GET_SPECIES = 8,   /* int32 [N] */
    MD_GET_IMAGE = 9      /* double [N][3]: the coordinates the force passes take, in the periodic
                             image of the last list build (wrapped into the box at the build and
                             followed continuously since): the FP32 copy of the mixed path converted
                             exactly to double, or the FP64 copy of the FP64 path (§2.2) */
};

/* Library ABI version (MD_ABI_VERSION). */
int32_t md_abi_version(void);

/* Short text for a status code (static storage). */
const char *md_status_string(md_status s);

/*
 * Create a context: copy the potential, the atoms' positions `pos` [N][3] (Å,
 * unwrapped), velocities `vel` [N][3] (Å/fs; NULL = zero) and species indices
 * `species` [N] (NULL = all 0), allocate the device buffers, and check the box
 * (orthorhombic, >= 3 link cells of width >= r_cut + skin per edge) and the
 * species (§3.1: halt before the run on an unsupported species).
 * On failure *out is NULL and the status says why.
 */
md_status md_create(const md_config *cfg, const md_potential *pot, const double *pos,
                    const double *vel, const int32_t *species, int32_t on_device, md_ctx **out);

/*
 * Create one context for a batch of n_replicas independent systems (the paper's use of many
 * runs for statistics, §2.6): replica r has cfgs[r].n_atoms atoms with positions pos[r],
 * velocities vel[r] (vel or vel[r] may be NULL) and species species[r] (may be NULL), in the
 * orthorhombic box cfgs[r].h.  The run settings (skin, k_max, dt_fs, precision,
 * rebuild_every, strain_rate_zz) must be equal in all cfgs; stream, strict_skin and
 * lanes_per_atom are taken from cfgs[0].  All replicas share the potential.  In the other
 * entry points a batch behaves as one system whose atoms are the replicas' atoms in order
 * (replica 0 first); md_step advances every replica in one launch; md_energy returns the
 * batch totals (temperature with 3N - 3 n_replicas degrees of freedom) and
 * md_replica_energies the values of each replica.  A list rebuild, when any replica needs
 * one, rebuilds every replica.
 */
md_status md_create_batch(int32_t n_replicas, const md_config *cfgs, const md_potential *pot,
                          const double *const *pos, const double *const *vel, const int32_t *const *species,
                          int32_t on_device, md_ctx **out);

/* Per-replica microstate values of the current state into out[n_replicas] (PE, KE, TE,
 * T with 3n - 3 degrees of freedom, momentum, box, volume; pressure_gpa is NaN: the virial
 * is reduced over the whole batch only).  A single system counts as one replica. */
md_status md_replica_energies(md_ctx *ctx, md_energies *out);

/* Bin the atoms into link cells (counting sort by cell, atoms renumbered in
 * cell order with a stable tie-break on atom id) and build the full Verlet list:
 * j is listed for i iff j != i and |r_ij|^2 < (r_cut + skin)^2 with the minimum
 * image (§2.2, §3.2.1).  Returns MD_ERR_NBR_OVERFLOW if an atom has > k_max. */
md_status md_build_neighbours(md_ctx *ctx);

/* Forces, per-atom density and energies at the current positions (pass 1 and
 * pass 2 of Eq. (1)); rebuilds the list first if it is missing or stale.  If
 * pe_out is not NULL it receives the total potential energy (FP64 sum). */
md_status md_eam_forces(md_ctx *ctx, double *pe_out);

/* Advance n_steps velocity-Verlet steps (§2.3): half kick, drift, [strain],
 * [list rebuild when scheduled or when an atom moved > skin/2], density pass,
 * force pass, half kick.  All n_steps run in ONE cooperative launch of a persistent
 * kernel (grid barriers between the phases, each wait bounded: a wait that gives up
 * returns MD_ERR_TIMEOUT).  FP64 contexts of at least 32,768 atoms run the call in
 * segments instead: the persistent launch stops at a step that needs a list rebuild, a
 * cooperative rebuild kernel with more warps per SM rebuilds, and a launch resumes at that
 * step (a few such segments are enqueued per call, from the rebuild interval seen so far;
 * rebuilds beyond them run inside the last launch).  Results are the same either way.
 * Energies of the final state are then available from md_energy.  Synchronises the stream
 * once, at the end. */
md_status md_step(md_ctx *ctx, int32_t n_steps);

/* Self-test of failure detection: runs one step in which one block of the persistent
 * kernel withholds its first barrier arrival, so the other blocks' bounded wait runs out
 * (about a millisecond of polling); every block then returns and the call reports
 * MD_ERR_TIMEOUT with no fault.  When the step kernel stages cell groups (MD_PASSES_STAGED,
 * CELLS or HALF, every group fitting), block 0's staging producer releases no group instead,
 * so that its consumers' bounded mbarrier waits run out.  Afterwards the state is not a clean
 * step boundary (positions have been drifted once); the next call recomputes forces. */
md_status md_selftest_timeout(md_ctx *ctx);

/* Graph mode (on = 1): md_step(n) records its device work for this n (the persistent
 * launch, the reduction, the copies back) as a CUDA graph the first time and replays the
 * graph afterwards.  Not used while profiling or under a strain ramp; on = 0 frees the
 * graphs.  md_tune or a change of link cells discards them. */
md_status md_set_graph(md_ctx *ctx, int32_t on);

/* Microstate thermodynamics of the current state (§2.1.2, §2.6), reduced in FP64
 * in a fixed order (bitwise reproducible). */
md_status md_energy(md_ctx *ctx, md_energies *out);

/* Copy one per-atom array (see MD_GET_*) into `dst` (caller's atom order). */
md_status md_get(md_ctx *ctx, int32_t what, void *dst, int32_t on_device);

/* Replace positions and velocities (caller's atom order); `force` may be NULL
 * (forces are then recomputed before the next step) or the forces at `pos`
 * (e.g. from a checkpoint, §4.1.3).  Any NULL of pos/vel keeps that array. */
md_status md_set_state(md_ctx *ctx, const double *pos, const double *vel, const double *force,
                       int32_t on_device);

/* A state kept by the caller, one call per stretch of steps: md_set_state(pos_in, vel_in,
 * force_in), md_step(n_steps), then md_get of positions, velocities and forces into pos_out,
 * vel_out, force_out and md_energy into *energies, with the copies and kernels in stream order
 * and the stream synchronised once (at the end).  Every argument but ctx may be NULL (that copy
 * is skipped); inputs and outputs may be the same buffers.  Results are bitwise those of the
 * separate calls.  Host buffers are best pinned (page-locked): the device then reads and writes
 * them itself over the host link, in caller order, inside the kernels that reorder the state
 * (no copy through a device stage); pageable buffers are copied through a device stage.  The
 * same holds for md_set_state's inputs.  on_device as for md_get. */
md_status md_step_io(md_ctx *ctx, int32_t n_steps, const double *pos_in, const double *vel_in,
                     const double *force_in, double *pos_out, double *vel_out, double *force_out,
                     md_energies *energies, int32_t on_device);

/* Autotuner: time 3 velocity-Verlet steps of the persistent step kernel from the current state
 * with each lanes_per_atom in {1, 2, 4, 8, 16, 32} (CUDA events; the trial steps rebuild no
 * list, and positions, velocities, forces and counters are put back after each), keep the
 * fastest for this context and return it in *lanes_out (nullable).  Computes the forces first
 * if needed.  Because the lane count fixes the summation order, results after md_tune are
 * reproducible but may differ in the last bits from those before it. */
md_status md_tune(md_ctx *ctx, int32_t *lanes_out);

/* Kernel timing of a context (tracing).  `launches` counts every kernel the context has
 * enqueued since md_create.  While profiling is on, the step kernel stamps the GPU clock
 * (%globaltimer) at each phase boundary and md_step adds the phase durations here (ms):
 * kick = the first half kick + drift of each md_step call (later ones are fused into the
 * force phase), rebuild = the list rebuild phases (0 when none is due), density and force
 * per step; the counts are the numbers of timed phases. */
typedef struct {
    int64_t launches;
    int64_t n_kick, n_rebuild, n_density, n_force;
    double ms_kick, ms_rebuild, ms_density, ms_force;
    double ms_rebuild_part[9]; /* bin, tile sums, top scan, apply, scatter, cell sort, gather,
                                  copyback, list build */
} md_profile;

/* Turn per-kernel event timing on (1) or off (0); turning it on clears the sums. */
md_status md_set_profiling(md_ctx *ctx, int32_t on);

/* Read the launch count and the timing sums. */
md_status md_get_profile(const md_ctx *ctx, md_profile *out);

/* The neighbour walk of the context's step kernel (see MD_PASSES_*); synchronises the stream. */
md_status md_get_passes(md_ctx *ctx, md_passes *out);

/*
 * Neighbour list without device allocation.  The paper has no counterpart: this entry
 * point serves callers that cannot allocate device memory - code running inside another
 * framework's memory pool or allocator hooks, or code that must not grow its device
 * footprint once it has started.  It builds the same full list as md_build_neighbours (the
 * same exact FP64 test, minimum image) for positions the caller already holds on the
 * device, and allocates nothing: no cudaMalloc or cudaFree and no allocating library call.
 * Its working memory is one fixed-size __device__ array inside the library (about 5.3 MB),
 * which every GPU that loads the library holds until the process exits.
 *   pos     device, [n_atoms][3] doubles (Å, may be unwrapped)
 *   box     host, the 3 edge lengths of an orthorhombic box (Å)
 *   r_list  list radius (Å): j is listed for i iff j != i and |r_ij|^2 < r_list^2
 *   count   device, [n_atoms] int32, out: neighbours of each atom (may exceed k_max)
 *   list    device, [n_atoms][k_max] int32, out: neighbour atom indices, then -1; the
 *           order inside a row is unspecified
 *   stream  cudaStream_t or NULL; the call synchronises it before returning.
 * The caller owns pos, count and list.  Returns MD_ERR_CAPACITY, launching nothing, if
 * n_atoms > MD_NOALLOC_MAX_ATOMS or the box holds more than MD_NOALLOC_MAX_CELLS link cells
 * of width >= r_list; MD_ERR_BOX if an edge holds fewer than 3 such cells;
 * MD_ERR_NBR_OVERFLOW if a row was cut at k_max; MD_ERR_ARG for bad arguments;
 * MD_ERR_CUDA on a CUDA error.
 * The first call on each device looks up the device address of the array (once per device,
 * with that device current): make that first call before any stream capture.  Every call
 * reuses the same array and leaves its contents there (each call clears what must start
 * at zero), so calls that overlap on the GPU - from two streams or two host threads - race.
 */
#define MD_NOALLOC_MAX_ATOMS 131072
#define MD_NOALLOC_MAX_CELLS 65536
md_status md_neighbours_noalloc(const double *pos, int64_t n_atoms, const double *box, double r_list,
                                int32_t k_max, int32_t *count, int32_t *list, void *stream);

/* Nose-Hoover thermostat (NVTp, §2.1.2), one per replica.  With it on, md_step integrates
 *   dp_i/dt = -dU/dq_i - pi_s p_i,   Q_s dpi_s/dt = sum_i p_i^2/m_i - g k_B T,   dxi/dt = pi_s,
 * g = 3 N - 3 for a replica of N atoms (the kinetic term is read as p^2/m, the standard form whose
 * fixed point is the section's temperature, sum p^2/2m = g k_B T / 2), by a thermostat half step
 * (length dt/2) before and after each velocity-Verlet step:
 *   pi += (dt/4)(2 KE - g kT)/Q;  v *= exp(-pi dt/2);  xi += pi dt/2;  pi += (dt/4)(2 KE' - g kT)/Q
 * (KE' after the scaling).  H' = KE + U + Q pi^2/2 + g k_B T xi is conserved.
 *   on: 1 = thermostat each replica r at t_kelvin[r] (K, > 0) with relaxation time tau_fs[r]
 *       (fs, > 0), starting from pi = xi = 0; the library sets the thermal inertia
 *       Q = g k_B T tau^2 (eV fs^2, read back with md_get_thermostat).  0 = plain NVE (the
 *       thermostat state is kept; t_kelvin and tau_fs may be NULL).  Host arrays of n_replicas,
 *       copied.
 * MD_ERR_ARG for a T or tau that is not positive and finite, or a Q that overflows; MD_ERR_STATE
 * for a surrogate context.  md_energy's te stays KE + U (§2.1: the reported total
 * energy excludes the thermostat's degree of freedom). */
md_status md_set_thermostat(md_ctx *ctx, int32_t on, const double *t_kelvin, const double *tau_fs);

/* Thermostat state per replica into out[n_replicas][4] (host): pi (1/fs), xi, Q (eV fs^2) and
 * the conserved H' (eV). */
md_status md_get_thermostat(md_ctx *ctx, double *out);

/* ------------------------------------------------------------------------------------
 * Learned surrogate of the per-atom energy.  This is an addition to the paper's method,
 * which has no counterpart: the force field of Eq. (1) is replaced by a small network of
 * each atom's neighbour environment, trained on forces and energies of the EAM model.
 *
 *   G_ik = sum_{j: r_ij < rd} b_k(r_ij),  k = 0..31,
 *   b_k(r) = exp(-(r - mu0 - k dmu)^2 / (2 width^2)) (cos(pi r / rd) + 1) / 2,
 *   x_i = (G_i - gmu) * ginv   (per-channel standardisation),
 *   E_i = w3 . s(W2 s(W1 x_i + b1) + b2) + b3,  s(z) = z / (1 + exp(-z)),
 *   U = sum_i E_i,  F_m = -dU/dr_m = sum_j [sum_k (g_mk + g_jk) b_k'(r_mj)] (r_j - r_m)/r_mj,
 *   g_i = dE_i/dG_i.
 * theta packs W1 [64][32], b1 [64], W2 [64][64], b2 [64], w3 [64], b3 (MD_SUR_PARAMS floats).
 * The list radius is r_cut + skin with r_cut = rd.  The forces are central pair forces, so
 * md_energy's virial and pressure keep their meaning.  md_eam_forces and md_step of a
 * MD_POT_SURROGATE context evaluate the surrogate; md_get(MD_GET_EATOM) gives E_i;
 * MD_GET_RHO and MD_GET_DF are not defined for it.
 * Network arithmetic (md_surrogate.net):
 *   MD_SUR_FP32  FP32 on the CUDA cores (the training path);
 *   MD_SUR_BF16  tensor cores (tcgen05): bf16 x and weights, FP32 accumulation, FP32 biases
 *                and activations, rounded to bf16 between layers.
 * Descriptors and gathers are FP32; positions, velocities and reductions FP64.
 */
#define MD_SUR_NB 32
#define MD_SUR_H1 64
#define MD_SUR_H2 64
#define MD_SUR_PARAMS 6337
enum { MD_SUR_FP32 = 0, MD_SUR_BF16 = 1 };
enum { MD_SUR_GET_G = 0, MD_SUR_GET_DEDG = 1 };

typedef struct {
    int32_t nb, h1, h2;  /* must be MD_SUR_NB, MD_SUR_H1, MD_SUR_H2 */
    int32_t net;         /* MD_SUR_FP32 or MD_SUR_BF16 */
    double mu0, dmu;     /* centre of channel k: mu0 + k dmu (Å) */
    double width;        /* Gaussian width (Å) */
    double rd;           /* cutoff (Å); must equal the potential's r_cut */
} md_surrogate;

/* Set the network of a MD_POT_SURROGATE context.  theta: host, MD_SUR_PARAMS floats;
 * gmu, ginv: host, MD_SUR_NB floats each, or NULL for 0 and 1.  Copied.  Resets the
 * optimiser state.  MD_ERR_STATE for another kind of context; MD_ERR_ARG for a bad spec. */
md_status md_set_surrogate(md_ctx *ctx, const md_surrogate *spec, const float *theta, const float *gmu,
                           const float *ginv);

/* Network parameters and standardisation into host arrays (any may be NULL). */
md_status md_sur_get_params(md_ctx *ctx, float *theta, float *gmu, float *ginv);

/* Per-channel mean and 1/standard deviation of G over all atoms at the current positions
 * become the standardisation; the network is re-expressed for it (the same function of G:
 * W1 and b1 change).  Resets the optimiser state. */
md_status md_sur_standardize(md_ctx *ctx);

/* md_sur_get: MD_SUR_GET_G, float [N][32] descriptors G; MD_SUR_GET_DEDG, float [N][32]
 * dE_i/dG_i of the last force evaluation; both in the caller's atom order. */
md_status md_sur_get(md_ctx *ctx, int32_t what, float *dst, int32_t on_device);

/* Training data: reference energies e_ref [n_replicas] (one per replica of a batch context)
 * and reference forces f_ref [N][3] (caller order) at the current positions, which are then
 * fixed (md_step or md_set_state invalidate them: MD_ERR_STATE).  Builds the neighbour
 * list and caches the descriptors of every atom. */
md_status md_sur_set_reference(md_ctx *ctx, const double *e_ref, const double *f_ref, int32_t on_device);

/* Loss over replicas [rep_begin, rep_end) (S replicas, Nb atoms):
 *   L = w_e/S sum_r ((E_r - Eref_r)/N_r)^2 + w_f/(3 Nb) sum_i |F_i - Fref_i|^2,
 * E_r = sum of E_i over replica r; loss[0], loss[1] = the two terms (host).  grad (host,
 * MD_SUR_PARAMS floats, or NULL) = dL/dtheta, from the FP32 network. */
md_status md_sur_loss_grad(md_ctx *ctx, int32_t rep_begin, int32_t rep_end, double w_e, double w_f,
                           double *loss, float *grad);

/* n_iter Adam steps (Kingma & Ba; beta1 0.9, beta2 0.999, eps 1e-8; learning rate lr) on
 * the loss of minibatches of batch_reps consecutive replicas of [rep_begin, rep_end); the
 * minibatch of step t starts at replica rep_begin + batch_reps * (h(seed + t) mod
 * floor((rep_end - rep_begin) / batch_reps)), h = SplitMix64.  loss (host, 2 doubles, or
 * NULL) = the terms of the last minibatch, before its update.  The optimiser state (moments,
 * step count) carries over between calls. */
md_status md_sur_train(md_ctx *ctx, int32_t n_iter, int32_t rep_begin, int32_t rep_end, int32_t batch_reps,
                       double lr, double w_e, double w_f, uint64_t seed, double *loss);

/* Measurement helper (the paper has no counterpart): the FP64 fused multiply-add rate of the
 * current device, from one launch of independent FMA chains (2 flop each) filling every SM,
 * timed with CUDA events on `stream` (cudaStream_t or NULL) after one short warm-up launch.
 * iters = FMA iterations per chain (each thread runs 8 chains).  *tflops = achieved TFLOP/s,
 * *ms (nullable) = the timed launch's duration.  Synchronises the stream.  MD_ERR_ARG for
 * iters < 1 or a NULL tflops; MD_ERR_CUDA on a CUDA error. */
md_status md_measure_fp64_peak(int64_t iters, double *tflops, double *ms, void *stream);

/* Text of the last error of this context ("" if none).  Valid until the next call. */
const char *md_last_error(const md_ctx *ctx);

/* Free the context and its device buffers (NULL is ignored). */
void md_destroy(md_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* MD_H */
