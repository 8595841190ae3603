/*
 * Plain FP64 CPU oracle for the EAM hot path of the MOLDY paper
 * (Ackland et al., "The MOLDY short-range molecular dynamics package").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check and the
 * benchmark's CPU-baseline leg may load or call this library.  It shares no code,
 * header, table or constant with the CUDA library: every formula here is written
 * out from the paper.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp (no FMA contraction, so that the
 * minimum-image distances are the same IEEE operations on every machine).
 *
 * What it computes (paper references by section / equation):
 *   - neighbour sets by brute force over all pairs with the minimum image (§2.2)
 *     and by the hybrid link-cell / neighbour-list method with padding (§3.2.1);
 *   - the cohesive energy of Eq. (1), U = sum_{i<j} V(r_ij) + sum_i F_i(rho_i),
 *     rho_i = sum_j phi_{s_i s_j}(r_ij) (asymmetric phi as in §2 and §3.1),
 *     and the forces F = -grad U, from a full (symmetric) neighbour list (§3.2.2,
 *     "calculate F_ij twice") and, as a cross-check, from the asymmetric half list
 *     with F_ij applied to both atoms (§3.2.2);
 *   - velocity-Verlet time integration (§2.3) in the units of §2.7;
 *   - microstate thermodynamics: KE, T with 3N-3 degrees of freedom (§2.1.2, §2.6),
 *     virial and pressure;
 *   - the strain-rate boundary condition: the box matrix is multiplied by a strain
 *     matrix each step with fractional coordinates fixed (§2.2).
 * Parity: pinned by closed-form lattice energies, finite differences, brute force,
 * Newton's third law and NVE energy conservation (tests/test_oracle_pins.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- units (§2.7): Å, amu, eV; user time in fs.  CODATA 2018. ---- */
#define ORC_AMU_KG 1.66053906660e-27
#define ORC_EV_J 1.602176634e-19
#define ORC_KB 8.617333262e-5 /* eV / K */
/* amu * (Å/fs)^2 in eV */
#define ORC_MVV2E (ORC_AMU_KG * 1.0e10 / ORC_EV_J)
#define ORC_EVA3_TO_GPA (ORC_EV_J * 1.0e30 / 1.0e9)

typedef struct {
    int32_t kind; /* 1: analytic Finnis-Sinclair (one species), 2: knot tables, 4: explicit knot sums */
    int32_t n_species;
    int32_t n_knots;
    int32_t pad;
    double fs[7]; /* d, c, A, beta, c0, c1, c2 */
    double r_min, r_cut, rho_min, rho_max;
    const double *tables; /* V[a][b], phi[a][b], F[a]; each n values then n slopes */
} orc_potential;

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------- */
/* Minimum image (§2.2): r_ij is the shortest vector from i to j or any of its
 * periodic images.  Orthorhombic box of lengths L: d - L*rint(d/L), with d/L
 * taken as d*(1/L).  Every operation separately rounded.                    */
static double orc_min_image(double d, double L, double invL) {
    return d - L * rint(d * invL);
}

static double orc_dist2(const double *pos, int64_t i, int64_t j, const double *L,
                        const double *invL, double *dv) {
    double dx = orc_min_image(pos[3 * j + 0] - pos[3 * i + 0], L[0], invL[0]);
    double dy = orc_min_image(pos[3 * j + 1] - pos[3 * i + 1], L[1], invL[1]);
    double dz = orc_min_image(pos[3 * j + 2] - pos[3 * i + 2], L[2], invL[2]);
    if (dv) { dv[0] = dx; dv[1] = dy; dv[2] = dz; }
    return (dx * dx + dy * dy) + dz * dz;
}

/* ------------------------------------------------------------------------- */
/* Neighbour sets.  j is a neighbour of i iff j != i and |r_ij|^2 < r_list^2,
 * r_list = potential range + padding (§3.2.1, Table 1 `rpad`).  The list is the
 * symmetric (full) one; each row is in ascending j.  Returns the largest count
 * (rows longer than k_max are truncated; the caller compares with k_max).     */
int32_t orc_neighbours_brute(int64_t n, const double *pos, const double *box, double r_list,
                             int32_t k_max, int32_t *count, int32_t *list) {
    double L[3] = {box[0], box[1], box[2]};
    double invL[3] = {1.0 / box[0], 1.0 / box[1], 1.0 / box[2]};
    double rl2 = r_list * r_list;
    int32_t maxc = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(max : maxc)
    for (int64_t i = 0; i < n; i++) {
        int32_t c = 0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            if (orc_dist2(pos, i, j, L, invL, NULL) < rl2) {
                if (c < k_max) list[i * k_max + c] = (int32_t)j;
                c++;
            }
        }
        count[i] = c;
        if (c > maxc) maxc = c;
    }
    return maxc;
}

static int orc_cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Hybrid link-cell / neighbour list (§3.2.1): link cells are fixed in fractional
 * coordinates, at least r_list wide; an atom's candidates are the atoms of its own
 * and the 26 adjacent cells.  Returns -1 if a box edge holds fewer than 3 cells.  */
int32_t orc_neighbours_cells(int64_t n, const double *pos, const double *box, double r_list,
                             int32_t k_max, int32_t *count, int32_t *list) {
    double L[3] = {box[0], box[1], box[2]};
    double invL[3] = {1.0 / box[0], 1.0 / box[1], 1.0 / box[2]};
    int nc[3];
    for (int k = 0; k < 3; k++) {
        nc[k] = (int)floor(L[k] / r_list);
        if (nc[k] < 3) return -1;
    }
    int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    int64_t *head = (int64_t *)malloc(sizeof(int64_t) * (ncell + 1));
    int64_t *cell_of = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    int64_t *members = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    memset(head, 0, sizeof(int64_t) * (ncell + 1));
    for (int64_t i = 0; i < n; i++) {
        int c[3];
        for (int k = 0; k < 3; k++) {
            double s = pos[3 * i + k] * invL[k];
            s = s - floor(s); /* wrapped fractional coordinate */
            c[k] = (int)(s * nc[k]);
            if (c[k] >= nc[k]) c[k] = nc[k] - 1;
            if (c[k] < 0) c[k] = 0;
        }
        cell_of[i] = ((int64_t)c[2] * nc[1] + c[1]) * nc[0] + c[0];
        head[cell_of[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; c++) head[c + 1] += head[c];
    {
        int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (ncell > 0 ? ncell : 1));
        memcpy(fill, head, sizeof(int64_t) * ncell);
        for (int64_t i = 0; i < n; i++) members[fill[cell_of[i]]++] = i; /* ascending i per cell */
        free(fill);
    }
    double rl2 = r_list * r_list;
    int32_t maxc = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(max : maxc)
    for (int64_t i = 0; i < n; i++) {
        int64_t ci = cell_of[i];
        int cx = (int)(ci % nc[0]), cy = (int)((ci / nc[0]) % nc[1]), cz = (int)(ci / ((int64_t)nc[0] * nc[1]));
        int32_t c = 0;
        for (int dz = -1; dz <= 1; dz++)
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    int x = (cx + dx + nc[0]) % nc[0], y = (cy + dy + nc[1]) % nc[1], z = (cz + dz + nc[2]) % nc[2];
                    int64_t cc = ((int64_t)z * nc[1] + y) * nc[0] + x;
                    for (int64_t m = head[cc]; m < head[cc + 1]; m++) {
                        int64_t j = members[m];
                        if (j == i) continue;
                        if (orc_dist2(pos, i, j, L, invL, NULL) < rl2) {
                            if (c < k_max) list[i * k_max + c] = (int32_t)j;
                            c++;
                        }
                    }
                }
        count[i] = c;
        if (c > maxc) maxc = c;
        qsort(list + i * k_max, (size_t)(c < k_max ? c : k_max), sizeof(int32_t), orc_cmp_i32);
    }
    free(head);
    free(cell_of);
    free(members);
    return maxc;
}

/* ------------------------------------------------------------------------- */
/* The potential interface (§3.1): V, phi and their derivatives per species pair,
 * F and F' per species.                                                     */

/* Knot table: values y_k and slopes y'_k at uniform knots x_k = x0 + k h on
 * [x0, x1]; cubic Hermite interpolation on each interval, written with the four
 * Hermite basis polynomials; the derivative is that of the same cubic.  Outside
 * [x0, x1]: linear extrapolation from the end knot, and a range count.       */
static double orc_table(const double *tab, int n, double x0, double x1, double x, double *dydx,
                        int64_t *viol) {
    const double *y = tab, *yp = tab + n;
    double h = (x1 - x0) / (double)(n - 1);
    if (x < x0) {
        (*viol)++;
        *dydx = yp[0];
        return y[0] + (x - x0) * yp[0];
    }
    if (x > x1) {
        (*viol)++;
        *dydx = yp[n - 1];
        return y[n - 1] + (x - x1) * yp[n - 1];
    }
    double u = (x - x0) / h;
    int k = (int)floor(u);
    if (k > n - 2) k = n - 2;
    if (k < 0) k = 0;
    double t = u - (double)k;
    double t2 = t * t, t3 = t2 * t;
    double h00 = 2.0 * t3 - 3.0 * t2 + 1.0, h10 = t3 - 2.0 * t2 + t;
    double h01 = -2.0 * t3 + 3.0 * t2, h11 = t3 - t2;
    double g00 = 6.0 * t2 - 6.0 * t, g10 = 3.0 * t2 - 4.0 * t + 1.0;
    double g01 = -6.0 * t2 + 6.0 * t, g11 = 3.0 * t2 - 2.0 * t;
    *dydx = (g00 * y[k] + g10 * h * yp[k] + g01 * y[k + 1] + g11 * h * yp[k + 1]) / h;
    return h00 * y[k] + h10 * h * yp[k] + h01 * y[k + 1] + h11 * h * yp[k + 1];
}

/* Explicit cubic knot sum of the generic potential files of §3.1.1:
 *   f(r) = sum_k c_k (r_k - r)^3 H(r_k - r),  f'(r) = -3 sum_k c_k (r_k - r)^2 H(r_k - r),
 * knot data = K coefficients c_k then K radii r_k. */
static double orc_knots(const double *kd, int K, double r, double *d) {
    double v = 0.0, g = 0.0;
    for (int k = 0; k < K; k++) {
        double u = kd[K + k] - r;
        if (u > 0.0) {
            v += kd[k] * u * u * u;
            g -= 3.0 * kd[k] * u * u;
        }
    }
    *d = g;
    return v;
}

/* which = 0: V_ab (pair), 1: phi_ab (density at an atom of species a from one of species b). */
static double orc_pair(const orc_potential *p, int which, int a, int b, double r, double *d,
                       int64_t *viol) {
    if (p->kind == 4) {
        int ns = p->n_species, K = p->n_knots;
        int t = which * ns * ns + a * ns + b;
        if (!(r < p->r_cut)) { *d = 0.0; return 0.0; }
        return orc_knots(p->tables + (size_t)t * 2 * K, K, r, d);
    }
    if (p->kind == 1) {
        const double dd = p->fs[0], c = p->fs[1], beta = p->fs[3];
        const double c0 = p->fs[4], c1 = p->fs[5], c2 = p->fs[6];
        if (which == 0) {
            if (!(r < c)) { *d = 0.0; return 0.0; }
            double q = c0 + c1 * r + c2 * r * r;
            *d = 2.0 * (r - c) * q + (r - c) * (r - c) * (c1 + 2.0 * c2 * r);
            return (r - c) * (r - c) * q;
        }
        if (!(r < dd)) { *d = 0.0; return 0.0; }
        *d = 2.0 * (r - dd) + 3.0 * beta * (r - dd) * (r - dd) / dd;
        return (r - dd) * (r - dd) + beta * (r - dd) * (r - dd) * (r - dd) / dd;
    }
    int ns = p->n_species, n = p->n_knots;
    int t = which * ns * ns + a * ns + b;
    return orc_table(p->tables + (size_t)t * 2 * n, n, p->r_min, p->r_cut, r, d, viol);
}

static double orc_embed(const orc_potential *p, int a, double rho, double *dF, int64_t *viol) {
    if (p->kind == 1 || p->kind == 4) {
        /* Finnis-Sinclair F = -A sqrt(rho); kind 4 keeps A_a after the 2 ns^2 knot functions */
        double A = p->kind == 1 ? p->fs[2]
                                : p->tables[(size_t)2 * p->n_species * p->n_species * 2 * p->n_knots + a];
        if (!(rho > 0.0)) { *dF = 0.0; return 0.0; } /* F(0) = 0 with F' = 0 (finite at rho = 0) */
        double s = sqrt(rho);
        *dF = -0.5 * A / s;
        return -A * s;
    }
    int ns = p->n_species, n = p->n_knots;
    int t = 2 * ns * ns + a;
    return orc_table(p->tables + (size_t)t * 2 * n, n, p->rho_min, p->rho_max, rho, dF, viol);
}

/* Expose the potential functions for the tests. */
double orc_pair_value(const orc_potential *p, int which, int a, int b, double r, double *d) {
    int64_t v = 0;
    return orc_pair(p, which, a, b, r, d, &v);
}
double orc_embed_value(const orc_potential *p, int a, double rho, double *dF) {
    int64_t v = 0;
    return orc_embed(p, a, rho, dF, &v);
}

/* ------------------------------------------------------------------------- */
/* Eq. (1) and its gradient from the full neighbour list.
 * Pass 1: rho_i = sum_j phi_{s_i s_j}(r_ij); F_i = F_{s_i}(rho_i), F'_i.
 * Pass 2: with d = r_j - r_i and r = |d|,
 *   force_i = sum_j [ V'_{s_i s_j}(r) + F'_i phi'_{s_i s_j}(r) + F'_j phi'_{s_j s_i}(r) ] d / r,
 *   E_i = F_i + 1/2 sum_j V(r)   (each pair's V counted once in U),
 *   W   = -1/2 sum_i sum_j g d (x) d / r   (virial; g is the bracket above).
 * Only pairs with r < r_cut contribute.  Per-atom sums run in list order; the
 * totals are summed over atoms in index order.  Returns the range count.       */
int64_t orc_eam_forces(int64_t n, const double *pos, const int32_t *species, const double *box,
                       const orc_potential *pot, const int32_t *count, const int32_t *list,
                       int32_t k_max, double *rho, double *dF, double *force, double *e_atom,
                       double *virial, double *pe) {
    double L[3] = {box[0], box[1], box[2]};
    double invL[3] = {1.0 / box[0], 1.0 / box[1], 1.0 / box[2]};
    double rc2 = pot->r_cut * pot->r_cut;
    int64_t viol = 0;
    double *w_atom = (double *)calloc((size_t)(n > 0 ? n : 1) * 6, sizeof(double));
#pragma omp parallel for schedule(static) reduction(+ : viol)
    for (int64_t i = 0; i < n; i++) {
        double s = 0.0;
        for (int32_t k = 0; k < count[i]; k++) {
            int64_t j = list[i * k_max + k];
            double r2 = orc_dist2(pos, i, j, L, invL, NULL);
            if (!(r2 < rc2)) continue;
            double dphi;
            s += orc_pair(pot, 1, species[i], species[j], sqrt(r2), &dphi, &viol);
        }
        rho[i] = s;
        e_atom[i] = orc_embed(pot, species[i], s, &dF[i], &viol);
    }
#pragma omp parallel for schedule(static) reduction(+ : viol)
    for (int64_t i = 0; i < n; i++) {
        double f[3] = {0.0, 0.0, 0.0}, ep = 0.0, w[6] = {0, 0, 0, 0, 0, 0};
        int a = species[i];
        for (int32_t k = 0; k < count[i]; k++) {
            int64_t j = list[i * k_max + k];
            double dv[3];
            double r2 = orc_dist2(pos, i, j, L, invL, dv);
            if (!(r2 < rc2)) continue;
            double r = sqrt(r2);
            int b = species[j];
            double dV, dphi_ab, dphi_ba;
            double v = orc_pair(pot, 0, a, b, r, &dV, &viol);
            orc_pair(pot, 1, a, b, r, &dphi_ab, &viol);
            orc_pair(pot, 1, b, a, r, &dphi_ba, &viol);
            double g = dV + dF[i] * dphi_ab + dF[j] * dphi_ba;
            double gr = g / r;
            for (int c = 0; c < 3; c++) f[c] += gr * dv[c];
            ep += 0.5 * v;
            w[0] -= 0.5 * gr * dv[0] * dv[0];
            w[1] -= 0.5 * gr * dv[1] * dv[1];
            w[2] -= 0.5 * gr * dv[2] * dv[2];
            w[3] -= 0.5 * gr * dv[1] * dv[2];
            w[4] -= 0.5 * gr * dv[0] * dv[2];
            w[5] -= 0.5 * gr * dv[0] * dv[1];
        }
        for (int c = 0; c < 3; c++) force[3 * i + c] = f[c];
        e_atom[i] += ep;
        for (int c = 0; c < 6; c++) w_atom[6 * i + c] = w[c];
    }
    double tot = 0.0, wt[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t i = 0; i < n; i++) {
        tot += e_atom[i];
        for (int c = 0; c < 6; c++) wt[c] += w_atom[6 * i + c];
    }
    free(w_atom);
    if (pe) *pe = tot;
    if (virial) { /* xx yy zz, then full 3x3 row-major */
        double m[9] = {wt[0], wt[5], wt[4], wt[5], wt[1], wt[3], wt[4], wt[3], wt[2]};
        memcpy(virial, m, sizeof(m));
    }
    return viol;
}

/* sum_k |3 c_k (r_k - r)^2| over the terms with r < r_k of explicit knot function t (kind 4). */
static double orc_knots_abs_slope(const orc_potential *p, int t, double r) {
    int K = p->n_knots;
    const double *kd = p->tables + (size_t)t * 2 * K;
    double g = 0.0;
    if (!(r < p->r_cut)) return 0.0;
    for (int k = 0; k < K; k++) {
        double u = kd[K + k] - r;
        if (u > 0.0) g += fabs(3.0 * kd[k] * u * u);
    }
    return g;
}

/* Scales of the force sum of Eq. (1)'s gradient, for the error bound of a reduced-precision
 * evaluation (test infrastructure).  For each atom i, over its list pairs with r < r_cut:
 *   m_i = sum_j ( |V'_ab| + |F'_i phi'_ab| + |F'_j phi'_ba| )                (eV/Å)
 *   q_i = sum_j r ( |V''_ab| + |F'_i phi''_ab| + |F'_j phi''_ba| )            (eV/Å)
 *   e_i = sum_j ( |F''_i phi'_ab| R_i + |F''_j phi'_ba| R_j ),
 *         R_a = sum_k ( phi_ak + r_ak |phi'_ak| )                             (eV/Å)
 *   c_i = sum_j ( k_V + |F'_i| k_ab + |F'_j| k_ba ),  k = orc_table_curv at r (tables only)
 * (a = s_i, b = s_j; for explicit knot sums |V'| and |phi'| are the sums of the absolute
 * terms |3 c_k (r_k - r)^2|).  m_i bounds the terms of the pair sum, q_i their change under a relative
 * change of r, and e_i the force change through F' under a relative change of every density
 * term.  Second derivatives are central differences of the first (step 1e-5 Å, and 1e-6 rho
 * for F), which is exact for a cubic within one table interval.  dF = F'(rho) of each atom. */
/* For knot tables (kind 2): the size (|2 c2| + |3 c3|) / h of the quadratic and cubic terms of
 * the derivative of the Hermite cubic of table t on the interval that holds r (c2, c3 the cubic's
 * coefficients in t = (r - r_k) / h); 0 outside the span and for other kinds. */
static double orc_table_curv(const orc_potential *p, int t, double r) {
    if (p->kind != 2) return 0.0;
    int nk = p->n_knots;
    const double *y = p->tables + (size_t)t * 2 * nk, *yp = y + nk;
    double h = (p->r_cut - p->r_min) / (double)(nk - 1);
    if (r < p->r_min || r > p->r_cut) return 0.0;
    int k = (int)floor((r - p->r_min) / h);
    if (k > nk - 2) k = nk - 2;
    double s0 = h * yp[k], s1 = h * yp[k + 1];
    double c2 = 3.0 * (y[k + 1] - y[k]) - 2.0 * s0 - s1;
    double c3 = 2.0 * (y[k] - y[k + 1]) + s0 + s1;
    return (fabs(2.0 * c2) + fabs(3.0 * c3)) / h;
}

void orc_eam_error_scales(int64_t n, const double *pos, const int32_t *species, const double *box,
                          const orc_potential *pot, const int32_t *count, const int32_t *list,
                          int32_t k_max, const double *dF, double *m, double *q, double *e, double *c) {
    double L[3] = {box[0], box[1], box[2]};
    double invL[3] = {1.0 / box[0], 1.0 / box[1], 1.0 / box[2]};
    double rc2 = pot->r_cut * pot->r_cut;
    const double h = 1e-5;
    double *R = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *d2F = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        int64_t viol = 0;
        double s = 0.0, rho = 0.0;
        for (int32_t k = 0; k < count[i]; k++) {
            int64_t j = list[i * k_max + k];
            double r2 = orc_dist2(pos, i, j, L, invL, NULL);
            if (!(r2 < rc2)) continue;
            double r = sqrt(r2), dphi;
            double phi = orc_pair(pot, 1, species[i], species[j], r, &dphi, &viol);
            rho += phi;
            s += fabs(phi) + r * fabs(dphi);
        }
        R[i] = s;
        double hr = 1e-6 * (rho > 0.0 ? rho : 1.0), dp, dm;
        orc_embed(pot, species[i], rho + hr, &dp, &viol);
        orc_embed(pot, species[i], rho - hr, &dm, &viol);
        d2F[i] = (dp - dm) / (2.0 * hr);
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        int64_t viol = 0;
        double sm = 0.0, sq = 0.0, se = 0.0, sc = 0.0;
        int a = species[i];
        for (int32_t k = 0; k < count[i]; k++) {
            int64_t j = list[i * k_max + k];
            double r2 = orc_dist2(pos, i, j, L, invL, NULL);
            if (!(r2 < rc2)) continue;
            double r = sqrt(r2);
            int b = species[j];
            double dV, dab, dba, p1, m1, vpp, abpp, bapp;
            orc_pair(pot, 0, a, b, r, &dV, &viol);
            orc_pair(pot, 1, a, b, r, &dab, &viol);
            orc_pair(pot, 1, b, a, r, &dba, &viol);
            if (pot->kind == 4) { /* explicit sums: the scale of a sum is the sum of |terms| */
                int ns = pot->n_species;
                dV = orc_knots_abs_slope(pot, 0 * ns * ns + a * ns + b, r);
                dab = orc_knots_abs_slope(pot, 1 * ns * ns + a * ns + b, r);
                dba = orc_knots_abs_slope(pot, 1 * ns * ns + b * ns + a, r);
            }
            orc_pair(pot, 0, a, b, r + h, &p1, &viol);
            orc_pair(pot, 0, a, b, r - h, &m1, &viol);
            vpp = (p1 - m1) / (2.0 * h);
            orc_pair(pot, 1, a, b, r + h, &p1, &viol);
            orc_pair(pot, 1, a, b, r - h, &m1, &viol);
            abpp = (p1 - m1) / (2.0 * h);
            orc_pair(pot, 1, b, a, r + h, &p1, &viol);
            orc_pair(pot, 1, b, a, r - h, &m1, &viol);
            bapp = (p1 - m1) / (2.0 * h);
            sm += fabs(dV) + fabs(dF[i] * dab) + fabs(dF[j] * dba);
            sq += r * (fabs(vpp) + fabs(dF[i] * abpp) + fabs(dF[j] * bapp));
            se += fabs(d2F[i] * dab) * R[i] + fabs(d2F[j] * dba) * R[j];
            {
                int ns = pot->n_species;
                sc += orc_table_curv(pot, a * ns + b, r) + fabs(dF[i]) * orc_table_curv(pot, ns * ns + a * ns + b, r) +
                      fabs(dF[j]) * orc_table_curv(pot, ns * ns + b * ns + a, r);
            }
        }
        m[i] = sm;
        q[i] = sq;
        e[i] = se;
        c[i] = sc;
    }
    free(R);
    free(d2F);
}

/* The paper's asymmetric (half) list with F_ij applied to i and j (§3.2.2), run
 * serially: a different order of operations for the same Eq. (1) gradient.
 * Uses the entries j > i of a full list.                                      */
int64_t orc_eam_forces_half(int64_t n, const double *pos, const int32_t *species, const double *box,
                            const orc_potential *pot, const int32_t *count, const int32_t *list,
                            int32_t k_max, double *force, double *pe) {
    double L[3] = {box[0], box[1], box[2]};
    double invL[3] = {1.0 / box[0], 1.0 / box[1], 1.0 / box[2]};
    double rc2 = pot->r_cut * pot->r_cut;
    int64_t viol = 0;
    double *rho = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *dF = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double u = 0.0;
    for (int64_t i = 0; i < n; i++)
        for (int32_t k = 0; k < count[i]; k++) {
            int64_t j = list[i * k_max + k];
            if (j <= i) continue;
            double r2 = orc_dist2(pos, i, j, L, invL, NULL);
            if (!(r2 < rc2)) continue;
            double r = sqrt(r2), dd;
            rho[i] += orc_pair(pot, 1, species[i], species[j], r, &dd, &viol);
            rho[j] += orc_pair(pot, 1, species[j], species[i], r, &dd, &viol);
        }
    for (int64_t i = 0; i < n; i++) {
        u += orc_embed(pot, species[i], rho[i], &dF[i], &viol);
        force[3 * i] = force[3 * i + 1] = force[3 * i + 2] = 0.0;
    }
    for (int64_t i = 0; i < n; i++)
        for (int32_t k = 0; k < count[i]; k++) {
            int64_t j = list[i * k_max + k];
            if (j <= i) continue;
            double dv[3];
            double r2 = orc_dist2(pos, i, j, L, invL, dv);
            if (!(r2 < rc2)) continue;
            double r = sqrt(r2);
            int a = species[i], b = species[j];
            double dV, dab, dba;
            u += orc_pair(pot, 0, a, b, r, &dV, &viol);
            orc_pair(pot, 1, a, b, r, &dab, &viol);
            orc_pair(pot, 1, b, a, r, &dba, &viol);
            double gr = (dV + dF[i] * dab + dF[j] * dba) / r;
            for (int c = 0; c < 3; c++) {
                force[3 * i + c] += gr * dv[c]; /* force on i: along +d (towards j) */
                force[3 * j + c] -= gr * dv[c]; /* Newton's third law on j           */
            }
        }
    free(rho);
    free(dF);
    if (pe) *pe = u;
    return viol;
}

/* ------------------------------------------------------------------------- */
/* Thermodynamics of a microstate (§2.1.2, §2.6): KE = sum m v^2 / 2,
 * T = 2 KE / ((3N-3) k_B), total momentum.                                    */
void orc_kinetic(int64_t n, const double *vel, const int32_t *species, const double *masses,
                 double *ke, double *temperature, double *momentum, double *kin_tensor) {
    double k = 0.0, p[3] = {0, 0, 0}, kt[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = 0; i < n; i++) {
        double m = masses[species[i]];
        const double *v = vel + 3 * i;
        k += 0.5 * m * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        for (int a = 0; a < 3; a++) {
            p[a] += m * v[a];
            for (int b = 0; b < 3; b++) kt[3 * a + b] += m * v[a] * v[b];
        }
    }
    k *= ORC_MVV2E;
    if (ke) *ke = k;
    if (temperature) *temperature = (n > 1) ? 2.0 * k / ((double)(3 * n - 3) * ORC_KB) : 0.0;
    if (momentum) memcpy(momentum, p, sizeof(p));
    if (kin_tensor) for (int a = 0; a < 9; a++) kin_tensor[a] = kt[a] * ORC_MVV2E;
}

/* Pressure (GPa) from the kinetic and virial tensors: P = (tr(K) + tr(W)) / (3 V). */
double orc_pressure_gpa(const double *kin_tensor, const double *virial, const double *box) {
    double vol = box[0] * box[1] * box[2];
    double tr = kin_tensor[0] + kin_tensor[4] + kin_tensor[8] + virial[0] + virial[4] + virial[8];
    return tr / (3.0 * vol) * ORC_EVA3_TO_GPA;
}

/* ------------------------------------------------------------------------- */
/* Velocity Verlet (§2.3) with the neighbour list rebuilt every `rebuild_every`
 * steps (Table 1 `nbrupdate`; 0 = never on a schedule) and whenever an atom has
 * moved more than skin/2 since the last build, so that the padded list stays
 * complete (§3.2.1).  Time step dt in fs; accelerations F/m converted from
 * eV/(Å amu) to Å/fs^2 (§2.7).  The strain-rate condition (§2.2): after each
 * drift, the box z edge and every z coordinate are multiplied by
 * (1 + strain_rate_zz * dt), fractional coordinates fixed.
 * `force` holds F(r) at the initial positions on entry (forces_valid = 1) or is
 * computed first; on exit it holds the forces at the final positions.
 * energies (if given) receives per step: PE, KE.                              */
int64_t orc_run_vv(int64_t n, double *pos, double *vel, const int32_t *species, const double *masses,
                   double *box, const orc_potential *pot, double dt_fs, int32_t n_steps, double skin,
                   int32_t k_max, int32_t rebuild_every, double strain_rate_zz, double *force,
                   int32_t forces_valid, double *energies, int32_t *n_rebuilds, int32_t *max_count) {
    double r_list = pot->r_cut + skin;
    int32_t *count = (int32_t *)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    int32_t *list = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1) * k_max);
    double *ref = (double *)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    double *rho = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    double *dF = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    double *ea = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    double acc = 1.0 / ORC_MVV2E; /* (eV/Å)/amu -> Å/fs^2 */
    int64_t viol = 0;
    int32_t rebuilds = 0, mc = 0;

#define ORC_BUILD()                                                                         \
    do {                                                                                    \
        int32_t m_ = orc_neighbours_cells(n, pos, box, r_list, k_max, count, list);         \
        if (m_ < 0) m_ = orc_neighbours_brute(n, pos, box, r_list, k_max, count, list);     \
        if (m_ > mc) mc = m_;                                                                \
        memcpy(ref, pos, sizeof(double) * 3 * n);                                           \
        rebuilds++;                                                                          \
    } while (0)

    ORC_BUILD();
    if (!forces_valid)
        viol += orc_eam_forces(n, pos, species, box, pot, count, list, k_max, rho, dF, force, ea, NULL, NULL);
    double half = 0.5 * dt_fs;
    double lim2 = 0.25 * skin * skin;
    for (int32_t step = 0; step < n_steps; step++) {
        for (int64_t i = 0; i < n; i++) {
            double im = acc / masses[species[i]];
            for (int c = 0; c < 3; c++) {
                vel[3 * i + c] += half * force[3 * i + c] * im;
                pos[3 * i + c] += dt_fs * vel[3 * i + c];
            }
        }
        if (strain_rate_zz != 0.0) {
            double s = 1.0 + strain_rate_zz * dt_fs * 1.0e-15;
            box[2] *= s;
            for (int64_t i = 0; i < n; i++) pos[3 * i + 2] *= s;
        }
        int rebuild = (rebuild_every > 0 && (step + 1) % rebuild_every == 0);
        for (int64_t i = 0; i < n && !rebuild; i++) {
            double dx = pos[3 * i] - ref[3 * i], dy = pos[3 * i + 1] - ref[3 * i + 1];
            double dz = pos[3 * i + 2] - ref[3 * i + 2];
            if ((dx * dx + dy * dy) + dz * dz > lim2) rebuild = 1;
        }
        if (rebuild) ORC_BUILD();
        double pe = 0.0;
        viol += orc_eam_forces(n, pos, species, box, pot, count, list, k_max, rho, dF, force, ea, NULL, &pe);
        for (int64_t i = 0; i < n; i++) {
            double im = acc / masses[species[i]];
            for (int c = 0; c < 3; c++) vel[3 * i + c] += half * force[3 * i + c] * im;
        }
        if (energies) {
            double ke;
            orc_kinetic(n, vel, species, masses, &ke, NULL, NULL, NULL);
            energies[2 * step] = pe;
            energies[2 * step + 1] = ke;
        }
    }
#undef ORC_BUILD
    if (n_rebuilds) *n_rebuilds = rebuilds;
    if (max_count) *max_count = mc;
    free(count);
    free(list);
    free(ref);
    free(rho);
    free(dF);
    free(ea);
    return viol;
}

/* ------------------------------------------------------------------------- */
/* Third-order predictor-corrector (§2.3, the paper's second integrator, after Gear), for the
 * second-order equations of motion r'' = F/m.  The state of each atom is the scaled Taylor
 * (Nordsieck) vector of its trajectory up to the third derivative,
 *   q0 = r,  q1 = dt v,  q2 = (dt^2/2) a,  q3 = (dt^3/6) b   (a = r'', b = da/dt),
 * and one step is:
 *   predict:  q0 <- q0 + q1 + q2 + q3,  q1 <- q1 + 2 q2 + 3 q3,  q2 <- q2 + 3 q3  (the Taylor
 *             series to third order; q3 is unchanged);
 *   evaluate: the forces at the predicted positions (the one force evaluation of the step);
 *   correct:  D = (dt^2/2) F/m - q2 (the error of the predicted acceleration term), then
 *             q_k <- q_k + c_k D with Gear's coefficients for a second-order equation and four
 *             values, c = (1/6, 5/6, 1, 1/3).
 * Start: q2 from the forces at the initial positions (computed unless forces_valid), and q3 from
 * `gear3` ([N][3], the third-derivative term of a previous call; zero to start afresh).  On exit
 * pos, vel hold q0 and q1 / dt, force the forces at the last predicted positions (so q2 =
 * (dt^2/2) F/m), gear3 the final q3.  energies[2 s ..] = (PE at the step's predicted positions,
 * KE of its corrected velocities).  The list is rebuilt as in orc_run_vv, from the predicted
 * positions.  No strain ramp.                                                                 */
int64_t orc_run_pc3(int64_t n, double *pos, double *vel, const int32_t *species, const double *masses,
                    const double *box, const orc_potential *pot, double dt_fs, int32_t n_steps, double skin,
                    int32_t k_max, int32_t rebuild_every, double *force, int32_t forces_valid, double *gear3,
                    double *energies, int32_t *n_rebuilds) {
    const double c0 = 1.0 / 6.0, c1 = 5.0 / 6.0, c3 = 1.0 / 3.0; /* c2 = 1 */
    double r_list = pot->r_cut + skin;
    size_t nn = (size_t)(n > 0 ? n : 1);
    int32_t *count = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *list = (int32_t *)malloc(sizeof(int32_t) * nn * k_max);
    double *ref = (double *)malloc(sizeof(double) * 3 * nn);
    double *rho = (double *)malloc(sizeof(double) * nn);
    double *dF = (double *)malloc(sizeof(double) * nn);
    double *ea = (double *)malloc(sizeof(double) * nn);
    double *q1 = (double *)malloc(sizeof(double) * 3 * nn);
    double *q2 = (double *)malloc(sizeof(double) * 3 * nn);
    double acc = 1.0 / ORC_MVV2E; /* (eV/Å)/amu -> Å/fs^2 */
    double h2 = 0.5 * dt_fs * dt_fs;
    double lim2 = 0.25 * skin * skin;
    int64_t viol = 0;
    int32_t rebuilds = 0;
    double L[3] = {box[0], box[1], box[2]};
#define ORC_BUILD3()                                                                            \
    do {                                                                                        \
        if (orc_neighbours_cells(n, pos, L, r_list, k_max, count, list) < 0)                    \
            orc_neighbours_brute(n, pos, L, r_list, k_max, count, list);                        \
        memcpy(ref, pos, sizeof(double) * 3 * n);                                               \
        rebuilds++;                                                                             \
    } while (0)
    ORC_BUILD3();
    if (!forces_valid)
        viol += orc_eam_forces(n, pos, species, L, pot, count, list, k_max, rho, dF, force, ea, NULL, NULL);
    for (int64_t i = 0; i < n; i++) {
        double im = acc / masses[species[i]];
        for (int c = 0; c < 3; c++) {
            q1[3 * i + c] = dt_fs * vel[3 * i + c];
            q2[3 * i + c] = h2 * force[3 * i + c] * im;
        }
    }
    for (int32_t step = 0; step < n_steps; step++) {
        for (size_t k = 0; k < 3 * (size_t)n; k++) { /* predict */
            pos[k] += q1[k] + q2[k] + gear3[k];
            q1[k] += 2.0 * q2[k] + 3.0 * gear3[k];
            q2[k] += 3.0 * gear3[k];
        }
        int rebuild = (rebuild_every > 0 && (step + 1) % rebuild_every == 0);
        for (int64_t i = 0; i < n && !rebuild; i++) {
            double dx = pos[3 * i] - ref[3 * i], dy = pos[3 * i + 1] - ref[3 * i + 1];
            double dz = pos[3 * i + 2] - ref[3 * i + 2];
            if ((dx * dx + dy * dy) + dz * dz > lim2) rebuild = 1;
        }
        if (rebuild) ORC_BUILD3();
        double pe = 0.0;
        viol += orc_eam_forces(n, pos, species, L, pot, count, list, k_max, rho, dF, force, ea, NULL, &pe);
        for (int64_t i = 0; i < n; i++) { /* correct */
            double im = acc / masses[species[i]];
            for (int c = 0; c < 3; c++) {
                size_t k = 3 * (size_t)i + c;
                double D = h2 * force[k] * im - q2[k];
                pos[k] += c0 * D;
                q1[k] += c1 * D;
                q2[k] += D;
                gear3[k] += c3 * D;
            }
        }
        if (energies) {
            for (size_t k = 0; k < 3 * (size_t)n; k++) vel[k] = q1[k] / dt_fs;
            double ke;
            orc_kinetic(n, vel, species, masses, &ke, NULL, NULL, NULL);
            energies[2 * step] = pe;
            energies[2 * step + 1] = ke;
        }
    }
#undef ORC_BUILD3
    for (size_t k = 0; k < 3 * (size_t)n; k++) vel[k] = q1[k] / dt_fs;
    if (n_rebuilds) *n_rebuilds = rebuilds;
    free(count);
    free(list);
    free(ref);
    free(rho);
    free(dF);
    free(ea);
    free(q1);
    free(q2);
    return viol;
}

/* ------------------------------------------------------------------------- */
/* Nose-Hoover thermostat (NVTp, §2.1.2): dp_i/dt = -dU/dq_i - pi_s p_i, Q_s dpi_s/dt = sum_i p_i^2/m_i
 * - g k_B T with g = 3N - 3 (the printed right-hand side writes the kinetic term as p^2/2m; the
 * reading taken here is the standard p^2/m, whose fixed point is the temperature the same section
 * defines, sum p^2/2m = g k_B T / 2).  The thermostat friction integrates to xi (dxi/dt = pi_s) and
 * H' = KE + U + Q_s pi_s^2 / 2 + g k_B T xi is conserved.  Integrator: a symmetric split, a
 * thermostat half step before and after each velocity-Verlet step of orc_run_vv; a thermostat half
 * step of length h = dt/2 is
 *   pi += (h/2) (2 KE - g kT) / Q;  v *= exp(-pi h);  xi += pi h;  pi += (h/2) (2 KE' - g kT) / Q
 * with KE' the kinetic energy of the scaled velocities.  Units: eV, fs, amu; Q in eV fs^2, pi in
 * 1/fs.  thermo[3] = {pi, xi, Q} in/out (Q is read only); energies[3 s ..] = (PE, KE, H'). */
static void orc_thermo_half(int64_t n, double *vel, const int32_t *species, const double *masses, double h,
                            double gkt, double *thermo) {
    double ke;
    orc_kinetic(n, vel, species, masses, &ke, NULL, NULL, NULL);
    double q = thermo[2];
    thermo[0] += 0.5 * h * (2.0 * ke - gkt) / q;
    double s = exp(-thermo[0] * h);
    for (int64_t i = 0; i < 3 * n; i++) vel[i] *= s;
    thermo[1] += thermo[0] * h;
    orc_kinetic(n, vel, species, masses, &ke, NULL, NULL, NULL);
    thermo[0] += 0.5 * h * (2.0 * ke - gkt) / q;
}

int64_t orc_run_nvt(int64_t n, double *pos, double *vel, const int32_t *species, const double *masses,
                    double *box, const orc_potential *pot, double dt_fs, int32_t n_steps, double skin, int32_t k_max,
                    double t_kelvin, double *thermo, double *force, int32_t forces_valid, double *energies) {
    const double gkt = (double)(3 * n - 3) * ORC_KB * t_kelvin;
    int64_t viol = 0;
    int32_t fv = forces_valid, nr = 0, mc = 0;
    for (int32_t step = 0; step < n_steps; step++) {
        orc_thermo_half(n, vel, species, masses, 0.5 * dt_fs, gkt, thermo);
        double e2[2];
        viol += orc_run_vv(n, pos, vel, species, masses, box, pot, dt_fs, 1, skin, k_max, 0, 0.0, force, fv, e2,
                           &nr, &mc);
        fv = 1;
        orc_thermo_half(n, vel, species, masses, 0.5 * dt_fs, gkt, thermo);
        if (energies) {
            double ke;
            orc_kinetic(n, vel, species, masses, &ke, NULL, NULL, NULL);
            energies[3 * step] = e2[0];
            energies[3 * step + 1] = ke;
            energies[3 * step + 2] = ke + e2[0] + 0.5 * thermo[2] * thermo[0] * thermo[0] + gkt * thermo[1];
        }
    }
    return viol;
}

/* ------------------------------------------------------------------------- */
/* Learned surrogate of the per-atom energy (not in the paper; the EAM oracle above is its
 * reference).  Descriptor of atom i: G_ik = sum_j b_k(r_ij) over neighbours with r < rd,
 *   b_k(r) = exp(-(r - mu_k)^2 / (2 w^2)) fc(r),  mu_k = mu0 + k dmu,
 *   fc(r) = (cos(pi r / rd) + 1) / 2.
 * Energy E_i = f(G_i), f a multilayer perceptron nb -> h1 -> h2 -> 1 with SiLU
 * s(z) = z / (1 + exp(-z)):  z1 = W1 G + b1, a1 = s(z1), z2 = W2 a1 + b2, a2 = s(z2),
 * E_i = w3 . a2 + b3.  Weights packed as W1 [h1][nb], b1 [h1], W2 [h2][h1], b2 [h2],
 * w3 [h2], b3.  With g_i = dE_i/dG_i, the force is F = -grad sum_i E_i:
 *   F_m = sum_j [ sum_k (g_mk + g_jk) b_k'(r_mj) ] (r_j - r_m) / r_mj.                       */
typedef struct {
    int32_t nb, h1, h2, pad;
    double mu0, dmu, width, rd;
} orc_sur_spec;

static double orc_silu(double z) { return z / (1.0 + exp(-z)); }
static double orc_dsilu(double z) {
    double s = 1.0 / (1.0 + exp(-z));
    return s * (1.0 + z * (1.0 - s));
}

static void orc_basis(const orc_sur_spec *sp, double r, double *b, double *db) {
    const double pi = 3.14159265358979323846;
    double fc = 0.5 * (cos(pi * r / sp->rd) + 1.0);
    double dfc = -0.5 * pi / sp->rd * sin(pi * r / sp->rd);
    double w2 = sp->width * sp->width;
    for (int k = 0; k < sp->nb; k++) {
        double a = r - (sp->mu0 + k * sp->dmu);
        double e = exp(-a * a / (2.0 * w2));
        b[k] = e * fc;
        db[k] = e * (dfc - a / w2 * fc);
    }
}

/* G [n][nb] from the full neighbour list. */
void orc_sur_descriptors(int64_t n, const double *pos, const double *box, const int32_t *count,
                         const int32_t *list, int32_t k_max, const orc_sur_spec *sp, double *G) {
    double L[3] = {box[0], box[1], box[2]};
    double invL[3] = {1.0 / box[0], 1.0 / box[1], 1.0 / box[2]};
    double rd2 = sp->rd * sp->rd;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        double b[256], db[256];
        double *g = G + i * sp->nb;
        for (int k = 0; k < sp->nb; k++) g[k] = 0.0;
        for (int32_t q = 0; q < count[i]; q++) {
            int64_t j = list[i * k_max + q];
            double r2 = orc_dist2(pos, i, j, L, invL, NULL);
            if (!(r2 < rd2)) continue;
            orc_basis(sp, sqrt(r2), b, db);
            for (int k = 0; k < sp->nb; k++) g[k] += b[k];
        }
    }
}

/* Per-atom energy E_i and input gradient g_i = dE_i/dG_i (backpropagation of the MLP). */
void orc_sur_mlp(int64_t n, const double *G, const orc_sur_spec *sp, const double *wts, double *E,
                 double *grad) {
    const int nb = sp->nb, h1 = sp->h1, h2 = sp->h2;
    const double *W1 = wts, *b1 = W1 + h1 * nb, *W2 = b1 + h1, *b2 = W2 + h2 * h1, *w3 = b2 + h2;
    const double b3 = w3[h2];
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        double z1[256], a1[256], z2[256], d2[256], d1[256];
        const double *x = G + i * nb;
        for (int p = 0; p < h1; p++) {
            double s = b1[p];
            for (int k = 0; k < nb; k++) s += W1[p * nb + k] * x[k];
            z1[p] = s;
            a1[p] = orc_silu(s);
        }
        double e = b3;
        for (int q = 0; q < h2; q++) {
            double s = b2[q];
            for (int p = 0; p < h1; p++) s += W2[q * h1 + p] * a1[p];
            z2[q] = s;
            e += w3[q] * orc_silu(s);
            d2[q] = w3[q] * orc_dsilu(s);
        }
        E[i] = e;
        for (int p = 0; p < h1; p++) {
            double s = 0.0;
            for (int q = 0; q < h2; q++) s += W2[q * h1 + p] * d2[q];
            d1[p] = s * orc_dsilu(z1[p]);
        }
        for (int k = 0; k < nb; k++) {
            double s = 0.0;
            for (int p = 0; p < h1; p++) s += W1[p * nb + k] * d1[p];
            grad[i * nb + k] = s;
        }
    }
}

/* Forces from the input gradients (see the header of this section). */
void orc_sur_forces(int64_t n, const double *pos, const double *box, const int32_t *count,
                    const int32_t *list, int32_t k_max, const orc_sur_spec *sp, const double *grad,
                    double *force) {
    double L[3] = {box[0], box[1], box[2]};
    double invL[3] = {1.0 / box[0], 1.0 / box[1], 1.0 / box[2]};
    double rd2 = sp->rd * sp->rd;
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < n; m++) {
        double b[256], db[256], f[3] = {0.0, 0.0, 0.0};
        for (int32_t q = 0; q < count[m]; q++) {
            int64_t j = list[m * k_max + q];
            double dv[3];
            double r2 = orc_dist2(pos, m, j, L, invL, dv);
            if (!(r2 < rd2)) continue;
            double r = sqrt(r2);
            orc_basis(sp, r, b, db);
            double c = 0.0;
            for (int k = 0; k < sp->nb; k++) c += (grad[m * sp->nb + k] + grad[j * sp->nb + k]) * db[k];
            for (int a = 0; a < 3; a++) f[a] += c * dv[a] / r;
        }
        for (int a = 0; a < 3; a++) force[3 * m + a] = f[a];
    }
}

/* Training loss of the surrogate over S frames (frame s holds atoms [off[s], off[s+1]), box
 * box[3s..3s+2]; list rows are stored per atom, and hold frame-local atom indices):
 *   L = wE/S sum_s ((E_s - Eref_s)/N_s)^2 + wF/(3 Ntot) sum_i |F_i - Fref_i|^2.
 * Gradient by the chain rule.  The energy term gives dL/dE_i = c_s = 2 wE (E_s - Eref_s)/(S N_s^2).
 * With phi_i = dL/dF_i = 2 wF (F_i - Fref_i)/(3 Ntot) and F_m = -sum_i g_i . dG_i/dr_m, the force
 * term of dL/dtheta is -sum_i d/dtheta (g_i . u_i), u_ik = sum_m dG_ik/dr_m . phi_m
 *   = sum_j b_k'(r_ij) (r_j - r_i)/r_ij . (phi_j - phi_i),
 * u held fixed.  g_i . u_i is the derivative of E_i along u_i (forward tangent), so each atom
 * contributes the parameter gradient of J_i = c_s E_i - (tangent of E_i along u_i), taken by a
 * reverse pass through the tangent-augmented network.  grad must hold the packed weight count. */
double orc_sur_loss_grad(int32_t n_frames, const int64_t *off, const double *pos, const double *box,
                         const int32_t *count, const int32_t *list, int32_t k_max,
                         const double *e_ref, const double *f_ref, const orc_sur_spec *sp,
                         const double *wts, double w_e, double w_f, double *grad, double *parts) {
    const int nb = sp->nb, h1 = sp->h1, h2 = sp->h2;
    const int64_t n = off[n_frames];
    const int64_t n_par = (int64_t)h1 * nb + h1 + (int64_t)h2 * h1 + h2 + h2 + 1;
    const double *W1 = wts, *b1 = W1 + h1 * nb, *W2 = b1 + h1, *b2 = W2 + h2 * h1, *w3 = b2 + h2;
    double *G = (double *)malloc(sizeof(double) * (n > 0 ? n : 1) * nb);
    double *g = (double *)malloc(sizeof(double) * (n > 0 ? n : 1) * nb);
    double *u = (double *)malloc(sizeof(double) * (n > 0 ? n : 1) * nb);
    double *E = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    double *F = (double *)malloc(sizeof(double) * (n > 0 ? n : 1) * 3);
    double *phi = (double *)malloc(sizeof(double) * (n > 0 ? n : 1) * 3);
    double *c = (double *)malloc(sizeof(double) * (n_frames > 0 ? n_frames : 1));
    double loss_e = 0.0, loss_f = 0.0;
    for (int64_t p = 0; p < n_par; p++) grad[p] = 0.0;

    for (int32_t s = 0; s < n_frames; s++) {
        const int64_t a = off[s], m = off[s + 1] - off[s];
        orc_sur_descriptors(m, pos + 3 * a, box + 3 * s, count + a, list + a * k_max, k_max, sp, G + a * nb);
    }
    orc_sur_mlp(n, G, sp, wts, E, g);
    for (int32_t s = 0; s < n_frames; s++) {
        const int64_t a = off[s], m = off[s + 1] - off[s];
        orc_sur_forces(m, pos + 3 * a, box + 3 * s, count + a, list + a * k_max, k_max, sp, g + a * nb, F + 3 * a);
        double es = 0.0;
        for (int64_t i = a; i < a + m; i++) es += E[i];
        double de = (es - e_ref[s]) / (double)m;
        loss_e += de * de;
        c[s] = 2.0 * w_e * (es - e_ref[s]) / ((double)n_frames * (double)m * (double)m);
    }
    loss_e *= w_e / (double)n_frames;
    for (int64_t i = 0; i < 3 * n; i++) {
        double d = F[i] - f_ref[i];
        loss_f += d * d;
        phi[i] = 2.0 * w_f * d / (3.0 * (double)n);
    }
    loss_f *= w_f / (3.0 * (double)n);

    /* u_i from the neighbour gather */
    for (int32_t s = 0; s < n_frames; s++) {
        const int64_t a = off[s], m = off[s + 1] - off[s];
        const double *ps = pos + 3 * a;
        double L[3] = {box[3 * s], box[3 * s + 1], box[3 * s + 2]};
        double invL[3] = {1.0 / L[0], 1.0 / L[1], 1.0 / L[2]};
        double b[256], db[256];
        for (int64_t i = 0; i < m; i++) {
            double *ui = u + (a + i) * nb;
            for (int k = 0; k < nb; k++) ui[k] = 0.0;
            for (int32_t q = 0; q < count[a + i]; q++) {
                int64_t j = list[(a + i) * k_max + q];
                double dv[3];
                double r2 = orc_dist2(ps, i, j, L, invL, dv);
                if (!(r2 < sp->rd * sp->rd)) continue;
                double r = sqrt(r2);
                orc_basis(sp, r, b, db);
                double t = 0.0;
                for (int x = 0; x < 3; x++) t += dv[x] / r * (phi[3 * (a + j) + x] - phi[3 * (a + i) + x]);
                for (int k = 0; k < nb; k++) ui[k] += db[k] * t;
            }
        }
    }

    /* per-atom reverse pass of J_i = c E_i - tangent(E_i; u_i) */
    double *gW1 = grad, *gb1 = gW1 + h1 * nb, *gW2 = gb1 + h1, *gb2 = gW2 + h2 * h1, *gw3 = gb2 + h2,
           *gb3 = gw3 + h2;
    for (int32_t s = 0; s < n_frames; s++) {
        for (int64_t i = off[s]; i < off[s + 1]; i++) {
            double z1[256], t1[256], a1[256], ta1[256], z2[256], t2[256], a2[256], ta2[256];
            double bz2[256], btz2[256], ba1[256], bta1[256], bz1[256], btz1[256];
            const double *x = G + i * nb, *v = u + i * nb;
            const double ce = c[s], ct = -1.0;
            for (int p = 0; p < h1; p++) {
                double sz = b1[p], st = 0.0;
                for (int k = 0; k < nb; k++) { sz += W1[p * nb + k] * x[k]; st += W1[p * nb + k] * v[k]; }
                z1[p] = sz; t1[p] = st;
                a1[p] = orc_silu(sz); ta1[p] = orc_dsilu(sz) * st;
            }
            for (int q = 0; q < h2; q++) {
                double sz = b2[q], st = 0.0;
                for (int p = 0; p < h1; p++) { sz += W2[q * h1 + p] * a1[p]; st += W2[q * h1 + p] * ta1[p]; }
                z2[q] = sz; t2[q] = st;
                a2[q] = orc_silu(sz); ta2[q] = orc_dsilu(sz) * st;
            }
            /* E = w3.a2 + b3, tangent = w3.ta2 */
            *gb3 += ce;
            for (int q = 0; q < h2; q++) {
                gw3[q] += ce * a2[q] + ct * ta2[q];
                double ba2 = ce * w3[q], bta2 = ct * w3[q];
                double sg = 1.0 / (1.0 + exp(-z2[q]));
                double d2s = sg * (1.0 - sg) * (2.0 + z2[q] * (1.0 - 2.0 * sg)); /* SiLU'' */
                bz2[q] = ba2 * orc_dsilu(z2[q]) + bta2 * d2s * t2[q];
                btz2[q] = bta2 * orc_dsilu(z2[q]);
                gb2[q] += bz2[q];
            }
            for (int q = 0; q < h2; q++)
                for (int p = 0; p < h1; p++) gW2[q * h1 + p] += bz2[q] * a1[p] + btz2[q] * ta1[p];
            for (int p = 0; p < h1; p++) {
                double sa = 0.0, st = 0.0;
                for (int q = 0; q < h2; q++) { sa += W2[q * h1 + p] * bz2[q]; st += W2[q * h1 + p] * btz2[q]; }
                ba1[p] = sa; bta1[p] = st;
                double sg = 1.0 / (1.0 + exp(-z1[p]));
                double d2s = sg * (1.0 - sg) * (2.0 + z1[p] * (1.0 - 2.0 * sg));
                bz1[p] = ba1[p] * orc_dsilu(z1[p]) + bta1[p] * d2s * t1[p];
                btz1[p] = bta1[p] * orc_dsilu(z1[p]);
                gb1[p] += bz1[p];
                for (int k = 0; k < nb; k++) gW1[p * nb + k] += bz1[p] * x[k] + btz1[p] * v[k];
            }
        }
    }
    if (parts) { parts[0] = loss_e; parts[1] = loss_f; }
    free(G); free(g); free(u); free(E); free(F); free(phi); free(c);
    return loss_e + loss_f;
}
