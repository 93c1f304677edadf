/*
 * pcms_oracle.c -- plain, slow, FP64 CPU oracle for the field-transfer hot path of
 * "PCMS: Parallel Coupler for Multimodel Simulations" (arXiv 2510.18838).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the independent definition that the CUDA
 * library is checked against. It is called by the test-suite, by the smoke check and
 * by the benchmark's CPU-baseline leg, and by nothing else. It shares no code, header,
 * table or constant with the CUDA path. Compile with -ffp-contract=off so that every
 * expression below is evaluated exactly as written (no fused multiply-add).
 *
 * What it computes (each function names the passage it follows):
 *
 *  - Radius selection (Sec. 3.2.1, selection function s^i = {s_j : phi_j > 0}; Table 1
 *    "0 for r > r_c"): source j is a neighbour of target t iff
 *        d2 = ((sx-tx)*(sx-tx) + (sy-ty)*(sy-ty)) [+ (sz-tz)*(sz-tz)]  <  r*r
 *    evaluated left to right in FP64, and phi(sqrt(d2)/r) > 0.
 *    Lists are returned in ascending source index.
 *  - Minimum-count radius growth (Sec. 3.2.1: with a minimum neighbour count the radius
 *    grows until the targets have enough sources). Per target (default): r <- 2 r until
 *    the count reaches max(min_neighbors, m). Global (option): one radius for every
 *    target, doubled until all of them reach that count.
 *  - Underdetermined check (Sec. 3.2.1: a fit with fewer equations than unknowns is an
 *    error): fewer neighbours than basis terms -> status UNDERDETERMINED, value NaN.
 *  - Local weighted polynomial fit (Sec. 3.2.1, Eq. 1): min_c ||Phi^(1/2)(A c - b)||^2 +
 *    lambda ||c||^2 with A the Vandermonde matrix of the basis centred at the target and
 *    scaled by 1/r, solved by unpivoted Householder QR of [diag(sqrt w) A; sqrt(lambda) I].
 *    The transferred value is c_0 (the basis is centred at the target, so p(0) = e_1).
 *    Shape functions N = diag(sqrt w) Q_1 R^-T e_1, so that value = sum_j N_j b_j.
 *  - Weights: Table 1 (Gaussian, C4, Const, No_Op, MQ, IMQ, TPS, cubic; a = 2) plus
 *    Wendland's C2 function (1-q)^4 (4q+1).
 *  - Point localization (Sec. 3.3): the element whose closure contains the point, by
 *    exact orientation signs, classified on the lowest-order entity; among all elements
 *    whose closure contains the point the smallest element id is reported; -1 if none.
 *  - Barycentric (parametric) linear interpolation in the located triangle (Sec. 3.3).
 *
 * Exact orientation: the 2x2 determinant is expanded into six products, each product is
 * split exactly into two doubles (Dekker's product with Veltkamp's split) and the twelve
 * doubles are summed exactly by growing a non-overlapping expansion (Knuth's two-sum),
 * after Shewchuk, "Adaptive Precision Floating-Point Arithmetic and Fast Robust Geometric
 * Predicates" (1997). The sign is the sign of the largest non-zero component.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_UNDERDETERMINED 1
#define ORC_ILL_CONDITIONED 2

/* weight kinds */
#define ORC_W_WENDLAND_C2 0
#define ORC_W_GAUSSIAN 1
#define ORC_W_C4 2
#define ORC_W_CONST 3
#define ORC_W_NOOP 4
#define ORC_W_MQ 5
#define ORC_W_IMQ 6
#define ORC_W_TPS 7
#define ORC_W_CUBIC 8

/* Rank test on the Householder R: column k is treated as dependent on columns 0..k-1
 * when |R_kk| <= ORC_RANK_TOL * ||column k of the (weighted, augmented) matrix||. */
#define ORC_RANK_TOL 1e-7
#define ORC_MAX_GROW 60
#define ORC_MAX_DIM 5     /* MLS in up to five dimensions (brute-force search above 3D) */
#define ORC_MAX_TERMS 21  /* quadratic basis in 5D */

int orc_version(void) { return 3; }

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------------------ */
/* Weights (Table 1, a = 2, plus Wendland C2). q = r / r_c, 0 <= q < 1.                  */
/* ------------------------------------------------------------------------------------ */
double orc_weight(int kind, double q) {
    const double a = 2.0;
    double aq = a * q;
    switch (kind) {
    case ORC_W_WENDLAND_C2: {
        double t = 1.0 - q;
        return t * t * t * t * (4.0 * q + 1.0);
    }
    case ORC_W_GAUSSIAN: return exp(-(aq * aq));
    case ORC_W_C4: {
        double t = 1.0 - q;
        double t6 = t * t * t * t * t * t;
        double poly = 5.0 * q * q * q * q * q + 30.0 * q * q * q * q + 72.0 * q * q * q +
                      82.0 * q * q + 36.0 * q + 6.0;
        return poly * t6;
    }
    case ORC_W_CONST: return 1.0;
    case ORC_W_NOOP: return 1.0;
    case ORC_W_MQ: return sqrt(1.0 + aq * aq);
    case ORC_W_IMQ: return 1.0 / sqrt(1.0 + aq * aq);
    case ORC_W_TPS: return (aq == 0.0) ? 0.0 : aq * aq * log(aq);
    case ORC_W_CUBIC: return aq * aq * aq;
    default: return NAN;
    }
}

/* Number of monomials of degree <= 2 in dim (2..5) variables: 1, dim + 1, or
 * 1 + dim + dim (dim + 1) / 2. */
int orc_num_terms(int dim, int degree) {
    if (dim < 2 || dim > ORC_MAX_DIM) return -1;
    if (degree == 0) return 1;
    if (degree == 1) return dim + 1;
    if (degree == 2) return 1 + dim + dim * (dim + 1) / 2;
    return -1;
}

/* Graded-lex monomials of u (degree <= 2): 1, then u_d, then u_d u_e (d <= e).
 * 2D [1, x, y, x^2, xy, y^2]; 3D [1, x, y, z, x^2, xy, xz, y^2, yz, z^2]; the same
 * rule in 4D and 5D. */
static void basis(int dim, int degree, const double* u, double* a) {
    int k = 0;
    a[k++] = 1.0;
    if (degree >= 1)
        for (int d = 0; d < dim; d++) a[k++] = u[d];
    if (degree >= 2)
        for (int d = 0; d < dim; d++)
            for (int e = d; e < dim; e++) a[k++] = u[d] * u[e];
}

/* ------------------------------------------------------------------------------------ */
/* Radius selection                                                                      */
/* ------------------------------------------------------------------------------------ */
/* ((dx*dx + dy*dy) + dz*dz) + ... summed left to right over the dimensions */
static double dist2(int dim, const double* src, int64_t ns, int64_t j, const double* t) {
    double dx = src[j] - t[0];
    double dy = src[ns + j] - t[1];
    double d2 = dx * dx + dy * dy;
    for (int d = 2; d < dim; d++) {
        double dz = src[d * ns + j] - t[d];
        d2 = d2 + dz * dz;
    }
    return d2;
}

static int selected(int dim, const double* src, int64_t ns, int64_t j, const double* t,
                    double r, double r2, int wkind) {
    double d2 = dist2(dim, src, ns, j, t);
    if (!(d2 < r2)) return 0;
    double q = sqrt(d2) / r;
    return orc_weight(wkind, q) > 0.0;
}

/* Uniform grid over the sources (Sec. 3.3 search structure), used by mode 1 only to
 * enumerate candidates; the decision is the same exact predicate. */
typedef struct {
    int dim;
    double lo[3], h;
    int64_t n[3], ncell;
    int64_t* start; /* ncell+1 */
    int64_t* item;  /* ns, ascending source index inside each cell */
} grid_t;

static int64_t cell_coord(double x, double lo, double h, int64_t n) {
    double f = floor((x - lo) / h);
    if (f < 0) return 0;
    if (f > (double)(n - 1)) return n - 1;
    return (int64_t)f;
}

static void grid_build(grid_t* g, int dim, const double* src, int64_t ns, double h) {
    g->dim = dim;
    double hi[3] = {0, 0, 0};
    for (int d = 0; d < dim; d++) {
        g->lo[d] = INFINITY;
        hi[d] = -INFINITY;
        for (int64_t j = 0; j < ns; j++) {
            double x = src[d * ns + j];
            if (x < g->lo[d]) g->lo[d] = x;
            if (x > hi[d]) hi[d] = x;
        }
        if (ns == 0) { g->lo[d] = 0; hi[d] = 0; }
    }
    /* keep the grid below ~2^24 cells by enlarging h if needed */
    for (;;) {
        int64_t tot = 1;
        for (int d = 0; d < dim; d++) {
            g->n[d] = (int64_t)floor((hi[d] - g->lo[d]) / h) + 1;
            tot *= g->n[d];
        }
        if (tot <= ((int64_t)1 << 24)) { g->ncell = tot; break; }
        h *= 2.0;
    }
    g->h = h;
    g->start = (int64_t*)calloc((size_t)g->ncell + 1, sizeof(int64_t));
    g->item = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ns > 0 ? ns : 1));
    int64_t* key = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ns > 0 ? ns : 1));
    for (int64_t j = 0; j < ns; j++) {
        int64_t c = 0, stride = 1;
        for (int d = 0; d < dim; d++) {
            c += stride * cell_coord(src[d * ns + j], g->lo[d], h, g->n[d]);
            stride *= g->n[d];
        }
        key[j] = c;
        g->start[c + 1]++;
    }
    for (int64_t c = 0; c < g->ncell; c++) g->start[c + 1] += g->start[c];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)g->ncell);
    memcpy(fill, g->start, sizeof(int64_t) * (size_t)g->ncell);
    for (int64_t j = 0; j < ns; j++) g->item[fill[key[j]]++] = j;
    free(fill);
    free(key);
}

static void grid_free(grid_t* g) {
    free(g->start);
    free(g->item);
}

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* Neighbours of one target at radius r; writes them (ascending) into out if non-NULL.
 * Returns the count. mode 0: every source; mode 1: grid candidates. */
static int64_t target_neighbors(int dim, const double* src, int64_t ns, const double* t,
                                double r, int wkind, int mode, const grid_t* g,
                                int32_t* out) {
    double r2 = r * r;
    int64_t cnt = 0;
    if (mode == 0 || g == NULL) {
        for (int64_t j = 0; j < ns; j++)
            if (selected(dim, src, ns, j, t, r, r2, wkind)) {
                if (out) out[cnt] = (int32_t)j;
                cnt++;
            }
        return cnt;
    }
    int64_t lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int d = 0; d < dim; d++) {
        double a = floor((t[d] - r - g->lo[d]) / g->h) - 1.0;
        double b = floor((t[d] + r - g->lo[d]) / g->h) + 1.0;
        if (b < 0 || a > (double)(g->n[d] - 1)) return 0;
        lo[d] = a < 0 ? 0 : (int64_t)a;
        hi[d] = b > (double)(g->n[d] - 1) ? g->n[d] - 1 : (int64_t)b;
    }
    int64_t zlo = dim == 3 ? lo[2] : 0, zhi = dim == 3 ? hi[2] : 0;
    for (int64_t cz = zlo; cz <= zhi; cz++)
        for (int64_t cy = lo[1]; cy <= hi[1]; cy++)
            for (int64_t cx = lo[0]; cx <= hi[0]; cx++) {
                int64_t c = cx + g->n[0] * (cy + g->n[1] * cz);
                for (int64_t p = g->start[c]; p < g->start[c + 1]; p++) {
                    int64_t j = g->item[p];
                    if (selected(dim, src, ns, j, t, r, r2, wkind)) {
                        if (out) out[cnt] = (int32_t)j;
                        cnt++;
                    }
                }
            }
    if (out && cnt > 1) qsort(out, (size_t)cnt, sizeof(int32_t), cmp_i32);
    return cnt;
}

static void load_target(int dim, const double* tgt, int64_t nt, int64_t i, double* t) {
    for (int d = 0; d < dim; d++) t[d] = tgt[d * nt + i];
    for (int d = dim; d < ORC_MAX_DIM; d++) t[d] = 0.0;
}

/* Per-target radius growth (Sec. 3.2.1). need <= 0: no growth. Returns count at the
 * final radius, and the doubling count in *kexp. */
static int64_t grow_radius(int dim, const double* src, int64_t ns, const double* t,
                           double radius, int wkind, int need, int mode, const grid_t* g,
                           int32_t* kexp) {
    int k = 0;
    int64_t cnt = target_neighbors(dim, src, ns, t, radius, wkind, mode, g, NULL);
    if (need > 0)
        while (cnt < need && k < ORC_MAX_GROW && cnt < ns) {
            k++;
            cnt = target_neighbors(dim, src, ns, t, ldexp(radius, k), wkind, mode, g, NULL);
        }
    *kexp = k;
    return cnt;
}

/* Counts (and growth exponents) for every target. need = max(min_neighbors, m) when
 * min_neighbors > 0, else 0 (no growth). Returns the total number of pairs. */
int64_t orc_count_neighbors(int dim, const double* src, int64_t ns, const double* tgt,
                            int64_t nt, double radius, int wkind, int need, int mode,
                            int32_t* counts, int32_t* kexp) {
    if (dim > 3) mode = 0; /* the grid is 2D/3D: brute force above */
    grid_t g;
    const grid_t* gp = NULL;
    if (mode == 1) {
        grid_build(&g, dim, src, ns, radius);
        gp = &g;
    }
    int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : total)
    for (int64_t i = 0; i < nt; i++) {
        double t[ORC_MAX_DIM];
        load_target(dim, tgt, nt, i, t);
        int32_t k = 0;
        int64_t c = grow_radius(dim, src, ns, t, radius, wkind, need, mode, gp, &k);
        counts[i] = (int32_t)c;
        kexp[i] = k;
        total += c;
    }
    if (gp) grid_free(&g);
    return total;
}

/* Global reading of the growth rule (Sec. 3.2.1): one radius for all targets, doubled
 * until every target has at least `need` neighbours (or already selects all ns sources),
 * at most ORC_MAX_GROW times. Returns the number of doublings; 0 when need <= 0. */
int orc_global_doublings(int dim, const double* src, int64_t ns, const double* tgt,
                         int64_t nt, double radius, int wkind, int need, int mode) {
    if (dim > 3) mode = 0; /* the grid is 2D/3D: brute force above */
    if (need <= 0 || nt <= 0) return 0;
    grid_t g;
    const grid_t* gp = NULL;
    if (mode == 1) {
        grid_build(&g, dim, src, ns, radius);
        gp = &g;
    }
    int k = 0;
    for (;;) {
        const double r = ldexp(radius, k);
        int64_t short_of = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : short_of)
        for (int64_t i = 0; i < nt; i++) {
            double t[ORC_MAX_DIM];
            load_target(dim, tgt, nt, i, t);
            int64_t c = target_neighbors(dim, src, ns, t, r, wkind, mode, gp, NULL);
            if (c < need && c < ns) short_of++;
        }
        if (short_of == 0 || k >= ORC_MAX_GROW) break;
        k++;
    }
    if (gp) grid_free(&g);
    return k;
}

/* Fill neighbour lists (ascending) given offsets from counts and the growth exponents. */
void orc_fill_neighbors(int dim, const double* src, int64_t ns, const double* tgt,
                        int64_t nt, double radius, int wkind, int mode,
                        const int32_t* kexp, const int64_t* offsets, int32_t* cols) {
    if (dim > 3) mode = 0; /* the grid is 2D/3D: brute force above */
    grid_t g;
    const grid_t* gp = NULL;
    if (mode == 1) {
        grid_build(&g, dim, src, ns, radius);
        gp = &g;
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < nt; i++) {
        double t[ORC_MAX_DIM];
        load_target(dim, tgt, nt, i, t);
        target_neighbors(dim, src, ns, t, ldexp(radius, kexp[i]), wkind, mode, gp,
                         cols + offsets[i]);
    }
    if (gp) grid_free(&g);
}

/* ------------------------------------------------------------------------------------ */
/* Weighted least squares by Householder QR (Eq. 1)                                      */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    double *B, *V, *rhs, *beta, *colnorm, *sw, *z, *y;
    int32_t* nbr;
    int64_t cap_rows, cap_nbr;
    int m, nf;
} work_t;

static void work_reserve(work_t* w, int64_t rows, int m, int nf) {
    if (rows <= w->cap_rows && m <= w->m && nf <= w->nf) return;
    int64_t R = rows > w->cap_rows ? rows * 2 : w->cap_rows;
    int M = m > w->m ? m : w->m;
    int F = nf > w->nf ? nf : w->nf;
    free(w->B); free(w->V); free(w->rhs); free(w->beta); free(w->colnorm);
    free(w->sw); free(w->z); free(w->y);
    w->B = (double*)malloc(sizeof(double) * (size_t)(R * M));
    w->V = (double*)malloc(sizeof(double) * (size_t)(R * M));
    w->rhs = (double*)malloc(sizeof(double) * (size_t)(R * (F > 0 ? F : 1)));
    w->beta = (double*)malloc(sizeof(double) * (size_t)M);
    w->colnorm = (double*)malloc(sizeof(double) * (size_t)M);
    w->sw = (double*)malloc(sizeof(double) * (size_t)R);
    w->z = (double*)malloc(sizeof(double) * (size_t)M);
    w->y = (double*)malloc(sizeof(double) * (size_t)R);
    w->cap_rows = R; w->m = M; w->nf = F;
}

static void work_free(work_t* w) {
    free(w->B); free(w->V); free(w->rhs); free(w->beta); free(w->colnorm);
    free(w->sw); free(w->z); free(w->y); free(w->nbr);
}

/* Solve one target. nbr[0..n-1] ascending. Writes values[f] (stride vstride) for each
 * field and, if shape != NULL, shape[0..n-1]. Returns the status. */
static int solve_target(int dim, int degree, int wkind, double lambda, const double* src,
                        int64_t ns, const double* t, double r, const int32_t* nbr, int64_t n,
                        const double* fields, int nf, double* values, int64_t vstride,
                        double* shape, work_t* w) {
    int m = orc_num_terms(dim, degree);
    if (n < m) {
        for (int f = 0; f < nf; f++) values[f * vstride] = NAN;
        if (shape) for (int64_t i = 0; i < n; i++) shape[i] = NAN;
        return ORC_UNDERDETERMINED;
    }
    int64_t rows = n + (lambda > 0.0 ? m : 0);
    work_reserve(w, rows, m, nf);
    double *B = w->B, *V = w->V, *rhs = w->rhs;
    /* B = [diag(sqrt w) A ; sqrt(lambda) I], column-major rows x m */
    for (int64_t i = 0; i < n; i++) {
        int64_t j = nbr[i];
        double u[ORC_MAX_DIM] = {0, 0, 0, 0, 0}, a[ORC_MAX_TERMS];
        for (int d = 0; d < dim; d++) u[d] = (src[d * ns + j] - t[d]) / r;
        double d2 = dist2(dim, src, ns, j, t);
        double wt = orc_weight(wkind, sqrt(d2) / r);
        double s = sqrt(wt);
        w->sw[i] = s;
        basis(dim, degree, u, a);
        for (int k = 0; k < m; k++) B[k * rows + i] = s * a[k];
        for (int f = 0; f < nf; f++) rhs[f * rows + i] = s * fields[(int64_t)f * ns + j];
    }
    if (lambda > 0.0) {
        double sl = sqrt(lambda);
        for (int64_t i = 0; i < m; i++) {
            for (int k = 0; k < m; k++) B[k * rows + n + i] = (k == i) ? sl : 0.0;
            for (int f = 0; f < nf; f++) rhs[f * rows + n + i] = 0.0;
        }
    }
    for (int k = 0; k < m; k++) {
        double s = 0.0;
        for (int64_t i = 0; i < rows; i++) s += B[k * rows + i] * B[k * rows + i];
        w->colnorm[k] = sqrt(s);
    }
    int status = ORC_OK;
    /* Householder: H_k = I - beta_k v_k v_k^T acting on rows k..rows-1 */
    for (int k = 0; k < m; k++) {
        double s = 0.0;
        for (int64_t i = k; i < rows; i++) s += B[k * rows + i] * B[k * rows + i];
        double nrm = sqrt(s);
        if (!(nrm > ORC_RANK_TOL * w->colnorm[k])) { status = ORC_ILL_CONDITIONED; break; }
        double alpha = B[k * rows + k] > 0.0 ? -nrm : nrm;
        double* v = V + (int64_t)k * rows;
        for (int64_t i = k; i < rows; i++) v[i] = B[k * rows + i];
        v[k] -= alpha;
        double vv = 0.0;
        for (int64_t i = k; i < rows; i++) vv += v[i] * v[i];
        double beta = 2.0 / vv;
        w->beta[k] = beta;
        B[k * rows + k] = alpha;
        for (int64_t i = k + 1; i < rows; i++) B[k * rows + i] = 0.0;
        for (int c = k + 1; c < m; c++) {
            double dot = 0.0;
            for (int64_t i = k; i < rows; i++) dot += v[i] * B[c * rows + i];
            dot *= beta;
            for (int64_t i = k; i < rows; i++) B[c * rows + i] -= dot * v[i];
        }
        for (int f = 0; f < nf; f++) {
            double dot = 0.0;
            for (int64_t i = k; i < rows; i++) dot += v[i] * rhs[f * rows + i];
            dot *= beta;
            for (int64_t i = k; i < rows; i++) rhs[f * rows + i] -= dot * v[i];
        }
    }
    if (status != ORC_OK) {
        for (int f = 0; f < nf; f++) values[f * vstride] = NAN;
        if (shape) for (int64_t i = 0; i < n; i++) shape[i] = NAN;
        return status;
    }
    /* values: back substitution R c = (Q^T rhs)[0:m]; value = c_0 */
    for (int f = 0; f < nf; f++) {
        double c[ORC_MAX_TERMS];
        for (int k = m - 1; k >= 0; k--) {
            double s = rhs[f * rows + k];
            for (int l = k + 1; l < m; l++) s -= B[l * rows + k] * c[l];
            c[k] = s / B[k * rows + k];
        }
        values[f * vstride] = c[0];
    }
    if (shape) {
        /* z = R^-T e_1 (forward substitution with R^T) */
        double* z = w->z;
        for (int k = 0; k < m; k++) {
            double s = (k == 0) ? 1.0 : 0.0;
            for (int l = 0; l < k; l++) s -= B[k * rows + l] * z[l];
            z[k] = s / B[k * rows + k];
        }
        /* y = Q [z; 0] = H_0 H_1 ... H_{m-1} [z; 0] */
        double* y = w->y;
        for (int64_t i = 0; i < rows; i++) y[i] = (i < m) ? z[i] : 0.0;
        for (int k = m - 1; k >= 0; k--) {
            double* v = V + (int64_t)k * rows;
            double dot = 0.0;
            for (int64_t i = k; i < rows; i++) dot += v[i] * y[i];
            dot *= w->beta[k];
            for (int64_t i = k; i < rows; i++) y[i] -= dot * v[i];
        }
        for (int64_t i = 0; i < n; i++) shape[i] = w->sw[i] * y[i];
    }
    return ORC_OK;
}

/* Full MLS transfer. fields: [nf][ns]; values: [nf][nt]; status, kexp: [nt].
 * need: see orc_count_neighbors. If offsets/cols/shape are non-NULL they receive the
 * neighbour lists and shape functions (offsets must come from a previous count with
 * the same arguments). */
void orc_mls(int dim, int degree, int wkind, double lambda, const double* src, int64_t ns,
             const double* tgt, int64_t nt, const double* fields, int nf, double radius,
             int need, int mode, double* values, int8_t* status, int32_t* kexp,
             const int64_t* offsets, int32_t* cols, double* shape) {
    if (dim > 3) mode = 0; /* the grid is 2D/3D: brute force above */
    grid_t g;
    const grid_t* gp = NULL;
    if (mode == 1) {
        grid_build(&g, dim, src, ns, radius);
        gp = &g;
    }
#pragma omp parallel
    {
        work_t w;
        memset(&w, 0, sizeof(w));
        w.cap_nbr = 0;
#pragma omp for schedule(dynamic, 8)
        for (int64_t i = 0; i < nt; i++) {
            double t[ORC_MAX_DIM];
            load_target(dim, tgt, nt, i, t);
            int32_t k = 0;
            int64_t cnt = grow_radius(dim, src, ns, t, radius, wkind, need, mode, gp, &k);
            kexp[i] = k;
            double r = ldexp(radius, k);
            if (cnt > w.cap_nbr) {
                free(w.nbr);
                w.cap_nbr = cnt * 2;
                w.nbr = (int32_t*)malloc(sizeof(int32_t) * (size_t)w.cap_nbr);
            }
            int32_t* nbr = w.nbr;
            int64_t n = cnt ? target_neighbors(dim, src, ns, t, r, wkind, mode, gp, nbr) : 0;
            if (cols) memcpy(cols + offsets[i], nbr, sizeof(int32_t) * (size_t)n);
            status[i] = (int8_t)solve_target(dim, degree, wkind, lambda, src, ns, t, r, nbr, n,
                                             fields, nf, values + i, nt,
                                             shape ? shape + offsets[i] : NULL, &w);
        }
        work_free(&w);
    }
    if (gp) grid_free(&g);
}

/* ------------------------------------------------------------------------------------ */
/* Exact orientation (Shewchuk 1997: two-sum, Dekker product, expansion growth)          */
/* ------------------------------------------------------------------------------------ */
static void two_sum(double a, double b, double* s, double* e) {
    double x = a + b;
    double bv = x - a;
    double av = x - bv;
    double br = b - bv;
    double ar = a - av;
    *s = x;
    *e = ar + br;
}

static void split(double a, double* hi, double* lo) {
    double c = 134217729.0 * a; /* 2^27 + 1 */
    double abig = c - a;
    *hi = c - abig;
    *lo = a - *hi;
}

static void two_product(double a, double b, double* p, double* e) {
    double x = a * b;
    double ah, al, bh, bl;
    split(a, &ah, &al);
    split(b, &bh, &bl);
    double e1 = x - ah * bh;
    double e2 = e1 - al * bh;
    double e3 = e2 - ah * bl;
    *p = x;
    *e = al * bl - e3;
}

/* e[0..n-1] non-overlapping, increasing magnitude; add b exactly; returns new length */
static int grow_expansion(double* e, int n, double b) {
    double q = b;
    for (int i = 0; i < n; i++) {
        double s, h;
        two_sum(q, e[i], &s, &h);
        e[i] = h;
        q = s;
    }
    e[n] = q;
    return n + 1;
}

/* sign of (ax-cx)(by-cy) - (ay-cy)(bx-cx), exactly: +1 left turn (CCW), -1, or 0 */
int orc_orient2d_sign(double ax, double ay, double bx, double by, double cx, double cy) {
    /* = ax*by - ax*cy - bx*ay + bx*cy + cx*ay - cx*by */
    double pa[6] = {ax, -ax, -bx, bx, cx, -cx};
    double pb[6] = {by, cy, ay, cy, ay, by};
    double e[16];
    int n = 0;
    for (int k = 0; k < 6; k++) {
        double p, err;
        two_product(pa[k], pb[k], &p, &err);
        n = grow_expansion(e, n, err);
        n = grow_expansion(e, n, p);
    }
    for (int i = n - 1; i >= 0; i--) {
        if (e[i] > 0.0) return 1;
        if (e[i] < 0.0) return -1;
    }
    return 0;
}

void orc_orient2d_sign_batch(int64_t n, const double* a, const double* b, const double* c,
                             int8_t* out) {
    /* a, b, c: [2][n] */
    for (int64_t i = 0; i < n; i++)
        out[i] = (int8_t)orc_orient2d_sign(a[i], a[n + i], b[i], b[n + i], c[i], c[n + i]);
}

/* plain FP64 signed double area, the fixed formula used for barycentric coordinates */
static double orient_fp(double ax, double ay, double bx, double by, double cx, double cy) {
    return (ax - cx) * (by - cy) - (ay - cy) * (bx - cx);
}

/* ------------------------------------------------------------------------------------ */
/* Point localization + barycentric interpolation (Sec. 3.3)                            */
/* ------------------------------------------------------------------------------------ */
/* closure test by exact signs; returns 1 if p is in the closed triangle and sets the
 * number of zero signs; degenerate (zero-area) triangles contain nothing */
static int tri_contains(const double* xy, int64_t nv, const int32_t* tri, int64_t ntri,
                        int64_t k, double px, double py, int* nzero) {
    int32_t i0 = tri[k], i1 = tri[ntri + k], i2 = tri[2 * ntri + k];
    double x0 = xy[i0], y0 = xy[nv + i0];
    double x1 = xy[i1], y1 = xy[nv + i1];
    double x2 = xy[i2], y2 = xy[nv + i2];
    int area = orc_orient2d_sign(x0, y0, x1, y1, x2, y2);
    if (area == 0) return 0;
    int o0 = orc_orient2d_sign(x1, y1, x2, y2, px, py);
    int o1 = orc_orient2d_sign(x2, y2, x0, y0, px, py);
    int o2 = orc_orient2d_sign(x0, y0, x1, y1, px, py);
    if (o0 * area < 0 || o1 * area < 0 || o2 * area < 0) return 0;
    *nzero = (o0 == 0) + (o1 == 0) + (o2 == 0);
    return 1;
}

static void interp(const double* xy, int64_t nv, const int32_t* tri, int64_t ntri, int64_t k,
                   double px, double py, const double* field, double* val) {
    int32_t i0 = tri[k], i1 = tri[ntri + k], i2 = tri[2 * ntri + k];
    double x0 = xy[i0], y0 = xy[nv + i0];
    double x1 = xy[i1], y1 = xy[nv + i1];
    double x2 = xy[i2], y2 = xy[nv + i2];
    double area = orient_fp(x0, y0, x1, y1, x2, y2);
    double l0 = orient_fp(px, py, x1, y1, x2, y2) / area;
    double l1 = orient_fp(x0, y0, px, py, x2, y2) / area;
    double l2 = 1.0 - l0 - l1;
    *val = l0 * field[i0] + l1 * field[i1] + l2 * field[i2];
}

/* mode 0: exhaustive over all triangles in ascending id (a bounding-box test first, which
 * only skips triangles that cannot contain the point); mode 1: uniform grid of triangle
 * bounding boxes, candidates in ascending id. elem[q] = smallest containing id or -1;
 * dimc[q] = dimension of the lowest-order entity (0 vertex, 1 edge, 2 face), -1 outside;
 * vals[q] (if field and vals are non-NULL) = barycentric value or NaN outside. */
void orc_locate(const double* xy, int64_t nv, const int32_t* tri, int64_t ntri,
                const double* pts, int64_t q, int mode, const double* field, int32_t* elem,
                int8_t* dimc, double* vals) {
    double* bb = (double*)malloc(sizeof(double) * 4 * (size_t)(ntri > 0 ? ntri : 1));
    double glo[2] = {INFINITY, INFINITY}, ghi[2] = {-INFINITY, -INFINITY};
    for (int64_t k = 0; k < ntri; k++) {
        double lo[2] = {INFINITY, INFINITY}, hi[2] = {-INFINITY, -INFINITY};
        for (int c = 0; c < 3; c++) {
            int32_t v = tri[c * ntri + k];
            for (int d = 0; d < 2; d++) {
                double x = xy[d * nv + v];
                if (x < lo[d]) lo[d] = x;
                if (x > hi[d]) hi[d] = x;
            }
        }
        bb[4 * k + 0] = lo[0]; bb[4 * k + 1] = lo[1];
        bb[4 * k + 2] = hi[0]; bb[4 * k + 3] = hi[1];
        for (int d = 0; d < 2; d++) {
            if (lo[d] < glo[d]) glo[d] = lo[d];
            if (hi[d] > ghi[d]) ghi[d] = hi[d];
        }
    }
    /* grid for mode 1 */
    int64_t gn[2] = {1, 1};
    double gh = 1.0;
    int64_t *gstart = NULL, *gitem = NULL;
    if (mode == 1 && ntri > 0) {
        double ex = ghi[0] - glo[0], ey = ghi[1] - glo[1];
        gh = sqrt((ex * ey > 0 ? ex * ey : 1.0) / ((double)ntri / 2.0 + 1.0));
        if (!(gh > 0)) gh = 1.0;
        gn[0] = (int64_t)floor(ex / gh) + 1;
        gn[1] = (int64_t)floor(ey / gh) + 1;
        int64_t nc = gn[0] * gn[1];
        gstart = (int64_t*)calloc((size_t)nc + 1, sizeof(int64_t));
        for (int pass = 0; pass < 2; pass++) {
            int64_t* fill = NULL;
            if (pass == 1) {
                for (int64_t c = 0; c < nc; c++) gstart[c + 1] += gstart[c];
                gitem = (int64_t*)malloc(sizeof(int64_t) * (size_t)(gstart[nc] + 1));
                fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)nc);
                memcpy(fill, gstart, sizeof(int64_t) * (size_t)nc);
            }
            for (int64_t k = 0; k < ntri; k++) {
                int64_t x0 = cell_coord(bb[4 * k + 0], glo[0], gh, gn[0]);
                int64_t y0 = cell_coord(bb[4 * k + 1], glo[1], gh, gn[1]);
                int64_t x1 = cell_coord(bb[4 * k + 2], glo[0], gh, gn[0]);
                int64_t y1 = cell_coord(bb[4 * k + 3], glo[1], gh, gn[1]);
                for (int64_t cy = y0; cy <= y1; cy++)
                    for (int64_t cx = x0; cx <= x1; cx++) {
                        int64_t c = cx + gn[0] * cy;
                        if (pass == 0) gstart[c + 1]++;
                        else gitem[fill[c]++] = k;
                    }
            }
            free(fill);
        }
    }
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < q; i++) {
        double px = pts[i], py = pts[q + i];
        int32_t found = -1;
        int nz = 0;
        if (ntri > 0 && px >= glo[0] && px <= ghi[0] && py >= glo[1] && py <= ghi[1]) {
            if (mode == 1) {
                int64_t c = cell_coord(px, glo[0], gh, gn[0]) +
                            gn[0] * cell_coord(py, glo[1], gh, gn[1]);
                for (int64_t p = gstart[c]; p < gstart[c + 1]; p++) {
                    int64_t k = gitem[p];
                    if (px < bb[4 * k] || px > bb[4 * k + 2] || py < bb[4 * k + 1] ||
                        py > bb[4 * k + 3])
                        continue;
                    if (tri_contains(xy, nv, tri, ntri, k, px, py, &nz)) { found = (int32_t)k; break; }
                }
            } else {
                for (int64_t k = 0; k < ntri; k++) {
                    if (px < bb[4 * k] || px > bb[4 * k + 2] || py < bb[4 * k + 1] ||
                        py > bb[4 * k + 3])
                        continue;
                    if (tri_contains(xy, nv, tri, ntri, k, px, py, &nz)) { found = (int32_t)k; break; }
                }
            }
        }
        elem[i] = found;
        if (dimc) dimc[i] = (int8_t)(found < 0 ? -1 : 2 - nz);
        if (field && vals) {
            if (found < 0) vals[i] = NAN;
            else interp(xy, nv, tri, ntri, found, px, py, field, &vals[i]);
        }
    }
    free(bb);
    free(gstart);
    free(gitem);
}
