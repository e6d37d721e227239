/*
 * mgard_oracle.c -- plain, slow FP64 CPU oracle of the multilevel L2
 * decomposition / recomposition of a structured 1D-3D grid
 * (Chen et al., "Accelerating Multigrid-based Hierarchical Scientific Data
 * Refactoring on GPUs", Section II-A, Eq. 1 and Eq. 2).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference for the
 * CUDA library: only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark may load it.  It shares no code, header, table or helper
 * with the GPU path.
 *
 * Everything is written the way the method is defined, level by level, with
 * no blocking or fusion:
 *   - the level-l nodal values are copied out of the full array (index stride
 *     2^(L-l)) into a compact level array,
 *   - coefficients c = v - Pi_{l-1} v on N_l \ N_{l-1} by multilinear
 *     interpolation from the N_{l-1} corners (Section II-A-1, Fig. 2),
 *   - load vector f = (R M_l) C one dimension at a time, C = c embedded with
 *     zeros on N_{l-1} (Section II-A-2: f_{l-1} = R_l M_l vec(C_l)),
 *   - correction z solves M_{l-1} z = f, one tridiagonal Thomas solve per line
 *     and dimension (Section III-A-3),
 *   - v(N_{l-1}) += z, coefficients stored in place (Fig. 3 layout).
 *
 * Readings of the paper used here:
 *   - M is the P1 mass matrix scaled by 6: M_ii = 2(h_{i-1}+h_i) with
 *     h_{-1} = h_{n-1} = 0, M_{i,i+1} = h_i (Section III-A-2 matrix M).
 *   - The transfer matrix R is the transpose of the multilinear prolongation
 *     P (the variational statement of Section II-A-2 forces R = P^T; the
 *     printed R and "mass-trans" K entries are not used).
 *   - Dimensions are processed fastest-varying first (Section II-A, the
 *     "prescribed order"; the result does not depend on it in exact
 *     arithmetic).
 *   - Per-dimension level counts (the *_per_dim entry points; the paper runs
 *     equal sides only, Section IV): dimension k coarsens in the first L_k
 *     steps from the finest level and keeps all its nodes after that, so a
 *     short side stops early while the others go on (L = max_k L_k levels).
 *     A dimension that does not coarsen in a step has P = I there: its nodes
 *     are all "coarse", its interpolation is the identity and its factor of
 *     the load vector is M alone, which the tensor-product solve with the
 *     same M then undoes (the spaces stay nested tensor products, so Eq. 1-2
 *     hold unchanged).  With every L_k = L this is exactly the plain map.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXD 3

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2 };

typedef struct {
    int d;              /* number of dimensions */
    long n[ORC_MAXD];   /* nodes per dimension, slowest first */
} shape_t;

static long shape_size(const shape_t *s)
{
    long t = 1;
    for (int k = 0; k < s->d; ++k) t *= s->n[k];
    return t;
}

/* ------------------------------------------------------------------------ */
/* One-dimensional line operators.  x holds the coordinates of the nodes of  */
/* the line at the level the operator acts on.                               */
/* ------------------------------------------------------------------------ */

/* out = M in, M the 6x-scaled P1 mass matrix on nodes x[0..n-1]. */
static void line_mass(long n, const double *x, const double *in, double *out)
{
    for (long i = 0; i < n; ++i) {
        double hl = (i > 0) ? x[i] - x[i - 1] : 0.0;
        double hr = (i < n - 1) ? x[i + 1] - x[i] : 0.0;
        double s = 2.0 * (hl + hr) * in[i];
        if (i > 0) s += hl * in[i - 1];
        if (i < n - 1) s += hr * in[i + 1];
        out[i] = s;
    }
}

/* Weights of linear interpolation at the odd fine node j from its two coarse
 * neighbours j-1 and j+1 (fine coordinates xf). */
static void interp_weights(const double *xf, long j, double *wl, double *wr)
{
    double span = xf[j + 1] - xf[j - 1];
    *wl = (xf[j + 1] - xf[j]) / span;
    *wr = (xf[j] - xf[j - 1]) / span;
}

/* out (nf) = P in (nc): prolongation from the coarse nodes (even fine
 * indices) to all nf = 2 nc - 1 fine nodes. */
static void line_prolong(long nf, const double *xf, const double *in, double *out)
{
    for (long j = 0; j < nf; ++j) {
        if (j % 2 == 0) {
            out[j] = in[j / 2];
        } else {
            double wl, wr;
            interp_weights(xf, j, &wl, &wr);
            out[j] = wl * in[(j - 1) / 2] + wr * in[(j + 1) / 2];
        }
    }
}

/* out (nc) = P^T in (nf): the transfer (restriction) matrix R = P^T. */
static void line_restrict(long nf, const double *xf, const double *in, double *out)
{
    long nc = (nf + 1) / 2;
    for (long i = 0; i < nc; ++i) out[i] = in[2 * i];
    for (long j = 1; j < nf; j += 2) {
        double wl, wr;
        interp_weights(xf, j, &wl, &wr);
        out[(j - 1) / 2] += wl * in[j];
        out[(j + 1) / 2] += wr * in[j];
    }
}

/* Solve M z = f on nodes x[0..n-1] with the textbook Thomas algorithm
 * (forward elimination, back substitution). */
static int line_mass_solve(long n, const double *x, const double *f, double *z)
{
    if (n < 1) return ORC_EINVAL;
    double *cp = (double *)malloc(sizeof(double) * (size_t)n);
    double *dp = (double *)malloc(sizeof(double) * (size_t)n);
    if (!cp || !dp) { free(cp); free(dp); return ORC_ENOMEM; }
    for (long i = 0; i < n; ++i) {
        double hl = (i > 0) ? x[i] - x[i - 1] : 0.0;
        double hr = (i < n - 1) ? x[i + 1] - x[i] : 0.0;
        double a = hl;              /* sub-diagonal   M_{i,i-1} */
        double b = 2.0 * (hl + hr); /* diagonal       M_{i,i}   */
        double c = hr;              /* super-diagonal M_{i,i+1} */
        if (i == 0) {
            cp[0] = c / b;
            dp[0] = f[0] / b;
        } else {
            double den = b - a * cp[i - 1];
            cp[i] = c / den;
            dp[i] = (f[i] - a * dp[i - 1]) / den;
        }
    }
    z[n - 1] = dp[n - 1];
    for (long i = n - 2; i >= 0; --i) z[i] = dp[i] - cp[i] * z[i + 1];
    free(cp);
    free(dp);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Applying a line operator along one dimension of a compact array.          */
/* ------------------------------------------------------------------------ */

enum { OP_MASS, OP_PROLONG, OP_RESTRICT, OP_SOLVE };

/* out (shape s with n[k] replaced by nout) = op applied to every line of
 * `in` (shape s) along dimension k.  x: coordinates used by the operator. */
static int apply_along(const shape_t *s, int k, long nout, int op, const double *x,
                       const double *in, double *out)
{
    long outer = 1, inner = 1;
    for (int q = 0; q < k; ++q) outer *= s->n[q];
    for (int q = k + 1; q < s->d; ++q) inner *= s->n[q];
    long nin = s->n[k];
    double *lin = (double *)malloc(sizeof(double) * (size_t)nin);
    double *lout = (double *)malloc(sizeof(double) * (size_t)nout);
    if (!lin || !lout) { free(lin); free(lout); return ORC_ENOMEM; }
    int rc = ORC_OK;
    for (long o = 0; o < outer && rc == ORC_OK; ++o) {
        for (long i = 0; i < inner; ++i) {
            for (long j = 0; j < nin; ++j) lin[j] = in[(o * nin + j) * inner + i];
            switch (op) {
            case OP_MASS: line_mass(nin, x, lin, lout); break;
            case OP_PROLONG: line_prolong(nout, x, lin, lout); break;
            case OP_RESTRICT: line_restrict(nin, x, lin, lout); break;
            default: rc = line_mass_solve(nin, x, lin, lout); break;
            }
            if (rc != ORC_OK) break;
            for (long j = 0; j < nout; ++j) out[(o * nout + j) * inner + i] = lout[j];
        }
    }
    free(lin);
    free(lout);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Level geometry                                                            */
/* ------------------------------------------------------------------------ */

typedef struct {
    shape_t fine;                 /* level-l nodes N_l                     */
    shape_t coarse;               /* level-(l-1) nodes N_{l-1}             */
    double *xf[ORC_MAXD];         /* coordinates of N_l per dimension      */
    double *xc[ORC_MAXD];         /* coordinates of N_{l-1} per dimension  */
    long stride[ORC_MAXD];        /* index stride of N_l in the full array */
    int coarsen[ORC_MAXD];        /* 1: the dimension coarsens in this step */
} level_t;

static void level_free(level_t *lv)
{
    for (int k = 0; k < ORC_MAXD; ++k) { free(lv->xf[k]); free(lv->xc[k]); lv->xf[k] = lv->xc[k] = NULL; }
}

/* Build level l (1 <= l <= L) of a grid with full shape s and coordinates x;
 * dimension k coarsens in the first Lk[k] steps from the finest level. */
static int level_make(const shape_t *s, const double *const *x, const int *Lk, int L, int l, level_t *lv)
{
    memset(lv, 0, sizeof(*lv));
    const int step = L - l;   /* steps taken from the finest level */
    lv->fine.d = lv->coarse.d = s->d;
    for (int k = 0; k < s->d; ++k) {
        lv->coarsen[k] = step < Lk[k];
        lv->stride[k] = 1L << (step < Lk[k] ? step : Lk[k]);
        long nf = (s->n[k] - 1) / lv->stride[k] + 1;
        long nc = lv->coarsen[k] ? (nf - 1) / 2 + 1 : nf;
        long cs = lv->coarsen[k] ? 2 : 1;
        lv->fine.n[k] = nf;
        lv->coarse.n[k] = nc;
        lv->xf[k] = (double *)malloc(sizeof(double) * (size_t)nf);
        lv->xc[k] = (double *)malloc(sizeof(double) * (size_t)nc);
        if (!lv->xf[k] || !lv->xc[k]) { level_free(lv); return ORC_ENOMEM; }
        for (long i = 0; i < nf; ++i) lv->xf[k][i] = x[k][i * lv->stride[k]];
        for (long i = 0; i < nc; ++i) lv->xc[k][i] = lv->xf[k][cs * i];
    }
    return ORC_OK;
}

/* Multi-index helpers for a compact array of shape s. */
static void unravel(const shape_t *s, long idx, long *ix)
{
    for (int k = s->d - 1; k >= 0; --k) { ix[k] = idx % s->n[k]; idx /= s->n[k]; }
}

static long ravel(const shape_t *s, const long *ix)
{
    long idx = 0;
    for (int k = 0; k < s->d; ++k) idx = idx * s->n[k] + ix[k];
    return idx;
}

/* Is level index i of dimension k on the coarse grid of the step? */
static int coarse_in_dim(const level_t *lv, int k, long i)
{
    return !lv->coarsen[k] || i % 2 == 0;
}

/* Is the level-l node ix in N_{l-1}? */
static int is_coarse(const level_t *lv, const long *ix)
{
    for (int k = 0; k < lv->fine.d; ++k) if (!coarse_in_dim(lv, k, ix[k])) return 0;
    return 1;
}

/* Index in the coarse array of a node of N_{l-1} given by its level index. */
static long coarse_at(const level_t *lv, const long *ix)
{
    long cx[ORC_MAXD];
    for (int k = 0; k < lv->fine.d; ++k) cx[k] = lv->coarsen[k] ? ix[k] / 2 : ix[k];
    return ravel(&lv->coarse, cx);
}

/* Copy the level-l nodes (index strides lv->stride) between u and v. */
static void level_gather(const shape_t *full, const level_t *lv, const double *u, double *v)
{
    long m = shape_size(&lv->fine), ix[ORC_MAXD], gx[ORC_MAXD];
    for (long i = 0; i < m; ++i) {
        unravel(&lv->fine, i, ix);
        for (int k = 0; k < full->d; ++k) gx[k] = ix[k] * lv->stride[k];
        v[i] = u[ravel(full, gx)];
    }
}

static void level_scatter(const shape_t *full, const level_t *lv, const double *v, double *u)
{
    long m = shape_size(&lv->fine), ix[ORC_MAXD], gx[ORC_MAXD];
    for (long i = 0; i < m; ++i) {
        unravel(&lv->fine, i, ix);
        for (int k = 0; k < full->d; ++k) gx[k] = ix[k] * lv->stride[k];
        u[ravel(full, gx)] = v[i];
    }
}

/* Multilinear interpolant Pi_{l-1} v at the level-l node ix, using only the
 * N_{l-1} corners (even indices) of the level array v. */
static double interp_at(const level_t *lv, const double *v, const long *ix)
{
    const shape_t *s = &lv->fine;
    int d = s->d;
    double total = 0.0;
    for (int combo = 0; combo < (1 << d); ++combo) {
        long cx[ORC_MAXD];
        double w = 1.0;
        int skip = 0;
        for (int k = 0; k < d; ++k) {
            int right = (combo >> k) & 1;
            if (coarse_in_dim(lv, k, ix[k])) {
                if (right) { skip = 1; break; }   /* even dimension: one corner */
                cx[k] = ix[k];
            } else {
                double wl, wr;
                interp_weights(lv->xf[k], ix[k], &wl, &wr);
                cx[k] = right ? ix[k] + 1 : ix[k] - 1;
                w *= right ? wr : wl;
            }
        }
        if (skip) continue;
        total += w * v[ravel(s, cx)];
    }
    return total;
}

/* Tensor-product application of the mass-then-transfer operator R M_l along
 * every dimension, fastest first: f (coarse shape) = (x)_k (P_k^T M_k) C. */
static int load_vector(const level_t *lv, const double *C, double *f)
{
    shape_t cur = lv->fine;
    long cap = shape_size(&lv->fine);
    double *a = (double *)malloc(sizeof(double) * (size_t)cap);
    double *b = (double *)malloc(sizeof(double) * (size_t)cap);
    if (!a || !b) { free(a); free(b); return ORC_ENOMEM; }
    memcpy(a, C, sizeof(double) * (size_t)cap);
    int rc = ORC_OK;
    for (int k = cur.d - 1; k >= 0 && rc == ORC_OK; --k) {
        rc = apply_along(&cur, k, cur.n[k], OP_MASS, lv->xf[k], a, b);
        if (rc != ORC_OK) break;
        if (lv->coarsen[k])
            rc = apply_along(&cur, k, lv->coarse.n[k], OP_RESTRICT, lv->xf[k], b, a);
        else  /* P = I along a dimension that does not coarsen */
            memcpy(a, b, sizeof(double) * (size_t)shape_size(&cur));
        cur.n[k] = lv->coarse.n[k];
    }
    if (rc == ORC_OK) memcpy(f, a, sizeof(double) * (size_t)shape_size(&lv->coarse));
    free(a);
    free(b);
    return rc;
}

/* In place: z = M_{l-1}^{-1} f, one dimension at a time, fastest first. */
static int coarse_solve(const level_t *lv, double *f)
{
    long m = shape_size(&lv->coarse);
    double *t = (double *)malloc(sizeof(double) * (size_t)m);
    if (!t) return ORC_ENOMEM;
    int rc = ORC_OK;
    for (int k = lv->coarse.d - 1; k >= 0 && rc == ORC_OK; --k) {
        rc = apply_along(&lv->coarse, k, lv->coarse.n[k], OP_SOLVE, lv->xc[k], f, t);
        if (rc == ORC_OK) memcpy(f, t, sizeof(double) * (size_t)m);
    }
    free(t);
    return rc;
}

/* In place: C (fine shape) = (x)_k (M_k P_k) z, z of coarse shape, fastest
 * first (prolongate then apply the fine mass matrix along each dimension). */
static int mass_prolong(const level_t *lv, const double *z, double *C)
{
    shape_t cur = lv->coarse;
    long cap = shape_size(&lv->fine);
    double *a = (double *)malloc(sizeof(double) * (size_t)cap);
    double *b = (double *)malloc(sizeof(double) * (size_t)cap);
    if (!a || !b) { free(a); free(b); return ORC_ENOMEM; }
    memcpy(a, z, sizeof(double) * (size_t)shape_size(&lv->coarse));
    int rc = ORC_OK;
    for (int k = cur.d - 1; k >= 0 && rc == ORC_OK; --k) {
        if (lv->coarsen[k])
            rc = apply_along(&cur, k, lv->fine.n[k], OP_PROLONG, lv->xf[k], a, b);
        else  /* P = I along a dimension that does not coarsen */
            memcpy(b, a, sizeof(double) * (size_t)shape_size(&cur));
        cur.n[k] = lv->fine.n[k];
        if (rc != ORC_OK) break;
        rc = apply_along(&cur, k, cur.n[k], OP_MASS, lv->xf[k], b, a);
    }
    if (rc == ORC_OK) memcpy(C, a, sizeof(double) * (size_t)cap);
    free(a);
    free(b);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* One level of the forward and inverse maps on a compact level array v.     */
/* ------------------------------------------------------------------------ */

/* Decomposition step l -> l-1 (Eq. 1): v holds Q_l u on N_l on entry; on
 * exit the odd nodes hold the coefficients (I - Pi_{l-1}) Q_l u and the even
 * nodes hold Q_{l-1} u, i.e. the unchanged coarse values plus the
 * correction z (Eq. 2). */
static int level_decompose(const level_t *lv, double *v)
{
    long m = shape_size(&lv->fine), mc = shape_size(&lv->coarse);
    long ix[ORC_MAXD];
    double *C = (double *)calloc((size_t)m, sizeof(double));
    double *f = (double *)malloc(sizeof(double) * (size_t)mc);
    if (!C || !f) { free(C); free(f); return ORC_ENOMEM; }
    for (long i = 0; i < m; ++i) {
        unravel(&lv->fine, i, ix);
        C[i] = is_coarse(lv, ix) ? 0.0 : v[i] - interp_at(lv, v, ix);
    }
    int rc = load_vector(lv, C, f);
    if (rc == ORC_OK) rc = coarse_solve(lv, f);
    if (rc == ORC_OK) {
        for (long i = 0; i < m; ++i) {
            unravel(&lv->fine, i, ix);
            if (is_coarse(lv, ix)) {
                v[i] += f[coarse_at(lv, ix)];
            } else {
                v[i] = C[i];
            }
        }
    }
    free(C);
    free(f);
    return rc;
}

/* Recomposition step l-1 -> l: exact inverse of level_decompose. */
static int level_recompose(const level_t *lv, double *v)
{
    long m = shape_size(&lv->fine), mc = shape_size(&lv->coarse);
    long ix[ORC_MAXD];
    double *C = (double *)calloc((size_t)m, sizeof(double));
    double *f = (double *)malloc(sizeof(double) * (size_t)mc);
    if (!C || !f) { free(C); free(f); return ORC_ENOMEM; }
    for (long i = 0; i < m; ++i) {
        unravel(&lv->fine, i, ix);
        C[i] = is_coarse(lv, ix) ? 0.0 : v[i];
    }
    int rc = load_vector(lv, C, f);
    if (rc == ORC_OK) rc = coarse_solve(lv, f);
    if (rc == ORC_OK) {
        /* coarse nodal values of Q_l u: Q_{l-1} u - z */
        for (long i = 0; i < m; ++i) {
            unravel(&lv->fine, i, ix);
            if (is_coarse(lv, ix)) {
                v[i] -= f[coarse_at(lv, ix)];
            }
        }
        /* new nodes: coefficient + interpolant of the corrected coarse values */
        for (long i = 0; i < m; ++i) {
            unravel(&lv->fine, i, ix);
            if (!is_coarse(lv, ix)) v[i] = C[i] + interp_at(lv, v, ix);
        }
    }
    free(C);
    free(f);
    return rc;
}

/* Transpose of level_decompose.  With o = odd part, e = even part, the step
 * is o' = o - Pi e, e' = e + A (o - Pi e), A = M_{l-1}^{-1} P^T M_l E_odd.
 * Its transpose: w = o_bar' + [M_l P M_{l-1}^{-1} e_bar']_odd,
 * o_bar = w, e_bar = e_bar' - Pi^T w. */
static int level_decompose_adjoint(const level_t *lv, double *v)
{
    long m = shape_size(&lv->fine), mc = shape_size(&lv->coarse);
    long ix[ORC_MAXD];
    double *z = (double *)malloc(sizeof(double) * (size_t)mc);
    double *G = (double *)malloc(sizeof(double) * (size_t)m);
    double *w = (double *)calloc((size_t)m, sizeof(double));
    if (!z || !G || !w) { free(z); free(G); free(w); return ORC_ENOMEM; }
    for (long i = 0; i < m; ++i) {
        unravel(&lv->fine, i, ix);
        if (is_coarse(lv, ix)) {
            z[coarse_at(lv, ix)] = v[i];
        }
    }
    int rc = coarse_solve(lv, z);
    if (rc == ORC_OK) rc = mass_prolong(lv, z, G);
    if (rc == ORC_OK) {
        for (long i = 0; i < m; ++i) {
            unravel(&lv->fine, i, ix);
            if (!is_coarse(lv, ix)) w[i] = v[i] + G[i];
        }
        /* e_bar = e_bar' - Pi^T w : every odd node sends its interpolation
         * weights times w back to its corners */
        for (long i = 0; i < m; ++i) {
            unravel(&lv->fine, i, ix);
            if (is_coarse(lv, ix)) continue;
            int d = lv->fine.d;
            for (int combo = 0; combo < (1 << d); ++combo) {
                long cx[ORC_MAXD];
                double wt = 1.0;
                int skip = 0;
                for (int k = 0; k < d; ++k) {
                    int right = (combo >> k) & 1;
                    if (coarse_in_dim(lv, k, ix[k])) {
                        if (right) { skip = 1; break; }
                        cx[k] = ix[k];
                    } else {
                        double wl, wr;
                        interp_weights(lv->xf[k], ix[k], &wl, &wr);
                        cx[k] = right ? ix[k] + 1 : ix[k] - 1;
                        wt *= right ? wr : wl;
                    }
                }
                if (skip) continue;
                v[ravel(&lv->fine, cx)] -= wt * w[i];
            }
        }
        for (long i = 0; i < m; ++i) {
            unravel(&lv->fine, i, ix);
            if (!is_coarse(lv, ix)) v[i] = w[i];
        }
    }
    free(z);
    free(G);
    free(w);
    return rc;
}

/* Transpose of level_recompose.  The step is e_new = e - A o,
 * o_new = o + Pi e_new.  Its transpose: e_tot = e_bar_new + Pi^T o_bar_new,
 * o_bar = o_bar_new - [M_l P M_{l-1}^{-1} e_tot]_odd, e_bar = e_tot. */
static int level_recompose_adjoint(const level_t *lv, double *v)
{
    long m = shape_size(&lv->fine), mc = shape_size(&lv->coarse);
    long ix[ORC_MAXD];
    double *z = (double *)malloc(sizeof(double) * (size_t)mc);
    double *G = (double *)malloc(sizeof(double) * (size_t)m);
    if (!z || !G) { free(z); free(G); return ORC_ENOMEM; }
    /* e_tot = e_bar_new + Pi^T o_bar_new, accumulated on the even nodes of v */
    for (long i = 0; i < m; ++i) {
        unravel(&lv->fine, i, ix);
        if (is_coarse(lv, ix)) continue;
        int d = lv->fine.d;
        for (int combo = 0; combo < (1 << d); ++combo) {
            long cx[ORC_MAXD];
            double wt = 1.0;
            int skip = 0;
            for (int k = 0; k < d; ++k) {
                int right = (combo >> k) & 1;
                if (coarse_in_dim(lv, k, ix[k])) {
                    if (right) { skip = 1; break; }
                    cx[k] = ix[k];
                } else {
                    double wl, wr;
                    interp_weights(lv->xf[k], ix[k], &wl, &wr);
                    cx[k] = right ? ix[k] + 1 : ix[k] - 1;
                    wt *= right ? wr : wl;
                }
            }
            if (skip) continue;
            v[ravel(&lv->fine, cx)] += wt * v[i];
        }
    }
    for (long i = 0; i < m; ++i) {
        unravel(&lv->fine, i, ix);
        if (is_coarse(lv, ix)) {
            z[coarse_at(lv, ix)] = v[i];
        }
    }
    int rc = coarse_solve(lv, z);
    if (rc == ORC_OK) rc = mass_prolong(lv, z, G);
    if (rc == ORC_OK) {
        for (long i = 0; i < m; ++i) {
            unravel(&lv->fine, i, ix);
            if (!is_coarse(lv, ix)) v[i] -= G[i];
        }
    }
    free(z);
    free(G);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Whole hierarchy                                                           */
/* ------------------------------------------------------------------------ */

static int check_args(int d, const long *n, const double *const *x, const int *Lk, shape_t *s)
{
    if (d < 1 || d > ORC_MAXD || !n || !x || !Lk) return ORC_EINVAL;
    s->d = d;
    for (int k = 0; k < d; ++k) {
        if (!x[k] || Lk[k] < 0 || Lk[k] > 30) return ORC_EINVAL;
        if (n[k] < 2) return ORC_EINVAL;
        if ((n[k] - 1) % (1L << Lk[k]) != 0) return ORC_EINVAL;
        s->n[k] = n[k];
    }
    return ORC_OK;
}

enum { DIR_DEC, DIR_REC, DIR_DEC_ADJ, DIR_REC_ADJ };

static int run(int d, const long *n, const double *const *x, const int *Lk, double *u, int dir)
{
    shape_t s;
    int rc = check_args(d, n, x, Lk, &s);
    if (rc != ORC_OK) return rc;
    int L = 0;
    for (int k = 0; k < d; ++k) if (Lk[k] > L) L = Lk[k];
    /* decompose and recompose-adjoint run finest first; the others coarsest first */
    int fine_first = (dir == DIR_DEC || dir == DIR_REC_ADJ);
    for (int step = 0; step < L && rc == ORC_OK; ++step) {
        int l = fine_first ? L - step : step + 1;
        level_t lv;
        rc = level_make(&s, x, Lk, L, l, &lv);
        if (rc != ORC_OK) break;
        double *v = (double *)malloc(sizeof(double) * (size_t)shape_size(&lv.fine));
        if (!v) { level_free(&lv); rc = ORC_ENOMEM; break; }
        level_gather(&s, &lv, u, v);
        switch (dir) {
        case DIR_DEC: rc = level_decompose(&lv, v); break;
        case DIR_REC: rc = level_recompose(&lv, v); break;
        case DIR_DEC_ADJ: rc = level_decompose_adjoint(&lv, v); break;
        default: rc = level_recompose_adjoint(&lv, v); break;
        }
        if (rc == ORC_OK) level_scatter(&s, &lv, v, u);
        free(v);
        level_free(&lv);
    }
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Exported entry points (called through ctypes by the tests).              */
/*   d      number of dimensions (1..3)                                     */
/*   n      nodes per dimension, slowest first; (n[k]-1) % 2^L == 0         */
/*   x      d coordinate arrays, x[k] of length n[k], strictly increasing   */
/*   L      number of levels to process (the *_per_dim forms: Lk, one       */
/*          level count per dimension)                                      */
/*   u      row-major array of prod(n) doubles, transformed in place        */
/* Return 0 on success, 1 on invalid arguments, 2 on allocation failure.    */
/* ------------------------------------------------------------------------ */

static int run_all(int d, const long *n, const double *const *x, int L, double *u, int dir)
{
    if (L < 0) return ORC_EINVAL;
    int Lk[ORC_MAXD] = {L, L, L};
    return run(d, n, x, Lk, u, dir);
}

int orc_decompose(int d, const long *n, const double *const *x, int L, double *u)
{
    return run_all(d, n, x, L, u, DIR_DEC);
}

int orc_recompose(int d, const long *n, const double *const *x, int L, double *u)
{
    return run_all(d, n, x, L, u, DIR_REC);
}

int orc_decompose_adjoint(int d, const long *n, const double *const *x, int L, double *u)
{
    return run_all(d, n, x, L, u, DIR_DEC_ADJ);
}

int orc_recompose_adjoint(int d, const long *n, const double *const *x, int L, double *u)
{
    return run_all(d, n, x, L, u, DIR_REC_ADJ);
}

/* The same maps with a level count per dimension: Lk[k] levels along
 * dimension k, (n[k]-1) % 2^Lk[k] == 0, L = max_k Lk[k] levels in all. */
int orc_decompose_per_dim(int d, const long *n, const double *const *x, const int *Lk, double *u)
{
    return run(d, n, x, Lk, u, DIR_DEC);
}

int orc_recompose_per_dim(int d, const long *n, const double *const *x, const int *Lk, double *u)
{
    return run(d, n, x, Lk, u, DIR_REC);
}

int orc_decompose_adjoint_per_dim(int d, const long *n, const double *const *x, const int *Lk, double *u)
{
    return run(d, n, x, Lk, u, DIR_DEC_ADJ);
}

int orc_recompose_adjoint_per_dim(int d, const long *n, const double *const *x, const int *Lk, double *u)
{
    return run(d, n, x, Lk, u, DIR_REC_ADJ);
}

/* Single-line operators, exported so the tests can pin them one by one. */
void orc_line_mass(long n, const double *x, const double *in, double *out)
{
    line_mass(n, x, in, out);
}

void orc_line_prolong(long nf, const double *xf, const double *in, double *out)
{
    line_prolong(nf, xf, in, out);
}

void orc_line_restrict(long nf, const double *xf, const double *in, double *out)
{
    line_restrict(nf, xf, in, out);
}

int orc_line_mass_solve(long n, const double *x, const double *f, double *z)
{
    return line_mass_solve(n, x, f, z);
}
