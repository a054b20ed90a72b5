/*
 * Plain FP64 CPU oracle for the discrete tangent-point energy and the discrete
 * Sobolev-Slobodeckij inner product of Yu, Schumacher & Crane, "Repulsive Curves"
 * (arXiv 2006.07859).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct reference that
 * the CUDA path is checked against.  Only the tests, the smoke check and the CPU
 * baseline of the benchmark may load it.  It shares no code, header or constant with
 * the CUDA library.
 *
 * Every quantity is computed literally from its definition in the paper:
 *   - edge length, unit tangent, midpoint ........ Sec. 5 "Notation"
 *   - tangent-point kernel k^alpha_beta .......... Eq. 3
 *   - discrete energy, 2x2 trapezoid kernel ...... Sec. 5.1, Eqs. 17-18
 *   - discrete differential ....................... Sec. 5.1 (partials of Eq. 17)
 *   - high-order Gram B by increments ............ Sec. 5.2.2, Eq. 21 and the increment table
 *   - low-order Gram B0 by increments ............ Sec. 5.2.3 (weight w0 and increment table)
 *   - the bilinear forms themselves .............. Eq. 21 and the B0 relation of Sec. 5.2.3
 * Pair sets are the ordered pairs (I, J) of edges that share no vertex (I cap J = empty).
 * Sums over pairs use Neumaier compensation; loops run I-major with J ascending.
 *
 * Status codes: 0 = ok, 1 = an edge of zero length (tangent undefined), 2 = bad argument.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- small helpers */

typedef struct {
    double s, c;
} orc_nsum; /* Neumaier compensated sum */

static void nsum_add(orc_nsum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

static double nsum_val(const orc_nsum *a) { return a->s + a->c; }

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void cross3(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

static void sub3(const double *a, const double *b, double *o)
{
    o[0] = a[0] - b[0];
    o[1] = a[1] - b[1];
    o[2] = a[2] - b[2];
}

/* I cap J = empty: the two edges share no vertex index (Sec. 5.1, Eq. 17). */
static int disjoint(const int *eI, const int *eJ)
{
    return eI[0] != eJ[0] && eI[0] != eJ[1] && eI[1] != eJ[0] && eI[1] != eJ[1];
}

/* Sec. 5 "Notation": l_I = |g_i1 - g_i2|, T_I = (g_i2 - g_i1)/l_I, x_I = (g_i1 + g_i2)/2. */
int orc_edge_quantities(int nV, const double *g, int nE, const int *E, double *ell, double *T, double *x)
{
    if (nV < 0 || nE < 0) return 2;
    for (int I = 0; I < nE; ++I) {
        int i1 = E[2 * I], i2 = E[2 * I + 1];
        if (i1 < 0 || i1 >= nV || i2 < 0 || i2 >= nV) return 2;
        double e[3];
        sub3(&g[3 * i2], &g[3 * i1], e);
        double l = sqrt(dot3(e, e));
        if (!(l > 0.0)) return 1;
        if (ell) ell[I] = l;
        if (T)
            for (int k = 0; k < 3; ++k) T[3 * I + k] = e[k] / l;
        if (x)
            for (int k = 0; k < 3; ++k) x[3 * I + k] = 0.5 * (g[3 * i1 + k] + g[3 * i2 + k]);
    }
    return 0;
}

/* Tangent-point kernel, Eq. 3: k(p, q, T) = |T x (p - q)|^alpha / |p - q|^beta. */
static double tp_kernel(const double *p, const double *q, const double *T, double alpha, double beta)
{
    double d[3], c[3];
    sub3(p, q, d);
    cross3(T, d, c);
    return pow(sqrt(dot3(c, c)), alpha) / pow(sqrt(dot3(d, d)), beta);
}

typedef struct {
    int nV, nE;
    const double *g;
    const int *E;
    double *ell, *T;
} orc_geom;

static int geom_init(orc_geom *G, int nV, const double *g, int nE, const int *E)
{
    G->nV = nV;
    G->nE = nE;
    G->g = g;
    G->E = E;
    G->ell = (double *)malloc(sizeof(double) * (size_t)(nE > 0 ? nE : 1));
    G->T = (double *)malloc(sizeof(double) * 3 * (size_t)(nE > 0 ? nE : 1));
    if (!G->ell || !G->T) return 2;
    return orc_edge_quantities(nV, g, nE, E, G->ell, G->T, NULL);
}

static void geom_free(orc_geom *G)
{
    free(G->ell);
    free(G->T);
}

/* Discrete kernel times lengths for one ordered pair, Eqs. 17-18:
 * E_IJ = l_I l_J * (1/4) sum_{i in I} sum_{j in J} k(g_i, g_j, T_I). */
static double pair_energy(const orc_geom *G, int I, int J, double alpha, double beta)
{
    const int *eI = &G->E[2 * I], *eJ = &G->E[2 * J];
    double s = 0.0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) s += tp_kernel(&G->g[3 * eI[a]], &G->g[3 * eJ[b]], &G->T[3 * I], alpha, beta);
    return 0.25 * s * G->ell[I] * G->ell[J];
}

/* ---------------------------------------------------------------- energy */

/* Eq. 17.  rows[I] = sum_{J disjoint from I} E_IJ (may be NULL); *total = sum_I rows[I]. */
int orc_energy(int nV, const double *g, int nE, const int *E, double alpha, double beta, double *rows,
               double *total)
{
    orc_geom G;
    int st = geom_init(&G, nV, g, nE, E);
    if (st) {
        geom_free(&G);
        return st;
    }
    double *r = (double *)malloc(sizeof(double) * (size_t)(nE > 0 ? nE : 1));
#pragma omp parallel for schedule(dynamic, 4)
    for (int I = 0; I < nE; ++I) {
        orc_nsum acc = {0.0, 0.0};
        for (int J = 0; J < nE; ++J)
            if (disjoint(&E[2 * I], &E[2 * J])) nsum_add(&acc, pair_energy(&G, I, J, alpha, beta));
        r[I] = nsum_val(&acc);
    }
    orc_nsum tot = {0.0, 0.0};
    for (int I = 0; I < nE; ++I) nsum_add(&tot, r[I]);
    if (rows) memcpy(rows, r, sizeof(double) * (size_t)nE);
    *total = nsum_val(&tot);
    free(r);
    geom_free(&G);
    return 0;
}

/* Energy rows for a subset of target edges only: rows[k] = sum_J E_{idx[k], J}. */
int orc_energy_rows(int nV, const double *g, int nE, const int *E, double alpha, double beta, int nidx,
                    const int *idx, double *rows)
{
    orc_geom G;
    int st = geom_init(&G, nV, g, nE, E);
    if (st) {
        geom_free(&G);
        return st;
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < nidx; ++k) {
        int I = idx[k];
        orc_nsum acc = {0.0, 0.0};
        for (int J = 0; J < nE; ++J)
            if (disjoint(&E[2 * I], &E[2 * J])) nsum_add(&acc, pair_energy(&G, I, J, alpha, beta));
        rows[k] = nsum_val(&acc);
    }
    geom_free(&G);
    return 0;
}

/* ---------------------------------------------------------------- differential */

/* Partial derivatives of k(p, q, T) = |c|^alpha |d|^-beta with d = p - q, c = T x d:
 *   dk/dd = alpha |c|^(alpha-2) |d|^-beta (c x T) - beta |c|^alpha |d|^(-beta-2) d
 *   dk/dT = alpha |c|^(alpha-2) |d|^-beta (d x c)
 * (d|c|^2/dd = 2 (c x T), d|c|^2/dT = 2 (d x c)).  When c = 0 the c-terms vanish for
 * alpha > 1, so they are dropped. */
static void tp_kernel_grad(const double *p, const double *q, const double *T, double alpha, double beta,
                           double *dk_dd, double *dk_dT)
{
    double d[3], c[3], cxT[3], dxc[3];
    sub3(p, q, d);
    cross3(T, d, c);
    double d2 = dot3(d, d), c2 = dot3(c, c);
    double dmb = pow(d2, -0.5 * beta);
    double f = pow(c2, 0.5 * alpha) * dmb;
    double a = (c2 > 0.0) ? alpha * pow(c2, 0.5 * alpha - 1.0) * dmb : 0.0;
    cross3(c, T, cxT);
    cross3(d, c, dxc);
    for (int k = 0; k < 3; ++k) {
        dk_dd[k] = a * cxT[k] - beta * f / d2 * d[k];
        dk_dT[k] = a * dxc[k];
    }
}

/* Accumulate d E_IJ / d gamma into out (Sec. 5.1): E_IJ = (1/4) l_I l_J sum_ab k(g_ia, g_jb, T_I).
 * Depends on g_i1, g_i2 through l_I, T_I and the points g_ia; on g_j1, g_j2 through l_J and g_jb.
 * dl_I/dg_i2 = T_I = -dl_I/dg_i1;  dT_I/dg_i2 = (Id - T T^t)/l_I = -dT_I/dg_i1.
 * If only_v >= 0, only the contribution to vertex only_v is accumulated (into out[0..2]). */
static void pair_energy_grad(const orc_geom *G, int I, int J, double alpha, double beta, double *out, int only_v)
{
    const int *eI = &G->E[2 * I], *eJ = &G->E[2 * J];
    const double *TI = &G->T[3 * I], *TJ = &G->T[3 * J];
    double lI = G->ell[I], lJ = G->ell[J];
    double K = 0.0, sumT[3] = {0, 0, 0}, gp[2][3] = {{0}}, gq[2][3] = {{0}};
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            const double *p = &G->g[3 * eI[a]], *q = &G->g[3 * eJ[b]];
            double dd[3], dT[3];
            K += tp_kernel(p, q, TI, alpha, beta);
            tp_kernel_grad(p, q, TI, alpha, beta, dd, dT);
            for (int k = 0; k < 3; ++k) {
                gp[a][k] += dd[k];  /* d/d p  = + dk/dd */
                gq[b][k] -= dd[k];  /* d/d q  = - dk/dd */
                sumT[k] += dT[k];
            }
        }
    /* (Id - T T^t) sumT / l_I */
    double tdot = dot3(TI, sumT), projT[3];
    for (int k = 0; k < 3; ++k) projT[k] = (sumT[k] - tdot * TI[k]) / lI;
    for (int a = 0; a < 2; ++a) {
        double sgn = (a == 0) ? -1.0 : 1.0; /* i1 gets the minus sign */
        int v = eI[a];
        if (only_v >= 0 && v != only_v) continue;
        double *o = (only_v >= 0) ? out : &out[3 * v];
        for (int k = 0; k < 3; ++k)
            o[k] += 0.25 * (sgn * TI[k] * lJ * K + lI * lJ * gp[a][k] + lI * lJ * sgn * projT[k]);
    }
    for (int b = 0; b < 2; ++b) {
        double sgn = (b == 0) ? -1.0 : 1.0;
        int v = eJ[b];
        if (only_v >= 0 && v != only_v) continue;
        double *o = (only_v >= 0) ? out : &out[3 * v];
        for (int k = 0; k < 3; ++k) o[k] += 0.25 * (lI * sgn * TJ[k] * K + lI * lJ * gq[b][k]);
    }
}

/* d(hat E)/d gamma in R^{3|V|}, vertex-major [nV][3] (Sec. 5.1). Serial scatter over all pairs. */
int orc_differential(int nV, const double *g, int nE, const int *E, double alpha, double beta, double *dE)
{
    orc_geom G;
    int st = geom_init(&G, nV, g, nE, E);
    if (st) {
        geom_free(&G);
        return st;
    }
    memset(dE, 0, sizeof(double) * 3 * (size_t)nV);
    for (int I = 0; I < nE; ++I)
        for (int J = 0; J < nE; ++J)
            if (disjoint(&E[2 * I], &E[2 * J])) pair_energy_grad(&G, I, J, alpha, beta, dE, -1);
    geom_free(&G);
    return 0;
}

/* The same differential at selected vertices only: every ordered pair (I, J) with v in I or v in J. */
int orc_differential_at(int nV, const double *g, int nE, const int *E, double alpha, double beta, int nidx,
                        const int *vidx, double *out)
{
    orc_geom G;
    int st = geom_init(&G, nV, g, nE, E);
    if (st) {
        geom_free(&G);
        return st;
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < nidx; ++k) {
        int v = vidx[k];
        double acc[3] = {0, 0, 0};
        /* the pairs that touch v: (X, Y) and (Y, X) for every edge X incident to v */
        for (int X = 0; X < nE; ++X) {
            if (E[2 * X] != v && E[2 * X + 1] != v) continue;
            for (int Y = 0; Y < nE; ++Y)
                if (disjoint(&E[2 * X], &E[2 * Y])) {
                    pair_energy_grad(&G, X, Y, alpha, beta, acc, v);
                    pair_energy_grad(&G, Y, X, alpha, beta, acc, v);
                }
        }
        for (int c = 0; c < 3; ++c) out[3 * k + c] = acc[c];
    }
    geom_free(&G);
    return 0;
}

/* ---------------------------------------------------------------- inner product weights */

/* Sec. 5.2.2: w_IJ = (1/4) l_I l_J sum_{i in I} sum_{j in J} |g_i - g_j|^-(2 sigma + 1).
 * Sec. 5.2.3: w0_IJ = (1/4) l_I l_J sum_i sum_j k^2_4(g_i, g_j, T_I) / |g_i - g_j|^(2 sigma + 1). */
static void pair_weights(const orc_geom *G, int I, int J, double sigma, double *w, double *w0)
{
    const int *eI = &G->E[2 * I], *eJ = &G->E[2 * J];
    double sw = 0.0, sw0 = 0.0, p = 2.0 * sigma + 1.0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            const double *gi = &G->g[3 * eI[a]], *gj = &G->g[3 * eJ[b]];
            double d[3];
            sub3(gi, gj, d);
            double r = sqrt(dot3(d, d));
            sw += 1.0 / pow(r, p);
            sw0 += tp_kernel(gi, gj, &G->T[3 * I], 2.0, 4.0) / pow(r, p);
        }
    *w = 0.25 * G->ell[I] * G->ell[J] * sw;
    *w0 = 0.25 * G->ell[I] * G->ell[J] * sw0;
}

/* The increments of Secs. 5.2.2-5.2.3 for one ordered pair, reported one at a time as
 * (row, col, value) through a callback, so that the dense build and the matrix-free
 * apply use the very same list. */
typedef void (*orc_incr_fn)(void *ctx, int row, int col, double val);

static void pair_increments(const orc_geom *G, int I, int J, double sigma, int want_B, int want_B0, orc_incr_fn fn,
                            void *ctx)
{
    const int *eI = &G->E[2 * I], *eJ = &G->E[2 * J];
    double w, w0;
    pair_weights(G, I, J, sigma, &w, &w0);
    double lI = G->ell[I], lJ = G->ell[J];
    double TIJ = dot3(&G->T[3 * I], &G->T[3 * J]);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            /* (-1)^{a+b} with a, b in {1, 2} */
            double sgn = ((a + b) % 2 == 0) ? 1.0 : -1.0;
            int ia = eI[a], ib = eI[b], ja = eJ[a], jb = eJ[b];
            if (want_B) {
                fn(ctx, ia, ib, sgn * w / (lI * lI));
                fn(ctx, ia, jb, -sgn * w * TIJ / (lI * lJ));
                fn(ctx, ja, jb, sgn * w / (lJ * lJ));
                fn(ctx, ja, ib, -sgn * w * TIJ / (lJ * lI));
            }
            if (want_B0) {
                fn(ctx, ia, ib, 0.25 * w0);
                fn(ctx, ia, jb, -0.25 * w0);
                fn(ctx, ja, ib, -0.25 * w0);
                fn(ctx, ja, jb, 0.25 * w0);
            }
        }
}

typedef struct {
    int n;
    double *M;
} dense_ctx;

static void dense_incr(void *c, int row, int col, double val)
{
    dense_ctx *d = (dense_ctx *)c;
    d->M[(size_t)row * d->n + col] += val;
}

/* Dense Gram matrices by the increment tables: B (Sec. 5.2.2) and B0 (Sec. 5.2.3), row-major nV x nV.
 * Either output may be NULL. */
int orc_gram_dense(int nV, const double *g, int nE, const int *E, double sigma, double *B, double *B0)
{
    orc_geom G;
    int st = geom_init(&G, nV, g, nE, E);
    if (st) {
        geom_free(&G);
        return st;
    }
    dense_ctx cb = {nV, B}, cb0 = {nV, B0};
    if (B) memset(B, 0, sizeof(double) * (size_t)nV * nV);
    if (B0) memset(B0, 0, sizeof(double) * (size_t)nV * nV);
    for (int I = 0; I < nE; ++I)
        for (int J = 0; J < nE; ++J)
            if (disjoint(&E[2 * I], &E[2 * J])) {
                if (B) pair_increments(&G, I, J, sigma, 1, 0, dense_incr, &cb);
                if (B0) pair_increments(&G, I, J, sigma, 0, 1, dense_incr, &cb0);
            }
    geom_free(&G);
    return 0;
}

typedef struct {
    const double *u; /* [nV][m] */
    double *out;     /* [nV][m] */
    int m;
    int only_row;    /* -1: all rows */
} apply_ctx;

static void apply_incr(void *c, int row, int col, double val)
{
    apply_ctx *a = (apply_ctx *)c;
    if (a->only_row >= 0 && row != a->only_row) return;
    double *o = (a->only_row >= 0) ? a->out : &a->out[(size_t)row * a->m];
    for (int k = 0; k < a->m; ++k) o[k] += val * a->u[(size_t)col * a->m + k];
}

/* Matrix-free (B + B0) u for u with m columns (vertex-major [nV][m]), applying the same
 * increments as orc_gram_dense directly to u.  Serial. */
int orc_gram_apply(int nV, const double *g, int nE, const int *E, double sigma, int m, const double *u, double *out)
{
    orc_geom G;
    int st = geom_init(&G, nV, g, nE, E);
    if (st) {
        geom_free(&G);
        return st;
    }
    memset(out, 0, sizeof(double) * (size_t)nV * m);
    apply_ctx ac = {u, out, m, -1};
    for (int I = 0; I < nE; ++I)
        for (int J = 0; J < nE; ++J)
            if (disjoint(&E[2 * I], &E[2 * J])) pair_increments(&G, I, J, sigma, 1, 1, apply_incr, &ac);
    geom_free(&G);
    return 0;
}

/* Rows of (B + B0) u at selected vertices: only the increments whose row is v. */
int orc_gram_apply_at(int nV, const double *g, int nE, const int *E, double sigma, int m, const double *u, int nidx,
                      const int *vidx, double *out)
{
    orc_geom G;
    int st = geom_init(&G, nV, g, nE, E);
    if (st) {
        geom_free(&G);
        return st;
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < nidx; ++k) {
        int v = vidx[k];
        apply_ctx ac = {u, &out[(size_t)k * m], m, v};
        for (int c = 0; c < m; ++c) out[(size_t)k * m + c] = 0.0;
        /* increments with row v come from the ordered pairs (X, Y) and (Y, X), X incident to v */
        for (int X = 0; X < nE; ++X) {
            if (E[2 * X] != v && E[2 * X + 1] != v) continue;
            for (int Y = 0; Y < nE; ++Y)
                if (disjoint(&E[2 * X], &E[2 * Y])) {
                    pair_increments(&G, X, Y, sigma, 1, 1, apply_incr, &ac);
                    pair_increments(&G, Y, X, sigma, 1, 1, apply_incr, &ac);
                }
        }
    }
    geom_free(&G);
    return 0;
}

/* The bilinear forms themselves, for scalar vertex functions u, v:
 *   u^T B v  = sum_{I,J disjoint} w_IJ < D_I u[I] - D_J u[J], D_I v[I] - D_J v[J] >   (Eq. 21)
 *   u^T B0 v = sum_{I,J disjoint} w0_IJ (u_I - u_J)(v_I - v_J)                          (Sec. 5.2.3)
 * with D_I u[I] = (u_i2 - u_i1)/l_I T_I (Sec. 5.2.1) and u_I = (u_i1 + u_i2)/2 (Sec. 5 "Notation"). */
int orc_bilinear(int nV, const double *g, int nE, const int *E, double sigma, const double *u, const double *v,
                 double *uBv, double *uB0v)
{
    orc_geom G;
    int st = geom_init(&G, nV, g, nE, E);
    if (st) {
        geom_free(&G);
        return st;
    }
    orc_nsum sb = {0, 0}, sb0 = {0, 0};
    for (int I = 0; I < nE; ++I)
        for (int J = 0; J < nE; ++J) {
            if (!disjoint(&E[2 * I], &E[2 * J])) continue;
            double w, w0;
            pair_weights(&G, I, J, sigma, &w, &w0);
            const int *eI = &E[2 * I], *eJ = &E[2 * J];
            const double *TI = &G.T[3 * I], *TJ = &G.T[3 * J];
            double Du[3], Dv[3];
            for (int k = 0; k < 3; ++k) {
                Du[k] = (u[eI[1]] - u[eI[0]]) / G.ell[I] * TI[k] - (u[eJ[1]] - u[eJ[0]]) / G.ell[J] * TJ[k];
                Dv[k] = (v[eI[1]] - v[eI[0]]) / G.ell[I] * TI[k] - (v[eJ[1]] - v[eJ[0]]) / G.ell[J] * TJ[k];
            }
            nsum_add(&sb, w * dot3(Du, Dv));
            double uI = 0.5 * (u[eI[0]] + u[eI[1]]), uJ = 0.5 * (u[eJ[0]] + u[eJ[1]]);
            double vI = 0.5 * (v[eI[0]] + v[eI[1]]), vJ = 0.5 * (v[eJ[0]] + v[eJ[1]]);
            nsum_add(&sb0, w0 * (uI - uJ) * (vI - vJ));
        }
    *uBv = nsum_val(&sb);
    *uB0v = nsum_val(&sb0);
    geom_free(&G);
    return 0;
}

/* Number of threads the OpenMP loops above use (1 without OpenMP). */
int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
