/*
 * tpe.h - C ABI of the GB300 (sm_103a) tangent-point energy / H^s descent library.
 *
 * Method: Yu, Schumacher & Crane, "Repulsive Curves" (arXiv 2006.07859).  A curve network
 * is a graph G = (V, E) with vertex positions gamma (Sec. 5 "Notation").  The library
 * evaluates, on one GPU,
 *   - the discrete tangent-point energy hat-E over ordered pairs of edges that share no
 *     vertex, with the 2x2 trapezoid kernel (Sec. 5.1, Eqs. 17-18, kernel of Eq. 3);
 *   - its differential d hat-E (Sec. 5.1);
 *   - the matrix-free product with A-bar = diag(A, A, A), A = B + B0 (Secs. 5.2-5.2.3, Eq. 19);
 *   - the projected H^s gradient g~ of Eq. 22, solved as P A-bar P y = P dE, g~ = P y (App. B.3.3);
 *   - one descent step with normalised gradient, backtracking from tau = 1 and constraint
 *     projection (Secs. 5.3.2 and 5.4, App. B.3.4).
 * Constraints are those of Sec. 8.1: the barycenter with either the total length or every edge length,
 * or the total length with pinned vertices, tangents and surface points (tp_params.constraint_set).
 *
 * Conventions shared by every entry point
 *   - Vertex arrays (gamma, dE, u, ...) are DEVICE pointers to double, vertex-major [nV][3].
 *   - Per-problem outputs (energies) are DEVICE pointers to double [n_problems].
 *   - Every call is enqueued on `stream` (a cudaStream_t; NULL = legacy default stream) and is
 *     asynchronous unless it says otherwise.  Calls that return host-side info structs
 *     synchronise the stream before returning.
 *   - The caller owns every pointer it passes; the context owns its own scratch memory,
 *     allocated once in tp_create and sized for the graph it was created with.  Only
 *     tp_set_params (switching a preconditioner, a constraint set or the line search on),
 *     tp_autotune (a larger work queue), the first tp_set_penalties, the first tp_set_pins,
 *     tp_set_tangents or tp_set_surface (and one that needs more solves than any before) and the
 *     first tp_collision_time allocate device memory after tp_create.
 *   - Every call returns a tp_status; nothing aborts or traps.  tp_last_error() gives a
 *     human-readable message for the last failing call on a context.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef TPE_H
#define TPE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TPE_API __attribute__((visibility("default")))
#else
#define TPE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st *tp_stream; /* same type as cudaStream_t */

typedef enum {
    TP_OK = 0,
    TP_ERR_INVALID_ARG = 1,     /* bad size, index, null pointer or parameter */
    TP_ERR_CUDA = 2,            /* a CUDA runtime call failed (message in tp_last_error) */
    TP_ERR_DEGENERATE_EDGE = 3, /* an edge has zero length, so its tangent is undefined */
    TP_ERR_NONFINITE = 4,       /* NaN/Inf in an input or result */
    TP_ERR_NOT_CONVERGED = 5,   /* CG stopped at cg_maxit above the tolerance (best iterate returned) */
    TP_ERR_BREAKDOWN = 6,       /* CG found p^T A p <= 0 (operator not SPD on range(P)) */
    TP_ERR_LINESEARCH = 7,      /* no step size passed Armijo + projection within max_halvings */
    TP_ERR_PROJECTION = 8,      /* constraint projection did not reach proj_tol */
    TP_ERR_OOM = 9,             /* device allocation failed in tp_create */
    TP_ERR_UNSUPPORTED = 10     /* option not available for this graph (e.g. spectral on open curves) */
} tp_status;

typedef enum {
    TP_FP64 = 0,  /* pair arithmetic in FP64 */
    TP_FP32 = 1,  /* pair arithmetic in FP32, per-tile partial sums folded into FP64 */
    TP_MIXED = 2  /* FP32 pairs on double-float positions, FP64 for pairs closer than near_cutoff */
} tp_precision;

typedef enum {
    TP_PRECOND_NONE = 0,
    TP_PRECOND_JACOBI = 1,   /* diag(A)^-1 */
    TP_PRECOND_SPECTRAL = 2, /* Jacobi-scaled circulant inverse per closed curve (not in the paper) */
    TP_PRECOND_SPECTRAL_RQ = 3, /* the same with the symbol corrected by Rayleigh quotients of the actual
                                   operator at sampled frequencies, rebuilt at every set-up (not in the paper) */
    TP_PRECOND_TWOLEVEL = 4,    /* TP_PRECOND_SPECTRAL_RQ plus an additive coarse-space correction
                                   Z (Z^T A Z)^-1 Z^T with coarse_dim periodic hat functions per curve */
    TP_PRECOND_LEARNED = 5,     /* TP_PRECOND_TWOLEVEL plus a learned SPD local term G_theta (tp_gnn_*);
                                   only for contexts created with it (not in the paper) */
    TP_PRECOND_TWOLEVEL_BALANCED = 6, /* the same spectral term S and coarse space Z in the balancing
                                   (multiplicative, symmetric) form Q r + (I - Q A) S (I - A Q) r,
                                   Q = Z (Z^T A Z)^-1 Z^T: exact on range(A Z).  Keeps the set-up's
                                   columns A Z (n (coarse_dim - 1) doubles per curve); every problem
                                   must be one closed curve (independent curves, or a one-curve graph),
                                   else TP_ERR_UNSUPPORTED (not in the paper) */
    TP_PRECOND_LEARNED_BALANCED = 7  /* the balancing form with the learned smoother W S W + G (tp_gnn_*) in
                                   place of S: Q r + (I - Q A)(W S W + G)(I - A Q) r; contexts created with
                                   it, every problem one closed curve (not in the paper) */
} tp_precond;

/* Constraint sets of Sec. 8.1 (Phi of the descent step; targets fixed by tp_set_constraints_from or at
 * the first call). */
typedef enum {
    TP_CONSTRAINTS_TOTAL_LENGTH = 0, /* barycenter (3 rows) + total length L0 - sum_I l_I (1 row) per problem */
    TP_CONSTRAINTS_EDGE_LENGTHS = 1, /* barycenter + one row l0_I - l_I per edge (isometric motions only).
                                        Every curve's edges must be one simple chain in storage order
                                        (i1 of edge I + 1 = i2 of edge I; closed when the last edge ends at
                                        the first one's start) and curves may not share vertices */
    TP_CONSTRAINTS_POINTS = 2        /* total length (1 row) + gamma_v - p_v (3 rows) per pinned vertex v
                                        (tp_set_pins, at least one in every problem), optional tangent rows
                                        (tp_set_tangents) and surface rows (tp_set_surface); no barycenter
                                        row (the pins fix the translations) */
} tp_constraint_set;

/* Start of the backtracking line search (Sec. 5.4). */
typedef enum {
    TP_LINESEARCH_UNIT = 0,    /* normalised gradient, tau = 1 (the paper's strategy for its applications) */
    TP_LINESEARCH_ISOTOPY = 1  /* tau = 2/3 tau_max, tau_max the first collision time of gamma - tau d in
                                  (0, ccd_horizon] (ccd_horizon when none comes first); every accepted
                                  step stays below the first collision along the straight path */
} tp_line_search;

/* Penalties of Sec. 8.1, added by descent_step to the energy and differential of the curve (tp_energy and
 * tp_differential stay the tangent-point energy alone; tp_penalty evaluates the penalties by themselves). */
typedef struct {
    double w_length;       /* weight of the total length sum_I l_I */
    double w_length_diff;  /* weight of sum over vertices of degree 2 of (l_I - l_J)^2, I, J its two edges */
    double w_field;        /* weight of the field potential sum_I l_I |T_I x X(x_I)|^2 */
    double field_M[9];     /* X(x) = u / |u| with u = M x + b (M row-major); X = 0 where u = 0 */
    double field_b[3];
} tp_penalties;

/* Shape of the learned preconditioner's edge-graph network (see tp_gnn_set_params). */
#define TP_GNN_HIDDEN 64
#define TP_GNN_FEATURES 8

typedef struct {
    double alpha, beta;   /* kernel exponents of Eq. 3; Lemma 1 needs alpha > 1, beta in [alpha+2, 2 alpha+1) */
    double sigma;         /* fractional order of B, B0; NaN => (beta - 1)/alpha - 1 (Sec. 4.2.2) */
    int precision;        /* tp_precision */
    double near_cutoff;   /* TP_MIXED: |x_I - x_J| < near_cutoff * mean edge length => FP64 pair */
    double cg_rtol;       /* stop when ||P(a - A-bar x)|| <= cg_rtol ||P a|| */
    int cg_maxit;
    int cg_check_every;   /* host polls the device-side convergence flag every k iterations */
    double proj_cg_rtol;  /* tolerance of the CG solve inside each constraint-projection iteration */
    int precond;          /* tp_precond */
    double armijo_c;      /* Armijo constant c in E(g - tau d) <= E(g) - c tau <dE, d> */
    double shrink;        /* backtracking factor */
    int max_halvings;
    double proj_tol;      /* success when max|Phi| <= proj_tol * max(1, L0) */
    int proj_maxit;
    int independent;      /* 1: every curve is its own problem (no cross-curve pairs, constraints per curve);
                             0: the whole graph is one problem (one barycenter + one total length) */
    int coarse_dim;       /* TP_PRECOND_TWOLEVEL*: hat functions per closed curve (default 128; at most 8192
                             and n / 4).  The set-up keeps n (m - 1) doubles of columns A Z per curve from
                             8 hats on (every two-level form) and 3 (m - 1)^2 doubles of coarse matrices */
    double far_cutoff;    /* TP_MIXED: source tiles farther than far_cutoff * (extent of the curve) from a
                             warp's targets use single-float positions (faster, less accurate); >= 10
                             keeps double-float positions everywhere */
    int use_graphs;       /* 1: CG runs blocks of cg_check_every iterations as captured CUDA graphs on a
                             context-owned stream joined to the caller's stream by events (the same
                             kernels in the same order as the direct launches); 0: direct launches */
    int precond_refresh;  /* rebuild the Rayleigh-quotient symbols and the coarse space every k-th
                             preconditioner set-up (1: every set-up); diag(A) and the learned term's
                             features are always rebuilt for the current curve */
    int constraint_set;   /* tp_constraint_set (default TP_CONSTRAINTS_TOTAL_LENGTH) */
    int line_search;      /* tp_line_search (default TP_LINESEARCH_UNIT) */
    double ccd_horizon;   /* TP_LINESEARCH_ISOTOPY: collision times are searched in (0, ccd_horizon]
                             (default 1.5, so that the start never exceeds tau = 1) */
    int warm_start;       /* 1 (default): the gradient solves start from the context's previous gradient
                             solutions and each projection solve from the previous one (a problem whose
                             guess does not lower the residual starts from zero); 0: every solve starts
                             from zero, so repeated calls on the same input give identical results */
} tp_params;

typedef struct {
    int iters;          /* CG iterations of the gradient solve (largest over problems, summed over the solves) */
    double rel_res;     /* final relative residual, recomputed with the working-precision operator (largest over problems) */
    int converged;      /* all problems reached cg_rtol */
    int n_converged;    /* problems whose solves all reached cg_rtol */
} tp_solve_info;

typedef struct {
    double E_before, E_after; /* summed over problems */
    double tau;               /* accepted step (0 if none) */
    double gnorm;             /* ||g~||_2 of the projected H^s gradient */
    int halvings;
    int proj_iters;           /* projection iterations of the accepted trial */
    int cg_iters;             /* gradient-solve CG iterations */
    int proj_cg_iters;        /* all CG iterations spent in constraint projections */
    int accepted;             /* problems whose step was accepted */
    double rel_res;           /* gradient-solve relative residual */
    int n_converged;          /* problems whose gradient solves reached cg_rtol */
} tp_step_info;

typedef struct tp_ctx tp_ctx;

/* Fill p with the defaults: (alpha, beta) = (2, 4.5), sigma = NaN, FP32, cg_rtol 1e-6,
 * cg_maxit 20000, cg_check_every 8, proj_cg_rtol 1e-6, spectral preconditioner,
 * Armijo c = 1e-4, shrink 0.5, 30 halvings, proj_tol 1e-10, proj_maxit 5, near_cutoff 4,
 * far_cutoff 10, independent 0, use_graphs 1, precond_refresh 1, coarse_dim 128,
 * constraint_set TP_CONSTRAINTS_TOTAL_LENGTH, line_search TP_LINESEARCH_UNIT,
 * ccd_horizon 1.5, warm_start 1. */
TPE_API void tp_default_params(tp_params *p);

/* Create a context for a fixed graph.  edges_host: HOST int32 [n_edges][2] (i1, i2), the edge
 * direction defines T_I.  vertex_offsets_host / edge_offsets_host: HOST int32 [n_curves + 1]
 * delimiting the curves (vertices and edges of curve c are contiguous); n_curves >= 1.
 * With p->independent = 1 every curve is its own problem.  Allocates all device scratch.
 * Curves of fewer than 4 edges have no disjoint pair: their energy, differential and A-bar are 0.
 * Errors: TP_ERR_INVALID_ARG (no edges at all, indices out of range, an edge outside its curve's
 * vertex range, bad parameters), TP_ERR_OOM, TP_ERR_CUDA. */
TPE_API tp_status tp_create(tp_ctx **ctx, int n_vertices, int n_edges, const int32_t *edges_host, int n_curves,
                    const int32_t *vertex_offsets_host, const int32_t *edge_offsets_host, const tp_params *p);
TPE_API void tp_destroy(tp_ctx *ctx);
TPE_API const char *tp_last_error(const tp_ctx *ctx);
TPE_API int tp_num_problems(const tp_ctx *ctx);
/* Replace the numeric parameters (not `independent`) of an existing context. */
TPE_API tp_status tp_set_params(tp_ctx *ctx, const tp_params *p);

/* Discrete energy hat-E (Sec. 5.1, Eq. 17) of every problem into E[n_problems] (device).
 * rows (device [n_edges], may be NULL) receives sum_J E_IJ per target edge I.
 * Errors: TP_ERR_DEGENERATE_EDGE if some l_I = 0 (checked on the device, reported on the
 * next synchronising call or by tp_check), TP_ERR_INVALID_ARG. */
TPE_API tp_status tp_energy(tp_ctx *ctx, const double *gamma, double *E, double *rows, tp_stream stream);

/* Differential d hat-E (Sec. 5.1) into dE [nV][3] (device); E (device [n_problems]) may be NULL. */
TPE_API tp_status tp_differential(tp_ctx *ctx, const double *gamma, double *dE, double *E, tp_stream stream);

/* Au = A-bar u with A = B + B0 of the curve gamma (Secs. 5.2.2-5.2.3, Eq. 19): u, Au device [nV][3]. */
TPE_API tp_status sobolev_apply(tp_ctx *ctx, const double *gamma, const double *u, double *Au, tp_stream stream);

/* AU_f = A-bar U_f for m vector fields at once (Secs. 5.2.2-5.2.3, Eq. 19 per field): U, AU device
 * double [m][nV][3] (field-major: field f starts at U + 3 nV f); m >= 0 (m = 0 does nothing).  Every
 * pair's Gram weights and tangent gap (about 220 of the 255 canonical FLOP of an apply) are computed
 * once per pass and applied to 4 fields (12 scalar columns); the per-column arithmetic is
 * sobolev_apply's (same precision mode).  Builds its work list, per-field records and partial sums at
 * the first call (about 4 nE records and slots x nE x 24 doubles).  U and AU must not overlap.
 * Errors: TP_ERR_INVALID_ARG (NULL pointers with m > 0, m < 0), TP_ERR_CUDA. */
TPE_API tp_status sobolev_apply_multi(tp_ctx *ctx, const double *gamma, const double *U, double *AU, int m,
                                      tp_stream stream);

/* The same product A-bar u in double-float arithmetic (every pair term as an unevaluated sum of two
 * floats, ~48 bits, from the FP64 positions, tangents, lengths and u): the accurate operator with which
 * the solves of TP_FP32 and TP_MIXED contexts judge their true residuals (FP64 contexts run their
 * FP64 pass).  About an order of magnitude slower than sobolev_apply.  Builds its own work list at the
 * first call (the only allocation, and it may grow the context's partial-sum buffer). */
TPE_API tp_status sobolev_apply_accurate(tp_ctx *ctx, const double *gamma, const double *u, double *Au,
                                         tp_stream stream);

/* diag(A) of the curve gamma into diag [nV] (device). */
TPE_API tp_status tp_gram_diagonal(tp_ctx *ctx, const double *gamma, double *diag, tp_stream stream);

/* Apply the configured preconditioner M^-1 (for the curve gamma) to r: z = M^-1 r, device [nV][3]. */
TPE_API tp_status tp_precond_apply(tp_ctx *ctx, const double *gamma, const double *r, double *z, tp_stream stream);

/* Symbols the spectral preconditioner currently divides by, for every curve at its vertex offset:
 * out DEVICE double [n_vertices].  rq = 0: regular-polygon symbols; rq = 1: the Rayleigh-quotient
 * corrected symbols of the last set-up (TP_PRECOND_SPECTRAL_RQ), which tp_precond_apply and the
 * solves rebuild for their curve. */
TPE_API tp_status tp_spectral_symbols(tp_ctx *ctx, int rq, double *out, tp_stream stream);

/* Regular-polygon symbol of the spectral preconditioner for a closed curve of n vertices
 * (eigenvalues of A of the regular n-gon divided by its diagonal, lambda_0 := lambda_1),
 * into lam (device [n]). */
TPE_API tp_status tp_spectral_symbol(tp_ctx *ctx, int n, double *lam, tp_stream stream);

/* Fix the constraint targets x0 (barycenter), L0 (total length) and, once the edge-length set has
 * been selected, every l0_I of every problem at their values on the curve gamma (Sec. 8.1).  Called
 * implicitly by the first sobolev_gradient or descent_step on a context. */
TPE_API tp_status tp_set_constraints_from(tp_ctx *ctx, const double *gamma, tp_stream stream);

/* Constraint values Phi (Sec. 8.1) of gamma into phi (device [4 * n_problems]):
 * rows 4q..4q+2 barycenter, row 4q+3 length of problem q: L0 - sum_I l_I, or with
 * TP_CONSTRAINTS_EDGE_LENGTHS max_I |l0_I - l_I| over the problem's edges.  With
 * TP_CONSTRAINTS_POINTS rows 4q..4q+2 hold instead, over the problem's constrained items, the largest
 * |gamma_v,k - p_v,k| (pins), |T_I,k - X_I,k| (tangents) and |f(gamma_v)| (surface points). */
TPE_API tp_status tp_constraints(tp_ctx *ctx, const double *gamma, double *phi, tp_stream stream);

/* Rows of TP_CONSTRAINTS_POINTS (Sec. 8.1).  All three calls copy their arrays, replace the previous
 * list of their kind (n = 0 removes it) and may be made in any order; a call whose list breaks a rule
 * returns TP_ERR_INVALID_ARG and leaves every list as it was.  Rules, per problem (each vertex or edge
 * belongs to the problem of its curve): at most 24 distinct constrained vertices (pinned vertices,
 * endpoints of tangent edges and surface vertices together) and at most 96 rows (3 per pin, 2 per
 * tangent, 1 per surface vertex); no surface vertex pinned; no tangent edge with both ends pinned.
 * The gradient takes one mean-free CG solve per three constrained vertices of the most constrained
 * problem (A-bar^+ e_v, reused by every constraint projection of the step) and a dense solve of
 * rows + 4 unknowns per problem.  The first call allocates the rows' scratch.
 *
 * Point constraints gamma_v = p_v: vertices HOST int32 [n], distinct, in [0, n_vertices); targets HOST
 * double [n][3], finite.  Every problem needs at least one pinned vertex. */
TPE_API tp_status tp_set_pins(tp_ctx *ctx, int n, const int32_t *vertices, const double *targets);

/* Tangent constraints T_I = X_I: edges HOST int32 [n], distinct, in [0, n_edges); X HOST double [n][3],
 * finite and nonzero (normalised by the library).  Each edge contributes the two rows b_a . T_I, with
 * (b_1, b_2) an orthonormal basis across X_I (the three rows T_I - X_I have a Jacobian of rank 2). */
TPE_API tp_status tp_set_tangents(tp_ctx *ctx, int n, const int32_t *edges, const double *X);

/* Surface constraints f(gamma_v) = 0 for one quadric f(x) = x^T Q x + b^T x + c (planes, spheres,
 * ellipsoids, cylinders, ...): quadric HOST double [13] = Q row-major (9), b (3), c, finite; vertices HOST
 * int32 [n], distinct, in [0, n_vertices). */
TPE_API tp_status tp_set_surface(tp_ctx *ctx, const double *quadric, int n, const int32_t *vertices);

/* Set (pen non-NULL, copied) or clear (NULL) the penalties the descent step adds (Sec. 8.1).  The first
 * call allocates their scratch.  Errors: TP_ERR_INVALID_ARG (a non-finite weight). */
TPE_API tp_status tp_set_penalties(tp_ctx *ctx, const tp_penalties *pen);

/* The penalties alone at gamma: E (DEVICE double [n_problems], may be NULL) and their gradient dE (DEVICE
 * [nV][3], may be NULL), both overwritten; zeros when none are set. */
TPE_API tp_status tp_penalty(tp_ctx *ctx, const double *gamma, double *E, double *dE, tp_stream stream);

/* Barnes-Hut comparator (App. B.1): the discrete energy and its differential approximated over a
 * bounding volume hierarchy of tangent-points (T_I, x_I), one tree per problem, in FP64.  The tree is
 * built on the host at every call (gamma is copied to the host; the call synchronises `stream`):
 * nodes with more than leaf_size edges split by the plane that minimises the two children's summed
 * squared 6-D box diameters; r_x, r_T are half the diagonals of a node's box of edge endpoints and of
 * its box of tangents.  A node is admissible for target I when r_x < eps |x_I - x_N| and r_T < eps and
 * it holds neither I nor an edge sharing a vertex with I; it then contributes
 * l_I L_N |T_I x (x_I - x_N)|^alpha / |x_I - x_N|^beta (Eq. BVHNodeTPE) to the energy and
 * L_N d/d gamma [l_I (k(x_I, x_N, T_I) + k(x_N, x_I, T_N))] to the target's endpoints in the
 * differential; leaves contribute their disjoint pairs exactly (the trapezoid kernel of Eq. 18).
 * eps = 0 gives the exact energy and differential.  A comparator for the exact tiled passes: the
 * library's solves and descent steps do not use it.
 *   eps >= 0, leaf_size in [1, 64] (else TP_ERR_INVALID_ARG).
 *   tp_bh_energy: E DEVICE double [n_problems] and/or rows DEVICE double [n_edges] (the per-edge
 *     sums), either may be NULL but not both.
 *   tp_bh_differential: dE DEVICE double [nV][3] (overwritten).
 *   TP_ERR_UNSUPPORTED when a vertex joins more than 15 edges or the tree is deeper than the
 *   traversal stack (94 levels).
 * tp_bh_stats reports the last pass's admissible nodes and leaf pairs summed over targets, the tree
 * depth and the host seconds of its hierarchy (copy of gamma to the host, build, upload); each output
 * may be NULL. */
TPE_API tp_status tp_bh_energy(tp_ctx *ctx, const double *gamma, double eps, int leaf_size, double *E, double *rows,
                               tp_stream stream);
TPE_API tp_status tp_bh_differential(tp_ctx *ctx, const double *gamma, double eps, int leaf_size, double *dE,
                                     tp_stream stream);
TPE_API tp_status tp_bh_stats(const tp_ctx *ctx, int64_t *admissible_nodes, int64_t *leaf_pairs, int32_t *depth,
                              double *build_seconds);

/* First collision time (Sec. 5.4): t (DEVICE double [n_problems]) receives, per problem, the first
 * tau in (0, horizon] at which two disjoint edges of gamma - tau d touch (segment distance at most
 * 1e-8 times the sum of their lengths), or horizon where none do.  gamma, d: DEVICE [nV][3].  Pairs
 * whose boxes swept over [0, horizon] are apart are skipped; the others solve the coplanarity cubic in
 * FP64.  The first call allocates the context's block-pair work list.  Errors: TP_ERR_INVALID_ARG
 * (horizon <= 0), TP_ERR_CUDA. */
TPE_API tp_status tp_collision_time(tp_ctx *ctx, const double *gamma, const double *d, double horizon, double *t,
                                    tp_stream stream);

/* Projected H^s gradient (Eq. 22 via the projected system of App. B.3.3): g = P y with
 * P A-bar P y = P dE, by preconditioned CG with device-resident scalars.  dE, g device [nV][3].
 * With TP_CONSTRAINTS_EDGE_LENGTHS, P is the orthogonal projector onto the mean-free velocities that
 * keep every edge length (one tridiagonal solve per curve and iteration), and a translation then
 * restores the barycenter row; the result is the same KKT solution of Eq. 22.
 * With TP_CONSTRAINTS_POINTS the KKT solution is formed from mean-free solves (A-bar^+ dE,
 * A-bar^+ C_len^T and A-bar^+ e_v for every constrained vertex v) and the Schur complement of the
 * constraint rows and the translations; info then sums the iterations of all of them.
 * info (host, may be NULL) is filled after a stream synchronisation.
 * Returns TP_ERR_NOT_CONVERGED (g holds the last iterate) or TP_ERR_BREAKDOWN on failure. */
TPE_API tp_status sobolev_gradient(tp_ctx *ctx, const double *gamma, const double *dE, double *g, tp_solve_info *info,
                           tp_stream stream);

/* One descent step in place on gamma (device [nV][3]) (Sec. 5.4) on the energy plus the penalties set
 * by tp_set_penalties: g~ by sobolev_gradient,
 * d = g~ / ||g~||_2, then tau = 1 (or 2/3 of the first collision time with TP_LINESEARCH_ISOTOPY),
 * shrink, ... until the constraint projection of gamma - tau d
 * (Sec. 5.3.2, App. B.3.4) succeeds and the Armijo condition holds.  Synchronises the stream
 * (the line search reads scalars on the host).  On TP_ERR_LINESEARCH gamma is unchanged. */
TPE_API tp_status descent_step(tp_ctx *ctx, double *gamma, tp_step_info *info, tp_stream stream);

/* Per-problem result of the context's last CG solve (the last one inside the last call that solved):
 * rel_res (HOST double [n_problems], may be NULL) the true relative residual recomputed with the
 * working-precision operator, iters (HOST int32 [n_problems], may be NULL) the iterations. */
TPE_API tp_status tp_last_solve(const tp_ctx *ctx, double *rel_res, int32_t *iters);

/* Number of kernel launches this context has issued since creation (all entry points). */
TPE_API int64_t tp_launch_count(const tp_ctx *ctx);

/* Ordered disjoint edge pairs (I, J) one pair pass of this context visits (Eq. 17's index set,
 * summed over problems): the algorithmic work unit of every pair kernel. */
TPE_API int64_t tp_pairs_per_pass(const tp_ctx *ctx);

/* Per-kernel timing with CUDA events recorded around every pair-kernel launch on its own stream.
 * enable = 1 starts (and clears) the record; op: 0 energy, 1 differential, 2 apply (full passes),
 * 3 diag, 4 apply inside CG solves (items of already converged problems skipped), 5 double-float
 * apply (tp_sobolev_apply_accurate and the refined solves' residuals), 6 the coarse-space pass that
 * assembles A Z for the two-level preconditioners, 7 the multi-field apply (sobolev_apply_multi and
 * the Rayleigh-quotient probes of the spectral set-up), one launch per 4 fields.
 * tp_profile_read synchronises the recorded events and returns the summed device time (ms) and
 * the number of launches of that pair kernel since profiling was enabled. */
TPE_API tp_status tp_profile(tp_ctx *ctx, int enable);
TPE_API tp_status tp_profile_read(tp_ctx *ctx, int op, double *total_ms, int64_t *launches);

/* Discrete energy (Eq. 17) of one curve network without any device allocation, for callers that
 * cannot call cudaMalloc (inside a region where allocation is forbidden, or with all free memory
 * handed to their own pool).  The paper has no counterpart: this is a variant of tp_energy's mixed
 * precision pair pass whose scratch (edge records, work items, partial sums; about 20 MB) lives in
 * fixed-size file-scope __device__ arrays that every GPU which loads the library keeps until exit.
 *   gamma  DEVICE double [n_vertices][3];  edges DEVICE int32 [n_edges][2] with indices in
 *          [0, n_vertices) (not checked: they are device data; may be NULL when n_edges = 0, which
 *          gives E = 0);  E DEVICE double [1].
 *   n_edges <= 65536, else TP_ERR_INVALID_ARG (the scratch has a fixed size).
 *   All pairs of disjoint edges of the whole graph form one problem (as independent = 0).
 * The first call on a device looks up the arrays' device addresses (cudaGetSymbolAddress).  Every
 * call synchronises `stream` once (to read the edge-length
 * statistics that set the near-pair cutoff) and then enqueues the pair pass.  All calls share the
 * same scratch and it keeps the last call's contents: calls that overlap on the GPU (other streams,
 * other host threads) race and must be serialised by the caller.
 * Errors: TP_ERR_INVALID_ARG, TP_ERR_DEGENERATE_EDGE, TP_ERR_NONFINITE, TP_ERR_CUDA. */
TPE_API tp_status tp_energy_static(const double *gamma, const int32_t *edges, int n_vertices, int n_edges,
                                   double alpha, double beta, double *E, tp_stream stream);

/* ------------------------------------------------------------------------------------------
 * Learned preconditioner (TP_PRECOND_LEARNED).  Not part of the paper: a 3-layer network on the
 * edge graph of the closed curves predicts three values (a_I, b_I, c_I) per edge that shape
 *   M^-1 r = W S W r + Z (Z^T A Z)^-1 Z^T r + G r,
 * W = D^-1/2 diag(exp(c_v)) with c_v the mean of c over the edges at vertex v (a learned rescaling of
 * the Jacobi-scaled circulant S of TP_PRECOND_TWOLEVEL, which c = 0 gives back), Z the coarse space,
 *   G = D^-1/2 (D_delta^T diag(e^{2a}) D_delta + D_sigma^T diag(e^{2b}) D_sigma) D^-1/2,
 * D = diag(A), (D_delta r)_I = r_i2 - r_i1, (D_sigma r)_I = r_i1 + r_i2.  M stays SPD for any
 * parameters, so CG with the exact operator remains the judge of the residual.
 * Network (per edge I, neighbours I-1 and I+1 along its curve; FP32 activations, BF16 weights):
 *   f_I = [log(l_I / mean l), 1 - T_{I-1}.T_I, 1 - T_I.T_{I+1}, log(d_i1 / mean d), log(d_i2 / mean d),
 *          log(l_{I-1} / l_I), log(l_{I+1} / l_I), 1]     (means over the edge's curve)
 *   h1 = relu(W1 f + b1),  h2 = relu(W2s h1 + W2n (h1[I-1] + h1[I+1]) / 2 + b2),
 *   h3 = relu(W3s h2 + W3n (h2[I-1] + h2[I+1]) / 2 + b3),  (a, b, c) = W4 h3 + b4.
 * Parameter vector theta: FP32, DEVICE, tp_gnn_num_params() values in the order
 *   W1 [64][8], b1 [64], W2s [64][64], W2n [64][64], b2, W3s, W3n, b3, W4 [3][64], b4 [3] (row-major).
 * Training: (r, e = A^+ r) pairs from the context's own CG solves (tp_cg_harvest), prepared once
 * (tp_gnn_prepare_pairs), then Adam steps (tp_gnn_train_step) on the A-norm error of the best
 * multiple of z = M^-1 r (preconditioned CG does not see the preconditioner's scale):
 *   L = min_a ||a z - e||_A^2 / ||e||_A^2 = 1 - (z^T r)^2 / ((z^T A z)(e^T r)),  in [0, 1].
 * Every tp_gnn_* call fails with TP_ERR_UNSUPPORTED on a context not created with
 * TP_PRECOND_LEARNED (only those hold the network's scratch, about 1.6 KB per edge). */
TPE_API int tp_gnn_num_params(void);

/* Load theta (DEVICE float [P]) as the FP32 master parameters and refresh their BF16 copy;
 * reset_optimizer = 1 also zeroes Adam's moments and step count. */
TPE_API tp_status tp_gnn_set_params(tp_ctx *ctx, const float *theta, int reset_optimizer, tp_stream stream);
/* Copy the FP32 master parameters into theta (DEVICE float [P]). */
TPE_API tp_status tp_gnn_get_params(tp_ctx *ctx, float *theta, tp_stream stream);

/* Bind the curve gamma: diag(A) by one pair pass and the edge features, kept for the forward,
 * backward, G-term and training calls until the next bind or preconditioner set-up. */
TPE_API tp_status tp_gnn_bind(tp_ctx *ctx, const double *gamma, tp_stream stream);

/* Network forward on the bound curve with the current BF16 weights.  features (DEVICE float
 * [n_edges][8]) and out (DEVICE float [n_edges][3]: a, b, c) may each be NULL. */
TPE_API tp_status tp_gnn_forward(tp_ctx *ctx, float *features, float *out, tp_stream stream);

/* Parameter gradient grad (DEVICE float [P]) of a scalar whose derivative with respect to the
 * outputs of the last forward pass is dout (DEVICE float [n_edges][3]).  The chain uses the BF16
 * weights the forward pass used; the sums are deterministic. */
TPE_API tp_status tp_gnn_backward(tp_ctx *ctx, const float *dout, float *grad, tp_stream stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the FP32 masters with gradient grad
 * (DEVICE float [P]) and learning rate lr; refreshes the BF16 copy. */
TPE_API tp_status tp_gnn_adam(tp_ctx *ctx, const float *grad, float lr, tp_stream stream);

/* z = G r (accumulate = 0) or z += G r (accumulate = 1) with the last forward's outputs and the
 * bound diag(A); r, z DEVICE double [nV][3]. */
TPE_API tp_status tp_gnn_g_apply(tp_ctx *ctx, const double *r, double *z, int accumulate, tp_stream stream);

/* dout (=, or += with accumulate = 1) the derivative of gz . (G r) with respect to the network
 * outputs (a, b): DEVICE float [n_edges][3] (the c column is set to 0, or left as it is when
 * accumulating); r, gz DEVICE double [nV][3]. */
TPE_API tp_status tp_gnn_out_grad(tp_ctx *ctx, const double *r, const double *gz, float *dout, int accumulate,
                                  tp_stream stream);

/* Solve A-bar y = P rhs by the configured preconditioned CG on the mean-free subspace (the solve
 * inside sobolev_gradient) and capture, every `every` iterations and at most max_pairs times, the
 * residual r_k into R[k] and the exact correction e_k = y* - y_k (y*: the final iterate) into E[k].
 * R, E: DEVICE double [max_pairs][nV][3].  *n_pairs (host) = pairs captured.  info (host, may be
 * NULL) as for sobolev_gradient.  Synchronises the stream. */
TPE_API tp_status tp_cg_harvest(tp_ctx *ctx, const double *gamma, const double *rhs, int every, int max_pairs,
                                double *R, double *E, int *n_pairs, tp_solve_info *info, tp_stream stream);

/* For n harvested pairs of the curve gamma: first R[k] := A-bar E[k] (CG's recursive residual drifts
 * below the true residual when the operator is inexact, so only A-bar e_k is exactly consistent with
 * e_k; on output every pair satisfies r = A-bar e), then ER[k] (DEVICE double [n][n_problems]) =
 * e_k . r_k per problem, B[k] = the part of the preconditioner that the parameters do not change,
 * applied to r_k and mean-projected, and AB[k] = A-bar B[k].  With ILAM (DEVICE double [nV], may be
 * NULL) the circulant is left to training (its scaling is learned): B[k] is the coarse term alone and
 * ILAM receives this curve's inverse circulant symbols; without it, B[k] is the whole two-level
 * preconditioner.  When the context's preconditioner is a balancing form (TP_PRECOND_TWOLEVEL_BALANCED
 * or TP_PRECOND_LEARNED_BALANCED), ILAM and R2 (DEVICE double [n][nV][3]) are required: B[k] = Q r_k and
 * R2[k] = (I - A Q) r_k, the vector the learned smoother acts on (R2 is ignored otherwise and may be
 * NULL).  R, E, B, AB DEVICE double [n][nV][3]; B may be the same buffer as E (ER is taken first).
 * Costs two A-bar applies per pair. */
TPE_API tp_status tp_gnn_prepare_pairs(tp_ctx *ctx, const double *gamma, int n, double *R, double *E,
                                       double *B, double *AB, double *ER, double *ILAM, double *R2,
                                       tp_stream stream);

/* One training step on n prepared pairs of the bound curve gamma, with the inverse symbols ILAM that
 * tp_gnn_prepare_pairs returned for it (NULL: the prepared B already holds the whole circulant):
 * z = B + W S W r + G r per pair (R2 NULL), or in the balancing form z = B + (I - Q A)(W S W r2 + G r2)
 * with r2 = R2[k] (the context's preconditioner must then be a balancing form, whose coarse space is the
 * one the pairs were prepared with); the loss at the current parameters, averaged over pairs and
 * problems, into *loss (host), the parameter gradient into grad (DEVICE float [P], may be NULL), then one
 * Adam step when lr > 0 (lr = 0: gradient only).  Costs one A-bar apply and two circulant applies per
 * pair.  Synchronises the stream. */
TPE_API tp_status tp_gnn_train_step(tp_ctx *ctx, const double *gamma, int n, const double *R, const double *B,
                                    const double *AB, const double *ER, const double *ILAM, const double *R2,
                                    float lr, double *loss, float *grad, tp_stream stream);

/* Autotuner of the pair passes (not in the paper).  For TP_MIXED contexts with the specialised
 * powers ((alpha, beta) = (2, 4.5)) it times, on the curve gamma, every candidate number of target
 * edges per thread of the energy (1, 2, 4), differential (1, 2) and apply / diag (1, 2, 4) gather
 * passes, and the symmetric energy, differential and apply passes (each unordered pair evaluated once, 1 or 2
 * targets per thread, when their partial sums fit in 32 GB and in half the free device memory), one
 * warm-up and three timed passes each
 * (CUDA events on `stream`), and keeps the fastest, rebuilding that op's work queue; other contexts
 * keep their defaults and are left unchanged.
 *   tpt (HOST int32 [6], may be NULL): the chosen targets per thread of the energy, differential and
 *       apply gather passes, then of the symmetric apply and energy, then the symmetric differential's
 *       variant (tp_set_diff_variant; 0: gather pass).
 *   ms  (HOST double [17], may be NULL): ms per pass for 1, 2, 4 targets per thread of the energy
 *       [0..2], differential [3..5] and apply [6..8] gather passes, then the symmetric apply [9..10],
 *       energy [11..12] with 1, 2, and the symmetric differential variants 1, 2 [13..14] and 3, 4
 *       [15..16] (0 where not a candidate).
 * May reallocate the context's partial-sum buffer (the only allocation after tp_create).
 * Synchronises the stream.  Errors: TP_ERR_INVALID_ARG, TP_ERR_CUDA, TP_ERR_DEGENERATE_EDGE. */
TPE_API tp_status tp_autotune(tp_ctx *ctx, const double *gamma, int32_t *tpt, double *ms, tp_stream stream);

/* Select the apply pass: symmetric_tpt = 0 the gather pass (every ordered pair, the default), 1 or 2
 * the symmetric pass (every unordered pair evaluated once; both rows receive their terms; TP_MIXED with
 * (alpha, beta) = (2, 4.5) only, else TP_ERR_UNSUPPORTED) with that many target edges per thread.  Both
 * are deterministic and differ only in summation order.  May grow the partial-sum buffer. */
TPE_API tp_status tp_set_apply_variant(tp_ctx *ctx, int symmetric_tpt);

/* The same choice for the energy pass (0: gather, 1 or 2: symmetric; the rows E_I are the same
 * sums in another order). */
TPE_API tp_status tp_set_energy_variant(tp_ctx *ctx, int symmetric_tpt);

/* The same choice for the differential pass (0: gather; 1 or 2: symmetric with that many targets per
 * thread; 3: symmetric, one target per thread with registers held to 4 resident CTAs per SM; 4: two
 * targets per thread held to 3 CTAs per SM.  Row J's terms of a pair are the mirror of row I's; near
 * pairs are FP64 on both sides). */
TPE_API tp_status tp_set_diff_variant(tp_ctx *ctx, int symmetric_tpt);

/* Throughput microbenchmarks on the current device (no context needed): FP32 FMA FLOP/s, MUFU
 * rsqrt op/s and FP64 FMA FLOP/s.  Returns 0 on success. */
TPE_API int tp_measure_peaks(double *fp32_flops, double *mufu_ops, double *fp64_flops);

#ifdef __cplusplus
}
#endif
#endif /* TPE_H */
