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
 * Constraints are the barycenter and total-length constraints of Sec. 8.1.
 *
 * Conventions shared by every entry point
 *   - Vertex arrays (gamma, dE, u, ...) are DEVICE pointers to double, vertex-major [nV][3].
 *   - Per-problem outputs (energies) are DEVICE pointers to double [n_problems].
 *   - Every call is enqueued on `stream` (a cudaStream_t; NULL = legacy default stream) and is
 *     asynchronous unless it says otherwise.  Calls that return host-side info structs
 *     synchronise the stream before returning.
 *   - The caller owns every pointer it passes; the context owns its own scratch memory,
 *     allocated once in tp_create and sized for the graph it was created with.  No entry
 *     point allocates device memory after tp_create.
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
    TP_PRECOND_SPECTRAL = 2  /* Jacobi-scaled circulant inverse per closed curve (not in the paper) */
} tp_precond;

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
    double far_cutoff;    /* TP_MIXED: source tiles farther than far_cutoff * (extent of the curve) from a
                             warp's targets use single-float positions (faster, less accurate); >= 10
                             keeps double-float positions everywhere */
} tp_params;

typedef struct {
    int iters;          /* CG iterations of the gradient solve */
    double rel_res;     /* final ||P(a - A-bar x)|| / ||P a||, recomputed with the exact operator */
    int converged;
} tp_solve_info;

typedef struct {
    double E_before, E_after; /* summed over problems */
    double tau;               /* accepted step (0 if none) */
    double gnorm;             /* ||g~||_2 of the projected H^s gradient */
    int halvings;
    int proj_iters;           /* projection iterations of the accepted trial */
    int cg_iters;             /* gradient-solve CG iterations */
    int proj_cg_iters;        /* all CG iterations spent in constraint projections */
    int accepted;
    double rel_res;           /* gradient-solve relative residual */
} tp_step_info;

typedef struct tp_ctx tp_ctx;

/* Fill p with the defaults: (alpha, beta) = (2, 4.5), sigma = NaN, FP32, cg_rtol 1e-6,
 * cg_maxit 20000, spectral preconditioner, Armijo c = 1e-4, shrink 0.5, 30 halvings,
 * proj_tol 1e-10, proj_maxit 5, near_cutoff 4. */
TPE_API void tp_default_params(tp_params *p);

/* Create a context for a fixed graph.  edges_host: HOST int32 [n_edges][2] (i1, i2), the edge
 * direction defines T_I.  vertex_offsets_host / edge_offsets_host: HOST int32 [n_curves + 1]
 * delimiting the curves (vertices and edges of curve c are contiguous); n_curves >= 1.
 * With p->independent = 1 every curve is its own problem.  Allocates all device scratch.
 * Errors: TP_ERR_INVALID_ARG (indices out of range, an edge outside its curve's vertex range,
 * bad parameters), TP_ERR_OOM, TP_ERR_CUDA. */
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

/* diag(A) of the curve gamma into diag [nV] (device). */
TPE_API tp_status tp_gram_diagonal(tp_ctx *ctx, const double *gamma, double *diag, tp_stream stream);

/* Apply the configured preconditioner M^-1 (for the curve gamma) to r: z = M^-1 r, device [nV][3]. */
TPE_API tp_status tp_precond_apply(tp_ctx *ctx, const double *gamma, const double *r, double *z, tp_stream stream);

/* Regular-polygon symbol of the spectral preconditioner for a closed curve of n vertices
 * (eigenvalues of A of the regular n-gon divided by its diagonal, lambda_0 := lambda_1),
 * into lam (device [n]). */
TPE_API tp_status tp_spectral_symbol(tp_ctx *ctx, int n, double *lam, tp_stream stream);

/* Fix the constraint targets x0 (barycenter) and L0 (total length) of every problem at their
 * values on the curve gamma (Sec. 8.1).  Called implicitly by the first sobolev_gradient or
 * descent_step on a context. */
TPE_API tp_status tp_set_constraints_from(tp_ctx *ctx, const double *gamma, tp_stream stream);

/* Constraint values Phi (Sec. 8.1) of gamma into phi (device [4 * n_problems]):
 * rows 4q..4q+2 barycenter, row 4q+3 length of problem q. */
TPE_API tp_status tp_constraints(tp_ctx *ctx, const double *gamma, double *phi, tp_stream stream);

/* Projected H^s gradient (Eq. 22 via the projected system of App. B.3.3): g = P y with
 * P A-bar P y = P dE, by preconditioned CG with device-resident scalars.  dE, g device [nV][3].
 * info (host, may be NULL) is filled after a stream synchronisation.
 * Returns TP_ERR_NOT_CONVERGED (g holds the last iterate) or TP_ERR_BREAKDOWN on failure. */
TPE_API tp_status sobolev_gradient(tp_ctx *ctx, const double *gamma, const double *dE, double *g, tp_solve_info *info,
                           tp_stream stream);

/* One descent step in place on gamma (device [nV][3]) (Sec. 5.4): g~ by sobolev_gradient,
 * d = g~ / ||g~||_2, then tau = 1, shrink, ... until the constraint projection of gamma - tau d
 * (Sec. 5.3.2, App. B.3.4) succeeds and the Armijo condition holds.  Synchronises the stream
 * (the line search reads scalars on the host).  On TP_ERR_LINESEARCH gamma is unchanged. */
TPE_API tp_status descent_step(tp_ctx *ctx, double *gamma, tp_step_info *info, tp_stream stream);

/* Number of kernel launches this context has issued since creation (all entry points). */
TPE_API int64_t tp_launch_count(const tp_ctx *ctx);

/* Ordered disjoint edge pairs (I, J) one pair pass of this context visits (Eq. 17's index set,
 * summed over problems): the algorithmic work unit of every pair kernel. */
TPE_API int64_t tp_pairs_per_pass(const tp_ctx *ctx);

/* Per-kernel timing with CUDA events recorded around every pair-kernel launch on its own stream.
 * enable = 1 starts (and clears) the record; op: 0 energy, 1 differential, 2 apply, 3 diag.
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
 *          [0, n_vertices) (not checked: they are device data);  E DEVICE double [1].
 *   n_edges <= 65536, else TP_ERR_INVALID_ARG (the scratch has a fixed size).
 *   All pairs of disjoint edges of the whole graph form one problem (as independent = 0).
 * The first call on a device looks up the arrays' device addresses (cudaGetSymbolAddress); make
 * it before any stream capture.  Every call synchronises `stream` once (to read the edge-length
 * statistics that set the near-pair cutoff) and then enqueues the pair pass.  All calls share the
 * same scratch and it keeps the last call's contents: calls that overlap on the GPU (other streams,
 * other host threads) race and must be serialised by the caller.
 * Errors: TP_ERR_INVALID_ARG, TP_ERR_DEGENERATE_EDGE, TP_ERR_NONFINITE, TP_ERR_CUDA. */
TPE_API tp_status tp_energy_static(const double *gamma, const int32_t *edges, int n_vertices, int n_edges,
                                   double alpha, double beta, double *E, tp_stream stream);

/* Throughput microbenchmarks on the current device (no context needed): FP32 FMA FLOP/s, MUFU
 * rsqrt op/s and FP64 FMA FLOP/s.  Returns 0 on success. */
TPE_API int tp_measure_peaks(double *fp32_flops, double *mufu_ops, double *fp64_flops);

#ifdef __cplusplus
}
#endif
#endif /* TPE_H */
