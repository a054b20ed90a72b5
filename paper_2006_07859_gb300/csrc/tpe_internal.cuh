// Internal declarations of the GB300 tangent-point library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/tpe.h"

namespace tpe {

struct SpecState;
struct SolverState;
struct CoarseState;
struct GnnState;
struct EdgeState;
struct CcdState;
struct PenState;
struct PinState;
struct BhState;

// Precision of the pair arithmetic.
enum Prec { P64 = 0, P32 = 1, PMIX = 2 };

// Which quantity a pair pass accumulates.
enum PairOp { OP_ENERGY = 0, OP_DIFF = 1, OP_APPLY = 2, OP_DIAG = 3 };

constexpr int kThreads = 128;  // threads per CTA of the pair passes
constexpr int kTile = 128;     // source edges staged in shared memory per tile

// One unit of the persistent pair-pass queue: targets [tgt0, tgt0 + ntgt) against sources
// [src0, src1); results go to partial slot `slot`.  [nb_lo, nb_hi] spans every edge that
// shares a vertex with some target of the item, so source tiles outside it skip the
// disjointness test.
struct WorkItem {
    int tgt0, ntgt, src0, src1, slot, nb_lo, nb_hi, pad;  // pad: problem index
};

// FP32 edge record (48 B): a = (g_i1, l), b = (g_i2, T.x), c = (T.y, T.z, i1, i2 as bits);
// lo = (low parts of g_i1 (3), low part of g_i2.x), lo2 = (g_i2.y low, g_i2.z low, 0, 0)
// (double-float positions, used by the mixed-precision pass only).
struct alignas(16) RecF {
    float4 a, b, c;
};
struct alignas(16) RecLo {
    float4 lo, lo2, lo3;  // lo2 = (g_i2.y lo, g_i2.z lo, T.x lo, T.y lo), lo3 = (T.z lo, 0, 0, 0)
};
// FP64 edge record (96 B).
struct alignas(16) RecD {
    double2 a0, a1;  // g_i1.xy, (g_i1.z, l)
    double2 b0, b1;  // g_i2.xy, (g_i2.z, T.x)
    double2 c0;      // T.y, T.z
    int i1, i2;
    int pad0, pad1;
};
// Per-edge data of the vector u in an apply: du = (u_j2 - u_j1)/l_J (3 comps), ub = (u_j1 + u_j2)/2,
// as double-float (hi + lo) so that the differences du_I - du_J, ub_I - ub_J are formed accurately.
// a = (du_hi.xyz, ub_hi.x), b = (ub_hi.yz, du_lo.xy), c = (du_lo.z, ub_lo.xyz).
struct alignas(16) URecF {
    float4 a, b, c;
};
struct alignas(16) URecD {
    double2 du0, du1, ub0, ub1;  // du.xy, (du.z, 0), ub.xy, (ub.z, 0)
};

struct KernelParams {
    double alpha, beta, p;  // kernel exponents and p = 2 sigma + 1
    int fast;               // (alpha, beta, p) == (2, 4.5, 2.5): specialised powers
    double near2;           // squared near-pair cutoff (mixed precision)
    float near2f;
    float near2f_diff;      // squared near cutoff of the differential (wider: its near terms cancel)
    float mid2f;            // squared distance below which a tile uses double-float differences
};

// Device-side scalars of one CG solve (all FP64) - one block per problem.
struct CGScalars {
    double rz, rz_new, pq, alpha, beta, bnorm2, rnorm2;
    double mq[3], mz[3];  // per-component means of q = A-bar p and z = M^-1 r (mean-free projector fused)
    int done, breakdown, iters;
};

// One captured block of CG iterations, reusable while everything it baked in is unchanged.
struct CgGraph {
    cudaGraphExec_t exec = nullptr;
    // key: the pointers and settings the captured launches depend on
    const double *gamma = nullptr;
    const void *items = nullptr;
    int which = -1, proj_mode = -1, precond = -1, every = 0, profile = 0, tpt = 0, sym = 0;
    double tol2 = -1.0;
    int64_t launches = 0;             // kernels per replay
    std::vector<cudaEvent_t> ev;      // profiling: (begin, end) per recorded pair kernel
    std::vector<int> prof_op;         // profiling: op of each (begin, end)
    int64_t stamp = 0;                // last use
};

struct Ctx {
    // graph
    int nV = 0, nE = 0, nCurves = 0, nProb = 0;
    int independent = 0;
    tp_params prm{};
    KernelParams kp{};
    std::vector<int32_t> h_edges, h_voff, h_eoff;
    std::vector<int32_t> h_prob_v, h_prob_e;  // per-problem vertex / edge offsets [nProb + 1]
    int32_t *d_edges = nullptr;                // [nE][2]
    int32_t *d_inc_ptr = nullptr;              // [nV + 1] incidence CSR
    int32_t *d_inc = nullptr;                  // [2 nE]: edge * 2 + slot (slot 1 <=> v is i2)
    int32_t *d_vprob = nullptr;                // [nV] problem of each vertex
    int32_t *d_eprob = nullptr;                // [nE] problem of each edge
    int32_t *d_prob_v = nullptr, *d_prob_e = nullptr;
    // spectral preconditioner (closed curves only)
    int spectral_ok = 0;
    std::vector<int32_t> h_curve_n;            // vertices of each curve
    int32_t *d_voff = nullptr;                 // [nCurves + 1]
    int max_curve_n = 0;
    SpecState *spec = nullptr;
    CoarseState *coarse = nullptr;
    // pair-pass work lists, one per pair op class (blocking depends on targets per thread)
    struct Plan {
        WorkItem *d_items = nullptr;
        int n_items = 0;
        int max_slots = 0;
        int grid = 0;
        int tpt = 0;
        int32_t *d_eslots = nullptr;  // [nE] number of partial slots of each target row
    };
    Plan plan_energy, plan_diff, plan_apply;
    int tpt[3] = {0, 0, 0};  // targets per thread chosen by tp_autotune (energy, diff, apply + diag); 0: default
    Plan plan_sym;           // symmetric apply (pairs_sym.cu): items over edge-block pairs (b, c >= b)
    int apply_sym = 0;       // > 0: the apply runs the symmetric pass with this many targets per thread
    Plan plan_sym_e;         // symmetric energy (pairs_sym.cu)
    int energy_sym = 0;      // > 0: the energy runs the symmetric pass with this many targets per thread
    Plan plan_sym_d;         // symmetric differential (pairs_sym.cu)
    int diff_sym = 0;        // > 0: the differential runs the symmetric pass
    Plan plan_df;            // double-float apply (pairs_df.cu), built at its first use
    Plan plan_multi;         // multi-field apply (pairs_multi.cu), built at its first use
    URecF *d_urecMF = nullptr;  // multi-field apply: per-edge records of kMultiG fields (FP32 contexts)
    URecD *d_urecMD = nullptr;  // the same in FP64 contexts
    double *d_partM = nullptr;  // multi-field apply: partial sums [slot][nE][6 kMultiG]
    int multi_ready = 0;
    int *d_counter = nullptr;  // persistent-queue counters [16]
    // edge records
    RecF *d_recF = nullptr, *d_recF2 = nullptr;
    RecLo *d_recLo = nullptr, *d_recLo2 = nullptr;
    RecD *d_recD = nullptr, *d_recD2 = nullptr;
    float *d_ell_lo[2] = {nullptr, nullptr};  // low parts of the edge lengths (double-float apply)
    // FP64 edge quantities of the two geometries (0: base curve, 1: trial curve): [nE], [nE][3], [nE][3]
    double *d_ellw[2] = {nullptr, nullptr}, *d_Tw[2] = {nullptr, nullptr}, *d_xw[2] = {nullptr, nullptr};
    double mean_ell = 0.0;
    double extent = 0.0;  // bounding-box diagonal of the first curve seen
    URecF *d_urecF = nullptr;
    URecD *d_urecD = nullptr;
    // partial results [max_slots][nE][6] (FP64)
    double *d_part = nullptr;
    size_t part_elems = 0;
    double *d_rows = nullptr;  // [nE]
    double *d_esum = nullptr;  // [nE][6] per-edge slot sums of the two-stage gather
    // constraints: per problem x0 (3) and L0
    double *d_x0L0 = nullptr;  // [nProb][4]
    int constraints_set = 0;
    double *d_Cv = nullptr;    // [nV][4][3] constraint Jacobian at the current curve
    double *d_G = nullptr;     // [nProb][16] C C^T
    double *d_Ginv = nullptr;  // [nProb][16]
    double *d_red = nullptr;   // reduction scratch [nProb][16]
    double *d_phi = nullptr;   // [nProb][4]
    // CG vectors [nV][3]
    double *d_y = nullptr, *d_r = nullptr, *d_z = nullptr, *d_p = nullptr, *d_q = nullptr, *d_diag = nullptr;
    double *d_t1 = nullptr, *d_t2 = nullptr, *d_t3 = nullptr, *d_t4 = nullptr;  // temporaries [nV][3]
    double *d_gam = nullptr;   // trial curve [nV][3]
    double *d_E = nullptr;     // [nProb]
    double *d_scal = nullptr;  // generic device scalars [64 + 8 nProb]
    CGScalars *d_cg = nullptr; // [nProb]
    int *d_err = nullptr;      // device error word
    double *h_pinned = nullptr;  // pinned host staging [64 + 8 nProb]
    int *h_pinned_i = nullptr;
    int64_t launches = 0;
    std::string err;
    int sm_count = 0;
    SolverState *sol = nullptr;
    double *d_best = nullptr;  // [nV][3] line-search result
    double *d_yw0 = nullptr, *d_yw1 = nullptr;  // [nV][3] last gradient solutions (warm starts of the next step)
    int warm_ok = 0;                            // d_yw0 / d_yw1 hold solutions of an earlier step
    int warm1_ok = 0;                           // total-length route: d_yw1 holds the last projection solution
    double *d_t5 = nullptr, *d_t6 = nullptr;
    int64_t pairs_per_pass = 0;
    const int *d_skip = nullptr;  // during a CG solve: per-problem converged flags (apply skips them)
    GnnState *gnn = nullptr;      // learned preconditioner term (contexts created with TP_PRECOND_LEARNED)
    EdgeState *edges = nullptr;   // edge-length constraint rows (edges.cu), allocated when first selected
    CcdState *ccd = nullptr;      // collision-time work list (ccd.cu), allocated when first used
    BhState *bh = nullptr;        // Barnes-Hut hierarchy (bh.cu), allocated when first used
    PenState *pen = nullptr;      // penalties of Sec. 8.1 (penalties.cu), allocated by tp_set_penalties
    PinState *pins = nullptr;     // point / tangent / surface rows of TP_CONSTRAINTS_POINTS (pins.cu)
    // captured CG iteration blocks
    cudaStream_t cg_stream = nullptr;
    cudaEvent_t cg_join[2] = {nullptr, nullptr};
    std::vector<CgGraph> graphs;
    CgGraph *capturing = nullptr;  // set while a block is being captured (profiling records into it)
    int64_t graph_clock = 0;
    int graphs_broken = 0;         // a capture failed: direct launches from then on
    int setups_since_full = -1;    // preconditioner set-ups since the last full one (-1: none yet)
    std::vector<double> last_rr;   // per problem: true relative residual of the last CG solve
    int last_refinements = 0;      // correction solves of the last CG solve (iterative refinement)
    double *d_rf = nullptr, *d_ef = nullptr;  // [nV][3] refinement residual and correction
    double *d_rs = nullptr;                   // [nV][3] refinement: the accurate residual before a correction
    std::vector<int> last_iters;   // per problem: its iterations
    // (residual, iterate) capture of a CG solve: every `every` iterations r -> R[n], y -> Y[n]
    struct Harvest {
        double *R = nullptr, *Y = nullptr;
        int every = 1, max = 0, n = 0;
    } hv;
    // per-kernel event timing (tp_profile)
    int profile = 0;
    std::vector<cudaEvent_t> prof_pool;
    std::vector<std::pair<int, int>> prof_pending;  // (op, slot)
    double prof_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int64_t prof_n[8] = {0, 0, 0, 0, 0, 0, 0, 0};
};

int prof_begin(Ctx &c, int op, cudaStream_t s);
void prof_end(Ctx &c, int slot, cudaStream_t s);
void prof_harvest(Ctx &c);
void graphs_free(Ctx &c);
void graphs_reset(Ctx &c);  // drop the captured blocks (their launches baked in parameters that changed)

// ------------------------------------------------------------------ pair passes (pairs.cu)
cudaError_t build_records(Ctx &c, const double *gamma, int which, cudaStream_t s);
cudaError_t build_urecs(Ctx &c, const double *u, int which_geom, cudaStream_t s);
// per-edge records of u into the given arrays (one of them NULL) instead of the context's
cudaError_t build_urecs_into(Ctx &c, const double *u, int which_geom, URecF *uf, URecD *ud, cudaStream_t s);
cudaError_t pair_energy(Ctx &c, const double *gamma, int which, double *rows_out, double *E_out, cudaStream_t s);
cudaError_t pair_diff(Ctx &c, const double *gamma, int which, double *dE, cudaStream_t s);
cudaError_t pair_apply(Ctx &c, const double *gamma_geom, int which, const double *u, double *Au, cudaStream_t s);
cudaError_t pair_diag(Ctx &c, const double *gamma_geom, int which, double *diag, cudaStream_t s);
// (pairs_df.cu) the apply in double-float arithmetic: the accurate operator of residual checks
cudaError_t pair_apply_acc(Ctx &c, const double *gamma_geom, int which, const double *u, double *Au, cudaStream_t s);
// AU_f = A-bar U_f for m vector fields ([m][nV][3] each), kMultiG fields per pair pass
constexpr int kMultiG = 4;
cudaError_t pair_apply_multi(Ctx &c, const double *gamma_geom, int which, const double *U, double *AU, int m,
                             cudaStream_t s);
void multi_free(Ctx &c);
void plan_pass(Ctx &c, Ctx::Plan &pl, int tpt, int occupancy);
void sym_plan_items(Ctx &c, Ctx::Plan &pl, int tpt, int occupancy);  // (pairs_sym.cu) items (b, c >= b)
cudaError_t gather_apply(Ctx &c, const Ctx::Plan &pl, double *Au, cudaStream_t s);
cudaError_t sym_select(Ctx &c, int tpt);  // (pairs_sym.cu) symmetric apply on (tpt 1, 2) or off (0)
cudaError_t sym_apply_pass(Ctx &c, int which, const double *gamma, const double *u, cudaStream_t s);
size_t sym_slots(const Ctx &c, int tpt);
cudaError_t sym_select_energy(Ctx &c, int tpt);
cudaError_t sym_energy_pass(Ctx &c, int which, const double *gamma, cudaStream_t s);
cudaError_t sym_select_diff(Ctx &c, int tpt);
cudaError_t sym_diff_pass(Ctx &c, int which, const double *gamma, cudaStream_t s);
void make_plans(Ctx &c);
cudaError_t replan(Ctx &c, int cls);  // rebuild the plan of one op class (0 energy, 1 diff, 2 apply/diag)
int tpt_default(const Ctx &c, int cls);
int tpt_candidates(const Ctx &c, int cls, int *out);  // the autotuner's search space; returns the count

// ------------------------------------------------------------------ solver pieces (solver.cu)
cudaError_t constraints_eval(Ctx &c, const double *gamma, int which, double *phi, cudaStream_t s);
cudaError_t constraints_jacobian(Ctx &c, int which, cudaStream_t s);
cudaError_t constraints_targets(Ctx &c, int which, cudaStream_t s);
cudaError_t project(Ctx &c, double *v, cudaStream_t s, const int *skip_flag);
cudaError_t pinv_apply(Ctx &c, const double *b_phi, double scale, double *out, cudaStream_t s);
cudaError_t spectral_setup(Ctx &c, cudaStream_t s);
cudaError_t spectral_rq_setup(Ctx &c, const double *gamma_geom, int which, cudaStream_t s);
cudaError_t coarse_setup(Ctx &c, const double *gamma_geom, int which, cudaStream_t s);
cudaError_t coarse_apply(Ctx &c, const double *r, double *z, cudaStream_t s);
cudaError_t coarse_balanced_apply(Ctx &c, const double *r, double *z, cudaStream_t s, const int *skip, bool learned);
cudaError_t coarse_balanced_part(Ctx &c, int which, const double *v, double *out, cudaStream_t s);
inline bool precond_learned(int p) { return p == TP_PRECOND_LEARNED || p == TP_PRECOND_LEARNED_BALANCED; }
inline bool precond_balanced(int p) { return p == TP_PRECOND_TWOLEVEL_BALANCED || p == TP_PRECOND_LEARNED_BALANCED; }
cudaError_t spectral_apply(Ctx &c, const double *r, double *z, cudaStream_t s, const int *skip);
void coarse_free(Ctx &c);
cudaError_t spectral_symbol_copy(Ctx &c, int rq, double *out, cudaStream_t s);
void spectral_free(Ctx &c);
cudaError_t precond_apply(Ctx &c, const double *r, double *z, cudaStream_t s, const int *skip_flag);
cudaError_t spectral_apply_ex(Ctx &c, const double *r, double *z, cudaStream_t s, const int *skip,
                              const double *diag, const double *ilam, const double *vlog);
const double *spectral_ilam(Ctx &c, cudaStream_t s);
cudaError_t precond_apply_base(Ctx &c, const double *r, double *z, cudaStream_t s, const int *skip_flag);
cudaError_t coarse_init(Ctx &c);
cudaError_t solver_setup(Ctx &c);
void solver_free(Ctx &c);
// x0 (optional, may alias x): initial guess; a problem whose initial residual is not below |P rhs| starts
// from zero instead.  The tolerance is always relative to |P rhs|.
cudaError_t cg_solve(Ctx &c, const double *gamma_geom, int which, const double *rhs, double *x, double rtol,
                     int maxit, int *iters, double *rel_res, int *converged, int *breakdown, cudaStream_t s,
                     int proj_mode, int *conv_flags = nullptr, const double *x0 = nullptr);
cudaError_t project_mean(Ctx &c, double *v, cudaStream_t s, const int *skip);
cudaError_t schur_shift(Ctx &c, double *out, const double *phi, double phi_scale, cudaStream_t s);
cudaError_t bary_rhs(Ctx &c, const double *dE, double *rhs, cudaStream_t s);
// edge-length constraints (edges.cu)
bool edges_chains_ok(const Ctx &c, std::string &why);
cudaError_t edges_init(Ctx &c);
void edges_free(Ctx &c);
cudaError_t edges_targets(Ctx &c, int which, cudaStream_t s);
cudaError_t edges_setup(Ctx &c, int which, cudaStream_t s);
cudaError_t edges_project(Ctx &c, double *v, cudaStream_t s, const int *skip);
cudaError_t edges_pinv(Ctx &c, double *out, cudaStream_t s);
cudaError_t edges_phi(Ctx &c, int which, double *phi, cudaStream_t s);
// penalties of Sec. 8.1 (penalties.cu)
cudaError_t penalties_set(Ctx &c, const tp_penalties *p);
void penalties_free(Ctx &c);
bool penalties_active(const Ctx &c);
cudaError_t penalties_add(Ctx &c, int which, double *E, double *dE, cudaStream_t s);
// first collision time along a direction (ccd.cu)
cudaError_t ccd_init(Ctx &c);
void ccd_free(Ctx &c);
// Barnes-Hut comparator (bh.cu): op OP_ENERGY (rows, E) or OP_DIFF (dE)
cudaError_t bh_pass(Ctx &c, const double *gamma, int op, double eps, int leaf_size, double *rows, double *E,
                    double *dE, cudaStream_t s, int &unsupported);
void bh_stats(const Ctx &c, unsigned long long *adm, unsigned long long *pairs, int *depth, double *build_s);
void bh_free(Ctx &c);
// E[q] = sum of rows over problem q's edges
cudaError_t segment_sum(Ctx &c, const double *rows, double *E, cudaStream_t s);
cudaError_t ccd_time(Ctx &c, const double *gamma, const double *d, double T, double *tmin, cudaStream_t s);
inline bool edge_constraints(const Ctx &c)
{
    return c.edges && c.prm.constraint_set == TP_CONSTRAINTS_EDGE_LENGTHS;
}
// point, tangent and surface constraints of Sec. 8.1 (pins.cu)
bool pins_ready(const Ctx &c);
cudaError_t pins_set(Ctx &c, int n, const int32_t *vertices, const double *targets, std::string &why);
cudaError_t tangents_set(Ctx &c, int n, const int32_t *edges, const double *X, std::string &why);
cudaError_t surface_set(Ctx &c, const double *quadric, int n, const int32_t *vertices, std::string &why);
void pins_free(Ctx &c);
cudaError_t pins_phi(Ctx &c, const double *gamma, int which, double *phi, cudaStream_t s);
cudaError_t pins_fields(Ctx &c, const double *gamma, double *rhs_scratch, int *iters, double *rr, int *conv,
                        int *bd, int *flags, cudaStream_t s);
cudaError_t pins_gradient(Ctx &c, const double *gamma, const double *dE, const double *y0, const double *y1,
                          double *g, cudaStream_t s);
cudaError_t pins_projection(Ctx &c, const double *y1, const double *gamma_t, const double *phi, double *x,
                            cudaStream_t s);
inline bool pin_constraints(const Ctx &c)
{
    return c.prm.constraint_set == TP_CONSTRAINTS_POINTS;
}
cudaError_t clen_rhs(Ctx &c, double *out, cudaStream_t s);
cudaError_t schur_gradient(Ctx &c, const double *y0, const double *y1, double *g, cudaStream_t s);
cudaError_t schur_projection(Ctx &c, const double *y1, const double *phi, double phi_scale, double *x,
                             cudaStream_t s);
cudaError_t vec_dot(Ctx &c, const double *a, const double *b, double *out_dev, cudaStream_t s);
cudaError_t vec_axpby(Ctx &c, double a, const double *x, double b, const double *y, double *out, cudaStream_t s);
cudaError_t vec_scale_dev(Ctx &c, const double *x, const double *num_dev, int invert_sqrt, double *out,
                          cudaStream_t s);
cudaError_t sum_problems(Ctx &c, const double *per_edge_or_vertex, int per_vertex, double *out, cudaStream_t s,
                         int add = 0);

// ------------------------------------------------------------------ learned preconditioner (gnn.cu)
int gnn_num_params();
cudaError_t gnn_alloc(Ctx &c);
void gnn_free(Ctx &c);
int gnn_ready(const Ctx &c);
int gnn_bound(const Ctx &c);
cudaError_t gnn_set_params(Ctx &c, const float *theta, int reset_adam, cudaStream_t s);
cudaError_t gnn_get_params(Ctx &c, float *theta, cudaStream_t s);
cudaError_t gnn_bind(Ctx &c, int which, const double *diag, cudaStream_t s);
double *gnn_diag_buffer(Ctx &c);
const float *gnn_features(const Ctx &c);
const float *gnn_outputs(const Ctx &c);
const float *gnn_last_grad(const Ctx &c);
cudaError_t gnn_forward(Ctx &c, cudaStream_t s);
cudaError_t gnn_backward(Ctx &c, const float *dout, float *grad, cudaStream_t s);
cudaError_t gnn_adam(Ctx &c, const float *grad, float lr, cudaStream_t s);
cudaError_t gnn_gapply(Ctx &c, const double *r, double *z, int accumulate, cudaStream_t s, const int *skip);
cudaError_t gnn_out_grad(Ctx &c, const double *r, const double *gz, double scale, int accumulate, float *dout,
                         cudaStream_t s);
cudaError_t gnn_problem_dot(Ctx &c, const double *a, const double *b, double *out, cudaStream_t s);
cudaError_t gnn_train_step(Ctx &c, const double *gamma, int n_pairs, const double *R, const double *B,
                           const double *AB, const double *ER, const double *ilam, const double *R2, float lr,
                           double *loss_dev, cudaStream_t s);
const double *gnn_vlog(const Ctx &c);

}  // namespace tpe

struct tp_ctx {
    tpe::Ctx c;
};
