// C ABI of the GB300 tangent-point library: context creation, the entry points of include/tpe.h,
// and the host orchestration of a descent step (Sec. 5.4): gradient solve, normalised direction,
// backtracking with constraint projection (Sec. 5.3.2 via App. B.3.4) and the Armijo test.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "tpe_internal.cuh"

using namespace tpe;

namespace {

tp_status fail(tp_ctx *ctx, tp_status st, const std::string &msg)
{
    if (ctx) ctx->c.err = msg;
    return st;
}

tp_status cuda_fail(tp_ctx *ctx, cudaError_t e, const char *where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return fail(ctx, TP_ERR_OOM, m);
    return fail(ctx, TP_ERR_CUDA, m);
}

#define CK(call)                                            \
    do {                                                    \
        cudaError_t e__ = (call);                           \
        if (e__ != cudaSuccess) return cuda_fail(ctx, e__, #call); \
    } while (0)

bool params_ok(const tp_params *p, std::string &why)
{
    if (!(p->alpha > 1.0)) {
        why = "alpha must be > 1";
        return false;
    }
    if (!(p->beta >= p->alpha + 2.0 - 1e-12 && p->beta < 2.0 * p->alpha + 1.0)) {
        why = "beta must lie in [alpha + 2, 2 alpha + 1)";
        return false;
    }
    if (p->precision < TP_FP64 || p->precision > TP_MIXED) {
        why = "bad precision";
        return false;
    }
    if (p->precond < TP_PRECOND_NONE || p->precond > TP_PRECOND_LEARNED_BALANCED) {
        why = "bad preconditioner";
        return false;
    }
    if (p->coarse_dim < 2) {
        why = "coarse_dim must be >= 2";
        return false;
    }
    if (p->constraint_set != TP_CONSTRAINTS_TOTAL_LENGTH && p->constraint_set != TP_CONSTRAINTS_EDGE_LENGTHS &&
        p->constraint_set != TP_CONSTRAINTS_POINTS) {
        why = "bad constraint_set";
        return false;
    }
    if ((p->line_search != TP_LINESEARCH_UNIT && p->line_search != TP_LINESEARCH_ISOTOPY) || !(p->ccd_horizon > 0.0)) {
        why = "bad line_search or ccd_horizon";
        return false;
    }
    if (p->precond_refresh < 1) {
        why = "precond_refresh must be >= 1";
        return false;
    }
    if (!(p->far_cutoff >= 0.0)) {
        why = "far_cutoff must be >= 0";
        return false;
    }
    if (!(p->cg_rtol > 0.0) || p->cg_maxit < 1 || !(p->shrink > 0.0 && p->shrink < 1.0) || p->max_halvings < 0 ||
        p->proj_maxit < 0 || !(p->proj_tol > 0.0)) {
        why = "bad solver or line-search parameter";
        return false;
    }
    return true;
}

void set_kernel_params(Ctx &c)
{
    const tp_params &p = c.prm;
    double sigma = std::isnan(p.sigma) ? (p.beta - 1.0) / p.alpha - 1.0 : p.sigma;
    c.kp.alpha = p.alpha;
    c.kp.beta = p.beta;
    c.kp.p = 2.0 * sigma + 1.0;
    c.kp.fast = (p.alpha == 2.0 && p.beta == 4.5 && c.kp.p == 2.5) ? 1 : 0;
    double rn = p.near_cutoff * c.mean_ell;
    c.kp.near2 = rn * rn;
    c.kp.near2f = (float)(rn * rn);
    // the differential's near-pair gradient terms are large and cancel between the two sides of a
    // vertex, so they get FP64 over a 4x wider band than the energy
    c.kp.near2f_diff = (float)(16.0 * rn * rn);
    // tiles closer than far_cutoff x the curve's extent use double-float differences (mixed path)
    double rm = std::max(p.far_cutoff * c.extent, rn);
    c.kp.mid2f = p.far_cutoff >= 10.0 ? 3.0e38f : (float)(rm * rm);
}

// Bounding-box diagonal of the vertex positions (host read; scales the double-float tile cutoff).
__global__ void k_extent(int nV, const double *g, double *out)
{
    __shared__ double sh[6][256];
    double b[6] = {1e300, 1e300, 1e300, -1e300, -1e300, -1e300};
    for (int i = threadIdx.x; i < nV; i += blockDim.x)
        for (int k = 0; k < 3; ++k) {
            b[k] = fmin(b[k], g[3 * i + k]);
            b[3 + k] = fmax(b[3 + k], g[3 * i + k]);
        }
    for (int k = 0; k < 6; ++k) sh[k][threadIdx.x] = b[k];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int k = 0; k < 6; ++k)
                sh[k][threadIdx.x] = k < 3 ? fmin(sh[k][threadIdx.x], sh[k][threadIdx.x + w])
                                           : fmax(sh[k][threadIdx.x], sh[k][threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < 3; ++k) s += (sh[3 + k][0] - sh[k][0]) * (sh[3 + k][0] - sh[k][0]);
        *out = sqrt(s);
    }
}

// FP64 mean edge length of geometry `which` (host read; used to scale the near-pair cutoff).
__global__ void k_sum_ell(int n, const double *ell, double *out)
{
    __shared__ double sh[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += ell[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

tp_status check_err_word(tp_ctx *ctx, cudaStream_t s)
{
    Ctx &c = ctx->c;
    int e = 0;
    CK(cudaMemcpyAsync(c.h_pinned_i + 1, c.d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    e = c.h_pinned_i[1];
    if (e) {
        CK(cudaMemsetAsync(c.d_err, 0, sizeof(int), s));
        if (e == TP_ERR_DEGENERATE_EDGE) return fail(ctx, TP_ERR_DEGENERATE_EDGE, "an edge has zero length");
        if (e == TP_ERR_NONFINITE) return fail(ctx, TP_ERR_NONFINITE, "non-finite vertex position");
        return fail(ctx, (tp_status)e, "device error");
    }
    return TP_OK;
}

// Build the edge records of `gamma` into geometry slot `which`; on the first call also fix the
// mean edge length that scales the near-pair cutoff.
tp_status records(tp_ctx *ctx, const double *gamma, int which, cudaStream_t s)
{
    Ctx &c = ctx->c;
    CK(build_records(c, gamma, which, s));
    if (c.mean_ell == 0.0 && c.nE > 0) {
        k_sum_ell<<<1, 256, 0, s>>>(c.nE, c.d_ellw[which], c.d_scal);
        k_extent<<<1, 256, 0, s>>>(c.nV, gamma, c.d_scal + 1);
        c.launches += 2;
        CK(cudaMemcpyAsync(c.h_pinned, c.d_scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        c.mean_ell = c.h_pinned[0] / c.nE;
        c.extent = c.h_pinned[1];
        set_kernel_params(c);
        tp_status st = check_err_word(ctx, s);
        if (st != TP_OK) {
            c.mean_ell = 0.0;
            return st;
        }
    }
    return TP_OK;
}

template <class T>
cudaError_t dalloc(T **p, size_t n)
{
    return cudaMalloc((void **)p, sizeof(T) * std::max<size_t>(1, n));
}

}  // namespace

extern "C" {

void tp_default_params(tp_params *p)
{
    if (!p) return;
    p->alpha = 2.0;
    p->beta = 4.5;
    p->sigma = NAN;
    p->precision = TP_FP32;
    p->near_cutoff = 4.0;
    p->cg_rtol = 1e-6;
    p->cg_maxit = 20000;
    p->cg_check_every = 8;
    p->proj_cg_rtol = 1e-6;
    p->precond = TP_PRECOND_SPECTRAL;
    p->armijo_c = 1e-4;
    p->shrink = 0.5;
    p->max_halvings = 30;
    p->proj_tol = 1e-10;
    p->proj_maxit = 5;
    p->independent = 0;
    p->far_cutoff = 10.0;
    p->use_graphs = 1;
    p->precond_refresh = 1;
    p->constraint_set = TP_CONSTRAINTS_TOTAL_LENGTH;
    p->line_search = TP_LINESEARCH_UNIT;
    p->ccd_horizon = 1.5;
    p->warm_start = 1;
    p->coarse_dim = 128;
}

const char *tp_last_error(const tp_ctx *ctx) { return ctx ? ctx->c.err.c_str() : "null context"; }

int tp_num_problems(const tp_ctx *ctx) { return ctx ? ctx->c.nProb : 0; }

int64_t tp_launch_count(const tp_ctx *ctx) { return ctx ? ctx->c.launches : 0; }

int64_t tp_pairs_per_pass(const tp_ctx *ctx) { return ctx ? ctx->c.pairs_per_pass : 0; }

tp_status tp_profile(tp_ctx *ctx, int enable)
{
    if (!ctx) return TP_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    prof_harvest(c);
    for (int k = 0; k < 8; ++k) {
        c.prof_ms[k] = 0.0;
        c.prof_n[k] = 0;
    }
    c.profile = enable ? 1 : 0;
    return TP_OK;
}

tp_status tp_profile_read(tp_ctx *ctx, int op, double *total_ms, int64_t *launches)
{
    if (!ctx || op < 0 || op > 7) return TP_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    prof_harvest(c);
    if (total_ms) *total_ms = c.prof_ms[op];
    if (launches) *launches = c.prof_n[op];
    return TP_OK;
}

void tp_destroy(tp_ctx *ctx)
{
    if (!ctx) return;
    Ctx &c = ctx->c;
    graphs_free(c);
    sym_select(c, 0);
    sym_select_energy(c, 0);
    sym_select_diff(c, 0);
    if (c.sol) solver_free(c);
    spectral_free(c);
    coarse_free(c);
    gnn_free(c);
    edges_free(c);
    ccd_free(c);
    penalties_free(c);
    pins_free(c);
    multi_free(c);
    bh_free(c);
    void *ptrs[] = {c.d_esum, c.d_edges, c.d_inc_ptr, c.d_inc, c.d_vprob, c.d_eprob, c.d_prob_v, c.d_prob_e, c.d_voff,
                    c.plan_energy.d_items, c.plan_diff.d_items, c.plan_apply.d_items, c.plan_energy.d_eslots,
                    c.plan_diff.d_eslots, c.plan_apply.d_eslots, c.d_counter, c.d_recF, c.d_recF2, c.d_recLo,
                    c.d_recLo2, c.d_recD, c.d_recD2, c.d_ellw[0], c.d_ellw[1], c.d_Tw[0], c.d_Tw[1], c.d_xw[0],
                    c.d_xw[1], c.d_urecF, c.d_urecD, c.d_part, c.d_rows, c.d_x0L0, c.d_Cv, c.d_G, c.d_Ginv,
                    c.d_red, c.d_phi, c.d_y, c.d_r, c.d_z, c.d_p, c.d_q, c.d_diag, c.d_t1, c.d_t2, c.d_t3, c.d_t4,
                    c.d_t5, c.d_t6, c.d_gam, c.d_best, c.d_yw0, c.d_yw1, c.d_E, c.d_scal, c.d_cg, c.d_err,
                    c.d_ell_lo[0], c.d_ell_lo[1], c.plan_df.d_items, c.plan_df.d_eslots, c.d_rf, c.d_ef, c.d_rs};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    prof_harvest(c);
    for (auto &e : c.prof_pool) cudaEventDestroy(e);
    if (c.h_pinned) cudaFreeHost(c.h_pinned);
    if (c.h_pinned_i) cudaFreeHost(c.h_pinned_i);
    delete ctx;
}

tp_status tp_create(tp_ctx **out, int nV, int nE, const int32_t *edges_host, int n_curves,
                    const int32_t *voff_host, const int32_t *eoff_host, const tp_params *p)
{
    if (!out) return TP_ERR_INVALID_ARG;
    *out = nullptr;
    tp_ctx *ctx = new (std::nothrow) tp_ctx();
    if (!ctx) return TP_ERR_OOM;
    *out = ctx;
    Ctx &c = ctx->c;
    tp_params prm;
    if (p)
        prm = *p;
    else
        tp_default_params(&prm);
    std::string why;
    if (!params_ok(&prm, why)) return fail(ctx, TP_ERR_INVALID_ARG, why);
    if (nV < 1 || nE < 0 || n_curves < 1 || (nE > 0 && !edges_host) || !voff_host || !eoff_host)
        return fail(ctx, TP_ERR_INVALID_ARG, "bad graph sizes or null pointers");
    if (nE == 0) return fail(ctx, TP_ERR_INVALID_ARG, "the graph has no edges (its energy is 0 and nothing moves)");
    if (voff_host[0] != 0 || eoff_host[0] != 0 || voff_host[n_curves] != nV || eoff_host[n_curves] != nE)
        return fail(ctx, TP_ERR_INVALID_ARG, "curve offsets must start at 0 and end at n_vertices / n_edges");
    for (int k = 0; k < n_curves; ++k)
        if (voff_host[k + 1] < voff_host[k] || eoff_host[k + 1] < eoff_host[k])
            return fail(ctx, TP_ERR_INVALID_ARG, "curve offsets must be non-decreasing");
    c.prm = prm;
    c.nV = nV;
    c.nE = nE;
    c.nCurves = n_curves;
    c.independent = prm.independent ? 1 : 0;
    c.h_edges.assign(edges_host, edges_host + 2 * (size_t)nE);
    c.h_voff.assign(voff_host, voff_host + n_curves + 1);
    c.h_eoff.assign(eoff_host, eoff_host + n_curves + 1);
    // validate edges: in range, two distinct endpoints, inside their curve's vertex range
    for (int k = 0; k < n_curves; ++k)
        for (int I = eoff_host[k]; I < eoff_host[k + 1]; ++I) {
            int a = edges_host[2 * I], b = edges_host[2 * I + 1];
            if (a < voff_host[k] || a >= voff_host[k + 1] || b < voff_host[k] || b >= voff_host[k + 1] || a == b)
                return fail(ctx, TP_ERR_INVALID_ARG, "edge " + std::to_string(I) + " is not a proper edge of its curve");
        }
    if (c.independent) {
        c.nProb = n_curves;
        c.h_prob_v = c.h_voff;
        c.h_prob_e = c.h_eoff;
    } else {
        c.nProb = 1;
        c.h_prob_v = {0, nV};
        c.h_prob_e = {0, nE};
    }
    // closed-curve check for the spectral preconditioner: curve k's edges are (v0+i, v0+(i+1) mod n)
    c.spectral_ok = 1;
    c.h_curve_n.resize(n_curves);
    for (int k = 0; k < n_curves; ++k) {
        int v0 = voff_host[k], n = voff_host[k + 1] - v0, e0 = eoff_host[k], m = eoff_host[k + 1] - e0;
        c.h_curve_n[k] = n;
        c.max_curve_n = std::max(c.max_curve_n, n);
        if (n != m || n < 4) {
            c.spectral_ok = 0;
            continue;
        }
        for (int i = 0; i < n; ++i)
            if (edges_host[2 * (e0 + i)] != v0 + i || edges_host[2 * (e0 + i) + 1] != v0 + (i + 1) % n) {
                c.spectral_ok = 0;
                break;
            }
    }
    if ((prm.precond >= TP_PRECOND_SPECTRAL) && !c.spectral_ok)
        return fail(ctx, TP_ERR_UNSUPPORTED,
                    "the spectral preconditioner needs every curve to be a closed polygon (i, i+1 mod n) of >= 4 vertices");
    if (precond_balanced(prm.precond) && c.nProb != n_curves)
        return fail(ctx, TP_ERR_UNSUPPORTED, "the balancing two-level form needs every problem to be one curve");
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&c.sm_count, cudaDevAttrMultiProcessorCount, dev));
    // incidence lists
    std::vector<int> deg(nV + 1, 0), inc(2 * (size_t)nE), vprob(nV), eprob(std::max(1, nE));
    for (int I = 0; I < nE; ++I) {
        deg[c.h_edges[2 * I] + 1]++;
        deg[c.h_edges[2 * I + 1] + 1]++;
    }
    for (int v = 0; v < nV; ++v) deg[v + 1] += deg[v];
    std::vector<int> fill(deg.begin(), deg.end() - 1);
    for (int I = 0; I < nE; ++I)
        for (int s = 0; s < 2; ++s) inc[fill[c.h_edges[2 * I + s]]++] = 2 * I + s;
    for (int q = 0; q < c.nProb; ++q) {
        for (int v = c.h_prob_v[q]; v < c.h_prob_v[q + 1]; ++v) vprob[v] = q;
        for (int I = c.h_prob_e[q]; I < c.h_prob_e[q + 1]; ++I) eprob[I] = q;
    }
    // ordered disjoint pairs per pass: n_q^2 minus, per edge, the edges sharing a vertex with it
    c.pairs_per_pass = 0;
    for (int q = 0; q < c.nProb; ++q) {
        int64_t n = c.h_prob_e[q + 1] - c.h_prob_e[q];
        int64_t excl = 0;
        for (int I = c.h_prob_e[q]; I < c.h_prob_e[q + 1]; ++I) {
            std::vector<int> nb;
            for (int s = 0; s < 2; ++s) {
                int v = c.h_edges[2 * I + s];
                for (int k = deg[v]; k < deg[v + 1]; ++k) nb.push_back(inc[k] >> 1);
            }
            std::sort(nb.begin(), nb.end());
            excl += std::unique(nb.begin(), nb.end()) - nb.begin();
        }
        c.pairs_per_pass += n * n - excl;
    }
    const bool p64 = prm.precision == TP_FP64, mix = prm.precision == TP_MIXED;
    CK(dalloc(&c.d_edges, 2 * (size_t)nE));
    CK(cudaMemcpy(c.d_edges, c.h_edges.data(), sizeof(int) * 2 * nE, cudaMemcpyHostToDevice));
    CK(dalloc(&c.d_inc_ptr, nV + 1));
    CK(cudaMemcpy(c.d_inc_ptr, deg.data(), sizeof(int) * (nV + 1), cudaMemcpyHostToDevice));
    CK(dalloc(&c.d_inc, 2 * (size_t)nE));
    CK(cudaMemcpy(c.d_inc, inc.data(), sizeof(int) * 2 * nE, cudaMemcpyHostToDevice));
    CK(dalloc(&c.d_vprob, nV));
    CK(cudaMemcpy(c.d_vprob, vprob.data(), sizeof(int) * nV, cudaMemcpyHostToDevice));
    CK(dalloc(&c.d_eprob, nE));
    CK(cudaMemcpy(c.d_eprob, eprob.data(), sizeof(int) * std::max(1, nE), cudaMemcpyHostToDevice));
    CK(dalloc(&c.d_prob_v, c.nProb + 1));
    CK(cudaMemcpy(c.d_prob_v, c.h_prob_v.data(), sizeof(int) * (c.nProb + 1), cudaMemcpyHostToDevice));
    CK(dalloc(&c.d_prob_e, c.nProb + 1));
    CK(cudaMemcpy(c.d_prob_e, c.h_prob_e.data(), sizeof(int) * (c.nProb + 1), cudaMemcpyHostToDevice));
    CK(dalloc(&c.d_voff, n_curves + 1));
    CK(cudaMemcpy(c.d_voff, c.h_voff.data(), sizeof(int) * (n_curves + 1), cudaMemcpyHostToDevice));
    for (int w = 0; w < 2; ++w) {
        CK(dalloc(&c.d_ellw[w], nE));
        CK(dalloc(&c.d_Tw[w], 3 * (size_t)nE));
        CK(dalloc(&c.d_xw[w], 3 * (size_t)nE));
    }
    if (p64) {
        CK(dalloc(&c.d_recD, nE));
        CK(dalloc(&c.d_recD2, nE));
        CK(dalloc(&c.d_urecD, nE));
    } else {
        CK(dalloc(&c.d_recF, nE));
        CK(dalloc(&c.d_recF2, nE));
        CK(dalloc(&c.d_urecF, nE));
        CK(dalloc(&c.d_recLo, nE));
        CK(dalloc(&c.d_recLo2, nE));
        CK(dalloc(&c.d_ell_lo[0], nE));
        CK(dalloc(&c.d_ell_lo[1], nE));
    }
    CK(dalloc(&c.d_counter, 16));
    CK(cudaMemset(c.d_counter, 0, sizeof(int) * 16));
    set_kernel_params(c);
    make_plans(c);
    CK(cudaGetLastError());
    int ms = std::max(std::max(c.plan_energy.max_slots, c.plan_diff.max_slots), c.plan_apply.max_slots);
    c.part_elems = (size_t)ms * std::max(1, nE) * 6;
    CK(dalloc(&c.d_part, c.part_elems));
    CK(dalloc(&c.d_rows, nE));
    CK(dalloc(&c.d_esum, 6 * (size_t)nE));
    CK(dalloc(&c.d_x0L0, 4 * (size_t)c.nProb));
    CK(dalloc(&c.d_Cv, 12 * (size_t)nV));
    CK(dalloc(&c.d_G, 16 * (size_t)c.nProb));
    CK(dalloc(&c.d_Ginv, 16 * (size_t)c.nProb));
    CK(dalloc(&c.d_red, 16 * (size_t)c.nProb));
    CK(dalloc(&c.d_phi, 4 * (size_t)c.nProb));
    double **vecs[] = {&c.d_y, &c.d_r, &c.d_z, &c.d_p, &c.d_q, &c.d_t1, &c.d_t2, &c.d_t3, &c.d_t4, &c.d_t5, &c.d_t6,
                       &c.d_gam, &c.d_best, &c.d_yw0, &c.d_yw1, &c.d_rf, &c.d_ef, &c.d_rs};
    for (double **v : vecs) CK(dalloc(v, 3 * (size_t)nV));
    CK(cudaMemset(c.d_z, 0, sizeof(double) * 3 * nV));
    CK(dalloc(&c.d_diag, nV));
    CK(dalloc(&c.d_E, c.nProb));
    CK(dalloc(&c.d_scal, 64 + 16 * (size_t)c.nProb));
    CK(dalloc(&c.d_cg, c.nProb));
    CK(dalloc(&c.d_err, 4));
    CK(cudaMemset(c.d_err, 0, sizeof(int) * 4));
    CK(cudaMallocHost(&c.h_pinned, sizeof(double) * (64 + 16 * (size_t)c.nProb)));
    CK(cudaMallocHost(&c.h_pinned_i, sizeof(int) * 64));
    CK(solver_setup(c));
    if (prm.precond >= TP_PRECOND_SPECTRAL) {
        cudaError_t e = spectral_setup(c, 0);
        if (e == cudaErrorNotSupported) return fail(ctx, TP_ERR_UNSUPPORTED, "spectral preconditioner not built");
        CK(e);
    }
    if (prm.precond >= TP_PRECOND_TWOLEVEL) CK(coarse_init(c));
    if (precond_learned(prm.precond)) CK(gnn_alloc(c));
    if (prm.constraint_set == TP_CONSTRAINTS_EDGE_LENGTHS) {
        if (!edges_chains_ok(c, why)) return fail(ctx, TP_ERR_INVALID_ARG, why);
        CK(edges_init(c));
    }
    if (prm.line_search == TP_LINESEARCH_ISOTOPY) CK(ccd_init(c));
    CK(cudaDeviceSynchronize());
    return TP_OK;
}

tp_status tp_set_params(tp_ctx *ctx, const tp_params *p)
{
    if (!ctx || !p) return TP_ERR_INVALID_ARG;
    std::string why;
    if (!params_ok(p, why)) return fail(ctx, TP_ERR_INVALID_ARG, why);
    Ctx &c = ctx->c;
    if (p->precision != c.prm.precision) return fail(ctx, TP_ERR_INVALID_ARG, "precision is fixed at creation");
    if ((p->precond >= TP_PRECOND_SPECTRAL) && !c.spectral_ok)
        return fail(ctx, TP_ERR_UNSUPPORTED, "the spectral preconditioner needs closed polygons");
    if (precond_learned(p->precond) && !c.gnn)
        return fail(ctx, TP_ERR_UNSUPPORTED, "the learned preconditioners need a context created with one of them");
    if (precond_balanced(p->precond) && c.nProb != c.nCurves)
        return fail(ctx, TP_ERR_UNSUPPORTED, "the balancing two-level form needs every problem to be one curve");
    if (p->constraint_set == TP_CONSTRAINTS_EDGE_LENGTHS && !c.edges) {
        if (!edges_chains_ok(c, why)) return fail(ctx, TP_ERR_INVALID_ARG, why);
        CK(edges_init(c));
        CK(cudaDeviceSynchronize());
    }
    if (p->line_search == TP_LINESEARCH_ISOTOPY && !c.ccd) {
        CK(ccd_init(c));
        CK(cudaDeviceSynchronize());
    }
    // a new constraint set takes its targets from the next curve solved, as on a fresh context
    if (p->constraint_set != c.prm.constraint_set) c.constraints_set = 0;
    int indep = c.prm.independent;
    int had_spectral = c.spec != nullptr;
    c.prm = *p;
    c.prm.independent = indep;
    set_kernel_params(c);
    graphs_reset(c);  // captured CG blocks baked in the old kernel parameters
    c.setups_since_full = -1;  // the next preconditioner set-up is a full one
    if (!c.kp.fast && (c.tpt[0] || c.tpt[1] || c.tpt[2] || c.apply_sym || c.energy_sym || c.diff_sym)) {
        // autotuned variants exist for the specialised powers only: back to the defaults
        for (int cls = 0; cls < 3; ++cls) {
            c.tpt[cls] = 0;
            CK(replan(c, cls));
        }
        CK(sym_select(c, 0));
        CK(sym_select_energy(c, 0));
        CK(sym_select_diff(c, 0));
    }
    if ((p->precond >= TP_PRECOND_SPECTRAL) && !had_spectral) {
        cudaError_t e = spectral_setup(c, 0);
        if (e == cudaErrorNotSupported) return fail(ctx, TP_ERR_UNSUPPORTED, "spectral preconditioner not built");
        CK(e);
        CK(cudaDeviceSynchronize());
    }
    if (p->precond >= TP_PRECOND_TWOLEVEL) CK(coarse_init(c));
    return TP_OK;
}

tp_status tp_energy(tp_ctx *ctx, const double *gamma, double *E, double *rows, tp_stream stream)
{
    if (!ctx || !gamma) return TP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    tp_status st = records(ctx, gamma, 0, s);
    if (st) return st;
    CK(pair_energy(ctx->c, gamma, 0, rows, E, s));
    return TP_OK;
}

tp_status tp_differential(tp_ctx *ctx, const double *gamma, double *dE, double *E, tp_stream stream)
{
    if (!ctx || !gamma || !dE) return TP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    tp_status st = records(ctx, gamma, 0, s);
    if (st) return st;
    CK(pair_diff(ctx->c, gamma, 0, dE, s));
    if (E) CK(pair_energy(ctx->c, gamma, 0, nullptr, E, s));
    return TP_OK;
}

tp_status sobolev_apply(tp_ctx *ctx, const double *gamma, const double *u, double *Au, tp_stream stream)
{
    if (!ctx || !gamma || !u || !Au) return TP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    tp_status st = records(ctx, gamma, 0, s);
    if (st) return st;
    CK(pair_apply(ctx->c, gamma, 0, u, Au, s));
    return TP_OK;
}

tp_status sobolev_apply_multi(tp_ctx *ctx, const double *gamma, const double *U, double *AU, int m, tp_stream stream)
{
    if (!ctx || !gamma || m < 0 || (m > 0 && (!U || !AU))) return TP_ERR_INVALID_ARG;
    if (m == 0) return TP_OK;
    cudaStream_t s = (cudaStream_t)stream;
    tp_status st = records(ctx, gamma, 0, s);
    if (st) return st;
    CK(pair_apply_multi(ctx->c, gamma, 0, U, AU, m, s));
    return TP_OK;
}

tp_status sobolev_apply_accurate(tp_ctx *ctx, const double *gamma, const double *u, double *Au, tp_stream stream)
{
    if (!ctx || !gamma || !u || !Au) return TP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    tp_status st = records(ctx, gamma, 0, s);
    if (st) return st;
    CK(pair_apply_acc(ctx->c, gamma, 0, u, Au, s));
    return check_err_word(ctx, s);
}

tp_status tp_gram_diagonal(tp_ctx *ctx, const double *gamma, double *diag, tp_stream stream)
{
    if (!ctx || !gamma || !diag) return TP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    tp_status st = records(ctx, gamma, 0, s);
    if (st) return st;
    CK(pair_diag(ctx->c, gamma, 0, diag, s));
    return TP_OK;
}

tp_status tp_set_constraints_from(tp_ctx *ctx, const double *gamma, tp_stream stream)
{
    if (!ctx || !gamma) return TP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    tp_status st = records(ctx, gamma, 0, s);
    if (st) return st;
    CK(constraints_targets(ctx->c, 0, s));
    ctx->c.constraints_set = 1;
    return TP_OK;
}

// TP_CONSTRAINTS_POINTS without pins has no constraint rows to solve with.
static tp_status need_pins(tp_ctx *ctx)
{
    if (pin_constraints(ctx->c) && !pins_ready(ctx->c))
        return fail(ctx, TP_ERR_INVALID_ARG, "TP_CONSTRAINTS_POINTS: no pinned vertices (tp_set_pins)");
    return TP_OK;
}

tp_status tp_set_pins(tp_ctx *ctx, int n, const int32_t *vertices, const double *targets)
{
    if (!ctx) return TP_ERR_INVALID_ARG;
    std::string why;
    cudaError_t e = pins_set(ctx->c, n, vertices, targets, why);
    if (e == cudaErrorInvalidValue && !why.empty()) return fail(ctx, TP_ERR_INVALID_ARG, why);
    CK(e);
    return TP_OK;
}

tp_status tp_set_tangents(tp_ctx *ctx, int n, const int32_t *edges, const double *X)
{
    if (!ctx) return TP_ERR_INVALID_ARG;
    std::string why;
    cudaError_t e = tangents_set(ctx->c, n, edges, X, why);
    if (e == cudaErrorInvalidValue && !why.empty()) return fail(ctx, TP_ERR_INVALID_ARG, why);
    CK(e);
    return TP_OK;
}

tp_status tp_set_surface(tp_ctx *ctx, const double *quadric, int n, const int32_t *vertices)
{
    if (!ctx) return TP_ERR_INVALID_ARG;
    std::string why;
    cudaError_t e = surface_set(ctx->c, quadric, n, vertices, why);
    if (e == cudaErrorInvalidValue && !why.empty()) return fail(ctx, TP_ERR_INVALID_ARG, why);
    CK(e);
    return TP_OK;
}

tp_status tp_constraints(tp_ctx *ctx, const double *gamma, double *phi, tp_stream stream)
{
    if (!ctx || !gamma || !phi) return TP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    tp_status st = need_pins(ctx);
    if (st) return st;
    st = records(ctx, gamma, 0, s);
    if (st) return st;
    if (!ctx->c.constraints_set) {
        CK(constraints_targets(ctx->c, 0, s));
        ctx->c.constraints_set = 1;
    }
    CK(constraints_eval(ctx->c, gamma, 0, phi, s));
    return TP_OK;
}

tp_status tp_set_penalties(tp_ctx *ctx, const tp_penalties *pen)
{
    if (!ctx) return TP_ERR_INVALID_ARG;
    if (pen) {
        bool ok = std::isfinite(pen->w_length) && std::isfinite(pen->w_length_diff) && std::isfinite(pen->w_field);
        for (int k = 0; k < 9; ++k) ok = ok && std::isfinite(pen->field_M[k]);
        for (int k = 0; k < 3; ++k) ok = ok && std::isfinite(pen->field_b[k]);
        if (!ok) return fail(ctx, TP_ERR_INVALID_ARG, "penalty weights and field must be finite");
    }
    CK(penalties_set(ctx->c, pen));
    return TP_OK;
}

tp_status tp_penalty(tp_ctx *ctx, const double *gamma, double *E, double *dE, tp_stream stream)
{
    if (!ctx || !gamma) return TP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Ctx &c = ctx->c;
    tp_status st = records(ctx, gamma, 0, s);
    if (st) return st;
    if (E) CK(cudaMemsetAsync(E, 0, sizeof(double) * c.nProb, s));
    if (dE) CK(cudaMemsetAsync(dE, 0, sizeof(double) * 3 * (size_t)c.nV, s));
    CK(penalties_add(c, 0, E, dE, s));
    return TP_OK;
}

static tp_status bh_call(tp_ctx *ctx, const double *gamma, int op, double eps, int leaf_size, double *rows,
                         double *E, double *dE, tp_stream stream)
{
    if (!(eps >= 0.0) || leaf_size < 1 || leaf_size > 64)
        return fail(ctx, TP_ERR_INVALID_ARG, "Barnes-Hut: eps must be >= 0 and leaf_size in [1, 64]");
    cudaStream_t s = (cudaStream_t)stream;
    tp_status st = records(ctx, gamma, 0, s);  // the degenerate-edge check
    if (st) return st;
    int unsupported = 0;
    CK(bh_pass(ctx->c, gamma, op, eps, leaf_size, rows, E, dE, s, unsupported));
    if (unsupported)
        return fail(ctx, TP_ERR_UNSUPPORTED, "Barnes-Hut: a vertex joins more than 15 edges, or the hierarchy is too deep");
    return TP_OK;
}

tp_status tp_bh_energy(tp_ctx *ctx, const double *gamma, double eps, int leaf_size, double *E, double *rows,
                       tp_stream stream)
{
    if (!ctx || !gamma || (!E && !rows)) return TP_ERR_INVALID_ARG;
    return bh_call(ctx, gamma, OP_ENERGY, eps, leaf_size, rows, E, nullptr, stream);
}

tp_status tp_bh_differential(tp_ctx *ctx, const double *gamma, double eps, int leaf_size, double *dE,
                             tp_stream stream)
{
    if (!ctx || !gamma || !dE) return TP_ERR_INVALID_ARG;
    return bh_call(ctx, gamma, OP_DIFF, eps, leaf_size, nullptr, nullptr, dE, stream);
}

tp_status tp_bh_stats(const tp_ctx *ctx, int64_t *admissible_nodes, int64_t *leaf_pairs, int32_t *depth,
                      double *build_seconds)
{
    if (!ctx) return TP_ERR_INVALID_ARG;
    unsigned long long a = 0, p = 0;
    int d = 0;
    double bs = 0.0;
    bh_stats(ctx->c, &a, &p, &d, &bs);
    if (admissible_nodes) *admissible_nodes = (int64_t)a;
    if (leaf_pairs) *leaf_pairs = (int64_t)p;
    if (depth) *depth = d;
    if (build_seconds) *build_seconds = bs;
    return TP_OK;
}

tp_status tp_collision_time(tp_ctx *ctx, const double *gamma, const double *d, double horizon, double *t,
                            tp_stream stream)
{
    if (!ctx || !gamma || !d || !t) return TP_ERR_INVALID_ARG;
    if (!(horizon > 0.0)) return fail(ctx, TP_ERR_INVALID_ARG, "horizon must be > 0");
    cudaStream_t s = (cudaStream_t)stream;
    tp_status st = records(ctx, gamma, 0, s);  // mean edge length (the box padding) and the degenerate-edge check
    if (st) return st;
    CK(ccd_time(ctx->c, gamma, d, horizon, t, s));
    return TP_OK;
}

// Preconditioner set-up for the geometry in slot 0: diag(A); the Rayleigh-quotient corrected
// symbols (TP_PRECOND_SPECTRAL_RQ and up); the coarse space (TP_PRECOND_TWOLEVEL and up); the
// learned term's features and network outputs (TP_PRECOND_LEARNED).
static tp_status precond_setup(tp_ctx *ctx, const double *gamma, cudaStream_t s)
{
    Ctx &c = ctx->c;
    if (precond_learned(c.prm.precond) && !gnn_ready(c))
        return fail(ctx, TP_ERR_INVALID_ARG, "learned preconditioner: no network parameters loaded (tp_gnn_set_params)");
    if (c.prm.precond != TP_PRECOND_NONE) CK(pair_diag(c, gamma, 0, c.d_diag, s));
    // the fitted symbols and the coarse space are rebuilt every precond_refresh-th set-up (any SPD
    // preconditioner keeps PCG exact; the curve moves little between consecutive descent steps)
    const bool full = c.setups_since_full < 0 || c.setups_since_full + 1 >= std::max(1, c.prm.precond_refresh);
    c.setups_since_full = full ? 0 : c.setups_since_full + 1;
    if (full && c.prm.precond >= TP_PRECOND_SPECTRAL_RQ) CK(spectral_rq_setup(c, gamma, 0, s));
    if (full && c.prm.precond >= TP_PRECOND_TWOLEVEL) CK(coarse_setup(c, gamma, 0, s));
    if (precond_learned(c.prm.precond)) {
        CK(gnn_bind(c, 0, c.d_diag, s));
        CK(gnn_forward(c, s));
    }
    return TP_OK;
}

tp_status tp_precond_apply(tp_ctx *ctx, const double *gamma, const double *r, double *z, tp_stream stream)
{
    if (!ctx || !gamma || !r || !z) return TP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Ctx &c = ctx->c;
    tp_status st = records(ctx, gamma, 0, s);
    if (st) return st;
    st = precond_setup(ctx, gamma, s);
    if (st) return st;
    CK(precond_apply(c, r, z, s, nullptr));
    return TP_OK;
}

tp_status tp_spectral_symbols(tp_ctx *ctx, int rq, double *out, tp_stream stream)
{
    if (!ctx || !out) return TP_ERR_INVALID_ARG;
    if (!ctx->c.spec) return fail(ctx, TP_ERR_UNSUPPORTED, "no spectral preconditioner in this context");
    CK(spectral_symbol_copy(ctx->c, rq, out, (cudaStream_t)stream));
    return TP_OK;
}


// H^s gradient of Eq. 22 by the mean-free route: y0 = A^+ dE, y1 = A^+ C_len^T (two CG solves on the
// mean-free subspace), then the 4x4 correction (schur_gradient).  dE first loses C_bary^T lambda_bary,
// the barycenter multiplier (zero for a translation-invariant dE).  Needs the Jacobian of `gamma` in
// c.d_Cv and the preconditioner set up.  Uses d_t3, d_t4, d_t5, d_t6 as scratch.
static cudaError_t gradient_solve(Ctx &c, const double *gamma, const double *dE_in, double *g, int *iters, double *rr,
                                  int *conv, int *bd, cudaStream_t s, int *n_conv = nullptr)
{
    std::vector<int> flags(c.nProb, 1);
    if (pin_constraints(c)) {
        // y0 = A^+ dE, y1 = A^+ C_len^T, the pins' fields A^+ e_v, then the Schur complement (pins.cu); no
        // barycenter multiplier: the pins' rows take up N^T dE
        int it = 0, cv = 1, b = 0;
        double r = 0.0;
        int i0 = 0, c0 = 0, b0 = 0;
        double r0 = 0.0;
        cudaError_t e = cg_solve(c, gamma, 0, dE_in, c.d_t3, c.prm.cg_rtol, c.prm.cg_maxit, &i0, &r0, &c0, &b0, s, 1,
                                 flags.data(), (c.warm_ok && c.prm.warm_start) ? c.d_yw0 : nullptr);
        if (e != cudaSuccess) return e;
        it += i0;
        r = std::max(r, r0);
        cv = cv && c0;
        b = b || b0;
        if ((e = clen_rhs(c, c.d_t6, s)) != cudaSuccess) return e;
        e = cg_solve(c, gamma, 0, c.d_t6, c.d_t4, c.prm.cg_rtol, c.prm.cg_maxit, &i0, &r0, &c0, &b0, s, 1,
                     flags.data(), (c.warm_ok && c.prm.warm_start) ? c.d_yw1 : nullptr);
        if (e != cudaSuccess) return e;
        it += i0;
        r = std::max(r, r0);
        cv = cv && c0;
        b = b || b0;
        if ((e = pins_fields(c, gamma, c.d_t6, &it, &r, &cv, &b, flags.data(), s)) != cudaSuccess) return e;
        const size_t vb = sizeof(double) * 3 * c.nV;
        if ((e = cudaMemcpyAsync(c.d_yw0, c.d_t3, vb, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(c.d_yw1, c.d_t4, vb, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
        c.warm_ok = 1;
        if (n_conv) {
            *n_conv = 0;
            for (int f : flags) *n_conv += f;
        }
        *iters = it;
        *rr = r;
        *conv = cv;
        *bd = b;
        return pins_gradient(c, gamma, dE_in, c.d_t3, c.d_t4, g, s);
    }
    {
        cudaError_t e = bary_rhs(c, dE_in, c.d_t5, s);
        if (e != cudaSuccess) return e;
    }
    const double *dE = c.d_t5;
    if (edge_constraints(c)) {
        // y on null(R) cap N-perp (projector mode 2), then the translation that restores the barycenter
        cudaError_t e = edges_setup(c, 0, s);
        if (e != cudaSuccess) return e;
        e = cg_solve(c, gamma, 0, dE, g, c.prm.cg_rtol, c.prm.cg_maxit, iters, rr, conv, bd, s, 2, flags.data(),
                     (c.warm_ok && c.prm.warm_start) ? c.d_yw0 : nullptr);
        if (e != cudaSuccess) return e;
        e = cudaMemcpyAsync(c.d_yw0, g, sizeof(double) * 3 * c.nV, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
        c.warm_ok = 1;
        if (n_conv) {
            *n_conv = 0;
            for (int f : flags) *n_conv += f;
        }
        return schur_shift(c, g, nullptr, 0.0, s);
    }
    if (precond_balanced(c.prm.precond)) {
        // One projected solve P A-bar P y = P dE with P = P_len P_N (the total-length row and the mean), then
        // the translation that restores the barycenter rows: the KKT solution of Eq. 22 (App. B.3.3 with
        // the translations handled apart).  It starts from the previous step's solution.  The balancing
        // preconditioner resolves the smooth modes through its coarse space, where C_len lives; the
        // one-level preconditioners amplify exactly those modes, and the projected operator then needs
        // thousands of iterations, so they keep the two mean-free solves below.
        cudaError_t e = cg_solve(c, gamma, 0, dE, g, c.prm.cg_rtol, c.prm.cg_maxit, iters, rr, conv, bd, s, 3,
                                 flags.data(), (c.warm_ok && c.prm.warm_start) ? c.d_yw0 : nullptr);
        if (e != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(c.d_yw0, g, sizeof(double) * 3 * c.nV, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
            return e;
        c.warm_ok = 1;
        if (n_conv) {
            *n_conv = 0;
            for (int f : flags) *n_conv += f;
        }
        return schur_shift(c, g, nullptr, 0.0, s);
    }
    int i0 = 0, i1 = 0, c0 = 0, c1 = 0, b0 = 0, b1 = 0;
    double r0 = 0, r1 = 0;
    // y0 = A^+ dE, y1 = A^+ C_len^T (mean-free), both from the previous step's solutions
    cudaError_t e = cg_solve(c, gamma, 0, dE, c.d_t3, c.prm.cg_rtol, c.prm.cg_maxit, &i0, &r0, &c0, &b0, s, 1,
                             flags.data(), (c.warm_ok && c.prm.warm_start) ? c.d_yw0 : nullptr);
    if (e != cudaSuccess) return e;
    e = clen_rhs(c, c.d_t6, s);
    if (e != cudaSuccess) return e;
    e = cg_solve(c, gamma, 0, c.d_t6, c.d_t4, c.prm.cg_rtol, c.prm.cg_maxit, &i1, &r1, &c1, &b1, s, 1, flags.data(),
                 (c.warm_ok && c.prm.warm_start) ? c.d_yw1 : nullptr);
    if (e != cudaSuccess) return e;
    const size_t vb = sizeof(double) * 3 * c.nV;
    if ((e = cudaMemcpyAsync(c.d_yw0, c.d_t3, vb, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(c.d_yw1, c.d_t4, vb, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
    c.warm_ok = 1;
    c.warm1_ok = 1;
    if (n_conv) {
        *n_conv = 0;
        for (int f : flags) *n_conv += f;
    }
    e = schur_gradient(c, c.d_t3, c.d_t4, g, s);
    *iters = i0 + i1;
    *rr = std::max(r0, r1);
    *conv = c0 && c1;
    *bd = b0 || b1;
    return e;
}

tp_status sobolev_gradient(tp_ctx *ctx, const double *gamma, const double *dE, double *g, tp_solve_info *info,
                           tp_stream stream)
{
    if (!ctx || !gamma || !dE || !g) return TP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Ctx &c = ctx->c;
    tp_status st = need_pins(ctx);
    if (st) return st;
    st = records(ctx, gamma, 0, s);
    if (st) return st;
    if (!c.constraints_set) {
        CK(constraints_targets(c, 0, s));
        c.constraints_set = 1;
    }
    CK(constraints_jacobian(c, 0, s));
    st = precond_setup(ctx, gamma, s);
    if (st) return st;
    int it = 0, conv = 0, bd = 0, nconv = 0;
    double rr = 0.0;
    CK(gradient_solve(c, gamma, dE, g, &it, &rr, &conv, &bd, s, &nconv));
    if (info) {
        info->iters = it;
        info->rel_res = rr;
        info->converged = conv;
        info->n_converged = nconv;
    }
    st = check_err_word(ctx, s);
    if (st) return st;
    if (bd) return fail(ctx, TP_ERR_BREAKDOWN, "CG breakdown: p^T A p <= 0");
    if (!conv) return fail(ctx, TP_ERR_NOT_CONVERGED, "CG did not reach cg_rtol within cg_maxit");
    return TP_OK;
}

// gamma_out = gamma_in - tau_q d (per problem)
__global__ void k_trial(int nV, const double *__restrict__ g, const double *__restrict__ d,
                        const double *__restrict__ tau, const int *__restrict__ vprob, double *__restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nV) return;
    double t = tau[vprob[i]];
    for (int k = 0; k < 3; ++k) out[3 * i + k] = g[3 * i + k] - t * d[3 * i + k];
}

// dst[v] = src[v] for the vertices of problems with mask[q] != 0
__global__ void k_copy_masked(int nV, const double *__restrict__ src, const int *__restrict__ mask,
                              const int *__restrict__ vprob, double *__restrict__ dst)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nV) return;
    if (!mask[vprob[i]]) return;
    for (int k = 0; k < 3; ++k) dst[3 * i + k] = src[3 * i + k];
}

// x += a - b (b may be NULL)
__global__ void k_add(int n, double *__restrict__ x, const double *__restrict__ a, const double *__restrict__ b)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] += a[i] - (b ? b[i] : 0.0);
}

tp_status descent_step(tp_ctx *ctx, double *gamma, tp_step_info *info, tp_stream stream)
{
    if (!ctx || !gamma) return TP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Ctx &c = ctx->c;
    const int nP = c.nProb, nV = c.nV;
    const size_t vb = sizeof(double) * 3 * nV;
    const int nb = (nV + 255) / 256;
    tp_status st = need_pins(ctx);
    if (st) return st;
    st = records(ctx, gamma, 0, s);
    if (st) return st;
    if (!c.constraints_set) {
        CK(constraints_targets(c, 0, s));
        c.constraints_set = 1;
    }
    // E(gamma), dE(gamma)
    double *E0 = c.d_scal + 64, *E1 = c.d_scal + 64 + nP, *gg = c.d_scal + 64 + 2 * nP,
           *slope = c.d_scal + 64 + 3 * nP, *tau_d = c.d_scal + 64 + 4 * nP;
    double *dE = c.d_t1, *g = c.d_t2, *dir = c.d_t3, *z = c.d_t4, *rhs = c.d_t5, *x = c.d_t6;
    // gradient_solve uses d_t3, d_t4, d_t6 as scratch before dir / z / x are written
    CK(pair_energy(c, gamma, 0, nullptr, E0, s));
    CK(pair_diff(c, gamma, 0, dE, s));
    CK(penalties_add(c, 0, E0, dE, s));  // Sec. 8.1 penalties, if any
    // g~ = projected H^s gradient
    CK(constraints_jacobian(c, 0, s));
    st = precond_setup(ctx, gamma, s);
    if (st) return st;
    int it = 0, conv = 0, bd = 0, nconv = 0;
    double rr = 0.0;
    CK(gradient_solve(c, gamma, dE, g, &it, &rr, &conv, &bd, s, &nconv));
    if (bd) return fail(ctx, TP_ERR_BREAKDOWN, "CG breakdown in the gradient solve");
    // d = g / |g| per problem, slope = <dE, d>
    CK(vec_dot(c, g, g, gg, s));
    CK(vec_scale_dev(c, g, gg, 1, dir, s));
    CK(vec_dot(c, dE, dir, slope, s));
    std::vector<double> hE0(nP), hgg(nP), hslope(nP), hE1(nP), hphi(4 * (size_t)nP), hx0L0(4 * (size_t)nP);
    CK(cudaMemcpyAsync(hE0.data(), E0, sizeof(double) * nP, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hgg.data(), gg, sizeof(double) * nP, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hslope.data(), slope, sizeof(double) * nP, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hx0L0.data(), c.d_x0L0, sizeof(double) * 4 * nP, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    st = check_err_word(ctx, s);
    if (st) return st;
    // per-problem line search state
    std::vector<double> tau(nP, 1.0), acc_tau(nP, 0.0);
    if (c.prm.line_search == TP_LINESEARCH_ISOTOPY) {
        // Sec. 5.4: start at 2/3 of the first collision time along gamma - tau d
        double *tcol = c.d_scal + 64 + 6 * nP;
        CK(ccd_time(c, gamma, dir, c.prm.ccd_horizon, tcol, s));
        std::vector<double> ht(nP);
        CK(cudaMemcpyAsync(ht.data(), tcol, sizeof(double) * nP, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int q = 0; q < nP; ++q) tau[q] = 2.0 / 3.0 * ht[q];
    }
    std::vector<int> pending(nP, 1), accepted(nP, 0), acc_halv(nP, 0), acc_pit(nP, 0);
    for (int q = 0; q < nP; ++q)
        if (!(hgg[q] > 0.0)) {
            pending[q] = 0;
            accepted[q] = 1;
            hE1[q] = hE0[q];
        }
    int proj_cg_total = 0;
    int *mask_dev = reinterpret_cast<int *>(c.d_scal + 64 + 5 * nP);  // nP ints fit in 8 nP doubles
    // the total-length route's projection solves start from the last projection solution of the previous
    // step (A-bar^+ C_len^T at a nearby curve)
    int have_z = 0;
    if (!pin_constraints(c) && !edge_constraints(c) && c.warm1_ok) {
        CK(cudaMemcpyAsync(z, c.d_yw1, vb, cudaMemcpyDeviceToDevice, s));
        have_z = 1;
    }
    CK(cudaMemcpyAsync(c.d_best, gamma, vb, cudaMemcpyDeviceToDevice, s));
    for (int h = 0; h <= c.prm.max_halvings; ++h) {
        int npend = 0;
        for (int q = 0; q < nP; ++q) npend += pending[q];
        if (npend == 0) break;
        // trial = gamma - tau d (problems not pending use tau 0)
        std::vector<double> tq(nP);
        for (int q = 0; q < nP; ++q) tq[q] = pending[q] ? tau[q] : 0.0;
        CK(cudaMemcpyAsync(tau_d, tq.data(), sizeof(double) * nP, cudaMemcpyHostToDevice, s));
        k_trial<<<nb, 256, 0, s>>>(nV, gamma, dir, tau_d, c.d_vprob, c.d_gam);
        c.launches++;
        // constraint projection
        std::vector<int> ok(nP, 0), pit(nP, 0);
        for (int pi = 0;; ++pi) {
            st = records(ctx, c.d_gam, 1, s);
            if (st) return st;
            CK(constraints_eval(c, c.d_gam, 1, c.d_phi, s));
            CK(cudaMemcpyAsync(hphi.data(), c.d_phi, sizeof(double) * 4 * nP, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            st = check_err_word(ctx, s);
            if (st) return st;
            int all = 1;
            for (int q = 0; q < nP; ++q) {
                double m = 0.0;
                for (int k = 0; k < 4; ++k) m = std::max(m, std::fabs(hphi[4 * q + k]));
                ok[q] = std::isfinite(m) && m <= c.prm.proj_tol * std::max(1.0, hx0L0[4 * q + 3]);
                if (pending[q] && !ok[q]) all = 0;
            }
            if (all || pi >= c.prm.proj_maxit) break;
            for (int q = 0; q < nP; ++q)
                if (pending[q] && !ok[q]) pit[q] = pi + 1;
            // x = argmin x^T A-bar(gamma) x / 2 s.t. C(trial) x = -Phi(trial) (Eq. 23) by the mean-free route:
            // y1 = A-bar(gamma)^+ C_len(trial)^T, then x = mu y1 + N t; trial += x
            CK(constraints_jacobian(c, 1, s));
            int pit_cg = 0, pconv = 0, pbd = 0;
            double prr = 0.0;
            if (edge_constraints(c)) {
                // App. B.3.4 with the edge rows R(trial): z0 = R^T (R R^T)^-1 (l0 - l) (so R z0 = l0 - l),
                // y = argmin |z0 - y|_A over null(R) cap N-perp, x = z0 - y, then the barycenter shift
                double *z0 = g;  // free after the direction was formed
                CK(edges_setup(c, 1, s));
                CK(edges_pinv(c, z0, s));
                CK(pair_apply(c, gamma, 0, z0, rhs, s));
                CK(cg_solve(c, gamma, 0, rhs, z, c.prm.proj_cg_rtol, c.prm.cg_maxit, &pit_cg, &prr, &pconv, &pbd,
                            s, 2));
                CK(vec_axpby(c, 1.0, z0, -1.0, z, x, s));
                CK(schur_shift(c, x, c.d_phi, -1.0, s));
            } else if (pin_constraints(c)) {
                // y1 = A-bar(gamma)^+ C_len(trial)^T; the pins' fields of the gradient step stay valid (their
                // rows do not depend on the curve); x from the Schur complement (pins.cu)
                CK(clen_rhs(c, rhs, s));
                CK(cg_solve(c, gamma, 0, rhs, z, c.prm.proj_cg_rtol, c.prm.cg_maxit, &pit_cg, &prr, &pconv, &pbd,
                            s, 1, nullptr, c.prm.warm_start ? z : nullptr));
                CK(pins_projection(c, z, c.d_gam, c.d_phi, x, s));
            } else {
                CK(clen_rhs(c, rhs, s));
                // starts from z: A-bar^+ C_len^T of the previous trial or of the last step's projection, both
                // close to this trial's solution
                CK(cg_solve(c, gamma, 0, rhs, z, c.prm.proj_cg_rtol, c.prm.cg_maxit, &pit_cg, &prr, &pconv, &pbd,
                            s, 1, nullptr, (c.prm.warm_start && have_z) ? z : nullptr));
                have_z = 1;
                CK(schur_projection(c, z, c.d_phi, -1.0, x, s));
            }
            proj_cg_total += pit_cg;
            k_add<<<(3 * nV + 255) / 256, 256, 0, s>>>(3 * nV, c.d_gam, x, nullptr);
            c.launches++;
        }
        // energy of the projected trial and the Armijo test
        st = records(ctx, c.d_gam, 1, s);
        if (st) return st;
        CK(pair_energy(c, c.d_gam, 1, nullptr, E1, s));
        CK(penalties_add(c, 1, E1, nullptr, s));
        std::vector<double> e1(nP);
        CK(cudaMemcpyAsync(e1.data(), E1, sizeof(double) * nP, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        std::vector<int> acc_now(nP, 0);
        for (int q = 0; q < nP; ++q) {
            if (!pending[q]) continue;
            if (ok[q] && std::isfinite(e1[q]) && e1[q] <= hE0[q] - c.prm.armijo_c * tau[q] * hslope[q]) {
                acc_now[q] = 1;
                accepted[q] = 1;
                pending[q] = 0;
                acc_tau[q] = tau[q];
                acc_halv[q] = h;
                acc_pit[q] = pit[q];
                hE1[q] = e1[q];
            } else {
                tau[q] *= c.prm.shrink;
            }
        }
        CK(cudaMemcpyAsync(mask_dev, acc_now.data(), sizeof(int) * nP, cudaMemcpyHostToDevice, s));
        k_copy_masked<<<nb, 256, 0, s>>>(nV, c.d_gam, mask_dev, c.d_vprob, c.d_best);
        c.launches++;
    }
    int nacc = 0;
    for (int q = 0; q < nP; ++q) {
        if (!accepted[q]) hE1[q] = hE0[q];
        nacc += accepted[q];
    }
    if (have_z && !pin_constraints(c) && !edge_constraints(c)) {
        CK(cudaMemcpyAsync(c.d_yw1, z, vb, cudaMemcpyDeviceToDevice, s));
        c.warm1_ok = 1;
    }
    CK(cudaMemcpyAsync(gamma, c.d_best, vb, cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
    if (info) {
        double a = 0, b = 0, gn = 0, tmax = 0;
        int hmax = 0, pmax = 0;
        for (int q = 0; q < nP; ++q) {
            a += hE0[q];
            b += hE1[q];
            gn += hgg[q];
            tmax = std::max(tmax, acc_tau[q]);
            hmax = std::max(hmax, acc_halv[q]);
            pmax = std::max(pmax, acc_pit[q]);
        }
        info->E_before = a;
        info->E_after = b;
        info->tau = tmax;
        info->gnorm = std::sqrt(gn);
        info->halvings = hmax;
        info->proj_iters = pmax;
        info->cg_iters = it;
        info->proj_cg_iters = proj_cg_total;
        info->accepted = nacc;
        info->rel_res = rr;
        info->n_converged = nconv;
    }
    if (nacc < nP) return fail(ctx, TP_ERR_LINESEARCH, "line search failed for some problem");
    return TP_OK;
}

// ---------------------------------------------------------------------------------- learned preconditioner

int tp_gnn_num_params(void) { return gnn_num_params(); }

static tp_status need_gnn(tp_ctx *ctx)
{
    if (!ctx) return TP_ERR_INVALID_ARG;
    if (!ctx->c.gnn) return fail(ctx, TP_ERR_UNSUPPORTED, "the context was not created with a learned preconditioner");
    return TP_OK;
}

tp_status tp_gnn_set_params(tp_ctx *ctx, const float *theta, int reset_optimizer, tp_stream stream)
{
    tp_status st = need_gnn(ctx);
    if (st) return st;
    if (!theta) return fail(ctx, TP_ERR_INVALID_ARG, "null parameter vector");
    CK(gnn_set_params(ctx->c, theta, reset_optimizer, (cudaStream_t)stream));
    return TP_OK;
}

tp_status tp_gnn_get_params(tp_ctx *ctx, float *theta, tp_stream stream)
{
    tp_status st = need_gnn(ctx);
    if (st) return st;
    if (!theta) return fail(ctx, TP_ERR_INVALID_ARG, "null parameter vector");
    if (!gnn_ready(ctx->c)) return fail(ctx, TP_ERR_INVALID_ARG, "no parameters loaded");
    CK(gnn_get_params(ctx->c, theta, (cudaStream_t)stream));
    return TP_OK;
}

tp_status tp_gnn_bind(tp_ctx *ctx, const double *gamma, tp_stream stream)
{
    tp_status st = need_gnn(ctx);
    if (st) return st;
    if (!gamma) return fail(ctx, TP_ERR_INVALID_ARG, "null curve");
    cudaStream_t s = (cudaStream_t)stream;
    Ctx &c = ctx->c;
    st = records(ctx, gamma, 0, s);
    if (st) return st;
    CK(pair_diag(c, gamma, 0, gnn_diag_buffer(c), s));
    CK(gnn_bind(c, 0, gnn_diag_buffer(c), s));
    return TP_OK;
}

tp_status tp_gnn_forward(tp_ctx *ctx, float *features, float *out, tp_stream stream)
{
    tp_status st = need_gnn(ctx);
    if (st) return st;
    Ctx &c = ctx->c;
    if (!gnn_ready(c) || !gnn_bound(c)) return fail(ctx, TP_ERR_INVALID_ARG, "parameters or geometry missing");
    cudaStream_t s = (cudaStream_t)stream;
    CK(gnn_forward(c, s));
    if (features) CK(cudaMemcpyAsync(features, gnn_features(c), sizeof(float) * TP_GNN_FEATURES * c.nE,
                                     cudaMemcpyDeviceToDevice, s));
    if (out) CK(cudaMemcpyAsync(out, gnn_outputs(c), sizeof(float) * 3 * c.nE, cudaMemcpyDeviceToDevice, s));
    return TP_OK;
}

tp_status tp_gnn_backward(tp_ctx *ctx, const float *dout, float *grad, tp_stream stream)
{
    tp_status st = need_gnn(ctx);
    if (st) return st;
    if (!dout || !grad) return fail(ctx, TP_ERR_INVALID_ARG, "null pointer");
    if (!gnn_ready(ctx->c) || !gnn_bound(ctx->c)) return fail(ctx, TP_ERR_INVALID_ARG, "parameters or geometry missing");
    CK(gnn_backward(ctx->c, dout, grad, (cudaStream_t)stream));
    return TP_OK;
}

tp_status tp_gnn_adam(tp_ctx *ctx, const float *grad, float lr, tp_stream stream)
{
    tp_status st = need_gnn(ctx);
    if (st) return st;
    if (!grad || !(lr >= 0.f)) return fail(ctx, TP_ERR_INVALID_ARG, "null gradient or bad learning rate");
    if (!gnn_ready(ctx->c)) return fail(ctx, TP_ERR_INVALID_ARG, "no parameters loaded");
    CK(gnn_adam(ctx->c, grad, lr, (cudaStream_t)stream));
    return TP_OK;
}

tp_status tp_gnn_g_apply(tp_ctx *ctx, const double *r, double *z, int accumulate, tp_stream stream)
{
    tp_status st = need_gnn(ctx);
    if (st) return st;
    if (!r || !z) return fail(ctx, TP_ERR_INVALID_ARG, "null pointer");
    if (!gnn_ready(ctx->c) || !gnn_bound(ctx->c)) return fail(ctx, TP_ERR_INVALID_ARG, "parameters or geometry missing");
    CK(gnn_gapply(ctx->c, r, z, accumulate, (cudaStream_t)stream, nullptr));
    return TP_OK;
}

tp_status tp_gnn_out_grad(tp_ctx *ctx, const double *r, const double *gz, float *dout, int accumulate,
                          tp_stream stream)
{
    tp_status st = need_gnn(ctx);
    if (st) return st;
    if (!r || !gz || !dout) return fail(ctx, TP_ERR_INVALID_ARG, "null pointer");
    if (!gnn_ready(ctx->c) || !gnn_bound(ctx->c)) return fail(ctx, TP_ERR_INVALID_ARG, "parameters or geometry missing");
    CK(gnn_out_grad(ctx->c, r, gz, 1.0, accumulate, dout, (cudaStream_t)stream));
    return TP_OK;
}

tp_status tp_cg_harvest(tp_ctx *ctx, const double *gamma, const double *rhs, int every, int max_pairs, double *R,
                        double *E, int *n_pairs, tp_solve_info *info, tp_stream stream)
{
    if (!ctx || !gamma || !rhs || !n_pairs || every < 1 || max_pairs < 0 || (max_pairs > 0 && (!R || !E)))
        return fail(ctx, TP_ERR_INVALID_ARG, "bad harvest arguments");
    cudaStream_t s = (cudaStream_t)stream;
    Ctx &c = ctx->c;
    tp_status st = records(ctx, gamma, 0, s);
    if (st) return st;
    st = precond_setup(ctx, gamma, s);
    if (st) return st;
    c.hv.R = max_pairs > 0 ? R : nullptr;
    c.hv.Y = E;
    c.hv.every = every;
    c.hv.max = max_pairs;
    c.hv.n = 0;
    int it = 0, conv = 0, bd = 0;
    double rr = 0.0;
    cudaError_t e = cg_solve(c, gamma, 0, rhs, c.d_t3, c.prm.cg_rtol, c.prm.cg_maxit, &it, &rr, &conv, &bd, s, 1);
    const int n = c.hv.n;
    c.hv = Ctx::Harvest{};
    CK(e);
    // exact corrections: e_k = y* - y_k (every iterate lies in the mean-free subspace)
    const size_t nv3 = 3 * (size_t)c.nV;
    for (int k = 0; k < n; ++k) CK(vec_axpby(c, 1.0, c.d_t3, -1.0, E + k * nv3, E + k * nv3, s));
    *n_pairs = n;
    if (info) {
        info->iters = it;
        info->rel_res = rr;
        info->converged = conv;
        info->n_converged = conv ? c.nProb : 0;
    }
    st = check_err_word(ctx, s);
    if (st) return st;
    if (bd) return fail(ctx, TP_ERR_BREAKDOWN, "CG breakdown: p^T A p <= 0");
    return TP_OK;
}

tp_status tp_gnn_prepare_pairs(tp_ctx *ctx, const double *gamma, int n, double *R, double *E, double *B,
                               double *AB, double *ER, double *ILAM, double *R2, tp_stream stream)
{
    if (!ctx || !gamma || n < 0 || (n > 0 && (!R || !E || !B || !AB || !ER)))
        return fail(ctx, TP_ERR_INVALID_ARG, "bad pair arguments");
    cudaStream_t s = (cudaStream_t)stream;
    Ctx &c = ctx->c;
    const bool balanced = precond_balanced(c.prm.precond);
    if (balanced && n > 0 && (!R2 || !ILAM || !c.spec))
        return fail(ctx, TP_ERR_INVALID_ARG, "the balancing form needs R2 and ILAM");
    tp_status st = records(ctx, gamma, 0, s);
    if (st) return st;
    st = precond_setup(ctx, gamma, s);
    if (st) return st;
    // with ILAM the circulant is left to the training step (its scaling is learned): B is the coarse
    // term alone and ILAM receives this geometry's inverse symbols
    const bool rescale = ILAM && c.spec;
    if (ILAM && !c.spec) return fail(ctx, TP_ERR_UNSUPPORTED, "no circulant preconditioner in this context");
    if (rescale) CK(cudaMemcpyAsync(ILAM, spectral_ilam(c, s), sizeof(double) * c.nV, cudaMemcpyDeviceToDevice, s));
    const size_t nv3 = 3 * (size_t)c.nV;
    for (int k = 0; k < n; ++k) {
        double *r = R + k * nv3;
        double *b = B + k * nv3;
        // r := A-bar e: the recursive CG residual drifts below the true residual of an inexact
        // operator, so only A-bar e is exactly consistent with e
        CK(pair_apply(c, gamma, 0, E + k * nv3, r, s));
        CK(gnn_problem_dot(c, E + k * nv3, r, ER + (size_t)k * c.nProb, s));  // before B may overwrite E
        if (balanced) {
            // z = Q r + (I - Q A) y with y the learned smoother of r2 = (I - A Q) r: B = Q r, R2 = r2
            CK(coarse_balanced_part(c, 0, r, b, s));
            CK(coarse_balanced_part(c, 1, r, R2 + k * nv3, s));
        } else if (rescale) {
            CK(cudaMemsetAsync(b, 0, sizeof(double) * nv3, s));
            if (c.prm.precond >= TP_PRECOND_TWOLEVEL) CK(coarse_apply(c, r, b, s));
        } else {
            CK(precond_apply_base(c, r, b, s, nullptr));
        }
        if (c.prm.precond != TP_PRECOND_NONE) CK(project_mean(c, b, s, nullptr));
        CK(pair_apply(c, gamma, 0, b, AB + k * nv3, s));
    }
    return TP_OK;
}

tp_status tp_gnn_train_step(tp_ctx *ctx, const double *gamma, int n, const double *R, const double *B,
                            const double *AB, const double *ER, const double *ILAM, const double *R2, float lr,
                            double *loss, float *grad, tp_stream stream)
{
    tp_status st = need_gnn(ctx);
    if (st) return st;
    if (!gamma || n < 1 || !R || !B || !AB || !ER || !(lr >= 0.f))
        return fail(ctx, TP_ERR_INVALID_ARG, "bad training arguments");
    Ctx &c = ctx->c;
    if (!gnn_ready(c) || !gnn_bound(c)) return fail(ctx, TP_ERR_INVALID_ARG, "parameters or geometry missing");
    cudaStream_t s = (cudaStream_t)stream;
    st = records(ctx, gamma, 0, s);
    if (st) return st;
    if (ILAM && !c.spec) return fail(ctx, TP_ERR_UNSUPPORTED, "no circulant preconditioner in this context");
    if (R2 && (!c.coarse || !precond_balanced(c.prm.precond)))
        return fail(ctx, TP_ERR_INVALID_ARG, "R2 needs a context in a balancing two-level preconditioner");
    CK(gnn_train_step(c, gamma, n, R, B, AB, ER, ILAM, R2, lr, c.d_scal, s));
    if (grad) CK(cudaMemcpyAsync(grad, gnn_last_grad(c), sizeof(float) * gnn_num_params(), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(c.h_pinned, c.d_scal, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (loss) *loss = c.h_pinned[0];
    return check_err_word(ctx, s);
}

tp_status tp_last_solve(const tp_ctx *ctx, double *rel_res, int32_t *iters)
{
    if (!ctx) return TP_ERR_INVALID_ARG;
    const Ctx &c = ctx->c;
    for (int q = 0; q < c.nProb; ++q) {
        if (rel_res) rel_res[q] = q < (int)c.last_rr.size() ? c.last_rr[q] : 0.0;
        if (iters) iters[q] = q < (int)c.last_iters.size() ? c.last_iters[q] : 0;
    }
    return TP_OK;
}

// ---------------------------------------------------------------------------------- autotuner

tp_status tp_set_diff_variant(tp_ctx *ctx, int symmetric_tpt)
{
    if (!ctx) return TP_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    if (symmetric_tpt < 0 || symmetric_tpt > 4) return fail(ctx, TP_ERR_INVALID_ARG, "the differential variant must be 0 .. 4");
    if (symmetric_tpt > 0 && !(c.prm.precision == TP_MIXED && c.kp.fast))
        return fail(ctx, TP_ERR_UNSUPPORTED, "the symmetric differential exists for TP_MIXED with (alpha, beta) = (2, 4.5)");
    CK(sym_select_diff(c, symmetric_tpt));
    return TP_OK;
}

tp_status tp_set_energy_variant(tp_ctx *ctx, int symmetric_tpt)
{
    if (!ctx) return TP_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    if (symmetric_tpt < 0 || symmetric_tpt > 2) return fail(ctx, TP_ERR_INVALID_ARG, "symmetric_tpt must be 0, 1 or 2");
    if (symmetric_tpt > 0 && !(c.prm.precision == TP_MIXED && c.kp.fast))
        return fail(ctx, TP_ERR_UNSUPPORTED, "the symmetric energy exists for TP_MIXED with (alpha, beta) = (2, 4.5)");
    CK(sym_select_energy(c, symmetric_tpt));
    return TP_OK;
}

tp_status tp_set_apply_variant(tp_ctx *ctx, int symmetric_tpt)
{
    if (!ctx) return TP_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    if (symmetric_tpt < 0 || symmetric_tpt > 2) return fail(ctx, TP_ERR_INVALID_ARG, "symmetric_tpt must be 0, 1 or 2");
    if (symmetric_tpt > 0 && !(c.prm.precision == TP_MIXED && c.kp.fast))
        return fail(ctx, TP_ERR_UNSUPPORTED, "the symmetric apply exists for TP_MIXED with (alpha, beta) = (2, 4.5)");
    CK(sym_select(c, symmetric_tpt));
    return TP_OK;
}

tp_status tp_autotune(tp_ctx *ctx, const double *gamma, int32_t *tpt, double *ms, tp_stream stream)
{
    if (!ctx || !gamma) return TP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Ctx &c = ctx->c;
    tp_status st = records(ctx, gamma, 0, s);
    if (st) return st;
    if (ms)
        for (int k = 0; k < 17; ++k) ms[k] = 0.0;
    if (tpt) tpt[3] = tpt[4] = tpt[5] = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int prof = c.profile;
    c.profile = 0;
    const int *skip = c.d_skip;
    c.d_skip = nullptr;
    auto run = [&](int cls) -> cudaError_t {
        if (cls == 0) return pair_energy(c, gamma, 0, c.d_rows, c.d_E, s);
        if (cls == 1) return pair_diff(c, gamma, 0, c.d_t2, s);
        return pair_apply(c, gamma, 0, gamma, c.d_t2, s);  // any u times the same
    };
    cudaError_t err = cudaSuccess;
    // a symmetric variant is a candidate while its partial sums fit in 32 GB and in half the free memory
    // (on top of what the partial buffer already holds); the buffer is shrunk to the winners' need below
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = 0;
    auto fits = [&](size_t bytes) {
        return bytes <= ((size_t)32 << 30) && bytes <= c.part_elems * sizeof(double) + free_b / 2;
    };
    for (int cls = 0; cls < 3 && err == cudaSuccess; ++cls) {
        int cand[4];
        const int nc = tpt_candidates(c, cls, cand);
        int best = cand[0];
        float best_ms = 1e30f;
        for (int i = 0; i < nc && nc > 1 && err == cudaSuccess; ++i) {
            c.tpt[cls] = cand[i];
            if ((err = replan(c, cls)) != cudaSuccess) break;
            if ((err = run(cls)) != cudaSuccess) break;  // warm-up
            cudaEventRecord(e0, s);
            for (int r = 0; r < 3 && err == cudaSuccess; ++r) err = run(cls);
            cudaEventRecord(e1, s);
            if (err == cudaSuccess) err = cudaEventSynchronize(e1);
            float t = 0.f;
            if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
            t /= 3.f;
            if (ms && cand[i] >= 1 && cand[i] <= 4) ms[3 * cls + (cand[i] == 4 ? 2 : cand[i] - 1)] = t;
            if (t < best_ms) {
                best_ms = t;
                best = cand[i];
            }
        }
        if (err == cudaSuccess && nc > 1) {
            c.tpt[cls] = best;
            err = replan(c, cls);
        }
        if (tpt) tpt[cls] = nc > 1 ? best : cand[0];
        // the differential also has the symmetric pass
        if (cls == 1 && nc > 1 && err == cudaSuccess) {
            int best_sym = 0;
            for (int t = 1; t <= 4 && err == cudaSuccess; ++t) {
                const int tpt_t = (t == 2 || t == 4) ? 2 : 1;
                if (!fits(sym_slots(c, tpt_t) * (size_t)c.nE * 6 * sizeof(double))) continue;
                if ((err = sym_select_diff(c, t)) != cudaSuccess) break;
                if ((err = run(cls)) != cudaSuccess) break;
                cudaEventRecord(e0, s);
                for (int r = 0; r < 3 && err == cudaSuccess; ++r) err = run(cls);
                cudaEventRecord(e1, s);
                if (err == cudaSuccess) err = cudaEventSynchronize(e1);
                float tm = 0.f;
                if (err == cudaSuccess) err = cudaEventElapsedTime(&tm, e0, e1);
                tm /= 3.f;
                if (ms) ms[t <= 2 ? 13 + t - 1 : 15 + t - 3] = tm;
                if (tm < best_ms) {
                    best_ms = tm;
                    best_sym = t;
                }
            }
            if (err == cudaSuccess) err = sym_select_diff(c, best_sym);
            if (tpt) tpt[5] = best_sym;
        }
        // the energy also has the symmetric pass (its rows are one double per edge and slot)
        if (cls == 0 && nc > 1 && err == cudaSuccess) {
            int best_sym = 0;
            for (int t = 1; t <= 2 && err == cudaSuccess; ++t) {
                if (!fits(sym_slots(c, t) * (size_t)c.nE * sizeof(double))) continue;
                if ((err = sym_select_energy(c, t)) != cudaSuccess) break;
                if ((err = run(cls)) != cudaSuccess) break;
                cudaEventRecord(e0, s);
                for (int r = 0; r < 3 && err == cudaSuccess; ++r) err = run(cls);
                cudaEventRecord(e1, s);
                if (err == cudaSuccess) err = cudaEventSynchronize(e1);
                float tm = 0.f;
                if (err == cudaSuccess) err = cudaEventElapsedTime(&tm, e0, e1);
                tm /= 3.f;
                if (ms) ms[11 + t - 1] = tm;
                if (tm < best_ms) {
                    best_ms = tm;
                    best_sym = t;
                }
            }
            if (err == cudaSuccess) err = sym_select_energy(c, best_sym);
            if (tpt) tpt[4] = best_sym;
        }
        // the apply also has the symmetric pass (each unordered pair once), if its partial slots fit
        if (cls == 2 && nc > 1 && err == cudaSuccess) {
            int best_sym = 0;
            for (int t = 1; t <= 2 && err == cudaSuccess; ++t) {
                if (!fits(sym_slots(c, t) * (size_t)c.nE * 6 * sizeof(double))) continue;
                if ((err = sym_select(c, t)) != cudaSuccess) break;
                if ((err = run(cls)) != cudaSuccess) break;
                cudaEventRecord(e0, s);
                for (int r = 0; r < 3 && err == cudaSuccess; ++r) err = run(cls);
                cudaEventRecord(e1, s);
                if (err == cudaSuccess) err = cudaEventSynchronize(e1);
                float tm = 0.f;
                if (err == cudaSuccess) err = cudaEventElapsedTime(&tm, e0, e1);
                tm /= 3.f;
                if (ms) ms[9 + t - 1] = tm;
                if (tm < best_ms) {
                    best_ms = tm;
                    best_sym = t;
                }
            }
            if (err == cudaSuccess) err = sym_select(c, best_sym);
            if (tpt) tpt[3] = best_sym;
        }
    }
    c.profile = prof;
    c.d_skip = skip;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(err);
    // keep only the partial buffer the chosen passes need (the candidates may have grown it)
    {
        const size_t nE1 = (size_t)std::max(1, c.nE);
        size_t need = (size_t)std::max(std::max(c.plan_energy.max_slots, c.plan_diff.max_slots), c.plan_apply.max_slots) *
                      nE1 * 6;
        if (c.apply_sym) need = std::max(need, (size_t)c.plan_sym.max_slots * nE1 * 6);
        if (c.energy_sym) need = std::max(need, (size_t)c.plan_sym_e.max_slots * nE1);
        if (c.diff_sym) need = std::max(need, (size_t)c.plan_sym_d.max_slots * nE1 * 6);
        if (need < c.part_elems) {
            graphs_reset(c);  // captured blocks hold the old buffer's address
            CK(cudaStreamSynchronize(s));
            CK(cudaFree(c.d_part));
            CK(cudaMalloc(&c.d_part, sizeof(double) * need));
            c.part_elems = need;
        }
    }
    return check_err_word(ctx, s);
}

}  // extern "C"
