// Sobolev apply in double-float arithmetic: the accurate operator that certifies the residuals of the
// mixed-precision solves.
//
// The product is the same as the gather pass of pairs.cu (Secs. 5.2.2-5.2.3): for every ordered pair
// (I, J) of disjoint edges
//   h_I += 2 w_IJ [(du_I - du_J) + (|T_I - T_J|^2 / 2) du_J],     l_I += (w0_IJ + w0_JI)(ub_I - ub_J),
// w_IJ = (1/4) l_I l_J sum_ab |d_ab|^-p, w0_IJ + w0_JI = (1/4) l_I l_J sum_ab (|T_I x d_ab|^2 + |T_J x d_ab|^2)
// |d_ab|^-(4+p), d_ab = g_ia - g_jb; (A u) at i1, i2 = -/+ h_I / l_I + l_I / 2.  Here every quantity is a
// double-float (hi + lo, ~48 bits) built from the FP64 positions, tangents, lengths and u: the chords,
// |d|^2, the powers (rsqrt and sqrt of the FP32 pipe, each refined by one exact-residual correction),
// |T x d|^2 = |d|^2 - (T . d)^2, the weights and the products with the u differences.  Each term is
// then correct to ~1e-13 relative, about 2^24 times better than the FP32 pair arithmetic of the mixed
// pass, so a residual b - A x formed with this pass is exact to far below the 1e-6 the solves certify.
// Row sums are double-float per tile and FP64 across tiles.  General exponents take the power in FP64.
//
// The pass is symmetric (as pairs_sym.cu): the Gram weights satisfy w_IJ = w_JI and enter the low-order
// form as w0_IJ + w0_JI, so one evaluation of an unordered pair {I, J} yields what row I receives from J
// and what row J receives from I.  Items are edge-block pairs (b, c >= b); lane l of a warp takes source
// (step + l) mod P at each step, and the source rows' terms go to per-warp double-float accumulators in
// shared memory (no atomics); target rows of block b write partial slot c, source rows of block c slot
// b, the diagonal item (b, b) is a plain gather writing slot b.  Every row receives one write per slot,
// so the result is deterministic.
#include <cuda_runtime.h>

#include "df.cuh"
#include "tpe_internal.cuh"

namespace tpe {

#define TPE_CHECK(x)                      \
    do {                                  \
        cudaError_t e_ = (x);             \
        if (e_ != cudaSuccess) return e_; \
    } while (0)

struct DfArgs {
    const WorkItem *items;
    int n_items;
    int *counter;
    const RecF *recF;
    const RecLo *recLo;
    const float *ell_lo;
    const URecF *urecF;
    const double *ell;  // FP64 edge lengths (output scaling)
    double *part;       // [slot][nE][6]
    int nE;
    double p;           // 2 sigma + 1
    const int *skip;
};

struct DfV3 {
    df x, y, z;
};

struct DfEdge {
    DfV3 p1, p2, T, du, ub;
    df ell;
    int i1, i2;
};

__device__ __forceinline__ void df_edge_load(DfEdge &e, const RecF &r, const RecLo &q, float ell_lo, const URecF &u)
{
    e.p1 = {df{r.a.x, q.lo.x}, df{r.a.y, q.lo.y}, df{r.a.z, q.lo.z}};
    e.p2 = {df{r.b.x, q.lo.w}, df{r.b.y, q.lo2.x}, df{r.b.z, q.lo2.y}};
    e.T = {df{r.b.w, q.lo2.z}, df{r.c.x, q.lo2.w}, df{r.c.y, q.lo3.x}};
    e.ell = df{r.a.w, ell_lo};
    e.i1 = __float_as_int(r.c.z);
    e.i2 = __float_as_int(r.c.w);
    e.du = {df{u.a.x, u.b.z}, df{u.a.y, u.b.w}, df{u.a.z, u.c.x}};
    e.ub = {df{u.a.w, u.c.y}, df{u.b.x, u.c.z}, df{u.b.y, u.c.w}};
}

__device__ __forceinline__ DfV3 df3_sub(const DfV3 &a, const DfV3 &b)
{
    return {df_sub(a.x, b.x), df_sub(a.y, b.y), df_sub(a.z, b.z)};
}

__device__ __forceinline__ df df3_dot(const DfV3 &a, const DfV3 &b)
{
    return df_add(df_add(df_mul(a.x, b.x), df_mul(a.y, b.y)), df_mul(a.z, b.z));
}

__device__ __forceinline__ df df3_norm2(const DfV3 &a) { return df_add(df_add(df_sqr(a.x), df_sqr(a.y)), df_sqr(a.z)); }

// F = |d|^-p and G = |d|^-(4+p) from d2 = |d|^2 (p = 2.5 in the fast path).
// r0 = rsqrt(d2.hi) has some ulp of error; rho = 1 - d2 r0^2 is formed exactly enough through fma
// (r0^2 = a + b exactly), and r = r0 (1 + eps), eps = rho / 2 + 3 rho^2 / 8.  sqrt(r0) = q0 + (r0 - q0^2)
// / (2 q0) likewise.  Then |d|^-2.5 = r0^2 sqrt(r0) (1 + eps)^2.5 and |d|^-2 = r0^2 (1 + eps)^2.
template <bool FAST>
__device__ __forceinline__ void df_powers(df d2, double p, df &F, df &G)
{
    if constexpr (FAST) {
        const float r0 = rsqrtf(d2.hi);
        const float a = __fmul_rn(r0, r0);
        const float b = __fmaf_rn(r0, r0, -a);
        float rho = __fmaf_rn(-d2.hi, a, 1.f);
        rho = __fmaf_rn(-d2.hi, b, rho);
        rho = __fmaf_rn(-d2.lo, a, rho);
        const float eps = rho * (0.5f + 0.375f * rho);
        const float q0 = sqrtf(r0);
        const float dq = __fmaf_rn(-q0, q0, r0) * (0.5f / q0);
        const df R2 = fast_two_sum(a, b);
        const df Q = fast_two_sum(q0, dq);
        F = df_scale1p(df_mul(R2, Q), eps * (2.5f + 1.875f * eps));
        const df Rsq = df_scale1p(R2, eps * (2.f + eps));  // |d|^-2
        G = df_mul(F, df_sqr(Rsq));
    } else {
        const double d2d = df_to_double(d2);
        const double f = pow(d2d, -0.5 * p);
        F = df_from_double(f);
        G = df_from_double(f / (d2d * d2d));
    }
}

// One unordered pair {I, J}: row I's terms into (A1, A2), row J's into (H, L) (all double-float).
template <bool FAST>
__device__ __forceinline__ void df_pair_both(const DfEdge &t, const DfEdge &s, double p, df (&A1)[3], df (&A2)[3],
                                             df (&H)[3], df (&L)[3])
{
    DfV3 d[4];
    d[0] = df3_sub(t.p1, s.p1);
    d[1] = df3_sub(t.p1, s.p2);
    d[2] = df3_sub(t.p2, s.p1);
    d[3] = df3_sub(t.p2, s.p2);
    df d2[4], F[4], G[4];
#pragma unroll
    for (int ab = 0; ab < 4; ++ab) {
        d2[ab] = df_add_pos(df_add_pos(df_sqr(d[ab].x), df_sqr(d[ab].y)), df_sqr(d[ab].z));
        df_powers<FAST>(d2[ab], p, F[ab], G[ab]);
    }
    // |T_I x d_ab|^2 depends on b only, |T_J x d_ab|^2 on a only (g_i2 = g_i1 + l_I T_I)
    const df tI1 = df3_dot(t.T, d[0]), tI2 = df3_dot(t.T, d[1]);
    const df tJ1 = df3_dot(s.T, d[0]), tJ2 = df3_dot(s.T, d[2]);
    const df cI1 = df_sub(d2[0], df_sqr(tI1)), cI2 = df_sub(d2[1], df_sqr(tI2));
    const df cJ1 = df_sub(d2[0], df_sqr(tJ1)), cJ2 = df_sub(d2[2], df_sqr(tJ2));
    const df sw = df_add_pos(df_add_pos(F[0], F[3]), df_add_pos(F[1], F[2]));
    const df sw0 = df_add_pos(df_add_pos(df_mul(cI1, df_add_pos(G[0], G[2])), df_mul(cI2, df_add_pos(G[1], G[3]))),
                              df_add_pos(df_mul(cJ1, df_add_pos(G[0], G[1])), df_mul(cJ2, df_add_pos(G[2], G[3]))));
    const df Wt = df_mul(s.ell, sw), W0t = df_mul(s.ell, sw0);
    const df Ws = df_mul(t.ell, sw), W0s = df_mul(t.ell, sw0);
    const DfV3 dT = df3_sub(t.T, s.T);
    const df omt = df_mul_f(df_add_pos(df_add_pos(df_sqr(dT.x), df_sqr(dT.y)), df_sqr(dT.z)), 0.5f);
    const df tdu[3] = {t.du.x, t.du.y, t.du.z}, sdu[3] = {s.du.x, s.du.y, s.du.z};
    const df tub[3] = {t.ub.x, t.ub.y, t.ub.z}, sub[3] = {s.ub.x, s.ub.y, s.ub.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const df ddv = df_sub(tdu[k], sdu[k]), dbv = df_sub(tub[k], sub[k]);
        // row I: (du_I - du_J) + omt du_J;  row J: (du_J - du_I) + omt du_I
        A1[k] = df_add(A1[k], df_mul(Wt, df_add(ddv, df_mul(omt, sdu[k]))));
        A2[k] = df_add(A2[k], df_mul(W0t, dbv));
        H[k] = df_add(H[k], df_mul(Ws, df_sub(df_mul(omt, tdu[k]), ddv)));
        L[k] = df_sub(L[k], df_mul(W0s, dbv));
    }
}

template <bool FAST>
__global__ void __launch_bounds__(kThreads, 2) k_apply_df_sym(const DfArgs a)
{
    constexpr int kW = kThreads / 32;
    __shared__ RecF sr[kTile];
    __shared__ RecLo sl[kTile];
    __shared__ URecF su[kTile];
    __shared__ float sel[kTile];
    __shared__ float2 sac[kW][6][kTile];  // per warp and source: double-float (hi, lo)
    __shared__ int s_item;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= a.n_items) break;
        const WorkItem w = a.items[it];
        if (a.skip && a.skip[w.pad]) continue;  // uniform over the block
        const int bslot = w.slot >> 16, cslot = w.slot & 0xffff;
        const bool diag = bslot == cslot;
        const bool valid = threadIdx.x < w.ntgt;  // clamped duplicates must not feed the source side
        const int I = w.tgt0 + min((int)threadIdx.x, w.ntgt - 1);
        DfEdge t;
        df_edge_load(t, a.recF[I], a.recLo[I], a.ell_lo[I], a.urecF[I]);
        double A64[6] = {0, 0, 0, 0, 0, 0};
        for (int s0 = w.src0; s0 < w.src1; s0 += kTile) {
            const int cnt = min(kTile, w.src1 - s0);
            __syncthreads();  // the previous tile's readers are done
            if (threadIdx.x < cnt) {
                const int J = s0 + threadIdx.x;
                sr[threadIdx.x] = a.recF[J];
                sl[threadIdx.x] = a.recLo[J];
                su[threadIdx.x] = a.urecF[J];
                sel[threadIdx.x] = a.ell_lo[J];
            }
            for (int j = lane; j < kTile; j += 32)
                for (int q = 0; q < 6; ++q) sac[wid][q][j] = make_float2(0.f, 0.f);
            __syncthreads();
            df A1[3] = {df_make(0.f), df_make(0.f), df_make(0.f)};
            df A2[3] = {df_make(0.f), df_make(0.f), df_make(0.f)};
            const int P = max(cnt, 32);
            for (int step = 0; step < P; ++step) {
                int j = step + lane;
                if (j >= P) j -= P;
                if (j < cnt) {
                    DfEdge s;
                    df_edge_load(s, sr[j], sl[j], sel[j], su[j]);
                    const bool keep = valid & (s.i1 != t.i1) & (s.i1 != t.i2) & (s.i2 != t.i1) & (s.i2 != t.i2);
                    if (keep) {
                        df H[3] = {df_make(0.f), df_make(0.f), df_make(0.f)};
                        df L[3] = {df_make(0.f), df_make(0.f), df_make(0.f)};
                        df_pair_both<FAST>(t, s, a.p, A1, A2, H, L);
                        if (!diag) {
#pragma unroll
                            for (int q = 0; q < 3; ++q) {
                                const float2 h = sac[wid][q][j], l = sac[wid][3 + q][j];
                                const df hh = df_add(df{h.x, h.y}, H[q]), ll = df_add(df{l.x, l.y}, L[q]);
                                sac[wid][q][j] = make_float2(hh.hi, hh.lo);
                                sac[wid][3 + q][j] = make_float2(ll.hi, ll.lo);
                            }
                        }
                    }
                }
                if (!diag) __syncwarp();  // the next step hands this lane's source to lane - 1
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                A64[k] += df_to_double(A1[k]);
                A64[3 + k] += df_to_double(A2[k]);
            }
            if (!diag) {
                __syncthreads();  // every warp's source accumulators are complete
                if (threadIdx.x < cnt) {
                    const int J = s0 + threadIdx.x;
                    double v[6];
                    for (int q = 0; q < 6; ++q) {
                        double x = 0.0;
                        for (int wv = 0; wv < kW; ++wv)
                            x += (double)sac[wv][q][threadIdx.x].x + (double)sac[wv][q][threadIdx.x].y;
                        v[q] = x;
                    }
                    const double l = a.ell[J];
                    double *o = a.part + ((size_t)bslot * a.nE + J) * 6;
                    for (int q = 0; q < 3; ++q) {
                        o[q] = 0.5 * v[q];
                        o[3 + q] = 0.125 * l * v[3 + q];
                    }
                }
            }
        }
        if (valid) {
            const double l = a.ell[I];
            double *o = a.part + ((size_t)cslot * a.nE + I) * 6;
            for (int k = 0; k < 3; ++k) {
                o[k] = 0.5 * A64[k];
                o[3 + k] = 0.125 * l * A64[3 + k];
            }
        }
    }
}

static int df_occupancy(bool fast)
{
    int occ = 0;
    if (fast)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_apply_df_sym<true>, kThreads, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_apply_df_sym<false>, kThreads, 0);
    return occ;
}

// Au = A-bar u in double-float arithmetic on the geometry slot `which` (records built for that curve).
// Contexts in FP64 run their own FP64 pass instead.  Uses its own work list of edge-block pairs (128-edge
// blocks) and the context's partial-sum buffer (one slot per block of the largest problem).
cudaError_t pair_apply_acc(Ctx &c, const double *gamma_geom, int which, const double *u, double *Au, cudaStream_t s)
{
    if (c.prm.precision == TP_FP64) return pair_apply(c, gamma_geom, which, u, Au, s);
    Ctx::Plan &pl = c.plan_df;
    if (!pl.d_items) {
        sym_plan_items(c, pl, 1, df_occupancy(c.kp.fast != 0));
        const size_t need = (size_t)pl.max_slots * std::max(1, c.nE) * 6;
        if (need > c.part_elems) {
            TPE_CHECK(cudaFree(c.d_part));
            TPE_CHECK(cudaMalloc(&c.d_part, sizeof(double) * need));
            c.part_elems = need;
            graphs_reset(c);  // captured blocks hold the old partial buffer
        }
    }
    TPE_CHECK(build_urecs(c, u, which, s));
    if (pl.n_items == 0) return cudaMemsetAsync(Au, 0, sizeof(double) * 3 * c.nV, s);
    TPE_CHECK(cudaMemsetAsync(c.d_counter + 7, 0, sizeof(int), s));
    DfArgs a;
    a.items = pl.d_items;
    a.n_items = pl.n_items;
    a.counter = c.d_counter + 7;
    a.recF = which ? c.d_recF2 : c.d_recF;
    a.recLo = which ? c.d_recLo2 : c.d_recLo;
    a.ell_lo = c.d_ell_lo[which];
    a.urecF = c.d_urecF;
    a.ell = c.d_ellw[which];
    a.part = c.d_part;
    a.nE = c.nE;
    a.p = c.kp.p;
    a.skip = c.d_skip;
    const int slot = c.profile ? prof_begin(c, 5, s) : -1;
    if (c.kp.fast)
        k_apply_df_sym<true><<<pl.grid, kThreads, 0, s>>>(a);
    else
        k_apply_df_sym<false><<<pl.grid, kThreads, 0, s>>>(a);
    if (slot >= 0 || slot <= -2) prof_end(c, slot, s);
    c.launches++;
    TPE_CHECK(cudaGetLastError());
    return gather_apply(c, pl, Au, s);
}

}  // namespace tpe
