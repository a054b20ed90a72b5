// Edge-length constraints of Sec. 8.1: Phi_I = l0_I - l_I for every edge, together with the barycenter.
//
// The rows r_I = d l_I / d gamma have -T_I at i1 and +T_I at i2.  Every edge length is invariant under
// translations, so the rows are orthogonal to N = span{e_x, e_y, e_z}, the null space of A-bar.  The
// Euclidean projector onto null(R) (P_E = I - R^T G^-1 R, G = R R^T) therefore commutes with the
// mean-free projector P_N, and P = P_E P_N is the orthogonal projector onto null(R) cap N-perp: the
// space on which the projected CG of App. B.3.3 runs.  The barycenter rows then only fix the
// translation (a 3x3 shift per problem), exactly as for the total-length set.
//
// G is tridiagonal per curve: G_II = |T_I|^2 + |T_I|^2 = 2 and, for consecutive edges I, J with
// i2(I) = i1(J), G_IJ = (+T_I) . (-T_J) = -T_I . T_J; closed curves add the corner between the last and
// the first edge.  It is solved per curve by parallel cyclic reduction (PCR):
//   * a closed curve's corner is removed by Sherman-Morrison: G = T + u w^T with u = (gam, 0.., g),
//     w = (1, 0.., g / gam), gam = -2, so that T = G + 2 w w^T is a plain tridiagonal SPD matrix;
//   * PCR on T takes ceil(log2 m) steps; step k (stride s = 2^k) replaces equation i by itself plus
//     alpha_i times equation i - s plus beta_i times equation i + s.  The multipliers depend only on
//     T, so they are computed once per set-up (one curve geometry) and each solve is a sequence of
//     stencil sweeps d_i += alpha_i d_{i-s} + beta_i d_{i+s}, then x_i = d_i / b_i;
//   * q = T^-1 u is computed at set-up, and G^-1 d = y - q (w . y) / (1 + w . q) with y = T^-1 d.
// One CTA solves one curve: in shared memory for curves of up to kSmemEdges edges, through a
// global-memory ping-pong buffer above that.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "tpe_internal.cuh"

namespace tpe {

#define TPE_CHECK(x)                      \
    do {                                  \
        cudaError_t e_ = (x);             \
        if (e_ != cudaSuccess) return e_; \
    } while (0)

constexpr int kEdgeThreads = 512;
constexpr int kSmemEdges = 12288;     // 2 x 12288 doubles = 192 KB of dynamic shared memory
constexpr double kSmGamma = -2.0;     // Sherman-Morrison shift of a closed curve's first pivot

struct ChainInfo {
    int e0, m, closed, K;  // first edge, edges, closed flag, PCR steps (2^K >= m)
    long long moff;        // offset of the chain's multipliers in d_mult (double2 units): [K][m]
    int prob, pad;
};

struct EdgeState {
    std::vector<ChainInfo> h_chain;
    std::vector<int> h_prob_chain;  // [nProb + 1] chains of each problem (chains are ordered by edge)
    int nSmall = 0, nLarge = 0, maxSmall = 0;
    ChainInfo *d_chain = nullptr;
    int *d_small = nullptr, *d_large = nullptr, *d_prob_chain = nullptr;
    double2 *d_mult = nullptr;  // PCR multipliers (alpha, beta)
    double *d_binv = nullptr;   // [nE] reciprocal final pivots
    double *d_q = nullptr;      // [nE] T^-1 u (closed chains)
    double *d_sm = nullptr;     // [nChains][2]: g / gam, 1 + w . q
    double *d_T = nullptr;      // [nE][3] tangents of the set-up geometry
    double *d_ws = nullptr;     // [6][nE] set-up scratch; [2][nE] ping-pong of the large-chain solves
    double *d_l0 = nullptr;     // [nE] target edge lengths
    double *d_phiE = nullptr;   // [nE] l0 - l of the last evaluated geometry
    double *d_cmax = nullptr;   // [nChains] max |l0 - l| per chain
};

__device__ __forceinline__ double dot3d(const double *a, const double *b)
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// max that keeps a NaN once it has been seen (fmax would drop it)
__device__ __forceinline__ double nanmax(double a, double b)
{
    return (b != b || b > a) ? b : a;
}

// Set-up, one CTA per chain: tridiagonal T from the tangents, PCR multipliers, reciprocal pivots, and
// for closed chains q = T^-1 u and the Sherman-Morrison scalars.
__global__ void __launch_bounds__(kEdgeThreads) k_edge_build(const ChainInfo *__restrict__ chains,
                                                             const double *__restrict__ Tg, double *__restrict__ Tc,
                                                             double2 *__restrict__ mult, double *__restrict__ binv,
                                                             double *__restrict__ q, double *__restrict__ sm,
                                                             double *__restrict__ ws, int nE)
{
    const ChainInfo ch = chains[blockIdx.x];
    const int m = ch.m, e0 = ch.e0;
    double *A = ws + e0, *B = ws + nE + e0, *C = ws + 2 * (size_t)nE + e0;
    double *An = ws + 3 * (size_t)nE + e0, *Bn = ws + 4 * (size_t)nE + e0, *Cn = ws + 5 * (size_t)nE + e0;
    const double gw = ch.closed ? -dot3d(Tg + 3 * (size_t)(e0 + m - 1), Tg + 3 * (size_t)e0) : 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const double *t = Tg + 3 * (size_t)(e0 + i);
        for (int k = 0; k < 3; ++k) Tc[3 * (size_t)(e0 + i) + k] = t[k];
        A[i] = i > 0 ? -dot3d(t - 3, t) : 0.0;
        C[i] = i + 1 < m ? -dot3d(t, t + 3) : 0.0;
        double b = 2.0;
        if (ch.closed && i == 0) b -= kSmGamma;
        if (ch.closed && i == m - 1) b -= gw * gw / kSmGamma;
        B[i] = b;
    }
    __syncthreads();
    double2 *mu = mult + ch.moff;
    for (int k = 0; k < ch.K; ++k) {
        const int s = 1 << k;
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            const bool lo = i - s >= 0, hi = i + s < m;
            const double al = lo ? -A[i] / B[i - s] : 0.0;
            const double be = hi ? -C[i] / B[i + s] : 0.0;
            An[i] = lo ? al * A[i - s] : 0.0;
            Cn[i] = hi ? be * C[i + s] : 0.0;
            Bn[i] = B[i] + (lo ? al * C[i - s] : 0.0) + (hi ? be * A[i + s] : 0.0);
            mu[(size_t)k * m + i] = make_double2(al, be);
        }
        __syncthreads();
        double *t;
        t = A, A = An, An = t;
        t = B, B = Bn, Bn = t;
        t = C, C = Cn, Cn = t;
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) binv[e0 + i] = 1.0 / B[i];
    if (!ch.closed) return;  // uniform per CTA: every thread leaves together
    // q = T^-1 u, u = (gam, 0, .., 0, g); the A / An buffers are free now
    double *D = A, *Dn = An;
    for (int i = threadIdx.x; i < m; i += blockDim.x) D[i] = (i == 0 ? kSmGamma : 0.0) + (i == m - 1 ? gw : 0.0);
    __syncthreads();
    for (int k = 0; k < ch.K; ++k) {
        const int s = 1 << k;
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            const double2 ab = mu[(size_t)k * m + i];
            Dn[i] = D[i] + (i - s >= 0 ? ab.x * D[i - s] : 0.0) + (i + s < m ? ab.y * D[i + s] : 0.0);
        }
        __syncthreads();
        double *t = D;
        D = Dn, Dn = t;
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) q[e0 + i] = D[i] / B[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        const double r = gw / kSmGamma;
        sm[2 * blockIdx.x] = r;
        sm[2 * blockIdx.x + 1] = 1.0 + q[e0] + r * q[e0 + m - 1];
    }
}

// One CTA per chain of the list: lambda = G^-1 d with d = R v (MODE 0) or d = phiE (MODE 1), then
// v -= R^T lambda (MODE 0) or out = R^T lambda (MODE 1).  SMEM: the PCR sweeps run in dynamic shared
// memory (2 m doubles), else in the global ping-pong buffer ws.
template <bool SMEM, int MODE>
__global__ void __launch_bounds__(kEdgeThreads) k_edge_solve(const ChainInfo *__restrict__ chains,
                                                             const int *__restrict__ list, int nE,
                                                             const int *__restrict__ edges,
                                                             const double *__restrict__ T,
                                                             const double2 *__restrict__ mult,
                                                             const double *__restrict__ binv,
                                                             const double *__restrict__ q,
                                                             const double *__restrict__ sm,
                                                             const double *__restrict__ phiE, double *ws,
                                                             double *v, const int *__restrict__ skip)
{
    extern __shared__ double shbuf[];
    const int cidx = list[blockIdx.x];
    const ChainInfo ch = chains[cidx];
    if (skip && skip[ch.prob]) return;  // uniform per CTA
    const int m = ch.m, e0 = ch.e0;
    double *D = SMEM ? shbuf : ws + e0;
    double *Dn = SMEM ? shbuf + m : ws + nE + e0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const int I = e0 + i;
        if (MODE == 0) {
            const int a = edges[2 * I], b = edges[2 * I + 1];
            const double *t = T + 3 * (size_t)I;
            D[i] = t[0] * (v[3 * (size_t)b] - v[3 * (size_t)a]) + t[1] * (v[3 * (size_t)b + 1] - v[3 * (size_t)a + 1]) +
                   t[2] * (v[3 * (size_t)b + 2] - v[3 * (size_t)a + 2]);
        } else {
            D[i] = phiE[I];
        }
    }
    __syncthreads();
    const double2 *mu = mult + ch.moff;
    for (int k = 0; k < ch.K; ++k) {
        const int s = 1 << k;
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            const double2 ab = mu[(size_t)k * m + i];
            Dn[i] = D[i] + (i - s >= 0 ? ab.x * D[i - s] : 0.0) + (i + s < m ? ab.y * D[i + s] : 0.0);
        }
        __syncthreads();
        double *t = D;
        D = Dn, Dn = t;
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) D[i] *= binv[e0 + i];
    __syncthreads();
    if (ch.closed) {
        const double corr = (D[0] + sm[2 * cidx] * D[m - 1]) / sm[2 * cidx + 1];
        __syncthreads();
        for (int i = threadIdx.x; i < m; i += blockDim.x) D[i] -= q[e0 + i] * corr;
        __syncthreads();
    }
    // R^T lambda at vertex i1(I): -lambda_I T_I + lambda_P T_P (P: the edge ending there)
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const int I = e0 + i;
        const double *t = T + 3 * (size_t)I;
        double z[3] = {-D[i] * t[0], -D[i] * t[1], -D[i] * t[2]};
        const int p = i > 0 ? i - 1 : (ch.closed ? m - 1 : -1);
        if (p >= 0) {
            const double *tp = T + 3 * (size_t)(e0 + p);
            for (int k = 0; k < 3; ++k) z[k] += D[p] * tp[k];
        }
        const int w = edges[2 * I];
        for (int k = 0; k < 3; ++k) {
            if (MODE == 0) v[3 * (size_t)w + k] -= z[k];
            else v[3 * (size_t)w + k] = z[k];
        }
        if (!ch.closed && i == m - 1) {  // the open end i2(last) has only the incoming edge
            const int w2 = edges[2 * I + 1];
            for (int k = 0; k < 3; ++k) {
                if (MODE == 0) v[3 * (size_t)w2 + k] -= D[i] * t[k];
                else v[3 * (size_t)w2 + k] = D[i] * t[k];
            }
        }
    }
}

// phiE = l0 - l per edge and the largest |phiE| of each chain (one CTA per chain).
__global__ void __launch_bounds__(256) k_edge_phi(const ChainInfo *__restrict__ chains, const double *__restrict__ ell,
                                                  const double *__restrict__ l0, double *__restrict__ phiE,
                                                  double *__restrict__ cmax)
{
    __shared__ double sh[256];
    const ChainInfo ch = chains[blockIdx.x];
    double mx = 0.0;
    for (int i = threadIdx.x; i < ch.m; i += blockDim.x) {
        const int I = ch.e0 + i;
        const double f = l0[I] - ell[I];
        phiE[I] = f;
        mx = nanmax(mx, fabs(f));
    }
    sh[threadIdx.x] = mx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] = nanmax(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) cmax[blockIdx.x] = sh[0];
}

// phi[4 q + 3] = max over the problem's chains (the slot of the total-length row).
__global__ void k_edge_phimax(int nProb, const int *__restrict__ prob_chain, const double *__restrict__ cmax,
                              double *__restrict__ phi)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nProb) return;
    double mx = 0.0;
    for (int k = prob_chain[q]; k < prob_chain[q + 1]; ++k) mx = nanmax(mx, cmax[k]);
    phi[4 * q + 3] = mx;
}

__global__ void k_copy_d(int n, const double *__restrict__ a, double *__restrict__ b)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i];
}

// ---------------------------------------------------------------------------------- host side

// Each curve's edges must form one simple chain in storage order (i1 of edge I + 1 = i2 of edge I; closed
// when the last edge ends where the first starts), and no two chains may share a vertex: one CTA owns
// each chain's vertices in the projection kernels.
bool edges_chains_ok(const Ctx &c, std::string &why)
{
    std::vector<int> owner(c.nV, -1);
    for (int k = 0; k < c.nCurves; ++k) {
        const int e0 = c.h_eoff[k], e1 = c.h_eoff[k + 1];
        if (e1 == e0) continue;
        const int head = c.h_edges[2 * (e1 - 1) + 1];
        const bool closed = e1 - e0 >= 3 && head == c.h_edges[2 * e0];
        for (int I = e0; I < e1; ++I) {
            if (I + 1 < e1 && c.h_edges[2 * (I + 1)] != c.h_edges[2 * I + 1]) {
                why = "edge-length constraints need every curve's edges stored in chain order (i1 of edge I + 1 = i2 of edge I)";
                return false;
            }
            const int a = c.h_edges[2 * I];
            if (owner[a] != -1) {
                why = "edge-length constraints need simple chains with disjoint vertices";
                return false;
            }
            owner[a] = k;
        }
        if (!closed) {
            if (owner[head] != -1) {
                why = "edge-length constraints need simple chains with disjoint vertices";
                return false;
            }
            owner[head] = k;
        }
    }
    return true;
}

static int ceil_log2(int m)
{
    int K = 0;
    while ((1 << K) < m) ++K;
    return K;
}

void edges_free(Ctx &c)
{
    if (!c.edges) return;
    EdgeState &E = *c.edges;
    void *ptrs[] = {E.d_chain, E.d_small, E.d_large, E.d_prob_chain, E.d_mult, E.d_binv, E.d_q, E.d_sm,
                    E.d_T, E.d_ws, E.d_l0, E.d_phiE, E.d_cmax};
    for (void *p : ptrs) cudaFree(p);
    delete c.edges;
    c.edges = nullptr;
}

template <class T>
static cudaError_t ealloc(T **p, size_t n)
{
    return cudaMalloc((void **)p, sizeof(T) * std::max<size_t>(1, n));
}

cudaError_t edges_init(Ctx &c)
{
    if (c.edges) return cudaSuccess;
    c.edges = new EdgeState();
    EdgeState &E = *c.edges;
    long long moff = 0;
    std::vector<int> small, large;
    E.h_prob_chain.assign(c.nProb + 1, 0);
    for (int k = 0; k < c.nCurves; ++k) {
        const int e0 = c.h_eoff[k], e1 = c.h_eoff[k + 1];
        if (e1 == e0) continue;
        ChainInfo ch{};
        ch.e0 = e0;
        ch.m = e1 - e0;
        ch.closed = (ch.m >= 3 && c.h_edges[2 * (e1 - 1) + 1] == c.h_edges[2 * e0]) ? 1 : 0;
        ch.K = ceil_log2(ch.m);
        ch.moff = moff;
        moff += (long long)ch.K * ch.m;
        int q = 0;
        while (q + 1 < c.nProb && c.h_prob_e[q + 1] <= e0) ++q;
        ch.prob = q;
        const int idx = (int)E.h_chain.size();
        (ch.m <= kSmemEdges ? small : large).push_back(idx);
        if (ch.m <= kSmemEdges) E.maxSmall = std::max(E.maxSmall, ch.m);
        E.h_chain.push_back(ch);
        E.h_prob_chain[q + 1]++;
    }
    for (int q = 0; q < c.nProb; ++q) E.h_prob_chain[q + 1] += E.h_prob_chain[q];
    const int nC = (int)E.h_chain.size();
    E.nSmall = (int)small.size();
    E.nLarge = (int)large.size();
    const size_t nE = std::max(1, c.nE);
    TPE_CHECK(ealloc(&E.d_chain, nC));
    TPE_CHECK(ealloc(&E.d_small, small.size()));
    TPE_CHECK(ealloc(&E.d_large, large.size()));
    TPE_CHECK(ealloc(&E.d_prob_chain, c.nProb + 1));
    TPE_CHECK(ealloc(&E.d_mult, (size_t)std::max(1LL, moff)));
    TPE_CHECK(ealloc(&E.d_binv, nE));
    TPE_CHECK(ealloc(&E.d_q, nE));
    TPE_CHECK(ealloc(&E.d_sm, 2 * (size_t)std::max(1, nC)));
    TPE_CHECK(ealloc(&E.d_T, 3 * nE));
    TPE_CHECK(ealloc(&E.d_ws, 6 * nE));
    TPE_CHECK(ealloc(&E.d_l0, nE));
    TPE_CHECK(ealloc(&E.d_phiE, nE));
    TPE_CHECK(ealloc(&E.d_cmax, nC));
    if (nC) TPE_CHECK(cudaMemcpy(E.d_chain, E.h_chain.data(), sizeof(ChainInfo) * nC, cudaMemcpyHostToDevice));
    if (!small.empty())
        TPE_CHECK(cudaMemcpy(E.d_small, small.data(), sizeof(int) * small.size(), cudaMemcpyHostToDevice));
    if (!large.empty())
        TPE_CHECK(cudaMemcpy(E.d_large, large.data(), sizeof(int) * large.size(), cudaMemcpyHostToDevice));
    TPE_CHECK(cudaMemcpy(E.d_prob_chain, E.h_prob_chain.data(), sizeof(int) * (c.nProb + 1), cudaMemcpyHostToDevice));
    TPE_CHECK(cudaMemset(E.d_sm, 0, sizeof(double) * 2 * std::max(1, nC)));
    const int smem = 2 * kSmemEdges * (int)sizeof(double);
    TPE_CHECK(cudaFuncSetAttribute(k_edge_solve<true, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    TPE_CHECK(cudaFuncSetAttribute(k_edge_solve<true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    return cudaSuccess;
}

cudaError_t edges_targets(Ctx &c, int which, cudaStream_t s)
{
    if (!c.edges || c.nE == 0) return cudaSuccess;
    k_copy_d<<<(c.nE + 255) / 256, 256, 0, s>>>(c.nE, c.d_ellw[which], c.edges->d_l0);
    c.launches++;
    return cudaGetLastError();
}

cudaError_t edges_setup(Ctx &c, int which, cudaStream_t s)
{
    EdgeState &E = *c.edges;
    const int nC = (int)E.h_chain.size();
    if (!nC) return cudaSuccess;
    k_edge_build<<<nC, kEdgeThreads, 0, s>>>(E.d_chain, c.d_Tw[which], E.d_T, E.d_mult, E.d_binv, E.d_q, E.d_sm,
                                             E.d_ws, c.nE);
    c.launches++;
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t edge_solve(Ctx &c, const double *phiE, double *v, cudaStream_t s, const int *skip)
{
    EdgeState &E = *c.edges;
    if (E.nSmall) {
        const size_t smem = 2 * (size_t)E.maxSmall * sizeof(double);
        k_edge_solve<true, MODE><<<E.nSmall, kEdgeThreads, smem, s>>>(E.d_chain, E.d_small, c.nE, c.d_edges, E.d_T,
                                                                      E.d_mult, E.d_binv, E.d_q, E.d_sm, phiE,
                                                                      E.d_ws, v, skip);
        c.launches++;
    }
    if (E.nLarge) {
        k_edge_solve<false, MODE><<<E.nLarge, kEdgeThreads, 0, s>>>(E.d_chain, E.d_large, c.nE, c.d_edges, E.d_T,
                                                                    E.d_mult, E.d_binv, E.d_q, E.d_sm, phiE,
                                                                    E.d_ws, v, skip);
        c.launches++;
    }
    return cudaGetLastError();
}

cudaError_t edges_project(Ctx &c, double *v, cudaStream_t s, const int *skip)
{
    return edge_solve<0>(c, nullptr, v, s, skip);
}

cudaError_t edges_pinv(Ctx &c, double *out, cudaStream_t s)
{
    TPE_CHECK(cudaMemsetAsync(out, 0, sizeof(double) * 3 * (size_t)c.nV, s));
    return edge_solve<1>(c, c.edges->d_phiE, out, s, nullptr);
}

cudaError_t edges_phi(Ctx &c, int which, double *phi, cudaStream_t s)
{
    EdgeState &E = *c.edges;
    const int nC = (int)E.h_chain.size();
    if (nC) {
        k_edge_phi<<<nC, 256, 0, s>>>(E.d_chain, c.d_ellw[which], E.d_l0, E.d_phiE, E.d_cmax);
        c.launches++;
    }
    k_edge_phimax<<<(c.nProb + 127) / 128, 128, 0, s>>>(c.nProb, E.d_prob_chain, E.d_cmax, phi);
    c.launches++;
    return cudaGetLastError();
}

}  // namespace tpe
