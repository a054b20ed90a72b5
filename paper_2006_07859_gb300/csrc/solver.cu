// Constraints, projection and the projected preconditioned CG of the H^s gradient.
//
//   Phi_bary = sum_I l_I (x_I - x0), Phi_len = L0 - sum_I l_I          (Sec. 8.1), per problem
//   C = d Phi, stored per vertex as C[v][4][3]
//   P v = v - C^T (C C^T)^-1 C v,  C^+ b = C^T (C C^T)^-1 b              (App. B.3.3, read as the
//                                                                         Euclidean projector onto null C)
//   CG on P A-bar P y = P a, x = P y                                     (App. B.3.3, Eq. "ProjectedSystem")
//
// Every reduction is deterministic: fixed chunks of vertices (never crossing problems) are reduced
// in shared memory, and the last block to finish sums the chunk partials of each problem in index
// order and runs the per-problem scalar update (CG alpha/beta, convergence flags) on the device.
// No scalar goes to the host inside an iteration; the host polls a pinned "active problems"
// counter every cg_check_every iterations.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "tpe_internal.cuh"

namespace tpe {

#define TPE_CHECK(x)                      \
    do {                                  \
        cudaError_t e_ = (x);             \
        if (e_ != cudaSuccess) return e_; \
    } while (0)

constexpr int kRedThreads = 256;

// ---------------------------------------------------------------------------------- reduction core

struct RedArgs {
    const int *chunk_lo;   // [nchunks + 1] element ranges of the chunks
    const int *prob_c0;    // [nprob + 1] first chunk of each problem
    int nchunks, nprob;
    double *partial;       // [nchunks][K]
    unsigned *counter;
    double *sums;          // [nprob][K]
};

// Block-reduce K values, publish the block partial, and in the last block sum the partials of
// every problem into sums[q][k].  Returns true in the last block (all threads).
template <int K>
__device__ bool reduce_phase(double (&s)[K], const RedArgs &ra)
{
    __shared__ double sh[K][kRedThreads];
    __shared__ bool last;
    for (int k = 0; k < K; ++k) sh[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int k = 0; k < K; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int k = 0; k < K; ++k) ra.partial[(size_t)blockIdx.x * K + k] = sh[k][0];
        __threadfence();
        last = (atomicAdd(ra.counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    for (int q = threadIdx.x; q < ra.nprob; q += blockDim.x) {
        for (int k = 0; k < K; ++k) {
            double acc = 0.0;
            for (int ch = ra.prob_c0[q]; ch < ra.prob_c0[q + 1]; ++ch) acc += __ldcg(&ra.partial[(size_t)ch * K + k]);
            ra.sums[(size_t)q * K + k] = acc;
        }
    }
    if (threadIdx.x == 0) *ra.counter = 0u;
    __threadfence();
    __syncthreads();
    return true;
}

// ---------------------------------------------------------------------------------- reduction plans



// Chunks of at most `cap` elements within each problem's range [off[q], off[q+1]).
static void make_red_plan(const std::vector<int32_t> &off, int cap, int **d_lo, int **d_c0, int *nch)
{
    std::vector<int> lo, c0;
    int nprob = (int)off.size() - 1;
    for (int q = 0; q < nprob; ++q) {
        c0.push_back((int)lo.size());
        int a = off[q], b = off[q + 1];
        if (b <= a) continue;
        for (int x = a; x < b; x += cap) lo.push_back(x);
    }
    c0.push_back((int)lo.size());
    int n = (int)lo.size();
    lo.push_back(off.back());
    cudaMalloc(d_lo, sizeof(int) * lo.size());
    cudaMemcpy(*d_lo, lo.data(), sizeof(int) * lo.size(), cudaMemcpyHostToDevice);
    cudaMalloc(d_c0, sizeof(int) * c0.size());
    cudaMemcpy(*d_c0, c0.data(), sizeof(int) * c0.size(), cudaMemcpyHostToDevice);
    *nch = n;
}

// The context keeps these in its generic scratch: see solver_setup.
}  // namespace tpe
struct tpe::SolverState {
    int *v_lo = nullptr, *v_c0 = nullptr, v_n = 0;  // vertex chunks
    int *e_lo = nullptr, *e_c0 = nullptr, e_n = 0;  // edge chunks
    double *partial = nullptr;                      // [max chunks][16]
    unsigned *counters = nullptr;                   // [8]
    double *sums = nullptr;                         // [nProb][16]
    double *mu = nullptr;                           // [nProb][4]
    int *done = nullptr;                            // [nProb] 1 = converged / inactive
    int *active = nullptr;                          // [1] number of active problems
    int *status = nullptr;                          // [nProb] 0 ok, 1 breakdown
};
namespace tpe {

static SolverState &S(Ctx &c) { return *c.sol; }

static inline RedArgs vargs(Ctx &c, int which_counter)
{
    SolverState &s = S(c);
    return RedArgs{s.v_lo, s.v_c0, s.v_n, c.nProb, s.partial, s.counters + which_counter, s.sums};
}
static inline RedArgs eargs(Ctx &c, int which_counter)
{
    SolverState &s = S(c);
    return RedArgs{s.e_lo, s.e_c0, s.e_n, c.nProb, s.partial, s.counters + which_counter, s.sums};
}

cudaError_t solver_setup(Ctx &c)
{
    c.sol = new SolverState();
    SolverState &s = S(c);
    // chunks of 2048 elements (8 per thread): measured faster on the benchmark step than chunks sized to
    // two per SM (more blocks, each with one element per thread, made the CG kernels slower)
    make_red_plan(c.h_prob_v, 2048, &s.v_lo, &s.v_c0, &s.v_n);
    make_red_plan(c.h_prob_e, 2048, &s.e_lo, &s.e_c0, &s.e_n);
    int mx = std::max(std::max(s.v_n, s.e_n), 1);
    TPE_CHECK(cudaMalloc(&s.partial, sizeof(double) * (size_t)mx * 16));
    TPE_CHECK(cudaMalloc(&s.counters, sizeof(unsigned) * 8));
    TPE_CHECK(cudaMemset(s.counters, 0, sizeof(unsigned) * 8));
    TPE_CHECK(cudaMalloc(&s.sums, sizeof(double) * (size_t)std::max(1, c.nProb) * 16));
    TPE_CHECK(cudaMalloc(&s.mu, sizeof(double) * (size_t)std::max(1, c.nProb) * 4));
    TPE_CHECK(cudaMalloc(&s.done, sizeof(int) * (size_t)std::max(1, c.nProb)));
    TPE_CHECK(cudaMalloc(&s.status, sizeof(int) * (size_t)std::max(1, c.nProb)));
    TPE_CHECK(cudaMalloc(&s.active, sizeof(int) * 4));
    return cudaSuccess;
}

void solver_free(Ctx &c)
{
    SolverState &s = S(c);
    cudaFree(s.v_lo);
    cudaFree(s.v_c0);
    cudaFree(s.e_lo);
    cudaFree(s.e_c0);
    cudaFree(s.partial);
    cudaFree(s.counters);
    cudaFree(s.sums);
    cudaFree(s.mu);
    cudaFree(s.done);
    cudaFree(s.status);
    cudaFree(s.active);
    delete c.sol;
    c.sol = nullptr;
}

// ---------------------------------------------------------------------------------- constraints

// Phi per problem from the FP64 edge quantities: sum l_I (x_I - x0) and L0 - sum l_I.
__global__ void k_phi(RedArgs ra, const double *__restrict__ ell, const double *__restrict__ x,
                      const double *__restrict__ x0L0, const int *__restrict__ eprob, double *__restrict__ phi)
{
    double s[4] = {0, 0, 0, 0};
    int lo = ra.chunk_lo[blockIdx.x], hi = ra.chunk_lo[blockIdx.x + 1];
    for (int I = lo + threadIdx.x; I < hi; I += blockDim.x) {
        int q = eprob[I];
        double l = ell[I];
        for (int k = 0; k < 3; ++k) s[k] += l * (x[3 * I + k] - x0L0[4 * q + k]);
        s[3] += l;
    }
    if (reduce_phase<4>(s, ra)) {
        for (int q = threadIdx.x; q < ra.nprob; q += blockDim.x) {
            for (int k = 0; k < 3; ++k) phi[4 * q + k] = ra.sums[4 * q + k];
            phi[4 * q + 3] = x0L0[4 * q + 3] - ra.sums[4 * q + 3];
        }
    }
}

// x0 = sum l_I x_I / sum l_I and L0 = sum l_I of the given curve.
__global__ void k_targets(RedArgs ra, const double *__restrict__ ell, const double *__restrict__ x,
                          double *__restrict__ x0L0)
{
    double s[4] = {0, 0, 0, 0};
    int lo = ra.chunk_lo[blockIdx.x], hi = ra.chunk_lo[blockIdx.x + 1];
    for (int I = lo + threadIdx.x; I < hi; I += blockDim.x) {
        double l = ell[I];
        for (int k = 0; k < 3; ++k) s[k] += l * x[3 * I + k];
        s[3] += l;
    }
    if (reduce_phase<4>(s, ra)) {
        for (int q = threadIdx.x; q < ra.nprob; q += blockDim.x) {
            double L = ra.sums[4 * q + 3];
            for (int k = 0; k < 3; ++k) x0L0[4 * q + k] = L > 0 ? ra.sums[4 * q + k] / L : 0.0;
            x0L0[4 * q + 3] = L;
        }
    }
}

// C[v][k][:] for the barycenter rows k < 3 and the length row k = 3:
//   d/dg_v [l_I (x_I,k - x0_k)] = s_v T_I (x_I,k - x0_k) + (l_I / 2) e_k,   d/dg_v [L0 - l_I] = -s_v T_I,
// with s_v = +1 if v = i2, -1 if v = i1.
__global__ void k_jacobian(int nV, const int *__restrict__ inc_ptr, const int *__restrict__ inc,
                           const double *__restrict__ ell, const double *__restrict__ T, const double *__restrict__ x,
                           const double *__restrict__ x0L0, const int *__restrict__ vprob, double *__restrict__ C)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nV) return;
    int q = vprob[v];
    double c[4][3] = {{0}};
    for (int k = inc_ptr[v]; k < inc_ptr[v + 1]; ++k) {
        int I = inc[k] >> 1;
        double sg = (inc[k] & 1) ? 1.0 : -1.0;
        double t[3] = {T[3 * I], T[3 * I + 1], T[3 * I + 2]};
        for (int r = 0; r < 3; ++r) {
            double xr = x[3 * I + r] - x0L0[4 * q + r];
            for (int cc = 0; cc < 3; ++cc) c[r][cc] += sg * t[cc] * xr;
            c[r][r] += 0.5 * ell[I];
        }
        for (int cc = 0; cc < 3; ++cc) c[3][cc] -= sg * t[cc];
    }
    for (int r = 0; r < 4; ++r)
        for (int cc = 0; cc < 3; ++cc) C[(size_t)v * 12 + r * 3 + cc] = c[r][cc];
}

// G = C C^T per problem, then G^-1 (4x4, Gauss-Jordan with partial pivoting in FP64).
__device__ void inv4(const double *G, double *Gi)
{
    double a[4][8];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 8; ++j) a[i][j] = j < 4 ? G[4 * i + j] : (j - 4 == i ? 1.0 : 0.0);
    for (int col = 0; col < 4; ++col) {
        int piv = col;
        for (int r = col + 1; r < 4; ++r)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (piv != col)
            for (int j = 0; j < 8; ++j) {
                double t = a[col][j];
                a[col][j] = a[piv][j];
                a[piv][j] = t;
            }
        double d = a[col][col];
        if (d == 0.0) d = 1e-300;
        for (int j = 0; j < 8; ++j) a[col][j] /= d;
        for (int r = 0; r < 4; ++r)
            if (r != col) {
                double f = a[r][col];
                for (int j = 0; j < 8; ++j) a[r][j] -= f * a[col][j];
            }
    }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) Gi[4 * i + j] = a[i][4 + j];
}

__global__ void k_gram_cc(RedArgs ra, const double *__restrict__ C, double *__restrict__ G, double *__restrict__ Gi)
{
    double s[10] = {0};
    int lo = ra.chunk_lo[blockIdx.x], hi = ra.chunk_lo[blockIdx.x + 1];
    for (int v = lo + threadIdx.x; v < hi; v += blockDim.x) {
        const double *c = C + (size_t)v * 12;
        int n = 0;
        for (int i = 0; i < 4; ++i)
            for (int j = i; j < 4; ++j) {
                s[n++] += c[3 * i] * c[3 * j] + c[3 * i + 1] * c[3 * j + 1] + c[3 * i + 2] * c[3 * j + 2];
            }
    }
    if (reduce_phase<10>(s, ra)) {
        for (int q = threadIdx.x; q < ra.nprob; q += blockDim.x) {
            double g[16];
            int n = 0;
            for (int i = 0; i < 4; ++i)
                for (int j = i; j < 4; ++j) {
                    g[4 * i + j] = g[4 * j + i] = ra.sums[(size_t)q * 10 + n];
                    ++n;
                }
            for (int k = 0; k < 16; ++k) G[16 * q + k] = g[k];
            inv4(g, Gi + 16 * q);
        }
    }
}

// mu = G^-1 (C v) per problem (skip problems whose flag is set).
__global__ void k_cv(RedArgs ra, const double *__restrict__ C, const double *__restrict__ v,
                     const double *__restrict__ Gi, double *__restrict__ mu, const int *__restrict__ skip)
{
    double s[4] = {0, 0, 0, 0};
    int lo = ra.chunk_lo[blockIdx.x], hi = ra.chunk_lo[blockIdx.x + 1];
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double *c = C + (size_t)i * 12;
        double a = v[3 * i], b = v[3 * i + 1], d = v[3 * i + 2];
        for (int k = 0; k < 4; ++k) s[k] += c[3 * k] * a + c[3 * k + 1] * b + c[3 * k + 2] * d;
    }
    if (reduce_phase<4>(s, ra)) {
        for (int q = threadIdx.x; q < ra.nprob; q += blockDim.x) {
            const double *g = Gi + 16 * q;
            const double *cv = ra.sums + 4 * q;
            for (int k = 0; k < 4; ++k)
                mu[4 * q + k] = g[4 * k] * cv[0] + g[4 * k + 1] * cv[1] + g[4 * k + 2] * cv[2] + g[4 * k + 3] * cv[3];
        }
    }
}

// v -= C^T mu (per vertex).
__global__ void k_sub_ctmu(int nV, const double *__restrict__ C, const double *__restrict__ mu,
                           const int *__restrict__ vprob, double *__restrict__ v, const int *__restrict__ skip)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nV) return;
    int q = vprob[i];
    if (skip && skip[q]) return;
    const double *c = C + (size_t)i * 12;
    const double *m = mu + 4 * q;
    for (int cc = 0; cc < 3; ++cc)
        v[3 * i + cc] -= c[cc] * m[0] + c[3 + cc] * m[1] + c[6 + cc] * m[2] + c[9 + cc] * m[3];
}

// out = scale * C^T G^-1 b  with b = phi (per problem).
__global__ void k_pinv(int nV, const double *__restrict__ C, const double *__restrict__ Gi,
                       const double *__restrict__ b, double scale, const int *__restrict__ vprob,
                       double *__restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nV) return;
    int q = vprob[i];
    const double *g = Gi + 16 * q;
    const double *bb = b + 4 * q;
    double m[4];
    for (int k = 0; k < 4; ++k) m[k] = scale * (g[4 * k] * bb[0] + g[4 * k + 1] * bb[1] + g[4 * k + 2] * bb[2] + g[4 * k + 3] * bb[3]);
    const double *c = C + (size_t)i * 12;
    for (int cc = 0; cc < 3; ++cc) out[3 * i + cc] = c[cc] * m[0] + c[3 + cc] * m[1] + c[6 + cc] * m[2] + c[9 + cc] * m[3];
}

// With TP_CONSTRAINTS_EDGE_LENGTHS the slot of the total-length row holds max_I |l0_I - l_I| over the
// problem's edges (edges.cu), so that one max over the four slots decides the projection's success.
// With TP_CONSTRAINTS_POINTS the barycenter slots hold the largest pin, tangent and surface residuals (pins.cu).
cudaError_t constraints_eval(Ctx &c, const double *gamma, int which, double *phi, cudaStream_t s)
{
    SolverState &st = S(c);
    k_phi<<<st.e_n, kRedThreads, 0, s>>>(eargs(c, 0), c.d_ellw[which], c.d_xw[which], c.d_x0L0, c.d_eprob, phi);
    c.launches++;
    TPE_CHECK(cudaGetLastError());
    if (edge_constraints(c)) TPE_CHECK(edges_phi(c, which, phi, s));
    if (pin_constraints(c) && pins_ready(c)) TPE_CHECK(pins_phi(c, gamma, which, phi, s));
    return cudaSuccess;
}

cudaError_t constraints_targets(Ctx &c, int which, cudaStream_t s)
{
    SolverState &st = S(c);
    k_targets<<<st.e_n, kRedThreads, 0, s>>>(eargs(c, 0), c.d_ellw[which], c.d_xw[which], c.d_x0L0);
    c.launches++;
    TPE_CHECK(cudaGetLastError());
    if (c.edges) TPE_CHECK(edges_targets(c, which, s));
    return cudaSuccess;
}

cudaError_t constraints_jacobian(Ctx &c, int which, cudaStream_t s)
{
    SolverState &st = S(c);
    k_jacobian<<<(c.nV + 255) / 256, 256, 0, s>>>(c.nV, c.d_inc_ptr, c.d_inc, c.d_ellw[which], c.d_Tw[which], c.d_xw[which], c.d_x0L0,
                                                  c.d_vprob, c.d_Cv);
    k_gram_cc<<<st.v_n, kRedThreads, 0, s>>>(vargs(c, 1), c.d_Cv, c.d_G, c.d_Ginv);
    c.launches += 2;
    return cudaGetLastError();
}

cudaError_t project(Ctx &c, double *v, cudaStream_t s, const int *skip)
{
    SolverState &st = S(c);
    k_cv<<<st.v_n, kRedThreads, 0, s>>>(vargs(c, 2), c.d_Cv, v, c.d_Ginv, st.mu, skip);
    k_sub_ctmu<<<(c.nV + 255) / 256, 256, 0, s>>>(c.nV, c.d_Cv, st.mu, c.d_vprob, v, skip);
    c.launches += 2;
    return cudaGetLastError();
}

cudaError_t pinv_apply(Ctx &c, const double *b_phi, double scale, double *out, cudaStream_t s)
{
    k_pinv<<<(c.nV + 255) / 256, 256, 0, s>>>(c.nV, c.d_Cv, c.d_Ginv, b_phi, scale, c.d_vprob, out);
    c.launches++;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------- vector helpers

// out[q] = sum over the problem's vertices of a . b
__global__ void k_dot(RedArgs ra, const double *__restrict__ a, const double *__restrict__ b, double *__restrict__ out)
{
    double s[1] = {0};
    int lo = ra.chunk_lo[blockIdx.x], hi = ra.chunk_lo[blockIdx.x + 1];
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x)
        s[0] += a[3 * i] * b[3 * i] + a[3 * i + 1] * b[3 * i + 1] + a[3 * i + 2] * b[3 * i + 2];
    if (reduce_phase<1>(s, ra))
        for (int q = threadIdx.x; q < ra.nprob; q += blockDim.x) out[q] = ra.sums[q];
}

cudaError_t vec_dot(Ctx &c, const double *a, const double *b, double *out_dev, cudaStream_t s)
{
    SolverState &st = S(c);
    k_dot<<<st.v_n, kRedThreads, 0, s>>>(vargs(c, 3), a, b, out_dev);
    c.launches++;
    return cudaGetLastError();
}

__global__ void k_axpby(int n, double a, const double *__restrict__ x, double b, const double *__restrict__ y,
                        double *__restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a * x[i] + (y ? b * y[i] : 0.0);
}

cudaError_t vec_axpby(Ctx &c, double a, const double *x, double b, const double *y, double *out, cudaStream_t s)
{
    int n = 3 * c.nV;
    k_axpby<<<(n + 255) / 256, 256, 0, s>>>(n, a, x, b, y, out);
    c.launches++;
    return cudaGetLastError();
}

// out = x * f(num[q]) per problem: f = 1/sqrt(num) if invert_sqrt else num.
__global__ void k_scale_prob(int nV, const double *__restrict__ x, const double *__restrict__ num, int invert_sqrt,
                             const int *__restrict__ vprob, double *__restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nV) return;
    double f = num[vprob[i]];
    if (invert_sqrt) f = f > 0.0 ? 1.0 / sqrt(f) : 0.0;
    for (int k = 0; k < 3; ++k) out[3 * i + k] = f * x[3 * i + k];
}

cudaError_t vec_scale_dev(Ctx &c, const double *x, const double *num_dev, int invert_sqrt, double *out,
                          cudaStream_t s)
{
    k_scale_prob<<<(c.nV + 255) / 256, 256, 0, s>>>(c.nV, x, num_dev, invert_sqrt, c.d_vprob, out);
    c.launches++;
    return cudaGetLastError();
}

// out[q] (+)= sum of x over problem q's vertices (per_vertex) or edges, in the fixed chunk order.
__global__ void k_sum_problems(RedArgs ra, const double *__restrict__ x, double *__restrict__ out, int add)
{
    double s[1] = {0};
    int lo = ra.chunk_lo[blockIdx.x], hi = ra.chunk_lo[blockIdx.x + 1];
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) s[0] += x[i];
    if (reduce_phase<1>(s, ra))
        for (int q = threadIdx.x; q < ra.nprob; q += blockDim.x) out[q] = (add ? out[q] : 0.0) + ra.sums[q];
}

cudaError_t sum_problems(Ctx &c, const double *x, int per_vertex, double *out, cudaStream_t s, int add)
{
    SolverState &st = S(c);
    if (per_vertex)
        k_sum_problems<<<st.v_n, kRedThreads, 0, s>>>(vargs(c, 0), x, out, add);
    else
        k_sum_problems<<<st.e_n, kRedThreads, 0, s>>>(eargs(c, 0), x, out, add);
    c.launches++;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------- preconditioners

__global__ void k_jacobi(int nV, const double *__restrict__ diag, const double *__restrict__ r,
                         double *__restrict__ z, const int *__restrict__ vprob, const int *__restrict__ skip)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nV) return;
    if (skip && skip[vprob[i]]) return;
    double d = diag[i];
    double f = d > 0.0 ? 1.0 / d : 0.0;
    for (int k = 0; k < 3; ++k) z[3 * i + k] = f * r[3 * i + k];
}

cudaError_t spectral_apply(Ctx &c, const double *r, double *z, cudaStream_t s, const int *skip);

// M^-1 r without the learned term (TP_PRECOND_LEARNED: the two-level part).
cudaError_t precond_apply_base(Ctx &c, const double *r, double *z, cudaStream_t s, const int *skip)
{
    switch (c.prm.precond) {
    case TP_PRECOND_JACOBI:
        k_jacobi<<<(c.nV + 255) / 256, 256, 0, s>>>(c.nV, c.d_diag, r, z, c.d_vprob, skip);
        c.launches++;
        return cudaGetLastError();
    case TP_PRECOND_SPECTRAL:
    case TP_PRECOND_SPECTRAL_RQ:
        return spectral_apply(c, r, z, s, skip);
    case TP_PRECOND_TWOLEVEL:
    case TP_PRECOND_LEARNED: {
        cudaError_t e = spectral_apply(c, r, z, s, skip);
        if (e != cudaSuccess) return e;
        return coarse_apply(c, r, z, s);
    }
    case TP_PRECOND_TWOLEVEL_BALANCED:
    case TP_PRECOND_LEARNED_BALANCED:
        return coarse_balanced_apply(c, r, z, s, skip, false);
    default:
        return cudaMemcpyAsync(z, r, sizeof(double) * 3 * c.nV, cudaMemcpyDeviceToDevice, s);
    }
}

// M^-1 r of the configured preconditioner.  TP_PRECOND_LEARNED: the circulant with the learned
// per-vertex rescaling, the coarse term and the learned local term G r.
cudaError_t precond_apply(Ctx &c, const double *r, double *z, cudaStream_t s, const int *skip)
{
    if (!precond_learned(c.prm.precond)) return precond_apply_base(c, r, z, s, skip);
    if (!gnn_ready(c) || !gnn_bound(c)) return cudaErrorNotReady;
    if (c.prm.precond == TP_PRECOND_LEARNED_BALANCED) return coarse_balanced_apply(c, r, z, s, skip, true);
    cudaError_t e = spectral_apply_ex(c, r, z, s, skip, c.d_diag, spectral_ilam(c, s), gnn_vlog(c));
    if (e != cudaSuccess) return e;
    if ((e = coarse_apply(c, r, z, s)) != cudaSuccess) return e;
    return gnn_gapply(c, r, z, 1, s, skip);
}

// ---------------------------------------------------------------------------------- CG

// Initialise: bb = r.r (r = P rhs already), rz = r.z; done flags for problems with zero rhs.
// Per problem |r|^2, r.z and |b|^2 (b = P rhs; r = b when the solve starts from zero).  A warm start
// that already meets the tolerance is done at once.
__global__ void k_cg_init(RedArgs ra, const double *__restrict__ r, const double *__restrict__ z,
                          const double *__restrict__ b, double tol2, CGScalars *__restrict__ cg,
                          int *__restrict__ done, int *__restrict__ active)
{
    double s[3] = {0, 0, 0};
    int lo = ra.chunk_lo[blockIdx.x], hi = ra.chunk_lo[blockIdx.x + 1];
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x)
        for (int k = 0; k < 3; ++k) {
            s[0] += r[3 * i + k] * r[3 * i + k];
            s[1] += r[3 * i + k] * z[3 * i + k];
            s[2] += b[3 * i + k] * b[3 * i + k];
        }
    if (reduce_phase<3>(s, ra)) {
        __shared__ int na;
        if (threadIdx.x == 0) na = 0;
        __syncthreads();
        for (int q = threadIdx.x; q < ra.nprob; q += blockDim.x) {
            CGScalars &g = cg[q];
            g.bnorm2 = ra.sums[3 * q + 2];
            g.rnorm2 = ra.sums[3 * q];
            g.rz = ra.sums[3 * q + 1];
            g.iters = 0;
            g.breakdown = 0;
            g.done = (g.bnorm2 == 0.0) || (g.rnorm2 <= tol2 * g.bnorm2);
            done[q] = g.done;
            if (!g.done) atomicAdd(&na, 1);
        }
        __syncthreads();
        if (threadIdx.x == 0) *active = na;
    }
}

// Warm start safeguard: per problem |r0|^2 and |b|^2; where the guess does not reduce the residual the
// problem restarts from y = 0, r = b.
__global__ void k_warm_norms(RedArgs ra, const double *__restrict__ r, const double *__restrict__ b,
                             double *__restrict__ out)
{
    double s[2] = {0, 0};
    int lo = ra.chunk_lo[blockIdx.x], hi = ra.chunk_lo[blockIdx.x + 1];
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x)
        for (int k = 0; k < 3; ++k) {
            s[0] += r[3 * i + k] * r[3 * i + k];
            s[1] += b[3 * i + k] * b[3 * i + k];
        }
    if (reduce_phase<2>(s, ra))
        for (int q = threadIdx.x; q < ra.nprob; q += blockDim.x) {
            out[2 * q] = ra.sums[2 * q];
            out[2 * q + 1] = ra.sums[2 * q + 1];
        }
}

__global__ void k_warm_reset(int nV, const int *__restrict__ vprob, const double *__restrict__ norms,
                             const double *__restrict__ b, double *__restrict__ y, double *__restrict__ r)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nV) return;
    const int q = vprob[i];
    if (!(norms[2 * q] < norms[2 * q + 1])) {
        for (int k = 0; k < 3; ++k) {
            y[3 * i + k] = 0.0;
            r[3 * i + k] = b[3 * i + k];
        }
    }
}

// alpha = rz / (p.q) per active problem.  fuse: q is not yet mean-free; its per-problem mean mq is
// taken here and p.(q - mq) = p.q - mq.sum(p) is used (the mean-free projector folded into the CG
// kernels: k_cg_update subtracts mq).
__global__ void k_cg_alpha(RedArgs ra, const double *__restrict__ p, const double *__restrict__ q_,
                           CGScalars *__restrict__ cg, int *__restrict__ done, const int *__restrict__ prob_v,
                           int fuse)
{
    double s[7] = {0, 0, 0, 0, 0, 0, 0};
    int lo = ra.chunk_lo[blockIdx.x], hi = ra.chunk_lo[blockIdx.x + 1];
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x)
        for (int k = 0; k < 3; ++k) {
            s[0] += p[3 * i + k] * q_[3 * i + k];
            s[1 + k] += q_[3 * i + k];
            s[4 + k] += p[3 * i + k];
        }
    if (reduce_phase<7>(s, ra)) {
        for (int q = threadIdx.x; q < ra.nprob; q += blockDim.x) {
            CGScalars &g = cg[q];
            if (g.done) continue;
            const double *S7 = ra.sums + 7 * q;
            double pq = S7[0];
            const double n = (double)(prob_v[q + 1] - prob_v[q]);
            for (int k = 0; k < 3; ++k) {
                g.mq[k] = (fuse && n > 0) ? S7[1 + k] / n : 0.0;
                pq -= g.mq[k] * S7[4 + k];
            }
            g.pq = pq;
            if (!(pq > 0.0)) {
                g.breakdown = 1;
                g.done = 1;
                done[q] = 1;
                g.alpha = 0.0;
            } else {
                g.alpha = g.rz / pq;
            }
        }
    }
}

// y += alpha p; r -= alpha q (active problems); then r.r
__global__ void k_cg_update(RedArgs ra, const int *__restrict__ vprob, const double *__restrict__ p,
                            const double *__restrict__ q_, double *__restrict__ y, double *__restrict__ r,
                            CGScalars *__restrict__ cg, int *__restrict__ done, double tol2, int *__restrict__ active)
{
    double s[1] = {0};
    int lo = ra.chunk_lo[blockIdx.x], hi = ra.chunk_lo[blockIdx.x + 1];
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        int pr = vprob[i];
        if (done[pr]) continue;
        double a = cg[pr].alpha;
        for (int k = 0; k < 3; ++k) {
            y[3 * i + k] += a * p[3 * i + k];
            double rv = r[3 * i + k] - a * (q_[3 * i + k] - cg[pr].mq[k]);
            r[3 * i + k] = rv;
            s[0] += rv * rv;
        }
    }
    if (reduce_phase<1>(s, ra)) {
        __shared__ int na;
        if (threadIdx.x == 0) na = 0;
        __syncthreads();
        for (int q = threadIdx.x; q < ra.nprob; q += blockDim.x) {
            CGScalars &g = cg[q];
            if (!g.done) {
                g.rnorm2 = ra.sums[q];
                g.iters += 1;
                if (g.rnorm2 <= tol2 * g.bnorm2) {
                    g.done = 1;
                    done[q] = 1;
                }
            }
            if (!g.done) atomicAdd(&na, 1);
        }
        __syncthreads();
        if (threadIdx.x == 0) *active = na;
    }
}

// rz_new = r.z; beta = rz_new / rz; rz = rz_new (active problems).  fuse: z is not yet mean-free; its
// mean mz is taken here, r.(z - mz) = r.z - mz.sum(r) is used, and k_cg_p subtracts mz.
__global__ void k_cg_beta(RedArgs ra, const double *__restrict__ r, const double *__restrict__ z,
                          CGScalars *__restrict__ cg, const int *__restrict__ done, const int *__restrict__ prob_v,
                          int fuse)
{
    double s[7] = {0, 0, 0, 0, 0, 0, 0};
    int lo = ra.chunk_lo[blockIdx.x], hi = ra.chunk_lo[blockIdx.x + 1];
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x)
        for (int k = 0; k < 3; ++k) {
            s[0] += r[3 * i + k] * z[3 * i + k];
            s[1 + k] += z[3 * i + k];
            s[4 + k] += r[3 * i + k];
        }
    if (reduce_phase<7>(s, ra)) {
        for (int q = threadIdx.x; q < ra.nprob; q += blockDim.x) {
            CGScalars &g = cg[q];
            if (g.done) continue;
            const double *S7 = ra.sums + 7 * q;
            double rzn = S7[0];
            const double n = (double)(prob_v[q + 1] - prob_v[q]);
            for (int k = 0; k < 3; ++k) {
                g.mz[k] = (fuse && n > 0) ? S7[1 + k] / n : 0.0;
                rzn -= g.mz[k] * S7[4 + k];
            }
            g.beta = g.rz != 0.0 ? rzn / g.rz : 0.0;
            g.rz = rzn;
        }
    }
}

// p = z + beta p (active problems)
__global__ void k_cg_p(int nV, const int *__restrict__ vprob, const double *__restrict__ z, double *__restrict__ p,
                       const CGScalars *__restrict__ cg, const int *__restrict__ done)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nV) return;
    int q = vprob[i];
    if (done[q]) return;
    double b = cg[q].beta;
    for (int k = 0; k < 3; ++k) p[3 * i + k] = (z[3 * i + k] - cg[q].mz[k]) + b * p[3 * i + k];
}

// Relative residual per problem: out[q] = sqrt(|r_true|^2 / |P rhs|^2), |P rhs|^2 from bn2[q] when given
// (the refinement keeps the first solve's norms), else from the solve's scalars.  bn2_out (may be NULL)
// receives the norms used.
__global__ void k_relres(RedArgs ra, const double *__restrict__ r, const CGScalars *__restrict__ cg,
                         double *__restrict__ out, const double *__restrict__ bn2, double *__restrict__ bn2_out)
{
    double s[1] = {0};
    int lo = ra.chunk_lo[blockIdx.x], hi = ra.chunk_lo[blockIdx.x + 1];
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x)
        s[0] += r[3 * i] * r[3 * i] + r[3 * i + 1] * r[3 * i + 1] + r[3 * i + 2] * r[3 * i + 2];
    if (reduce_phase<1>(s, ra))
        for (int q = threadIdx.x; q < ra.nprob; q += blockDim.x) {
            const double b = bn2 ? bn2[q] : cg[q].bnorm2;
            out[q] = b > 0.0 ? sqrt(ra.sums[q] / b) : 0.0;
            if (bn2_out) bn2_out[q] = b;
        }
}

// v[i] = 0 on the vertices of problems whose keep[q] is 0
__global__ void k_zero_problems(int nV, const int *__restrict__ vprob, const int *__restrict__ keep,
                                double *__restrict__ v)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nV || keep[vprob[i]]) return;
    v[3 * i] = v[3 * i + 1] = v[3 * i + 2] = 0.0;
}

// Solve P A-bar P y = P rhs (A-bar of the geometry `which`), x = P y.  The constraint Jacobian
// (c.d_Cv, c.d_Ginv) must describe the projector to use.  rhs and x may not alias the CG scratch.
cudaError_t project_mean(Ctx &c, double *v, cudaStream_t s, const int *skip);

// v -= C_len (C_len . v) / (C_len . C_len) per problem (the total-length row of the Jacobian at the base
// curve, row 3 of c.d_Cv); C_len sums to zero over every problem, so this commutes with the mean removal.
__global__ void k_len_red(RedArgs ra, const double *__restrict__ C, const double *__restrict__ v,
                          double *__restrict__ out)
{
    double s[2] = {0, 0};
    int lo = ra.chunk_lo[blockIdx.x], hi = ra.chunk_lo[blockIdx.x + 1];
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x)
        for (int k = 0; k < 3; ++k) {
            const double cl = C[(size_t)i * 12 + 9 + k];
            s[0] += cl * v[3 * i + k];
            s[1] += cl * cl;
        }
    if (reduce_phase<2>(s, ra))
        for (int q = threadIdx.x; q < ra.nprob; q += blockDim.x)
            out[q] = ra.sums[2 * q + 1] > 0.0 ? ra.sums[2 * q] / ra.sums[2 * q + 1] : 0.0;
}

__global__ void k_len_sub(int nV, const double *__restrict__ C, const double *__restrict__ coef,
                          const int *__restrict__ vprob, double *__restrict__ v, const int *__restrict__ skip)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nV) return;
    const int q = vprob[i];
    if (skip && skip[q]) return;
    const double a = coef[q];
    for (int k = 0; k < 3; ++k) v[3 * i + k] -= a * C[(size_t)i * 12 + 9 + k];
}

static cudaError_t project_len(Ctx &c, double *v, cudaStream_t s, const int *skip)
{
    SolverState &st = S(c);
    k_len_red<<<st.v_n, kRedThreads, 0, s>>>(vargs(c, 2), c.d_Cv, v, st.mu);
    k_len_sub<<<(c.nV + 255) / 256, 256, 0, s>>>(c.nV, c.d_Cv, st.mu, c.d_vprob, v, skip);
    c.launches += 2;
    return cudaGetLastError();
}

// proj_mode 0: P = I - C^T (C C^T)^-1 C (constraint projector); 1: P = subtract the per-problem mean;
// 2: the mean, then the edge-length rows (P = P_E P_N, the two commute; edges.cu, set up by edges_setup);
// 3: the mean, then the total-length row (P = P_len P_N; the projected system of App. B.3.3 for the
// total-length row, with the translations left to the barycenter shift).
static cudaError_t projector(Ctx &c, int mode, double *v, cudaStream_t s, const int *skip)
{
    if (mode == 2) {
        TPE_CHECK(project_mean(c, v, s, skip));
        return edges_project(c, v, s, skip);
    }
    if (mode == 3) {
        TPE_CHECK(project_mean(c, v, s, skip));
        return project_len(c, v, s, skip);
    }
    return mode ? project_mean(c, v, s, skip) : project(c, v, s, skip);
}

// What the CG iteration still applies outside its kernels: mode 0 the whole constraint projector, mode 1
// nothing, mode 2 the edge rows, mode 3 the length row (both commute with the mean removal).
static cudaError_t projector_rest(Ctx &c, int mode, double *v, cudaStream_t s, const int *skip)
{
    if (mode == 0) return project(c, v, s, skip);
    if (mode == 2) return edges_project(c, v, s, skip);
    if (mode == 3) return project_len(c, v, s, skip);
    return cudaSuccess;
}

// ---------------------------------------------------------------------------------- CUDA graphs of CG blocks

static cudaError_t graph_stream(Ctx &c)
{
    if (c.cg_stream) return cudaSuccess;
    TPE_CHECK(cudaStreamCreateWithFlags(&c.cg_stream, cudaStreamNonBlocking));
    TPE_CHECK(cudaEventCreateWithFlags(&c.cg_join[0], cudaEventDisableTiming));
    TPE_CHECK(cudaEventCreateWithFlags(&c.cg_join[1], cudaEventDisableTiming));
    return cudaSuccess;
}

static void graph_destroy(CgGraph &g)
{
    if (g.exec) cudaGraphExecDestroy(g.exec);
    for (cudaEvent_t e : g.ev)
        if (e) cudaEventDestroy(e);
    g = CgGraph{};
}

void graphs_reset(Ctx &c)
{
    for (auto &g : c.graphs) graph_destroy(g);
    c.graphs.clear();
}

void graphs_free(Ctx &c)
{
    for (auto &g : c.graphs) graph_destroy(g);
    c.graphs.clear();
    if (c.cg_stream) cudaStreamDestroy(c.cg_stream);
    for (auto &e : c.cg_join)
        if (e) cudaEventDestroy(e);
    c.cg_stream = nullptr;
    c.cg_join[0] = c.cg_join[1] = nullptr;
}

// Profiled pair-kernel times of the last replay of g into the context's per-op totals.
static void graph_prof_harvest(Ctx &c, CgGraph &g)
{
    for (size_t k = 0; k < g.prof_op.size(); ++k) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, g.ev[2 * k], g.ev[2 * k + 1]) == cudaSuccess) {
            c.prof_ms[g.prof_op[k]] += ms;
            c.prof_n[g.prof_op[k]] += 1;
        }
    }
}

// The cached graph of `every` CG iterations for this solve's settings, captured on first use.  A
// failed capture leaves *out = NULL and switches the context to direct launches.
template <class Body>
static cudaError_t graph_block(Ctx &c, const double *gamma_geom, int which, int proj_mode, int every, double tol2,
                               Body &body, cudaStream_t cs, CgGraph **out)
{
    *out = nullptr;
    const void *items = c.plan_apply.d_items;
    for (auto &g : c.graphs)
        if (g.exec && g.gamma == gamma_geom && g.which == which && g.proj_mode == proj_mode &&
            g.precond == c.prm.precond && g.every == every && g.profile == c.profile && g.items == items &&
            g.tpt == c.plan_apply.tpt && g.tol2 == tol2 && g.sym == c.apply_sym) {
            g.stamp = ++c.graph_clock;
            *out = &g;
            return cudaSuccess;
        }
    if (c.graphs.size() < 4) c.graphs.emplace_back();
    CgGraph *slot = &c.graphs[0];
    for (auto &g : c.graphs)
        if (g.stamp < slot->stamp) slot = &g;
    graph_destroy(*slot);
    CgGraph &g = *slot;
    g.gamma = gamma_geom;
    g.which = which;
    g.proj_mode = proj_mode;
    g.precond = c.prm.precond;
    g.every = every;
    g.profile = c.profile;
    g.items = items;
    g.tpt = c.plan_apply.tpt;
    g.tol2 = tol2;
    g.sym = c.apply_sym;
    g.stamp = ++c.graph_clock;
    if (c.profile) {
        g.ev.resize(4 * every + 8);
        for (auto &e : g.ev) TPE_CHECK(cudaEventCreate(&e));
    }
    if (c.profile) prof_harvest(c);  // nothing recorded on the stream may be waited on during capture
    const int64_t l0 = c.launches;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        c.capturing = &g;
        for (int k = 0; k < every && e == cudaSuccess; ++k) e = body(cs);
        c.capturing = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) e = e2;
    }
    g.launches = c.launches - l0;
    c.launches = l0;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();  // clear the capture error; the solve continues with direct launches
        graph_destroy(g);
        c.graphs_broken = 1;
        return cudaSuccess;
    }
    *out = &g;
    return cudaSuccess;
}

// Per-problem outcome of one preconditioned CG run.
struct PcgOut {
    std::vector<int> iters, done, bd;
    std::vector<double> rr;  // true relative residual of x (when computed)
};

// Preconditioned CG on P A-bar P y = P rhs (the working-precision operator), x = P y.  residual: 0 none,
// 1 with the working-precision operator, 2 with the accurate (double-float) one; r = P (rhs - A-bar x) is
// then left in c.d_r and the norms |P rhs|^2 in bn2 (device [nProb], may be NULL).
static cudaError_t pcg_run(Ctx &c, const double *gamma_geom, int which, const double *rhs, double *x, double rtol,
                           int maxit, cudaStream_t s, int proj_mode, const double *x0, int residual, PcgOut &out,
                           double *bn2)
{
    SolverState &st = S(c);
    const size_t vb = sizeof(double) * 3 * c.nV;
    const int nb = (c.nV + 255) / 256;
    double *r = c.d_r, *z = c.d_z, *p = c.d_p, *q = c.d_q, *y = c.d_y;
    const double tol2 = rtol * rtol;
    // b = P rhs (kept in q until the iterations start)
    TPE_CHECK(cudaMemcpyAsync(q, rhs, vb, cudaMemcpyDeviceToDevice, s));
    TPE_CHECK(projector(c, proj_mode, q, s, nullptr));
    if (x0) {
        // y = P x0, r = b - P A-bar y; problems the guess does not help restart from zero
        TPE_CHECK(cudaMemcpyAsync(y, x0, vb, cudaMemcpyDeviceToDevice, s));
        TPE_CHECK(projector(c, proj_mode, y, s, nullptr));
        TPE_CHECK(pair_apply(c, gamma_geom, which, y, z, s));
        TPE_CHECK(projector(c, proj_mode, z, s, nullptr));
        TPE_CHECK(vec_axpby(c, 1.0, q, -1.0, z, r, s));
        double *norms = c.d_scal + 64 + 12 * (size_t)c.nProb;  // [nProb][2]
        k_warm_norms<<<st.v_n, kRedThreads, 0, s>>>(vargs(c, 4), r, q, norms);
        k_warm_reset<<<nb, 256, 0, s>>>(c.nV, c.d_vprob, norms, q, y, r);
        c.launches += 2;
    } else {
        TPE_CHECK(cudaMemcpyAsync(r, q, vb, cudaMemcpyDeviceToDevice, s));
        TPE_CHECK(cudaMemsetAsync(y, 0, vb, s));
    }
    TPE_CHECK(precond_apply(c, r, z, s, nullptr));
    if (c.prm.precond != TP_PRECOND_NONE) TPE_CHECK(projector(c, proj_mode, z, s, nullptr));
    TPE_CHECK(cudaMemcpyAsync(p, z, vb, cudaMemcpyDeviceToDevice, s));
    k_cg_init<<<st.v_n, kRedThreads, 0, s>>>(vargs(c, 4), r, z, q, tol2, c.d_cg, st.done, st.active);
    c.launches++;
    const int every = std::max(1, c.prm.cg_check_every);
    const int fuse = proj_mode != 0;  // projector modes 1, 2: their mean removal runs inside the CG kernels
    int it = 0;
    int *h_active = c.h_pinned_i;
    // one CG iteration enqueued on stream ss
    auto body = [&](cudaStream_t ss) -> cudaError_t {
        // q = P A-bar p (work items of converged problems are skipped)
        c.d_skip = st.done;
        cudaError_t ea = pair_apply(c, gamma_geom, which, p, q, ss);
        c.d_skip = nullptr;
        TPE_CHECK(ea);
        // the mean-free part of the projector is folded into the CG kernels (fuse); the rest runs here
        TPE_CHECK(projector_rest(c, proj_mode, q, ss, st.done));
        k_cg_alpha<<<st.v_n, kRedThreads, 0, ss>>>(vargs(c, 5), p, q, c.d_cg, st.done, c.d_prob_v, fuse);
        k_cg_update<<<st.v_n, kRedThreads, 0, ss>>>(vargs(c, 6), c.d_vprob, p, q, y, r, c.d_cg, st.done, tol2,
                                                    st.active);
        c.launches += 2;
        TPE_CHECK(precond_apply(c, r, z, ss, st.done));
        if (c.prm.precond != TP_PRECOND_NONE) TPE_CHECK(projector_rest(c, proj_mode, z, ss, st.done));
        k_cg_beta<<<st.v_n, kRedThreads, 0, ss>>>(vargs(c, 7), r, c.prm.precond != TP_PRECOND_NONE ? z : r,
                                                  c.d_cg, st.done, c.d_prob_v, fuse);
        k_cg_p<<<nb, 256, 0, ss>>>(c.nV, c.d_vprob, c.prm.precond != TP_PRECOND_NONE ? z : r, p, c.d_cg, st.done);
        c.launches += 2;
        return cudaGetLastError();
    };
    // Blocks of `every` iterations between host polls run as captured graphs (not while pairs are
    // being harvested, which copies per iteration).
    const bool graphs = c.prm.use_graphs && !c.graphs_broken && !c.hv.R && maxit >= every;
    cudaStream_t rs = s;
    if (graphs) {
        TPE_CHECK(graph_stream(c));
        rs = c.cg_stream;
        TPE_CHECK(cudaEventRecord(c.cg_join[0], s));
        TPE_CHECK(cudaStreamWaitEvent(rs, c.cg_join[0], 0));
    }
    for (; it < maxit;) {
        if (graphs && !c.graphs_broken && maxit - it >= every) {
            CgGraph *g = nullptr;
            TPE_CHECK(graph_block(c, gamma_geom, which, proj_mode, every, tol2, body, rs, &g));
            if (g) {
                TPE_CHECK(cudaGraphLaunch(g->exec, rs));
                c.launches += g->launches;
                it += every;
                TPE_CHECK(cudaMemcpyAsync(h_active, st.active, sizeof(int), cudaMemcpyDeviceToHost, rs));
                TPE_CHECK(cudaStreamSynchronize(rs));
                graph_prof_harvest(c, *g);
                if (*h_active == 0) break;
                continue;
            }
        }
        TPE_CHECK(body(rs));
        ++it;
        if (c.hv.R && c.hv.n < c.hv.max && it % c.hv.every == 0) {
            const size_t off = (size_t)c.hv.n * 3 * c.nV;
            TPE_CHECK(cudaMemcpyAsync(c.hv.R + off, r, vb, cudaMemcpyDeviceToDevice, rs));
            TPE_CHECK(cudaMemcpyAsync(c.hv.Y + off, y, vb, cudaMemcpyDeviceToDevice, rs));
            c.hv.n++;
        }
        if (it % every == 0 || it == maxit) {
            TPE_CHECK(cudaMemcpyAsync(h_active, st.active, sizeof(int), cudaMemcpyDeviceToHost, rs));
            TPE_CHECK(cudaStreamSynchronize(rs));
            if (*h_active == 0) break;
        }
    }
    if (graphs) {  // join: the caller's stream waits for the iterations
        TPE_CHECK(cudaEventRecord(c.cg_join[1], rs));
        TPE_CHECK(cudaStreamWaitEvent(s, c.cg_join[1], 0));
    }
    // x = P y; true residual r = P (rhs - A-bar x)
    TPE_CHECK(cudaMemcpyAsync(x, y, vb, cudaMemcpyDeviceToDevice, s));
    TPE_CHECK(projector(c, proj_mode, x, s, nullptr));
    double *rr = c.d_scal + 64 + 10 * (size_t)c.nProb;  // [nProb]
    if (residual) {
        if (residual == 2)
            TPE_CHECK(pair_apply_acc(c, gamma_geom, which, x, q, s));
        else
            TPE_CHECK(pair_apply(c, gamma_geom, which, x, q, s));
        TPE_CHECK(vec_axpby(c, 1.0, rhs, -1.0, q, r, s));
        TPE_CHECK(projector(c, proj_mode, r, s, nullptr));
        k_relres<<<st.v_n, kRedThreads, 0, s>>>(vargs(c, 3), r, c.d_cg, rr, nullptr, bn2);
        c.launches++;
    }
    std::vector<CGScalars> hcg(c.nProb);
    out.rr.assign(c.nProb, 0.0);
    TPE_CHECK(cudaMemcpyAsync(hcg.data(), c.d_cg, sizeof(CGScalars) * c.nProb, cudaMemcpyDeviceToHost, s));
    if (residual) TPE_CHECK(cudaMemcpyAsync(out.rr.data(), rr, sizeof(double) * c.nProb, cudaMemcpyDeviceToHost, s));
    TPE_CHECK(cudaStreamSynchronize(s));
    out.iters.resize(c.nProb);
    out.done.resize(c.nProb);
    out.bd.resize(c.nProb);
    for (int qq = 0; qq < c.nProb; ++qq) {
        out.iters[qq] = hcg[qq].iters;
        out.done[qq] = hcg[qq].done;
        out.bd[qq] = hcg[qq].breakdown;
    }
    return cudaSuccess;
}

// Solves below this relative tolerance in FP32 / mixed contexts are refined against the double-float
// operator: the FP32 pair arithmetic's rounding sets a floor on the true residual (~1e-5 on curves of
// 4,096 vertices, ~3e-4 on smooth vectors at 262,144, growing like n^2) that the recursive residual does
// not see.  Looser solves (the constraint projections at 1e-3) keep the working-precision residual.
constexpr double kRefineBelow = 5e-4;
constexpr int kRefineMax = 4;        // correction solves at most
constexpr double kUpdateBelow = 1e-2; // residuals below this are updated with the working-precision A-bar e
constexpr double kCorrectionTol = 1e-2;

cudaError_t cg_solve(Ctx &c, const double *gamma_geom, int which, const double *rhs, double *x, double rtol,
                     int maxit, int *iters, double *rel_res, int *converged, int *breakdown, cudaStream_t s,
                     int proj_mode, int *conv_flags, const double *x0)
{
    SolverState &st = S(c);
    const bool refine = c.prm.precision != TP_FP64 && rtol < kRefineBelow && !c.hv.R;
    double *bn2 = c.d_scal + 64 + 11 * (size_t)c.nProb;  // [nProb] |P rhs|^2 of this solve
    PcgOut o;
    TPE_CHECK(pcg_run(c, gamma_geom, which, rhs, x, rtol, maxit, s, proj_mode, x0, refine ? 2 : 1, o, bn2));
    std::vector<int> it = o.iters, bd = o.bd, done = o.done;
    std::vector<double> rr = o.rr;
    int rounds = 0;
    if (refine) {
        // Iterative refinement: the residual r = P (rhs - A-bar_acc x) of the accurate operator is solved
        // for a correction e with the working-precision PCG (to kCorrectionTol relative), x += e, and the
        // residual of the new x follows, until every problem's true relative residual is within rtol.
        // The new residual is r - P A-bar_w e with the working-precision product when every residual
        // was below kUpdateBelow: A-bar_w's relative error on e (its rounding floor, ~3e-4 on smooth
        // vectors at 262,144 edges) then multiplies |A-bar e| ~ |r| <= kUpdateBelow |P rhs|, and adds at
        // most ~3e-6 |P rhs| against the accurate evaluation of A-bar x it replaces.  Otherwise the
        // accurate operator forms it again.
        const int nb = (c.nV + 255) / 256;
        int *keep = reinterpret_cast<int *>(c.d_scal + 64 + 14 * (size_t)c.nProb);  // nProb ints
        double *rr_d = c.d_scal + 64 + 10 * (size_t)c.nProb;
        std::vector<double> prev(c.nProb, 0.0);
        for (; rounds < kRefineMax; ++rounds) {
            std::vector<int> need(c.nProb, 0);
            int any = 0;
            for (int q = 0; q < c.nProb; ++q) {
                // a problem whose last correction did not halve its residual has reached the accurate
                // operator's own evaluation floor: further rounds cannot help it
                const bool stalled = rounds > 0 && rr[q] > 0.5 * prev[q];
                need[q] = !bd[q] && rr[q] > rtol && !stalled;
                any |= need[q];
            }
            if (!any) break;
            prev = rr;
            double mx = 0.0;
            for (int q = 0; q < c.nProb; ++q) mx = std::max(mx, rr[q]);
            const bool update = mx <= kUpdateBelow;
            TPE_CHECK(cudaMemcpyAsync(keep, need.data(), sizeof(int) * c.nProb, cudaMemcpyHostToDevice, s));
            TPE_CHECK(cudaMemcpyAsync(c.d_rf, c.d_r, sizeof(double) * 3 * c.nV, cudaMemcpyDeviceToDevice, s));
            if (update) TPE_CHECK(cudaMemcpyAsync(c.d_rs, c.d_r, sizeof(double) * 3 * c.nV, cudaMemcpyDeviceToDevice, s));
            k_zero_problems<<<nb, 256, 0, s>>>(c.nV, c.d_vprob, keep, c.d_rf);
            c.launches++;
            PcgOut oc;
            TPE_CHECK(pcg_run(c, gamma_geom, which, c.d_rf, c.d_ef, kCorrectionTol, maxit, s, proj_mode, nullptr, 0, oc,
                              nullptr));
            TPE_CHECK(vec_axpby(c, 1.0, x, 1.0, c.d_ef, x, s));
            for (int q = 0; q < c.nProb; ++q)
                if (need[q]) {
                    it[q] += oc.iters[q];
                    bd[q] |= oc.bd[q];
                }
            // r = P (rhs - A-bar_acc x), relative to the first solve's |P rhs|: updated by the correction's
            // working-precision product, or formed again with the accurate operator
            if (update) {
                TPE_CHECK(pair_apply(c, gamma_geom, which, c.d_ef, c.d_q, s));
                TPE_CHECK(projector(c, proj_mode, c.d_q, s, nullptr));
                TPE_CHECK(vec_axpby(c, 1.0, c.d_rs, -1.0, c.d_q, c.d_r, s));
            } else {
                TPE_CHECK(pair_apply_acc(c, gamma_geom, which, x, c.d_q, s));
                TPE_CHECK(vec_axpby(c, 1.0, rhs, -1.0, c.d_q, c.d_r, s));
                TPE_CHECK(projector(c, proj_mode, c.d_r, s, nullptr));
            }
            k_relres<<<st.v_n, kRedThreads, 0, s>>>(vargs(c, 3), c.d_r, c.d_cg, rr_d, bn2, nullptr);
            c.launches++;
            TPE_CHECK(cudaMemcpyAsync(rr.data(), rr_d, sizeof(double) * c.nProb, cudaMemcpyDeviceToHost, s));
            TPE_CHECK(cudaStreamSynchronize(s));
        }
    }
    c.last_rr = rr;
    c.last_iters = it;
    c.last_refinements = rounds;
    // converged: CG met the tolerance and the true relative residual is within rtol when it was judged by
    // the accurate operator (refined solves), or within 10 rtol when judged by the working-precision
    // operator after CG stopped on its recursive residual (FP64 solves, whose rounding can leave the true
    // residual a little above a tolerance near 1e-11; and the loose projection solves)
    const double lim = refine ? rtol : 10.0 * rtol;
    int mx_it = 0, b = 0, conv = 1;
    double mx_rr = 0.0;
    for (int q = 0; q < c.nProb; ++q) {
        mx_it = std::max(mx_it, it[q]);
        b |= bd[q];
        const int ok = (done[q] || refine) && !bd[q] && rr[q] <= lim;
        conv &= ok;
        if (conv_flags) conv_flags[q] &= ok;
        mx_rr = std::max(mx_rr, rr[q]);
    }
    if (iters) *iters = mx_it;
    if (rel_res) *rel_res = mx_rr;
    if (converged) *converged = conv;
    if (breakdown) *breakdown = b;
    return cudaSuccess;
}

}  // namespace tpe

namespace tpe {

// ---------------------------------------------------------------------------------- mean-free route
//
// For the barycenter + total-length constraint set the KKT systems of Eqs. 22-23 reduce to solves
// on the mean-free subspace.  null(A-bar) = span{e_x, e_y, e_z} (translations), and C_bary N = L Id,
// C_len N = 0 (N: the translation basis).  Solvability of A-bar g + C^T lambda = dE needs
// N^T C^T lambda = 0, i.e. lambda_bary = 0, hence
//   g = A^+ dE - lambda_len A^+ C_len^T + N t,   lambda_len = <C_len, A^+ dE> / <C_len, A^+ C_len^T>,
//   t = -(C_bary N)^-1 C_bary (A^+ dE - lambda_len A^+ C_len^T),
// and the constraint projection min x^T A-bar x / 2 s.t. C x = b has x = mu A^+ C_len^T + N t with
// mu = b_len / <C_len, A^+ C_len^T>, t = (C_bary N)^-1 (b_bary - mu C_bary A^+ C_len^T).
// A^+ is applied by CG on the mean-free subspace (projector: subtract the per-problem mean).

// per-problem mean of each component
__global__ void k_mean(RedArgs ra, const double *__restrict__ v, const int *__restrict__ prob_v,
                       double *__restrict__ mean)
{
    double s[3] = {0, 0, 0};
    int lo = ra.chunk_lo[blockIdx.x], hi = ra.chunk_lo[blockIdx.x + 1];
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x)
        for (int k = 0; k < 3; ++k) s[k] += v[3 * i + k];
    if (reduce_phase<3>(s, ra))
        for (int q = threadIdx.x; q < ra.nprob; q += blockDim.x) {
            double n = (double)(prob_v[q + 1] - prob_v[q]);
            for (int k = 0; k < 3; ++k) mean[3 * q + k] = n > 0 ? ra.sums[3 * q + k] / n : 0.0;
        }
}

__global__ void k_sub_mean(int nV, const double *__restrict__ mean, const int *__restrict__ vprob,
                           double *__restrict__ v, const int *__restrict__ skip)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nV) return;
    int q = vprob[i];
    if (skip && skip[q]) return;
    for (int k = 0; k < 3; ++k) v[3 * i + k] -= mean[3 * q + k];
}

cudaError_t project_mean(Ctx &c, double *v, cudaStream_t s, const int *skip)
{
    SolverState &st = S(c);
    k_mean<<<st.v_n, kRedThreads, 0, s>>>(vargs(c, 2), v, c.d_prob_v, st.mu);
    k_sub_mean<<<(c.nV + 255) / 256, 256, 0, s>>>(c.nV, st.mu, c.d_vprob, v, skip);
    c.launches += 2;
    return cudaGetLastError();
}

// out[v] = C_len row (row 3 of C) at vertex v
__global__ void k_clen(int nV, const double *__restrict__ C, double *__restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nV) return;
    for (int k = 0; k < 3; ++k) out[3 * i + k] = C[(size_t)i * 12 + 9 + k];
}

cudaError_t clen_rhs(Ctx &c, double *out, cudaStream_t s)
{
    k_clen<<<(c.nV + 255) / 256, 256, 0, s>>>(c.nV, c.d_Cv, out);
    c.launches++;
    return cudaGetLastError();
}

// Reductions per problem: s[0] = <C_len, a>, s[1] = <C_len, b>, s[2..4] = C_bary_k . b,
// s[5..13] = (C_bary N)_kj = sum_v C[v][k][j].
__global__ void k_schur_red(RedArgs ra, const double *__restrict__ C, const double *__restrict__ a,
                            const double *__restrict__ b, double *__restrict__ out)
{
    double s[14] = {0};
    int lo = ra.chunk_lo[blockIdx.x], hi = ra.chunk_lo[blockIdx.x + 1];
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double *cv = C + (size_t)i * 12;
        for (int j = 0; j < 3; ++j) {
            double av = a ? a[3 * i + j] : 0.0, bv = b[3 * i + j];
            s[0] += cv[9 + j] * av;
            s[1] += cv[9 + j] * bv;
            for (int k = 0; k < 3; ++k) {
                s[2 + k] += cv[3 * k + j] * bv;
                s[5 + 3 * k + j] += cv[3 * k + j];
            }
        }
    }
    if (reduce_phase<14>(s, ra))
        for (int q = threadIdx.x; q < ra.nprob; q += blockDim.x)
            for (int k = 0; k < 14; ++k) out[14 * q + k] = ra.sums[14 * q + k];
}

__device__ void solve3(const double *M, const double *r, double *x)
{
    double a = M[0], b = M[1], c = M[2], d = M[3], e = M[4], f = M[5], g = M[6], h = M[7], k = M[8];
    double det = a * (e * k - f * h) - b * (d * k - f * g) + c * (d * h - e * g);
    if (det == 0.0) det = 1e-300;
    double inv[9] = {(e * k - f * h), -(b * k - c * h), (b * f - c * e), -(d * k - f * g), (a * k - c * g),
                     -(a * f - c * d), (d * h - e * g), -(a * h - b * g), (a * e - b * d)};
    for (int i = 0; i < 3; ++i) x[i] = (inv[3 * i] * r[0] + inv[3 * i + 1] * r[1] + inv[3 * i + 2] * r[2]) / det;
}

// g' = y0 - lambda y1 with lambda = s0 / s1 (per problem), written to out.
__global__ void k_schur_lin(int nV, const double *__restrict__ red, const double *__restrict__ y0,
                            const double *__restrict__ y1, const int *__restrict__ vprob, double *__restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nV) return;
    const double *r = red + 14 * vprob[i];
    double lam = r[1] != 0.0 ? r[0] / r[1] : 0.0;
    for (int k = 0; k < 3; ++k) out[3 * i + k] = y0[3 * i + k] - lam * y1[3 * i + k];
}

// out += t with (C_bary N) t = target - C_bary out  (target: -phi_bary scaled, or 0)
__global__ void k_schur_shift(int nV, const double *__restrict__ red, const double *__restrict__ phi, double phi_scale,
                              const int *__restrict__ vprob, double *__restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nV) return;
    int q = vprob[i];
    const double *r = red + 14 * q;
    double rhs[3], t[3];
    for (int k = 0; k < 3; ++k) rhs[k] = (phi ? phi_scale * phi[4 * q + k] : 0.0) - r[2 + k];
    solve3(r + 5, rhs, t);
    for (int k = 0; k < 3; ++k) out[3 * i + k] += t[k];
}

// x = mu y1 with mu = b_len / <C_len, y1>, b = phi_scale * phi (per problem).
__global__ void k_proj_lin(int nV, const double *__restrict__ red, const double *__restrict__ phi, double phi_scale,
                           const double *__restrict__ y1, const int *__restrict__ vprob, double *__restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nV) return;
    int q = vprob[i];
    const double *r = red + 14 * q;
    double mu = r[1] != 0.0 ? phi_scale * phi[4 * q + 3] / r[1] : 0.0;
    for (int k = 0; k < 3; ++k) out[3 * i + k] = mu * y1[3 * i + k];
}

// g = A^+ dE - lambda A^+ C_len^T + N t from y0 = A^+ dE and y1 = A^+ C_len^T (Jacobian in c.d_Cv).
cudaError_t schur_gradient(Ctx &c, const double *y0, const double *y1, double *g, cudaStream_t s)
{
    SolverState &st = S(c);
    double *red = st.sums + 0;  // scratch reused below
    double *red_out = c.d_red;  // [nProb][14] (d_red holds 16 per problem)
    (void)red;
    const int nb = (c.nV + 255) / 256;
    k_schur_red<<<st.v_n, kRedThreads, 0, s>>>(vargs(c, 3), c.d_Cv, y0, y1, red_out);
    k_schur_lin<<<nb, 256, 0, s>>>(c.nV, red_out, y0, y1, c.d_vprob, g);
    k_schur_red<<<st.v_n, kRedThreads, 0, s>>>(vargs(c, 3), c.d_Cv, nullptr, g, red_out);
    k_schur_shift<<<nb, 256, 0, s>>>(c.nV, red_out, nullptr, 0.0, c.d_vprob, g);
    c.launches += 4;
    return cudaGetLastError();
}

// Barycenter multiplier of Eq. 22: translations are in null(A-bar) and null(C_len), null(C_edges), so
// N^T (A-bar g + C^T lambda) = N^T dE leaves (C_bary N)^T lambda_bary = N^T dE per problem.  rhs =
// dE - C_bary^T lambda_bary is then consistent on the mean-free subspace.  lambda_bary = 0 when dE is
// translation invariant (the tangent-point differential); penalties with a non-constant field are not.
__global__ void k_bary_red(RedArgs ra, const double *__restrict__ C, const double *__restrict__ dE,
                           double *__restrict__ out)
{
    double s[12] = {0};
    int lo = ra.chunk_lo[blockIdx.x], hi = ra.chunk_lo[blockIdx.x + 1];
    for (int v = lo + threadIdx.x; v < hi; v += blockDim.x) {
        const double *cv = C + (size_t)v * 12;
        for (int j = 0; j < 3; ++j) {
            s[j] += dE[3 * (size_t)v + j];
            for (int k = 0; k < 3; ++k) s[3 + 3 * k + j] += cv[3 * k + j];
        }
    }
    if (reduce_phase<12>(s, ra))
        for (int q = threadIdx.x; q < ra.nprob; q += blockDim.x)
            for (int k = 0; k < 12; ++k) out[12 * q + k] = ra.sums[12 * q + k];
}

__global__ void k_bary_rhs(int nV, const double *__restrict__ red, const double *__restrict__ C,
                           const double *__restrict__ dE, const int *__restrict__ vprob, double *__restrict__ rhs)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nV) return;
    const double *r = red + 12 * vprob[v];
    double Mt[9], lam[3];
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) Mt[3 * j + k] = r[3 + 3 * k + j];  // (C_bary N)^T
    solve3(Mt, r, lam);
    const double *cv = C + (size_t)v * 12;
    for (int j = 0; j < 3; ++j)
        rhs[3 * (size_t)v + j] = dE[3 * (size_t)v + j] - (lam[0] * cv[j] + lam[1] * cv[3 + j] + lam[2] * cv[6 + j]);
}

cudaError_t bary_rhs(Ctx &c, const double *dE, double *rhs, cudaStream_t s)
{
    SolverState &st = S(c);
    k_bary_red<<<st.v_n, kRedThreads, 0, s>>>(vargs(c, 3), c.d_Cv, dE, c.d_red);
    k_bary_rhs<<<(c.nV + 255) / 256, 256, 0, s>>>(c.nV, c.d_red, c.d_Cv, dE, c.d_vprob, rhs);
    c.launches += 2;
    return cudaGetLastError();
}

// out += N t with C_bary (out + N t) = phi_scale * phi_bary (phi null: 0); the barycenter step of the
// edge-length route, where the edge rows are already satisfied by out.
cudaError_t schur_shift(Ctx &c, double *out, const double *phi, double phi_scale, cudaStream_t s)
{
    SolverState &st = S(c);
    const int nb = (c.nV + 255) / 256;
    k_schur_red<<<st.v_n, kRedThreads, 0, s>>>(vargs(c, 3), c.d_Cv, nullptr, out, c.d_red);
    k_schur_shift<<<nb, 256, 0, s>>>(c.nV, c.d_red, phi, phi_scale, c.d_vprob, out);
    c.launches += 2;
    return cudaGetLastError();
}

// x = mu y1 + N t solving C x = phi_scale * phi with y1 = A^+ C_len^T (Jacobian in c.d_Cv).
cudaError_t schur_projection(Ctx &c, const double *y1, const double *phi, double phi_scale, double *x,
                             cudaStream_t s)
{
    SolverState &st = S(c);
    double *red_out = c.d_red;
    const int nb = (c.nV + 255) / 256;
    k_schur_red<<<st.v_n, kRedThreads, 0, s>>>(vargs(c, 3), c.d_Cv, nullptr, y1, red_out);
    k_proj_lin<<<nb, 256, 0, s>>>(c.nV, red_out, phi, phi_scale, y1, c.d_vprob, x);
    k_schur_red<<<st.v_n, kRedThreads, 0, s>>>(vargs(c, 3), c.d_Cv, nullptr, x, red_out);
    k_schur_shift<<<nb, 256, 0, s>>>(c.nV, red_out, phi, phi_scale, c.d_vprob, x);
    c.launches += 4;
    return cudaGetLastError();
}

// Reductions per problem for the pinned-point route (pins.cu): out[5q] = <C_len, a> (0 if a is NULL),
// out[5q + 1] = <C_len, b>, out[5q + 2..4] = sum over the problem's vertices of dE (0 if dE is NULL).
__global__ void k_pin_red(RedArgs ra, const double *__restrict__ C, const double *__restrict__ a,
                          const double *__restrict__ b, const double *__restrict__ dE, double *__restrict__ out)
{
    double s[5] = {0, 0, 0, 0, 0};
    int lo = ra.chunk_lo[blockIdx.x], hi = ra.chunk_lo[blockIdx.x + 1];
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double *cv = C + (size_t)i * 12 + 9;
        for (int j = 0; j < 3; ++j) {
            if (a) s[0] += cv[j] * a[3 * (size_t)i + j];
            s[1] += cv[j] * b[3 * (size_t)i + j];
            if (dE) s[2 + j] += dE[3 * (size_t)i + j];
        }
    }
    if (reduce_phase<5>(s, ra))
        for (int q = threadIdx.x; q < ra.nprob; q += blockDim.x)
            for (int k = 0; k < 5; ++k) out[5 * q + k] = ra.sums[5 * q + k];
}

cudaError_t pin_reduce(Ctx &c, const double *a, const double *b, const double *dE, double *out, cudaStream_t s)
{
    SolverState &st = S(c);
    k_pin_red<<<st.v_n, kRedThreads, 0, s>>>(vargs(c, 3), c.d_Cv, a, b, dE, out);
    c.launches++;
    return cudaGetLastError();
}

}  // namespace tpe
