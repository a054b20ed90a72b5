// Coarse-space correction of the spectral preconditioner (TP_PRECOND_TWOLEVEL; not from the paper).
//
// The Rayleigh-quotient corrected circulant fixes the spectrum of A mode by mode, but A is not
// circulant: its slowest modes on a knotted curve are global low-frequency deformations whose
// stiffness depends on where the curve comes close to itself.  An additive two-level term fixes them:
//
//   M^-1 = M_spectral^-1 + Z (Z^T A Z)^-1 Z^T,
//
// Z = the m - 1 first of m periodic hat functions per closed curve (centres i = j n / m, support of
// two hat widths; the m hats sum to 1, so the dropped one is implied on the mean-free subspace).
// Z^T A Z comes from the columns A Z, which one dedicated pair pass assembles (coarse_az.cu); coarse
// spaces below 8 hats are probed instead, with (m - 1) / 3 applies of the pair kernel (three hats per
// apply, one per component).  It is Cholesky-factored per curve in FP64 and inverted explicitly
// (L^-T L^-1) at set-up.
// Per CG iteration the term costs three small kernels: restriction Z^T r, the (m - 1) x (m - 1)
// mat-vec with the inverse (all rows and components in parallel), prolongation Z y.
//
// Balancing form (TP_PRECOND_TWOLEVEL_BALANCED, when every problem is one closed curve): with
// Q = Z E^-1 Z^T, E = Z^T A Z and S the spectral term,
//   M^-1 r = Q r + (I - Q A) S (I - A Q) r,
// the symmetric multiplicative combination: it is exact on range(A Z) and leaves S only the complement.
// The columns A Z of the set-up are kept (n (m - 1) doubles per curve) so that A Q r = (A Z) E^-1 Z^T r
// and Q A y = Z E^-1 (A Z)^T y cost two dense passes over them and no pair pass.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "coarse.cuh"

namespace tpe {

#define TPE_CHECK(x)                      \
    do {                                  \
        cudaError_t e_ = (x);             \
        if (e_ != cudaSuccess) return e_; \
    } while (0)

__global__ void k_coarse_probe(int nV, int b, const CoarseCurve *__restrict__ cc, const int *__restrict__ vcurve,
                               double *__restrict__ y)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nV) return;
    const CoarseCurve C = cc[vcurve[v]];
    int i = v - C.v0;
    for (int q = 0; q < 3; ++q) {
        int l = 3 * b + q;
        y[3 * v + q] = (l < C.m - 1) ? hat(i, l, C.n, C.m) : 0.0;
    }
}

// Ac[j][3b + q] = Z_j^T (A Z_{3b+q}): one block per (curve, j)
__global__ void k_coarse_gram(int b, const CoarseCurve *__restrict__ cc, const double *__restrict__ AZ,
                              double *__restrict__ L)
{
    const CoarseCurve C = cc[blockIdx.x];
    const int j = blockIdx.y;
    const int mm = C.m - 1;
    if (j >= mm) return;
    int lo, len;
    hat_support(j, C.n, C.m, lo, len);
    __shared__ double sh[3][128];
    double s[3] = {0, 0, 0};
    for (int k = threadIdx.x; k < len; k += blockDim.x) {
        int i = ((lo + k) % C.n + C.n) % C.n;
        double z = hat(i, j, C.n, C.m);
        for (int q = 0; q < 3; ++q) s[q] += z * AZ[3 * (C.v0 + i) + q];
    }
    for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] = s[q];
    __syncthreads();
    for (int w = 64; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 3; ++q) {
            int l = 3 * b + q;
            if (l < mm) L[C.aoff + (long long)j * mm + l] = sh[q][0];
        }
}

// symmetrise, Cholesky-factor and invert in place every curve's coarse matrix of at most 127 rows, in
// shared memory (one block per curve; larger ones go to the tiled kernels of coarse_factor.cu);
// Li: scratch of the same layout for L^-1
__global__ void k_coarse_factor(const CoarseCurve *__restrict__ cc, double *__restrict__ L, double *__restrict__ Li)
{
    const CoarseCurve C = cc[blockIdx.x];
    const int mm = C.m - 1;
    if (mm > kSmemCoarse - 1) return;
    extern __shared__ double a[];  // [mm][mm] (dynamic shared memory)
    double *g = L + C.aoff;
    for (int t = threadIdx.x; t < mm * mm; t += blockDim.x) {
        int r = t / mm, col = t % mm;
        a[r * mm + col] = 0.5 * (g[r * mm + col] + g[col * mm + r]);
    }
    __syncthreads();
    for (int k = 0; k < mm; ++k) {
        if (threadIdx.x == 0) {
            double d = a[k * mm + k];
            a[k * mm + k] = d > 0.0 ? sqrt(d) : 1e-150;
        }
        __syncthreads();
        double dk = a[k * mm + k];
        for (int r = k + 1 + threadIdx.x; r < mm; r += blockDim.x) a[r * mm + k] /= dk;
        __syncthreads();
        for (int t = threadIdx.x; t < (mm - k - 1) * (mm - k - 1); t += blockDim.x) {
            int r = k + 1 + t / (mm - k - 1), col = k + 1 + t % (mm - k - 1);
            if (col <= r) a[r * mm + col] -= a[r * mm + k] * a[col * mm + k];
        }
        __syncthreads();
    }
    // L^-1 by forward substitution, one column per thread, then (Z^T A Z)^-1 = L^-T L^-1
    double *li = Li + C.aoff;
    for (int col = threadIdx.x; col < mm; col += blockDim.x) {
        for (int r = 0; r < mm; ++r) {
            double v = (r == col) ? 1.0 : 0.0;
            for (int k = col; k < r; ++k) v -= a[r * mm + k] * li[k * mm + col];
            li[r * mm + col] = r < col ? 0.0 : v / a[r * mm + r];
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < mm * mm; t += blockDim.x) {
        const int r = t / mm, col = t % mm;
        double v = 0.0;
        for (int k = max(r, col); k < mm; ++k) v += li[k * mm + r] * li[k * mm + col];
        g[t] = v;
    }
}

// w[j][q] = Z_j^T r: one block per (curve, j)
__global__ void k_coarse_restrict(const CoarseCurve *__restrict__ cc, const double *__restrict__ r,
                                  double *__restrict__ w)
{
    const CoarseCurve C = cc[blockIdx.x];
    const int j = blockIdx.y;
    if (j >= C.m - 1) return;
    int lo, len;
    hat_support(j, C.n, C.m, lo, len);
    __shared__ double sh[3][128];
    double s[3] = {0, 0, 0};
    for (int k = threadIdx.x; k < len; k += blockDim.x) {
        int i = ((lo + k) % C.n + C.n) % C.n;
        double z = hat(i, j, C.n, C.m);
        for (int q = 0; q < 3; ++q) s[q] += z * r[3 * (C.v0 + i) + q];
    }
    for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] = s[q];
    __syncthreads();
    for (int wv = 64; wv > 0; wv >>= 1) {
        if (threadIdx.x < wv)
            for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + wv];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 3; ++q) w[C.woff + 3 * j + q] = sh[q][0];
}

// y = (Z^T A Z)^-1 w per curve: one warp per row (8 rows per block, blockIdx.y the curve).  The lanes
// split the row's entries (contiguous, so the loads coalesce) and a warp-shuffle sum finishes each of
// the three components.  w and y are separate buffers: several blocks serve one curve.
constexpr int kSolveRows = 8;
__global__ void __launch_bounds__(32 * kSolveRows) k_coarse_solve(const CoarseCurve *__restrict__ cc,
                                                                  const double *__restrict__ Ainv,
                                                                  const double *__restrict__ w,
                                                                  double *__restrict__ y)
{
    const CoarseCurve C = cc[blockIdx.y];
    const int mm = C.m - 1;
    const int r0 = blockIdx.x * kSolveRows;
    if (r0 >= mm) return;  // uniform per block
    extern __shared__ double sw[];  // [3 (max_m - 1)] the curve's coarse vector
    for (int t = threadIdx.x; t < 3 * mm; t += blockDim.x) sw[t] = w[C.woff + t];
    __syncthreads();
    const int r = r0 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (r >= mm) return;  // whole warps leave; no barrier follows
    const double *a = Ainv + C.aoff + (size_t)r * mm;
    double s[3] = {0.0, 0.0, 0.0};
    for (int k = lane; k < mm; k += 32) {
        const double v = a[k];
        s[0] += v * sw[3 * k];
        s[1] += v * sw[3 * k + 1];
        s[2] += v * sw[3 * k + 2];
    }
    for (int o = 16; o > 0; o >>= 1)
        for (int q = 0; q < 3; ++q) s[q] += __shfl_xor_sync(0xffffffffu, s[q], o);
    if (lane == 0)
        for (int q = 0; q < 3; ++q) y[C.woff + 3 * r + q] = s[q];
}

// z[v] += sum_j Z_j(i) y_j (each vertex lies in at most two hats)
__global__ void k_coarse_prolong(int nV, const CoarseCurve *__restrict__ cc, const int *__restrict__ vcurve,
                                 const double *__restrict__ w, double *__restrict__ z)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nV) return;
    const CoarseCurve C = cc[vcurve[v]];
    int i = v - C.v0;
    double t = (double)i * C.m / C.n;
    int j0 = (int)floor(t);
    double acc[3] = {0, 0, 0};
    for (int dj = 0; dj <= 1; ++dj) {
        int j = (j0 + dj) % C.m;
        if (j >= C.m - 1) continue;
        double h = hat(i, j, C.n, C.m);
        for (int q = 0; q < 3; ++q) acc[q] += h * w[C.woff + 3 * j + q];
    }
    for (int q = 0; q < 3; ++q) z[3 * v + q] += acc[q];
}

// AZ[curve][3b + q][i] = (A z_{3b+q})(v0 + i): the probe of batch b carries hat 3b + q in component q
__global__ void k_az_store(int nV, int b, const CoarseCurve *__restrict__ cc, const int *__restrict__ vcurve,
                           const double *__restrict__ AY, double *__restrict__ AZ)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nV) return;
    const CoarseCurve C = cc[vcurve[v]];
    const int i = v - C.v0;
    for (int q = 0; q < 3; ++q) {
        const int l = 3 * b + q;
        if (l < C.m - 1) AZ[C.zoff + (long long)l * C.n + i] = AY[3 * v + q];
    }
}

// out[v] = r[v] - sum_j AZ[j][v] w[j] (three components; each vertex reads its curve's column entries,
// consecutive vertices read consecutive addresses of a column).  The coefficients w of a chunk of
// columns are staged in shared memory, and the column loop is unrolled so that every thread keeps
// several independent loads in flight (the pass streams n (m - 1) doubles from memory).
constexpr int kAzChunk = 512;
__global__ void __launch_bounds__(256) k_az_prolong_sub(int nV, const CoarseCurve *__restrict__ cc,
                                                        const int *__restrict__ vcurve, const double *__restrict__ AZ,
                                                        const double *__restrict__ w, const double *__restrict__ r,
                                                        double *__restrict__ out, int max_mm)
{
    __shared__ double sw[3 * kAzChunk];
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    const int vc = min(v, nV - 1);
    const CoarseCurve C = cc[vcurve[vc]];
    const int i = vc - C.v0, mm = C.m - 1;
    const double *az = AZ + C.zoff + i;
    // the block's vertices may span curves: each stages its own curve's coefficients chunk by chunk
    const CoarseCurve C0 = cc[vcurve[min((int)(blockIdx.x * blockDim.x), nV - 1)]];
    const bool uniform = C0.woff == C.woff;
    const double *wc = w + C.woff;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int j0 = 0; j0 < max_mm; j0 += kAzChunk) {
        const int cnt = min(kAzChunk, max(0, (C0.m - 1) - j0));
        __syncthreads();
        for (int t = threadIdx.x; t < 3 * cnt; t += blockDim.x) sw[t] = w[C0.woff + 3 * (long long)j0 + t];
        __syncthreads();
        const int hi = min(mm, j0 + kAzChunk);
        if (uniform) {
#pragma unroll 8
            for (int j = j0; j < hi; ++j) {
                const double a = az[(long long)j * C.n];
                s0 += a * sw[3 * (j - j0)];
                s1 += a * sw[3 * (j - j0) + 1];
                s2 += a * sw[3 * (j - j0) + 2];
            }
        } else {
            for (int j = j0; j < hi; ++j) {
                const double a = az[(long long)j * C.n];
                s0 += a * wc[3 * j];
                s1 += a * wc[3 * j + 1];
                s2 += a * wc[3 * j + 2];
            }
        }
    }
    if (v >= nV) return;
    out[3 * v] = r[3 * v] - s0;
    out[3 * v + 1] = r[3 * v + 1] - s1;
    out[3 * v + 2] = r[3 * v + 2] - s2;
}

// w[j][q] = sum_i AZ[j][i] y[v0 + i][q]: one block per (curve, kAzCols consecutive columns), so that each
// pass over y serves several columns; fixed-order sums (per thread, then warp shuffles, then warps)
constexpr int kAzCols = 8;
__global__ void __launch_bounds__(256) k_az_restrict(const CoarseCurve *__restrict__ cc, const double *__restrict__ AZ,
                                                     const double *__restrict__ y, double *__restrict__ w)
{
    const CoarseCurve C = cc[blockIdx.x];
    const int j0 = blockIdx.y * kAzCols, mm = C.m - 1;
    if (j0 >= mm) return;  // uniform per block
    const int nc = min(kAzCols, mm - j0);
    const double *az = AZ + C.zoff + (long long)j0 * C.n;
    double s[kAzCols][3];
#pragma unroll
    for (int c = 0; c < kAzCols; ++c) s[c][0] = s[c][1] = s[c][2] = 0.0;
    for (int i = threadIdx.x; i < C.n; i += blockDim.x) {
        const double *yy = y + 3 * (size_t)(C.v0 + i);
        const double y0 = yy[0], y1 = yy[1], y2 = yy[2];
#pragma unroll
        for (int c = 0; c < kAzCols; ++c)
            if (c < nc) {
                const double a = az[(long long)c * C.n + i];
                s[c][0] += a * y0;
                s[c][1] += a * y1;
                s[c][2] += a * y2;
            }
    }
    __shared__ double sh[8][kAzCols * 3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < kAzCols; ++c)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            double x = s[c][q];
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0) sh[warp][3 * c + q] = x;
        }
    __syncthreads();
    if (threadIdx.x < 3 * nc) {
        double x = 0.0;
        for (int k = 0; k < 8; ++k) x += sh[k][threadIdx.x];
        w[C.woff + 3 * (long long)j0 + threadIdx.x] = x;
    }
}

__global__ void k_coarse_sub(long long n, const double *__restrict__ a, double *__restrict__ b)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i] - b[i];
}

// The balancing form's extra storage (the A Z columns and two coarse vectors), allocated when that
// preconditioner is selected on a context whose problems are single curves.
static cudaError_t coarse_balanced_alloc(Ctx &c)
{
    CoarseState &S = *c.coarse;
    S.balanced = (c.prm.precond == TP_PRECOND_TWOLEVEL_BALANCED || c.prm.precond == TP_PRECOND_LEARNED_BALANCED) &&
                 c.nCurves == c.nProb;
    if (!S.balanced || S.d_w3) return cudaSuccess;
    const CoarseCurve &L = S.curves.back();
    const long long woff = L.woff + 3LL * (L.m - 1), zoff = L.zoff + (long long)(L.m - 1) * L.n;
    TPE_CHECK(cudaMalloc(&S.d_w3, sizeof(double) * std::max<long long>(1, woff)));
    TPE_CHECK(cudaMalloc(&S.d_w4, sizeof(double) * std::max<long long>(1, woff)));
    if (!S.d_AZ) TPE_CHECK(cudaMalloc(&S.d_AZ, sizeof(double) * std::max<long long>(1, zoff)));
    TPE_CHECK(cudaMalloc(&S.d_r2, sizeof(double) * 3 * (size_t)c.nV));
    S.ready = 0;  // the next set-up fills the A Z columns
    return cudaSuccess;
}

// The A Z pass's per-edge hat records, its work items (blocks of 128 target rows, biggest curves
// first) and the A Z columns it writes.
static cudaError_t coarse_pass_alloc(Ctx &c)
{
    CoarseState &S = *c.coarse;
    const CoarseCurve &L = S.curves.back();
    const long long zoff = L.zoff + (long long)(L.m - 1) * L.n;
    TPE_CHECK(cudaMalloc(&S.d_AZ, sizeof(double) * std::max<long long>(1, zoff)));
    TPE_CHECK(cudaMalloc(&S.d_hbase, sizeof(int) * std::max(1, c.nE)));
    if (c.prm.precision == TP_FP64)
        TPE_CHECK(cudaMalloc(&S.d_hatD, sizeof(URecD) * std::max(1, c.nE)));
    else
        TPE_CHECK(cudaMalloc(&S.d_hatF, sizeof(URecF) * std::max(1, c.nE)));
    std::vector<int> order(S.curves.size());
    for (size_t k = 0; k < order.size(); ++k) order[k] = (int)k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return S.curves[a].n > S.curves[b].n; });
    std::vector<int2> items;
    for (int k : order)
        for (int r = 0; r < S.curves[k].n; r += kThreads) items.push_back(make_int2(k, r));
    S.n_items = (int)items.size();
    TPE_CHECK(cudaMalloc(&S.d_items, sizeof(int2) * std::max<size_t>(1, items.size())));
    TPE_CHECK(cudaMemcpy(S.d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice));
    return cudaSuccess;
}

cudaError_t coarse_init(Ctx &c)
{
    if (c.coarse) return coarse_balanced_alloc(c);
    c.coarse = new CoarseState();
    CoarseState &S = *c.coarse;
    long long aoff = 0, woff = 0, zoff = 0;
    std::vector<int> vc(c.nV);
    for (int k = 0; k < c.nCurves; ++k) {
        CoarseCurve C{};
        C.v0 = c.h_voff[k];
        C.n = c.h_voff[k + 1] - C.v0;
        C.m = std::max(2, std::min(std::min(c.prm.coarse_dim, kMaxCoarse), C.n / 4));
        C.e0 = c.h_eoff[k];
        C.aoff = aoff;
        C.woff = woff;
        C.zoff = zoff;
        aoff += (long long)(C.m - 1) * (C.m - 1);
        woff += 3LL * (C.m - 1);
        zoff += (long long)(C.m - 1) * C.n;
        S.max_m = std::max(S.max_m, C.m);
        S.curves.push_back(C);
        for (int v = C.v0; v < C.v0 + C.n; ++v) vc[v] = k;
    }
    TPE_CHECK(cudaMalloc(&S.d_curves, sizeof(CoarseCurve) * S.curves.size()));
    TPE_CHECK(cudaMemcpy(S.d_curves, S.curves.data(), sizeof(CoarseCurve) * S.curves.size(), cudaMemcpyHostToDevice));
    TPE_CHECK(cudaMalloc(&S.d_vcurve, sizeof(int) * c.nV));
    TPE_CHECK(cudaMemcpy(S.d_vcurve, vc.data(), sizeof(int) * c.nV, cudaMemcpyHostToDevice));
    TPE_CHECK(cudaMalloc(&S.d_L, sizeof(double) * std::max<long long>(1, aoff)));
    TPE_CHECK(cudaMalloc(&S.d_Li, sizeof(double) * std::max<long long>(1, aoff)));
    TPE_CHECK(cudaMalloc(&S.d_W, sizeof(double) * std::max<long long>(1, aoff)));
    TPE_CHECK(cudaMalloc(&S.d_w, sizeof(double) * std::max<long long>(1, woff)));
    TPE_CHECK(cudaMalloc(&S.d_w2, sizeof(double) * std::max<long long>(1, woff)));
    // the A Z pass needs hats of a few edges each on chain-ordered closed curves (which the spectral
    // preconditioner under every two-level one already requires); small coarse spaces are probed
    S.az_pass = c.spectral_ok && !S.curves.empty();
    for (const CoarseCurve &C : S.curves) S.az_pass = S.az_pass && C.m >= kMinPassCoarse;
    if (S.az_pass) TPE_CHECK(coarse_pass_alloc(c));
    // balancing form: each problem must be one curve, so that E = Z^T A Z is the exact Galerkin matrix
    TPE_CHECK(coarse_balanced_alloc(c));
    TPE_CHECK(cudaFuncSetAttribute(k_coarse_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, kFactorSmem));
    TPE_CHECK(cudaFuncSetAttribute(k_coarse_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(sizeof(double) * 3 * (kMaxCoarse - 1))));
    return cudaSuccess;
}

void coarse_free(Ctx &c)
{
    if (!c.coarse) return;
    cudaFree(c.coarse->d_curves);
    cudaFree(c.coarse->d_vcurve);
    cudaFree(c.coarse->d_L);
    cudaFree(c.coarse->d_Li);
    cudaFree(c.coarse->d_W);
    cudaFree(c.coarse->d_w);
    cudaFree(c.coarse->d_w2);
    cudaFree(c.coarse->d_w3);
    cudaFree(c.coarse->d_w4);
    cudaFree(c.coarse->d_AZ);
    cudaFree(c.coarse->d_r2);
    cudaFree(c.coarse->d_items);
    cudaFree(c.coarse->d_hbase);
    cudaFree(c.coarse->d_hatF);
    cudaFree(c.coarse->d_hatD);
    delete c.coarse;
    c.coarse = nullptr;
}

// Z^T A Z of the curve `gamma_geom` (geometry slot `which`) and its factors; uses c.d_y, c.d_q.
cudaError_t coarse_setup(Ctx &c, const double *gamma_geom, int which, cudaStream_t s)
{
    TPE_CHECK(coarse_init(c));
    CoarseState &S = *c.coarse;
    const int nb = (c.nV + 255) / 256;
    const int nbatch = S.az_pass ? 0 : (S.max_m - 1 + 2) / 3;
    if (S.az_pass) TPE_CHECK(coarse_az_pass(c, which, s));
    for (int b = 0; b < nbatch; ++b) {
        k_coarse_probe<<<nb, 256, 0, s>>>(c.nV, b, S.d_curves, S.d_vcurve, c.d_y);
        c.launches++;
        TPE_CHECK(pair_apply(c, gamma_geom, which, c.d_y, c.d_q, s));
        k_coarse_gram<<<dim3(c.nCurves, S.max_m), 128, 0, s>>>(b, S.d_curves, c.d_q, S.d_L);
        c.launches++;
        if (S.balanced) {
            k_az_store<<<nb, 256, 0, s>>>(c.nV, b, S.d_curves, S.d_vcurve, c.d_q, S.d_AZ);
            c.launches++;
        }
    }
    const int msm = std::min(S.max_m, kSmemCoarse) - 1;
    k_coarse_factor<<<c.nCurves, 256, (size_t)msm * msm * sizeof(double), s>>>(S.d_curves, S.d_L, S.d_Li);
    c.launches++;
    for (const CoarseCurve &C : S.curves)
        if (C.m - 1 > kSmemCoarse - 1)
            TPE_CHECK(coarse_factor_tiled(c, C.m - 1, S.d_L + C.aoff, S.d_W + C.aoff, S.d_Li + C.aoff, s));
    S.ready = 1;
    return cudaGetLastError();
}

// z += Z (Z^T A Z)^-1 Z^T r
cudaError_t coarse_apply(Ctx &c, const double *r, double *z, cudaStream_t s)
{
    if (!c.coarse || !c.coarse->ready) return cudaSuccess;
    CoarseState &S = *c.coarse;
    k_coarse_restrict<<<dim3(c.nCurves, S.max_m), 128, 0, s>>>(S.d_curves, r, S.d_w);
    k_coarse_solve<<<dim3((S.max_m - 1 + kSolveRows - 1) / kSolveRows, c.nCurves), 32 * kSolveRows,
                     sizeof(double) * 3 * (S.max_m - 1), s>>>(S.d_curves, S.d_L, S.d_w, S.d_w2);
    k_coarse_prolong<<<(c.nV + 255) / 256, 256, 0, s>>>(c.nV, S.d_curves, S.d_vcurve, S.d_w2, z);
    c.launches += 3;
    return cudaGetLastError();
}

// z = Q r + (I - Q A) S (I - A Q) r (balancing form).  S = spectral_apply with the skip flags, or with
// `learned` the learned smoother W S W + G of TP_PRECOND_LEARNED_BALANCED (the network's per-vertex
// rescaling of the circulant and its local term).  r must not alias z.
cudaError_t coarse_balanced_apply(Ctx &c, const double *r, double *z, cudaStream_t s, const int *skip, bool learned)
{
    if (!c.coarse || !c.coarse->ready || !c.coarse->balanced) return cudaErrorNotReady;
    CoarseState &S = *c.coarse;
    const dim3 gsolve((S.max_m - 1 + kSolveRows - 1) / kSolveRows, c.nCurves);
    const size_t smem = sizeof(double) * 3 * (S.max_m - 1);
    const int nb = (c.nV + 255) / 256;
    // c1 = E^-1 Z^T r,  r2 = r - (A Z) c1
    k_coarse_restrict<<<dim3(c.nCurves, S.max_m), 128, 0, s>>>(S.d_curves, r, S.d_w);
    k_coarse_solve<<<gsolve, 32 * kSolveRows, smem, s>>>(S.d_curves, S.d_L, S.d_w, S.d_w2);
    k_az_prolong_sub<<<nb, 256, 0, s>>>(c.nV, S.d_curves, S.d_vcurve, S.d_AZ, S.d_w2, r, S.d_r2, S.max_m - 1);
    c.launches += 3;
    // y = S r2 (into z)
    if (learned) {
        TPE_CHECK(spectral_apply_ex(c, S.d_r2, z, s, skip, c.d_diag, spectral_ilam(c, s), gnn_vlog(c)));
        TPE_CHECK(gnn_gapply(c, S.d_r2, z, 1, s, skip));
    } else {
        TPE_CHECK(spectral_apply(c, S.d_r2, z, s, skip));
    }
    // c2 = E^-1 (A Z)^T y;  z = y + Z (c1 - c2)
    k_az_restrict<<<dim3(c.nCurves, (S.max_m - 1 + kAzCols - 1) / kAzCols), 256, 0, s>>>(S.d_curves, S.d_AZ, z, S.d_w3);
    k_coarse_solve<<<gsolve, 32 * kSolveRows, smem, s>>>(S.d_curves, S.d_L, S.d_w3, S.d_w4);
    const long long nw = (long long)S.curves.back().woff + 3LL * (S.curves.back().m - 1);
    k_coarse_sub<<<(unsigned)((nw + 255) / 256), 256, 0, s>>>(nw, S.d_w2, S.d_w4);
    k_coarse_prolong<<<nb, 256, 0, s>>>(c.nV, S.d_curves, S.d_vcurve, S.d_w4, z);
    c.launches += 4;
    return cudaGetLastError();
}

__global__ void k_coarse_neg(long long n, double *__restrict__ a)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = -a[i];
}

// The pieces of the balancing form that training needs, for the A Z columns and E of the last set-up:
//   which 0: out = Q v = Z E^-1 Z^T v;   1: out = (I - A Q) v;   2: out = (I - Q A) v.
// out may alias v for 1 and 2.
cudaError_t coarse_balanced_part(Ctx &c, int which, const double *v, double *out, cudaStream_t s)
{
    if (!c.coarse || !c.coarse->ready || !c.coarse->balanced) return cudaErrorNotReady;
    CoarseState &S = *c.coarse;
    const dim3 gsolve((S.max_m - 1 + kSolveRows - 1) / kSolveRows, c.nCurves);
    const size_t smem = sizeof(double) * 3 * (S.max_m - 1);
    const int nb = (c.nV + 255) / 256;
    const long long nw = (long long)S.curves.back().woff + 3LL * (S.curves.back().m - 1);
    if (which == 2)
        k_az_restrict<<<dim3(c.nCurves, (S.max_m - 1 + kAzCols - 1) / kAzCols), 256, 0, s>>>(S.d_curves, S.d_AZ, v, S.d_w3);
    else
        k_coarse_restrict<<<dim3(c.nCurves, S.max_m), 128, 0, s>>>(S.d_curves, v, S.d_w3);
    k_coarse_solve<<<gsolve, 32 * kSolveRows, smem, s>>>(S.d_curves, S.d_L, S.d_w3, S.d_w4);
    c.launches += 2;
    if (which == 0) {
        TPE_CHECK(cudaMemsetAsync(out, 0, sizeof(double) * 3 * c.nV, s));
        k_coarse_prolong<<<nb, 256, 0, s>>>(c.nV, S.d_curves, S.d_vcurve, S.d_w4, out);
        c.launches++;
    } else if (which == 1) {
        k_az_prolong_sub<<<nb, 256, 0, s>>>(c.nV, S.d_curves, S.d_vcurve, S.d_AZ, S.d_w4, v, out, S.max_m - 1);
        c.launches++;
    } else {
        if (out != v) TPE_CHECK(cudaMemcpyAsync(out, v, sizeof(double) * 3 * c.nV, cudaMemcpyDeviceToDevice, s));
        k_coarse_neg<<<(unsigned)((nw + 255) / 256), 256, 0, s>>>(nw, S.d_w4);
        k_coarse_prolong<<<nb, 256, 0, s>>>(c.nV, S.d_curves, S.d_vcurve, S.d_w4, out);
        c.launches += 2;
    }
    return cudaGetLastError();
}

}  // namespace tpe
