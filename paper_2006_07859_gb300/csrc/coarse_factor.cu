// Tiled FP64 Cholesky factorisation and explicit inverse of a coarse matrix E = Z^T A Z with more than
// 127 rows (smaller ones are factored by one CTA in shared memory, coarse.cu).
//
// E is symmetric positive definite, row-major mm x mm.  With 32 x 32 tiles:
//   1. W = (E + E^T) / 2;
//   2. right-looking Cholesky W = L L^T: per tile column k, the diagonal tile (one CTA), the panel
//      below it (one CTA per tile row: X L_kk^T = W_ik) and the rank-32 update of the trailing lower
//      tiles (one CTA per tile);
//   3. Y = L^-1 one tile row at a time: L_ii Y_ij = -sum_{k=j}^{i-1} L_ik Y_kj for j < i and
//      L_ii Y_ii = I (one CTA per tile of the row);
//   4. E^-1 = Y^T Y: tile (a, b) = sum_{k >= max(a, b)} Y_ka^T Y_kb (one CTA per lower tile, written to
//      both triangles).
// Every step costs O(mm^3 / 6) FMAs spread over (mm / 32)^2 / 2 CTAs.  The one-CTA kernel takes
// about mm^3 / 3 sequential steps of global-memory latency, which is 0.55 s at 1023 rows.
// Zero or negative pivots (E singular in floating point) are replaced by 1e-150, as in the one-CTA
// kernel, so a degenerate coarse space yields huge but finite entries instead of NaN.
#include <cuda_runtime.h>

#include "coarse.cuh"

namespace tpe {

#define TPE_CHECK(x)                      \
    do {                                  \
        cudaError_t e_ = (x);             \
        if (e_ != cudaSuccess) return e_; \
    } while (0)

constexpr int kFB = 32;  // tile edge

// element (r, c) of tile (ti, tj) of a row-major mm x mm matrix, or `pad` outside it
__device__ __forceinline__ double tile_ld(const double *A, int mm, int ti, int tj, int r, int c, double pad)
{
    const int R = ti * kFB + r, C = tj * kFB + c;
    return (R < mm && C < mm) ? A[(long long)R * mm + C] : pad;
}

__device__ __forceinline__ void tile_st(double *A, int mm, int ti, int tj, int r, int c, double v)
{
    const int R = ti * kFB + r, C = tj * kFB + c;
    if (R < mm && C < mm) A[(long long)R * mm + C] = v;
}

// lower tile number idx -> (ti, tj), tj <= ti
__device__ __forceinline__ void lower_tile(long long idx, int &ti, int &tj)
{
    int t = (int)((sqrt(8.0 * (double)idx + 1.0) - 1.0) * 0.5);
    while ((long long)(t + 1) * (t + 2) / 2 <= idx) ++t;
    while ((long long)t * (t + 1) / 2 > idx) --t;
    ti = t;
    tj = (int)(idx - (long long)t * (t + 1) / 2);
}

__global__ void k_fac_sym(int mm, const double *__restrict__ E, double *__restrict__ W)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)mm * mm) return;
    const int r = (int)(t / mm), c = (int)(t % mm);
    W[t] = 0.5 * (E[t] + E[(long long)c * mm + r]);
}

// Cholesky of the diagonal tile (k, k) in place; rows / columns past mm are padded with the identity
__global__ void __launch_bounds__(256) k_fac_diag(int mm, int k, double *__restrict__ W)
{
    __shared__ double t[kFB][kFB + 1];
    for (int e = threadIdx.x; e < kFB * kFB; e += blockDim.x) {
        const int r = e / kFB, c = e % kFB;
        t[r][c] = tile_ld(W, mm, k, k, r, c, r == c ? 1.0 : 0.0);
    }
    __syncthreads();
    for (int c = 0; c < kFB; ++c) {
        if (threadIdx.x == 0) {
            const double d = t[c][c];
            t[c][c] = d > 0.0 ? sqrt(d) : 1e-150;
        }
        __syncthreads();
        const double dc = t[c][c];
        for (int r = c + 1 + threadIdx.x; r < kFB; r += blockDim.x) t[r][c] /= dc;
        __syncthreads();
        const int w = kFB - 1 - c;
        for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
            const int r = c + 1 + e / w, q = c + 1 + e % w;
            if (q <= r) t[r][q] -= t[r][c] * t[q][c];
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < kFB * kFB; e += blockDim.x) {
        const int r = e / kFB, c = e % kFB;
        if (c <= r) tile_st(W, mm, k, k, r, c, t[r][c]);
    }
}

// panel tile (i, k), i = k + 1 + blockIdx.x: solve X L_kk^T = W_ik in place (one thread per row)
__global__ void __launch_bounds__(kFB) k_fac_panel(int mm, int k, double *__restrict__ W)
{
    const int i = k + 1 + blockIdx.x;
    __shared__ double L[kFB][kFB + 1], X[kFB][kFB + 1];
    const int r = threadIdx.x;
    for (int c = 0; c < kFB; ++c) {
        L[r][c] = tile_ld(W, mm, k, k, r, c, r == c ? 1.0 : 0.0);
        X[r][c] = tile_ld(W, mm, i, k, r, c, 0.0);
    }
    __syncthreads();
    for (int c = 0; c < kFB; ++c) {
        double v = X[r][c];
        for (int q = 0; q < c; ++q) v -= X[r][q] * L[c][q];
        X[r][c] = v / L[c][c];
    }
    for (int c = 0; c < kFB; ++c) tile_st(W, mm, i, k, r, c, X[r][c]);
}

// out(r, c) of a 32 x 32 tile product, 4 outputs per thread (256 threads): rows r = tid / 8,
// columns c = (tid % 8) + 8 q
#define FAC_OUT_LOOP for (int q = 0; q < 4; ++q)

// trailing update: W_ij -= W_ik W_jk^T for the lower tiles k < j <= i
__global__ void __launch_bounds__(256) k_fac_update(int mm, int k, double *__restrict__ W)
{
    int ti, tj;
    lower_tile(blockIdx.x, ti, tj);
    const int i = k + 1 + ti, j = k + 1 + tj;
    __shared__ double P[kFB][kFB + 1], Q[kFB][kFB + 1];
    for (int e = threadIdx.x; e < kFB * kFB; e += blockDim.x) {
        const int r = e / kFB, c = e % kFB;
        P[r][c] = tile_ld(W, mm, i, k, r, c, 0.0);
        Q[r][c] = tile_ld(W, mm, j, k, r, c, 0.0);
    }
    __syncthreads();
    const int r = threadIdx.x >> 3, c0 = threadIdx.x & 7;
    double acc[4] = {0, 0, 0, 0};
    for (int p = 0; p < kFB; ++p) {
        const double a = P[r][p];
        FAC_OUT_LOOP acc[q] += a * Q[c0 + 8 * q][p];
    }
    FAC_OUT_LOOP
    {
        const int R = i * kFB + r, C = j * kFB + c0 + 8 * q;
        if (R < mm && C < mm) W[(long long)R * mm + C] -= acc[q];
    }
}

// tile (i, j), j = blockIdx.x <= i, of Y = L^-1 (rows above i already done)
__global__ void __launch_bounds__(256) k_fac_inv_row(int mm, int i, const double *__restrict__ Lf,
                                                     double *__restrict__ Y)
{
    const int j = blockIdx.x;
    __shared__ double Lii[kFB][kFB + 1], S[kFB][kFB + 1], P[kFB][kFB + 1], Q[kFB][kFB + 1];
    for (int e = threadIdx.x; e < kFB * kFB; e += blockDim.x) {
        const int r = e / kFB, c = e % kFB;
        Lii[r][c] = tile_ld(Lf, mm, i, i, r, c, r == c ? 1.0 : 0.0);
    }
    // S = -sum_{k=j}^{i-1} L_ik Y_kj  (identity when j == i)
    const int r = threadIdx.x >> 3, c0 = threadIdx.x & 7;
    double acc[4] = {0, 0, 0, 0};
    for (int k = j; k < i; ++k) {
        __syncthreads();
        for (int e = threadIdx.x; e < kFB * kFB; e += blockDim.x) {
            const int rr = e / kFB, cc = e % kFB;
            P[rr][cc] = tile_ld(Lf, mm, i, k, rr, cc, 0.0);
            Q[rr][cc] = tile_ld(Y, mm, k, j, rr, cc, 0.0);
        }
        __syncthreads();
        for (int p = 0; p < kFB; ++p) {
            const double a = P[r][p];
            FAC_OUT_LOOP acc[q] += a * Q[p][c0 + 8 * q];
        }
    }
    FAC_OUT_LOOP S[r][c0 + 8 * q] = (j == i) ? ((r == c0 + 8 * q) ? 1.0 : 0.0) : -acc[q];
    __syncthreads();
    // L_ii Y_ij = S by forward substitution, one thread per column
    if (threadIdx.x < kFB) {
        const int c = threadIdx.x;
        for (int rr = 0; rr < kFB; ++rr) {
            double v = S[rr][c];
            for (int q = 0; q < rr; ++q) v -= Lii[rr][q] * S[q][c];
            S[rr][c] = v / Lii[rr][rr];
        }
        for (int rr = 0; rr < kFB; ++rr) tile_st(Y, mm, i, j, rr, c, S[rr][c]);
    }
}

// E^-1 = Y^T Y: lower tile (a, b) and its mirror
__global__ void __launch_bounds__(256) k_fac_gram(int mm, int nb, const double *__restrict__ Y,
                                                  double *__restrict__ Ainv)
{
    int a, b;
    lower_tile(blockIdx.x, a, b);
    __shared__ double P[kFB][kFB + 1], Q[kFB][kFB + 1];
    const int r = threadIdx.x >> 3, c0 = threadIdx.x & 7;
    double acc[4] = {0, 0, 0, 0};
    for (int k = a; k < nb; ++k) {
        __syncthreads();
        for (int e = threadIdx.x; e < kFB * kFB; e += blockDim.x) {
            const int rr = e / kFB, cc = e % kFB;
            P[rr][cc] = tile_ld(Y, mm, k, a, rr, cc, 0.0);
            Q[rr][cc] = tile_ld(Y, mm, k, b, rr, cc, 0.0);
        }
        __syncthreads();
        for (int p = 0; p < kFB; ++p) {
            const double x = P[p][r];
            FAC_OUT_LOOP acc[q] += x * Q[p][c0 + 8 * q];
        }
    }
    FAC_OUT_LOOP
    {
        const int R = a * kFB + r, C = b * kFB + c0 + 8 * q;
        if (R < mm && C < mm) {
            Ainv[(long long)R * mm + C] = acc[q];
            Ainv[(long long)C * mm + R] = acc[q];
        }
    }
}

// E (row-major mm x mm at E) -> E^-1 in place; W and Y are scratch of the same size
cudaError_t coarse_factor_tiled(Ctx &c, int mm, double *E, double *W, double *Y, cudaStream_t s)
{
    const int nb = (mm + kFB - 1) / kFB;
    const long long n2 = (long long)mm * mm;
    k_fac_sym<<<(unsigned)((n2 + 255) / 256), 256, 0, s>>>(mm, E, W);
    c.launches++;
    for (int k = 0; k < nb; ++k) {
        k_fac_diag<<<1, 256, 0, s>>>(mm, k, W);
        c.launches++;
        const int T = nb - k - 1;
        if (T == 0) break;
        k_fac_panel<<<T, kFB, 0, s>>>(mm, k, W);
        k_fac_update<<<(unsigned)((long long)T * (T + 1) / 2), 256, 0, s>>>(mm, k, W);
        c.launches += 2;
    }
    TPE_CHECK(cudaMemsetAsync(Y, 0, sizeof(double) * n2, s));
    for (int i = 0; i < nb; ++i) {
        k_fac_inv_row<<<i + 1, 256, 0, s>>>(mm, i, W, Y);
        c.launches++;
    }
    k_fac_gram<<<(unsigned)((long long)nb * (nb + 1) / 2), 256, 0, s>>>(mm, nb, Y, E);
    c.launches++;
    return cudaGetLastError();
}

}  // namespace tpe
