// Learned preconditioner term (TP_PRECOND_LEARNED; this library's extension, not in the paper).
//
// A 3-layer network on the edge graph of the closed curves (width 64, BF16 weights, FP32
// accumulation; the 64-wide layers on the tensor cores) maps local geometry to three values (a_I, b_I, c_I) per edge that shape an SPD
// preconditioner around the two-level one:
//   M^-1 r = W S W r + Z (Z^T A Z)^-1 Z^T r + G r,
//   W = D^-1/2 diag(exp(c_v)), c_v = mean of c over the two edges at vertex v, S the circulant of the
//   Rayleigh-quotient symbol (c = 0: the two-level preconditioner), and the local term
//   r~ = r / sqrt(d),  delta_I = r~_i2 - r~_i1,  sigma_I = r~_i1 + r~_i2,
//   (G r)_i2 += (e^{2a} delta_I + e^{2b} sigma_I) / sqrt(d_i2),
//   (G r)_i1 += (-e^{2a} delta_I + e^{2b} sigma_I) / sqrt(d_i1),
// that is, G = D^-1/2 (D_delta^T E_a D_delta + D_sigma^T E_b D_sigma) D^-1/2 with d = diag(A).
// Features of edge I (I-1, I+1: its neighbours on the curve):
//   [log(l / mean l), 1 - T_{I-1}.T_I, 1 - T_I.T_{I+1}, log(d_i1 / mean d), log(d_i2 / mean d),
//    log(l_{I-1} / l_I), log(l_{I+1} / l_I), 1]
// Layers: h1 = relu(W1 f + b1); h2 = relu(W2s h1 + W2n avg(h1[I-1], h1[I+1]) + b2);
//         h3 = relu(W3s h2 + W3n avg(h2[I-1], h2[I+1]) + b3); (a, b, c) = W4 h3 + b4.
// Training minimises, over (residual, correction) pairs harvested from the CG solves (e = A^+ r), the
// A-norm error of the best multiple of z = M^-1 r + G r (preconditioned CG ignores the scale of M):
//   L = min_a ||a z - e||_A^2 / ||e||_A^2 = 1 - s^2 / (q e^T r),  s = z^T r,  q = z^T A z,
//   dL/dz = -2 s / (q e^T r) (r - (s / q) A z),
// and through the rescaling (S symmetric), with z_S = W S W r and z2 = W S W (dL/dz):
//   dL/dc_v = sum over components of ((dL/dz)_v (z_S)_v + r_v (z2)_v).
// Parameters are FP32 masters with a BF16 copy; the forward and backward passes read the BF16
// values (so the gradient is that of the network actually evaluated), Adam updates the masters.
// The parameter-gradient reductions are deterministic (fixed block partials, fixed-order sums).
#include <cuda_bf16.h>
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

constexpr int kH = TP_GNN_HIDDEN, kF = TP_GNN_FEATURES, kO = 3;
// parameter layout: W1 [64][8], b1, W2s [64][64], W2n, b2, W3s, W3n, b3, W4 [3][64], b4 [3]
constexpr int oW1 = 0, ob1 = oW1 + kH * kF, oW2s = ob1 + kH, oW2n = oW2s + kH * kH, ob2 = oW2n + kH * kH,
              oW3s = ob2 + kH, oW3n = oW3s + kH * kH, ob3 = oW3n + kH * kH, oW4 = ob3 + kH, ob4 = oW4 + kO * kH,
              kNParams = ob4 + kO;
constexpr int kWgBlocks = 256;  // blocks of the weight-gradient kernels (fixed: deterministic sums)
constexpr int kWgSub = 32;      // edges staged per sub-tile
constexpr int kWgMax = kH * kH + kH;

struct GnnState {
    float *master = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;  // [P]
    __nv_bfloat16 *wb = nullptr;                                            // [P] BF16 copy
    float *feat = nullptr;                                                  // [nE][8]
    float *z1 = nullptr, *z2 = nullptr, *z3 = nullptr;                      // pre-activations [nE][64]
    float *bA = nullptr, *bB = nullptr, *bC = nullptr;                      // backward scratch [nE][64]
    float *out = nullptr, *dout = nullptr;                                  // [nE][3]: a, b, c
    double *vlog = nullptr;                                                 // [nV] c_v
    double *zs = nullptr, *zg = nullptr, *w = nullptr, *dcv = nullptr;      // [nV][3], [nV][3], [nV][3], [nV]
    double *ew = nullptr;                                                   // [nE][2]: e^{2a}, e^{2b}
    double *diag = nullptr;                                                 // [nV] diag(A) of the bound curve
    double *cstat = nullptr;                                                // [nCurves][2]: mean l, mean d
    float *wpart = nullptr;                                                 // [kWgBlocks][kWgMax]
    double *loss = nullptr;                                                 // [nProb]
    double *sq = nullptr;                                                   // [nProb][2]: z^T r, z^T A z
    double *g = nullptr, *Ag = nullptr, *gz = nullptr, *gy = nullptr;       // [nV][3]
    int *eprev = nullptr, *enext = nullptr, *ecurve = nullptr;              // [nE]
    int loaded = 0, bound = 0, adam_t = 0;
};

// ---------------------------------------------------------------------------------- forward

__device__ __forceinline__ float bf(const __nv_bfloat16 *w, int i) { return __bfloat162float(w[i]); }

// per-curve mean edge length and mean diag(A) (one block per curve; closed curves: edges = vertices)
__global__ void k_gnn_cstat(const int *__restrict__ voff, const double *__restrict__ ell,
                            const double *__restrict__ diag, double *__restrict__ cstat)
{
    const int c = blockIdx.x, v0 = voff[c], v1 = voff[c + 1];
    __shared__ double sh[2][256];
    double a = 0, b = 0;
    for (int i = v0 + threadIdx.x; i < v1; i += blockDim.x) {
        a += ell[i];
        b += diag[i];
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double n = (double)(v1 - v0);
        cstat[2 * c] = sh[0][0] / n;
        cstat[2 * c + 1] = sh[1][0] / n;
    }
}

__global__ void k_gnn_features(int nE, const int *__restrict__ ecurve, const int *__restrict__ eprev,
                               const int *__restrict__ enext, const int *__restrict__ E,
                               const double *__restrict__ ell, const double *__restrict__ T,
                               const double *__restrict__ diag, const double *__restrict__ cstat,
                               float *__restrict__ f)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nE) return;
    const int c = ecurve[I], P = eprev[I], N = enext[I];
    const double ml = cstat[2 * c], md = cstat[2 * c + 1];
    const double tp = T[3 * P] * T[3 * I] + T[3 * P + 1] * T[3 * I + 1] + T[3 * P + 2] * T[3 * I + 2];
    const double tn = T[3 * I] * T[3 * N] + T[3 * I + 1] * T[3 * N + 1] + T[3 * I + 2] * T[3 * N + 2];
    const int i1 = E[2 * I], i2 = E[2 * I + 1];
    float *o = f + (size_t)I * kF;
    o[0] = (float)log(ell[I] / ml);
    o[1] = (float)(1.0 - tp);
    o[2] = (float)(1.0 - tn);
    o[3] = (float)log(diag[i1] / md);
    o[4] = (float)log(diag[i2] / md);
    o[5] = (float)log(ell[P] / ell[I]);
    o[6] = (float)log(ell[N] / ell[I]);
    o[7] = 1.0f;
}

// z1 = W1 f + b1 (one thread per edge)
__global__ void __launch_bounds__(128) k_gnn_l1(int nE, const float *__restrict__ f,
                                                const __nv_bfloat16 *__restrict__ w, float *__restrict__ z1)
{
    __shared__ float W[kH * kF + kH];
    for (int t = threadIdx.x; t < kH * kF + kH; t += blockDim.x) W[t] = bf(w, oW1 + t);
    __syncthreads();
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nE) return;
    float x[kF];
#pragma unroll
    for (int k = 0; k < kF; ++k) x[k] = f[(size_t)I * kF + k];
    float4 *zo = reinterpret_cast<float4 *>(z1 + (size_t)I * kH);
#pragma unroll 4
    for (int o = 0; o < kH; o += 4) {
        float s[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            s[q] = W[kH * kF + o + q];
#pragma unroll
            for (int k = 0; k < kF; ++k) s[q] = fmaf(W[(o + q) * kF + k], x[k], s[q]);
        }
        zo[o / 4] = make_float4(s[0], s[1], s[2], s[3]);
    }
}

// ---------------------------------------------------------------------------------- tensor-core layers
//
// The two 64-wide contractions per layer run on the tensor cores with mma.sync m16n8k16 (BF16 operands,
// FP32 accumulation): the forward message-passing layer z = [Ws | Wn] [h; m] + b (K = 128, N = 64) and
// its data gradient [dh | dm] = dz [Ws | Wn] (K = 64, N = 128).  The weights are BF16 already; each FP32
// activation is split into three BF16 terms (x = x1 + x2 + x3 to ~2^-24), so the products carry the
// FP32 activations' digits and the layers compute what the CUDA-core form computes, up to the order of
// the FP32 sums.  A block of 64 threads (two warps of 16 rows) takes 32 edges; the operand tiles sit in
// shared memory with padded rows.
constexpr int kTcRows = 32;

__device__ __forceinline__ uint32_t bf_pack(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// x = h + m + l in BF16 terms (each the rounding of the remainder)
__device__ __forceinline__ void bf_split3(float x, __nv_bfloat16 (&t)[3])
{
    t[0] = __float2bfloat16_rn(x);
    float r = x - __bfloat162float(t[0]);
    t[1] = __float2bfloat16_rn(r);
    r -= __bfloat162float(t[1]);
    t[2] = __float2bfloat16_rn(r);
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// acc[n-tile][4] += X[rows r0 .. r0 + 15][0 .. K) x B (B given transposed: Bt[n][k]), one warp.
// Fragment layouts of m16n8k16 (g = lane / 4, q = lane % 4): A rows g and g + 8, columns 2q, 2q + 1 and
// 2q + 8, 2q + 9; B column g, rows 2q, 2q + 1 and 2q + 8, 2q + 9; C rows g and g + 8, columns 2q, 2q + 1.
template <int K, int N, int LDX, int LDB>
__device__ __forceinline__ void tc_rows16(const float *X, int r0, const __nv_bfloat16 *Bt, float (&acc)[N / 8][4])
{
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
#pragma unroll
    for (int kk = 0; kk < K; kk += 16) {
        const int c0 = kk + 2 * q;
        const float x[8] = {X[(r0 + g) * LDX + c0],         X[(r0 + g) * LDX + c0 + 1],
                            X[(r0 + g + 8) * LDX + c0],     X[(r0 + g + 8) * LDX + c0 + 1],
                            X[(r0 + g) * LDX + c0 + 8],     X[(r0 + g) * LDX + c0 + 9],
                            X[(r0 + g + 8) * LDX + c0 + 8], X[(r0 + g + 8) * LDX + c0 + 9]};
        __nv_bfloat16 t[8][3];
#pragma unroll
        for (int e = 0; e < 8; ++e) bf_split3(x[e], t[e]);
        uint32_t a[3][4];
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int r = 0; r < 4; ++r) a[p][r] = bf_pack(t[2 * r][p], t[2 * r + 1][p]);
#pragma unroll
        for (int nt = 0; nt < N / 8; ++nt) {
            const __nv_bfloat16 *bc = Bt + (nt * 8 + g) * LDB + c0;
            const uint32_t b0 = bf_pack(bc[0], bc[1]), b1 = bf_pack(bc[8], bc[9]);
            // smallest terms first
            mma_bf16_16816(acc[nt], a[2], b0, b1);
            mma_bf16_16816(acc[nt], a[1], b0, b1);
            mma_bf16_16816(acc[nt], a[0], b0, b1);
        }
    }
}

// zout = Ws relu(zin) + Wn avg(relu(zin[I-1]), relu(zin[I+1])) + b on the tensor cores
__global__ void __launch_bounds__(64) k_gnn_lmp_tc(int nE, const int *__restrict__ eprev, const int *__restrict__ enext,
                                                   const float *__restrict__ zin, const __nv_bfloat16 *__restrict__ w,
                                                   int oWs, int oWn, int ob, float *__restrict__ zout)
{
    constexpr int K = 2 * kH, LDX = K + 4, LDB = K + 8;
    __shared__ __align__(16) float X[kTcRows * LDX];
    __shared__ __align__(16) __nv_bfloat16 Bt[kH * LDB];
    __shared__ float bias[kH];
    for (int t = threadIdx.x; t < kH * K; t += blockDim.x) {
        const int n = t / K, k = t % K;
        Bt[n * LDB + k] = k < kH ? w[oWs + n * kH + k] : w[oWn + n * kH + (k - kH)];
    }
    for (int t = threadIdx.x; t < kH; t += blockDim.x) bias[t] = bf(w, ob + t);
    const int I0 = blockIdx.x * kTcRows;
    for (int t = threadIdx.x; t < kTcRows * K; t += blockDim.x) {
        const int r = t / K, k = t % K, I = I0 + r;
        float v = 0.f;
        if (I < nE) {
            if (k < kH)
                v = fmaxf(zin[(size_t)I * kH + k], 0.f);
            else
                v = 0.5f * (fmaxf(zin[(size_t)eprev[I] * kH + k - kH], 0.f) +
                            fmaxf(zin[(size_t)enext[I] * kH + k - kH], 0.f));
        }
        X[r * LDX + k] = v;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    float acc[kH / 8][4];
#pragma unroll
    for (int nt = 0; nt < kH / 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
    tc_rows16<K, kH, LDX, LDB>(X, 16 * warp, Bt, acc);
#pragma unroll
    for (int nt = 0; nt < kH / 8; ++nt)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int I = I0 + 16 * warp + g + 8 * h;
            if (I >= nE) continue;
            const int col = nt * 8 + 2 * q;
            float2 o = make_float2(acc[nt][2 * h] + bias[col], acc[nt][2 * h + 1] + bias[col + 1]);
            *reinterpret_cast<float2 *>(zout + (size_t)I * kH + col) = o;
        }
}

// dh = dz Ws, dm = dz Wn on the tensor cores (dh[k] = sum_o dz[o] Ws[o][k])
__global__ void __launch_bounds__(64) k_gnn_bmat_tc(int nE, const float *__restrict__ dz,
                                                    const __nv_bfloat16 *__restrict__ w, int oWs, int oWn,
                                                    float *__restrict__ dh, float *__restrict__ dm)
{
    constexpr int K = kH, N = 2 * kH, LDX = K + 4, LDB = K + 8;
    __shared__ __align__(16) float X[kTcRows * LDX];
    __shared__ __align__(16) __nv_bfloat16 Bt[N * LDB];
    for (int t = threadIdx.x; t < N * K; t += blockDim.x) {
        const int n = t / K, o = t % K;  // Bt[n][o] = Ws[o][n] (n < 64), Wn[o][n - 64]
        Bt[n * LDB + o] = n < kH ? w[oWs + o * kH + n] : w[oWn + o * kH + (n - kH)];
    }
    const int I0 = blockIdx.x * kTcRows;
    for (int t = threadIdx.x; t < kTcRows * K; t += blockDim.x) {
        const int r = t / K, k = t % K, I = I0 + r;
        X[r * LDX + k] = I < nE ? dz[(size_t)I * kH + k] : 0.f;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    float acc[N / 8][4];
#pragma unroll
    for (int nt = 0; nt < N / 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
    tc_rows16<K, N, LDX, LDB>(X, 16 * warp, Bt, acc);
#pragma unroll
    for (int nt = 0; nt < N / 8; ++nt)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int I = I0 + 16 * warp + g + 8 * h;
            if (I >= nE) continue;
            const int col = nt * 8 + 2 * q;
            float *out = col < kH ? dh + (size_t)I * kH + col : dm + (size_t)I * kH + (col - kH);
            *reinterpret_cast<float2 *>(out) = make_float2(acc[nt][2 * h], acc[nt][2 * h + 1]);
        }
}

// (a, b, c) = W4 relu(z3) + b4; also e^{2a}, e^{2b} in FP64 for the G term
__global__ void k_gnn_out(int nE, const float *__restrict__ z3, const __nv_bfloat16 *__restrict__ w,
                          float *__restrict__ out, double *__restrict__ ew)
{
    __shared__ float W[kO * kH + kO];
    for (int t = threadIdx.x; t < kO * kH + kO; t += blockDim.x) W[t] = bf(w, oW4 + t);
    __syncthreads();
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nE) return;
    float o[kO];
#pragma unroll
    for (int q = 0; q < kO; ++q) o[q] = W[kO * kH + q];
    const float4 *z = reinterpret_cast<const float4 *>(z3 + (size_t)I * kH);
#pragma unroll
    for (int k = 0; k < kH / 4; ++k) {
        const float4 v = z[k];
        const float hv[4] = {fmaxf(v.x, 0.f), fmaxf(v.y, 0.f), fmaxf(v.z, 0.f), fmaxf(v.w, 0.f)};
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int c = 0; c < kO; ++c) o[c] = fmaf(W[c * kH + 4 * k + q], hv[q], o[c]);
    }
    for (int c = 0; c < kO; ++c) out[kO * I + c] = o[c];
    ew[2 * I] = exp(2.0 * (double)o[0]);
    ew[2 * I + 1] = exp(2.0 * (double)o[1]);
}

// c_v = mean over the edges incident to v of their output c
__global__ void k_gnn_vlog(int nV, const int *__restrict__ inc_ptr, const int *__restrict__ inc,
                           const float *__restrict__ out, double *__restrict__ vlog)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nV) return;
    double s = 0.0;
    const int k0 = inc_ptr[v], k1 = inc_ptr[v + 1];
    for (int k = k0; k < k1; ++k) s += (double)out[kO * (inc[k] >> 1) + 2];
    vlog[v] = k1 > k0 ? s / (k1 - k0) : 0.0;
}

// ---------------------------------------------------------------------------------- backward

// dz3 = (dout W4) * [z3 > 0]
__global__ void k_gnn_bout(int nE, const float *__restrict__ dout, const float *__restrict__ z3,
                           const __nv_bfloat16 *__restrict__ w, float *__restrict__ dz3)
{
    __shared__ float W[kO * kH];
    for (int t = threadIdx.x; t < kO * kH; t += blockDim.x) W[t] = bf(w, oW4 + t);
    __syncthreads();
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nE) return;
    const float da = dout[kO * I], db = dout[kO * I + 1], dc = dout[kO * I + 2];
    for (int k = 0; k < kH; ++k) {
        const float z = z3[(size_t)I * kH + k];
        dz3[(size_t)I * kH + k] = z > 0.f ? fmaf(da, W[k], fmaf(db, W[kH + k], dc * W[2 * kH + k])) : 0.f;
    }
}

// Block partials of grad_W[o][k] = sum_I dz[I][o] x_I[k] and grad_b[o] = sum_I dz[I][o] over one
// contiguous edge range per block.  x_I = relu(xin[I]) (mode 0), avg(relu(xin[I-1]), relu(xin[I+1]))
// (mode 1) or xin[I] itself (mode 2: the features).
template <int O, int K>
__global__ void __launch_bounds__(256) k_gnn_wgrad(int nE, const float *__restrict__ dz, const float *__restrict__ xin,
                                                   const int *__restrict__ eprev, const int *__restrict__ enext,
                                                   int mode, float *__restrict__ wpart)
{
    constexpr int NE = O * K + O;          // entries: weights then biases
    constexpr int PER = (NE + 255) / 256;  // entries per thread
    __shared__ float sd[kWgSub][O], sx[kWgSub][K];
    const int per_blk = (nE + gridDim.x - 1) / gridDim.x;
    const int e0 = blockIdx.x * per_blk, e1 = min(nE, e0 + per_blk);
    float acc[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) acc[q] = 0.f;
    for (int base = e0; base < e1; base += kWgSub) {
        for (int t = threadIdx.x; t < kWgSub * O; t += blockDim.x) {
            const int e = t / O, o = t % O, I = base + e;
            sd[e][o] = I < e1 ? dz[(size_t)I * O + o] : 0.f;
        }
        for (int t = threadIdx.x; t < kWgSub * K; t += blockDim.x) {
            const int e = t / K, k = t % K, I = base + e;
            float xv = 0.f;
            if (I < e1) {
                if (mode == 0)
                    xv = fmaxf(xin[(size_t)I * K + k], 0.f);
                else if (mode == 1)
                    xv = 0.5f * (fmaxf(xin[(size_t)eprev[I] * K + k], 0.f) + fmaxf(xin[(size_t)enext[I] * K + k], 0.f));
                else
                    xv = xin[(size_t)I * K + k];
            }
            sx[e][k] = xv;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int ent = threadIdx.x + 256 * q;
            if (ent < O * K) {
                const int o = ent / K, k = ent % K;
                float s = acc[q];
#pragma unroll 8
                for (int e = 0; e < kWgSub; ++e) s = fmaf(sd[e][o], sx[e][k], s);
                acc[q] = s;
            } else if (ent < NE) {
                const int o = ent - O * K;
                float s = acc[q];
                for (int e = 0; e < kWgSub; ++e) s += sd[e][o];
                acc[q] = s;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int ent = threadIdx.x + 256 * q;
        if (ent < NE) wpart[(size_t)blockIdx.x * kWgMax + ent] = acc[q];
    }
}

// grad[oW + e] (and the biases at ob) = sum of the block partials, in block order
__global__ void k_gnn_wreduce(int nW, int nB, int nblk, const float *__restrict__ wpart, int oW, int ob,
                              float *__restrict__ grad)
{
    const int ent = blockIdx.x * blockDim.x + threadIdx.x;
    if (ent >= nW + nB) return;
    float s = 0.f;
    for (int b = 0; b < nblk; ++b) s += wpart[(size_t)b * kWgMax + ent];
    if (ent < nW)
        grad[oW + ent] = s;
    else
        grad[ob + ent - nW] = s;
}

// dzin = (dh + (dm[I+1] + dm[I-1]) / 2) * [zin > 0], written over dh (m[J] averages h[J-1], h[J+1])
__global__ void k_gnn_bcombine(int nE, const int *__restrict__ eprev, const int *__restrict__ enext,
                               const float *__restrict__ dm, const float *__restrict__ zin, float *__restrict__ dh)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nE) return;
    const int P = eprev[I], N = enext[I];
    for (int k = 0; k < kH; ++k) {
        const float g = dh[(size_t)I * kH + k] + 0.5f * (dm[(size_t)N * kH + k] + dm[(size_t)P * kH + k]);
        dh[(size_t)I * kH + k] = zin[(size_t)I * kH + k] > 0.f ? g : 0.f;
    }
}

__global__ void k_gnn_adam(int P, float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                           const float *__restrict__ g, float lr, float b1, float b2, float eps, float c1, float c2,
                           __nv_bfloat16 *__restrict__ wb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi, vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    wb[i] = __float2bfloat16(wi);
}

__global__ void k_gnn_tobf16(int P, const float *__restrict__ w, __nv_bfloat16 *__restrict__ wb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < P) wb[i] = __float2bfloat16(w[i]);
}

// ---------------------------------------------------------------------------------- the G term

// z[v] (+)= (G r)[v] over the edges incident to v (incidence CSR: edge * 2 + slot, slot 1 <=> v = i2)
__global__ void k_gnn_gapply(int nV, const int *__restrict__ inc_ptr, const int *__restrict__ inc,
                             const int *__restrict__ E, const double *__restrict__ ew, const double *__restrict__ diag,
                             const double *__restrict__ r, double *__restrict__ z, int accumulate,
                             const int *__restrict__ vprob, const int *__restrict__ skip)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nV) return;
    if (skip && skip[vprob[v]]) return;
    double acc[3] = {0, 0, 0};
    for (int k = inc_ptr[v]; k < inc_ptr[v + 1]; ++k) {
        const int e = inc[k] >> 1, sl = inc[k] & 1;
        const int a = E[2 * e], b = E[2 * e + 1];
        const double ea = ew[2 * e], eb = ew[2 * e + 1];
        const double sa = 1.0 / sqrt(diag[a]), sb = 1.0 / sqrt(diag[b]);
        const double sg = sl ? ea : -ea;
        for (int q = 0; q < 3; ++q) {
            const double ra = r[3 * a + q] * sa, rb = r[3 * b + q] * sb;
            acc[q] += sg * (rb - ra) + eb * (ra + rb);
        }
    }
    const double s = 1.0 / sqrt(diag[v]);
    for (int q = 0; q < 3; ++q) z[3 * v + q] = (accumulate ? z[3 * v + q] : 0.0) + acc[q] * s;
}

// dout (+)= scale * d(gz . G r)/d(a, b) = scale * [2 e^{2a} (g~_i2 - g~_i1).delta, 2 e^{2b} (g~_i1 + g~_i2).sigma]
__global__ void k_gnn_doutput(int nE, const int *__restrict__ E, const double *__restrict__ ew,
                              const double *__restrict__ diag, const double *__restrict__ r,
                              const double *__restrict__ gz, double scale, int accumulate, float *__restrict__ dout)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nE) return;
    const int a = E[2 * I], b = E[2 * I + 1];
    const double sa = 1.0 / sqrt(diag[a]), sb = 1.0 / sqrt(diag[b]);
    double dea = 0, deb = 0;
    for (int q = 0; q < 3; ++q) {
        const double ra = r[3 * a + q] * sa, rb = r[3 * b + q] * sb;
        const double ga = gz[3 * a + q] * sa, gb = gz[3 * b + q] * sb;
        dea += (gb - ga) * (rb - ra);
        deb += (ga + gb) * (ra + rb);
    }
    const float da = (float)(scale * 2.0 * ew[2 * I] * dea), db = (float)(scale * 2.0 * ew[2 * I + 1] * deb);
    if (accumulate) {
        dout[kO * I] += da;
        dout[kO * I + 1] += db;
    } else {
        dout[kO * I] = da;
        dout[kO * I + 1] = db;
        dout[kO * I + 2] = 0.f;
    }
}

// dc_v = sum over components of gz_v . zs_v + r_v . z2_v (the rescaling's gradient at vertex v)
__global__ void k_gnn_dcv(int nV, const double *__restrict__ gz, const double *__restrict__ zs,
                          const double *__restrict__ r, const double *__restrict__ z2, double *__restrict__ dcv)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nV) return;
    double s = 0.0;
    for (int q = 0; q < 3; ++q) s += gz[3 * v + q] * zs[3 * v + q] + r[3 * v + q] * z2[3 * v + q];
    dcv[v] = s;
}

// dout_c[I] += scale * (dc_{i1} + dc_{i2}) / 2   (c_v averages the two edges at v; closed curves)
__global__ void k_gnn_dc_edges(int nE, const int *__restrict__ E, const double *__restrict__ dcv, double scale,
                               float *__restrict__ dout)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nE) return;
    dout[kO * I + 2] += (float)(scale * 0.5 * (dcv[E[2 * I]] + dcv[E[2 * I + 1]]));
}

// w = a + b
__global__ void k_gnn_add(int n, const double *__restrict__ a, const double *__restrict__ b, double *__restrict__ w)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) w[i] = a[i] + b[i];
}

// ---------------------------------------------------------------------------------- training loss

// gz = -2 s / (q er) (r - (s / q) (Ab + Ag)) with (s, q) = sq[problem]
__global__ void k_gnn_gz(int nV, const int *__restrict__ vprob, const double *__restrict__ r,
                         const double *__restrict__ Ab, const double *__restrict__ Ag, const double *__restrict__ er,
                         const double *__restrict__ sq, double *__restrict__ gz)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nV) return;
    const int p = vprob[i];
    const double e = er[p], sv = sq[2 * p], qv = sq[2 * p + 1];
    const bool ok = e > 0.0 && qv > 0.0;
    const double f = ok ? -2.0 * sv / (qv * e) : 0.0, ratio = ok ? sv / qv : 0.0;
    for (int k = 0; k < 3; ++k) gz[3 * i + k] = f * (r[3 * i + k] - ratio * (Ab[3 * i + k] + Ag[3 * i + k]));
}

// per problem (one block each): s = z.r, q = z.(Ab + Ag) with z = b + g into sq; loss[q] += scale (1 - s^2 / (q er))
__global__ void k_gnn_loss(const int *__restrict__ prob_v, const double *__restrict__ r, const double *__restrict__ b,
                           const double *__restrict__ g, const double *__restrict__ Ab, const double *__restrict__ Ag,
                           const double *__restrict__ er, double scale, double *__restrict__ sq,
                           double *__restrict__ loss)
{
    const int q = blockIdx.x, v0 = prob_v[q], v1 = prob_v[q + 1];
    double s1 = 0, s2 = 0;
    for (int i = 3 * v0 + threadIdx.x; i < 3 * v1; i += blockDim.x) {
        const double z = b[i] + g[i];
        s1 += z * (Ab[i] + Ag[i]);
        s2 += z * r[i];
    }
    __shared__ double sh[2][256];
    sh[0][threadIdx.x] = s1;
    sh[1][threadIdx.x] = s2;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double e = er[q], qz = sh[0][0], sz = sh[1][0];
        sq[2 * q] = sz;
        sq[2 * q + 1] = qz;
        loss[q] += (e > 0.0 && qz > 0.0) ? scale * (1.0 - sz * sz / (qz * e)) : 0.0;
    }
}

// out[q] = sum over the vertices of problem q of a . b (one block per problem)
__global__ void k_gnn_pdot(const int *__restrict__ prob_v, const double *__restrict__ a, const double *__restrict__ b,
                           double *__restrict__ out)
{
    const int q = blockIdx.x, v0 = prob_v[q], v1 = prob_v[q + 1];
    double s = 0;
    for (int i = 3 * v0 + threadIdx.x; i < 3 * v1; i += blockDim.x) s += a[i] * b[i];
    __shared__ double sh[256];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = sh[0];
}

// out[0] = sum_i x[i] (one block)
__global__ void k_gnn_sum(int n, const double *__restrict__ x, double *__restrict__ out)
{
    double s = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
    __shared__ double sh[256];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0];
}

// ---------------------------------------------------------------------------------- host side

int gnn_num_params() { return kNParams; }

cudaError_t gnn_alloc(Ctx &c)
{
    if (c.gnn) return cudaSuccess;
    c.gnn = new GnnState();
    GnnState &G = *c.gnn;
    const size_t nE = std::max(1, c.nE), nV = std::max(1, c.nV);
    TPE_CHECK(cudaMalloc(&G.master, sizeof(float) * kNParams));
    TPE_CHECK(cudaMalloc(&G.m, sizeof(float) * kNParams));
    TPE_CHECK(cudaMalloc(&G.v, sizeof(float) * kNParams));
    TPE_CHECK(cudaMalloc(&G.grad, sizeof(float) * kNParams));
    TPE_CHECK(cudaMalloc(&G.wb, sizeof(__nv_bfloat16) * kNParams));
    TPE_CHECK(cudaMemset(G.m, 0, sizeof(float) * kNParams));
    TPE_CHECK(cudaMemset(G.v, 0, sizeof(float) * kNParams));
    TPE_CHECK(cudaMalloc(&G.feat, sizeof(float) * nE * kF));
    float **acts[] = {&G.z1, &G.z2, &G.z3, &G.bA, &G.bB, &G.bC};
    for (float **p : acts) TPE_CHECK(cudaMalloc(p, sizeof(float) * nE * kH));
    TPE_CHECK(cudaMalloc(&G.out, sizeof(float) * nE * kO));
    TPE_CHECK(cudaMalloc(&G.dout, sizeof(float) * nE * kO));
    TPE_CHECK(cudaMalloc(&G.vlog, sizeof(double) * nV));
    TPE_CHECK(cudaMemset(G.vlog, 0, sizeof(double) * nV));
    TPE_CHECK(cudaMalloc(&G.zs, sizeof(double) * 3 * nV));
    TPE_CHECK(cudaMalloc(&G.zg, sizeof(double) * 3 * nV));
    TPE_CHECK(cudaMalloc(&G.w, sizeof(double) * 3 * nV));
    TPE_CHECK(cudaMalloc(&G.dcv, sizeof(double) * nV));
    TPE_CHECK(cudaMalloc(&G.ew, sizeof(double) * nE * 2));
    TPE_CHECK(cudaMalloc(&G.diag, sizeof(double) * nV));
    TPE_CHECK(cudaMalloc(&G.cstat, sizeof(double) * 2 * c.nCurves));
    TPE_CHECK(cudaMalloc(&G.wpart, sizeof(float) * kWgBlocks * kWgMax));
    TPE_CHECK(cudaMalloc(&G.loss, sizeof(double) * std::max(1, c.nProb)));
    TPE_CHECK(cudaMalloc(&G.sq, sizeof(double) * 2 * std::max(1, c.nProb)));
    TPE_CHECK(cudaMalloc(&G.g, sizeof(double) * 3 * nV));
    TPE_CHECK(cudaMalloc(&G.Ag, sizeof(double) * 3 * nV));
    TPE_CHECK(cudaMalloc(&G.gz, sizeof(double) * 3 * nV));
    TPE_CHECK(cudaMalloc(&G.gy, sizeof(double) * 3 * nV));
    // neighbours along the closed curves: edge v0 + i = (v0 + i, v0 + (i + 1) mod n)
    std::vector<int> ep(nE), en(nE), ec(nE);
    for (int k = 0; k < c.nCurves; ++k) {
        const int v0 = c.h_voff[k], n = c.h_voff[k + 1] - v0;
        for (int i = 0; i < n; ++i) {
            ep[v0 + i] = v0 + (i + n - 1) % n;
            en[v0 + i] = v0 + (i + 1) % n;
            ec[v0 + i] = k;
        }
    }
    TPE_CHECK(cudaMalloc(&G.eprev, sizeof(int) * nE));
    TPE_CHECK(cudaMalloc(&G.enext, sizeof(int) * nE));
    TPE_CHECK(cudaMalloc(&G.ecurve, sizeof(int) * nE));
    TPE_CHECK(cudaMemcpy(G.eprev, ep.data(), sizeof(int) * nE, cudaMemcpyHostToDevice));
    TPE_CHECK(cudaMemcpy(G.enext, en.data(), sizeof(int) * nE, cudaMemcpyHostToDevice));
    TPE_CHECK(cudaMemcpy(G.ecurve, ec.data(), sizeof(int) * nE, cudaMemcpyHostToDevice));
    return cudaSuccess;
}

void gnn_free(Ctx &c)
{
    if (!c.gnn) return;
    GnnState &G = *c.gnn;
    void *p[] = {G.master, G.m,     G.v,     G.grad, G.wb, G.feat, G.z1, G.z2,    G.z3,    G.bA,
                 G.bB,     G.bC,    G.out,   G.dout, G.ew, G.diag, G.cstat, G.wpart, G.loss, G.sq, G.vlog, G.zs, G.zg, G.w, G.dcv, G.g,
                 G.Ag,     G.gz,    G.gy,    G.eprev, G.enext, G.ecurve};
    for (void *q : p)
        if (q) cudaFree(q);
    delete c.gnn;
    c.gnn = nullptr;
}

int gnn_ready(const Ctx &c) { return c.gnn && c.gnn->loaded; }
int gnn_bound(const Ctx &c) { return c.gnn && c.gnn->bound; }

cudaError_t gnn_set_params(Ctx &c, const float *theta, int reset_adam, cudaStream_t s)
{
    GnnState &G = *c.gnn;
    TPE_CHECK(cudaMemcpyAsync(G.master, theta, sizeof(float) * kNParams, cudaMemcpyDeviceToDevice, s));
    if (reset_adam) {
        TPE_CHECK(cudaMemsetAsync(G.m, 0, sizeof(float) * kNParams, s));
        TPE_CHECK(cudaMemsetAsync(G.v, 0, sizeof(float) * kNParams, s));
        G.adam_t = 0;
    }
    k_gnn_tobf16<<<(kNParams + 255) / 256, 256, 0, s>>>(kNParams, G.master, G.wb);
    c.launches++;
    G.loaded = 1;
    return cudaGetLastError();
}

cudaError_t gnn_get_params(Ctx &c, float *theta, cudaStream_t s)
{
    return cudaMemcpyAsync(theta, c.gnn->master, sizeof(float) * kNParams, cudaMemcpyDeviceToDevice, s);
}

// Bind the geometry whose FP64 edge quantities are in slot `which` and whose diag(A) is `diag`:
// the features, kept until the next bind.
cudaError_t gnn_bind(Ctx &c, int which, const double *diag, cudaStream_t s)
{
    GnnState &G = *c.gnn;
    if (diag != G.diag) TPE_CHECK(cudaMemcpyAsync(G.diag, diag, sizeof(double) * c.nV, cudaMemcpyDeviceToDevice, s));
    k_gnn_cstat<<<c.nCurves, 256, 0, s>>>(c.d_voff, c.d_ellw[which], G.diag, G.cstat);
    k_gnn_features<<<(c.nE + 127) / 128, 128, 0, s>>>(c.nE, G.ecurve, G.eprev, G.enext, c.d_edges, c.d_ellw[which],
                                                      c.d_Tw[which], G.diag, G.cstat, G.feat);
    c.launches += 2;
    G.bound = 1;
    return cudaGetLastError();
}

double *gnn_diag_buffer(Ctx &c) { return c.gnn->diag; }
const float *gnn_features(const Ctx &c) { return c.gnn->feat; }
const float *gnn_outputs(const Ctx &c) { return c.gnn->out; }
const double *gnn_vlog(const Ctx &c) { return c.gnn->vlog; }

// Network forward on the bound features with the current BF16 weights: outputs and e^{2a}, e^{2b}.
cudaError_t gnn_forward(Ctx &c, cudaStream_t s)
{
    GnnState &G = *c.gnn;
    const int nb = (c.nE + 127) / 128;
    k_gnn_l1<<<nb, 128, 0, s>>>(c.nE, G.feat, G.wb, G.z1);
    const int ntc = (c.nE + kTcRows - 1) / kTcRows;
    k_gnn_lmp_tc<<<ntc, 64, 0, s>>>(c.nE, G.eprev, G.enext, G.z1, G.wb, oW2s, oW2n, ob2, G.z2);
    k_gnn_lmp_tc<<<ntc, 64, 0, s>>>(c.nE, G.eprev, G.enext, G.z2, G.wb, oW3s, oW3n, ob3, G.z3);
    k_gnn_out<<<nb, 128, 0, s>>>(c.nE, G.z3, G.wb, G.out, G.ew);
    k_gnn_vlog<<<(c.nV + 255) / 256, 256, 0, s>>>(c.nV, c.d_inc_ptr, c.d_inc, G.out, G.vlog);
    c.launches += 5;
    return cudaGetLastError();
}

template <int O, int K>
static cudaError_t wgrad(Ctx &c, const float *dz, const float *x, int mode, int oW, int ob, float *grad,
                         cudaStream_t s)
{
    GnnState &G = *c.gnn;
    const int nblk = std::max(1, std::min(kWgBlocks, (c.nE + kWgSub - 1) / kWgSub));
    k_gnn_wgrad<O, K><<<nblk, 256, 0, s>>>(c.nE, dz, x, G.eprev, G.enext, mode, G.wpart);
    const int nb = ob >= 0 ? O : 0, n = O * K + nb;
    k_gnn_wreduce<<<(n + 255) / 256, 256, 0, s>>>(O * K, nb, nblk, G.wpart, oW, ob, grad);
    c.launches += 2;
    return cudaGetLastError();
}

// Parameter gradient (FP32, [P]) of a scalar whose derivative with respect to the outputs of the
// last forward pass is dout [nE][2].
cudaError_t gnn_backward(Ctx &c, const float *dout, float *grad, cudaStream_t s)
{
    GnnState &G = *c.gnn;
    const int nb = (c.nE + 127) / 128;
    // read-out: W4, b4, then dz3 into bA
    TPE_CHECK((wgrad<kO, kH>(c, dout, G.z3, 0, oW4, ob4, grad, s)));
    k_gnn_bout<<<nb, 128, 0, s>>>(c.nE, dout, G.z3, G.wb, G.bA);
    c.launches++;
    // layer 3: x = h2 (self) and avg h2 (neighbours)
    TPE_CHECK((wgrad<kH, kH>(c, G.bA, G.z2, 0, oW3s, ob3, grad, s)));
    TPE_CHECK((wgrad<kH, kH>(c, G.bA, G.z2, 1, oW3n, -1, grad, s)));
    k_gnn_bmat_tc<<<(c.nE + kTcRows - 1) / kTcRows, 64, 0, s>>>(c.nE, G.bA, G.wb, oW3s, oW3n, G.bB, G.bC);
    k_gnn_bcombine<<<nb, 128, 0, s>>>(c.nE, G.eprev, G.enext, G.bC, G.z2, G.bB);  // dz2 in bB
    c.launches += 2;
    // layer 2
    TPE_CHECK((wgrad<kH, kH>(c, G.bB, G.z1, 0, oW2s, ob2, grad, s)));
    TPE_CHECK((wgrad<kH, kH>(c, G.bB, G.z1, 1, oW2n, -1, grad, s)));
    k_gnn_bmat_tc<<<(c.nE + kTcRows - 1) / kTcRows, 64, 0, s>>>(c.nE, G.bB, G.wb, oW2s, oW2n, G.bA, G.bC);
    k_gnn_bcombine<<<nb, 128, 0, s>>>(c.nE, G.eprev, G.enext, G.bC, G.z1, G.bA);  // dz1 in bA
    c.launches += 2;
    // layer 1: x = the features
    TPE_CHECK((wgrad<kH, kF>(c, G.bA, G.feat, 2, oW1, ob1, grad, s)));
    return cudaGetLastError();
}

cudaError_t gnn_adam(Ctx &c, const float *grad, float lr, cudaStream_t s)
{
    GnnState &G = *c.gnn;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    G.adam_t++;
    const float c1 = 1.f - powf(b1, (float)G.adam_t), c2 = 1.f - powf(b2, (float)G.adam_t);
    k_gnn_adam<<<(kNParams + 255) / 256, 256, 0, s>>>(kNParams, G.master, G.m, G.v, grad, lr, b1, b2, eps, c1, c2,
                                                      G.wb);
    c.launches++;
    return cudaGetLastError();
}

cudaError_t gnn_gapply(Ctx &c, const double *r, double *z, int accumulate, cudaStream_t s, const int *skip)
{
    GnnState &G = *c.gnn;
    k_gnn_gapply<<<(c.nV + 255) / 256, 256, 0, s>>>(c.nV, c.d_inc_ptr, c.d_inc, c.d_edges, G.ew, G.diag, r, z,
                                                    accumulate, c.d_vprob, skip);
    c.launches++;
    return cudaGetLastError();
}

cudaError_t gnn_out_grad(Ctx &c, const double *r, const double *gz, double scale, int accumulate, float *dout,
                         cudaStream_t s)
{
    GnnState &G = *c.gnn;
    k_gnn_doutput<<<(c.nE + 127) / 128, 128, 0, s>>>(c.nE, c.d_edges, G.ew, G.diag, r, gz, scale, accumulate, dout);
    c.launches++;
    return cudaGetLastError();
}

cudaError_t gnn_problem_dot(Ctx &c, const double *a, const double *b, double *out, cudaStream_t s)
{
    k_gnn_pdot<<<c.nProb, 256, 0, s>>>(c.d_prob_v, a, b, out);
    c.launches++;
    return cudaGetLastError();
}

// One training step over n_pairs prepared pairs of the bound geometry (edge records in slot 0):
// r_i, b_i (the parameter-independent part of M^-1 r_i: the coarse term), Ab_i = A b_i, er_i = e_i . r_i
// per problem, and ilam (the inverse circulant symbols of the geometry, [nV]; NULL: no rescaled
// circulant).  Additive form (R2 NULL): z = b + W S W r + G r.  Balancing form (R2 given, r2_i =
// (I - A Q) r_i, b_i = Q r_i): z = b + (I - Q A) y, y = W S W r2 + G r2, and dL/dy = (I - A Q) dL/dz.
// Per pair: one A apply of the parameter-dependent part, the loss, dL/dz, the output gradients of G and,
// through one more circulant apply, of the rescaling.  The loss at the current parameters (mean over
// pairs and problems) goes to loss_dev; then, for lr > 0, one Adam step.  The parameter gradient is left
// in the context (gnn_last_grad).
cudaError_t gnn_train_step(Ctx &c, const double *gamma, int n_pairs, const double *R, const double *B,
                           const double *AB, const double *ER, const double *ilam, const double *R2, float lr,
                           double *loss_dev, cudaStream_t s)
{
    GnnState &G = *c.gnn;
    const size_t nv3 = 3 * (size_t)c.nV;
    const double scale = 1.0 / ((double)n_pairs * c.nProb);
    const int nbv = (int)((nv3 + 255) / 256);
    TPE_CHECK(gnn_forward(c, s));
    TPE_CHECK(cudaMemsetAsync(G.loss, 0, sizeof(double) * c.nProb, s));
    for (int i = 0; i < n_pairs; ++i) {
        const double *r = R + i * nv3, *b = B + i * nv3, *Ab = AB + i * nv3, *er = ER + (size_t)i * c.nProb;
        const double *x = R2 ? R2 + i * nv3 : r;  // what the learned terms act on
        TPE_CHECK(gnn_gapply(c, x, G.g, 0, s, nullptr));
        if (ilam) {
            TPE_CHECK(spectral_apply_ex(c, x, G.zs, s, nullptr, G.diag, ilam, G.vlog));
            k_gnn_add<<<nbv, 256, 0, s>>>((int)nv3, G.g, G.zs, G.w);
            c.launches++;
        } else if (R2) {
            TPE_CHECK(cudaMemcpyAsync(G.w, G.g, sizeof(double) * nv3, cudaMemcpyDeviceToDevice, s));
        }
        double *w = (ilam || R2) ? G.w : G.g;
        if (R2) TPE_CHECK(coarse_balanced_part(c, 2, w, w, s));  // w = (I - Q A) y
        TPE_CHECK(pair_apply(c, gamma, 0, w, G.Ag, s));
        k_gnn_loss<<<c.nProb, 256, 0, s>>>(c.d_prob_v, r, b, w, Ab, G.Ag, er, scale, G.sq, G.loss);
        k_gnn_gz<<<(c.nV + 255) / 256, 256, 0, s>>>(c.nV, c.d_vprob, r, Ab, G.Ag, er, G.sq, G.gz);
        c.launches += 2;
        const double *gy = G.gz;
        if (R2) {
            TPE_CHECK(coarse_balanced_part(c, 1, G.gz, G.gy, s));  // dL/dy = (I - A Q) dL/dz
            gy = G.gy;
        }
        TPE_CHECK(gnn_out_grad(c, x, gy, scale, i > 0, G.dout, s));
        if (ilam) {
            TPE_CHECK(spectral_apply_ex(c, gy, G.zg, s, nullptr, G.diag, ilam, G.vlog));
            k_gnn_dcv<<<(c.nV + 255) / 256, 256, 0, s>>>(c.nV, gy, G.zs, x, G.zg, G.dcv);
            k_gnn_dc_edges<<<(c.nE + 127) / 128, 128, 0, s>>>(c.nE, c.d_edges, G.dcv, scale, G.dout);
            c.launches += 2;
        }
    }
    TPE_CHECK(gnn_backward(c, G.dout, G.grad, s));
    if (lr > 0.f) TPE_CHECK(gnn_adam(c, G.grad, lr, s));
    if (loss_dev) {
        k_gnn_sum<<<1, 256, 0, s>>>(c.nProb, G.loss, loss_dev);
        c.launches++;
    }
    return cudaGetLastError();
}

const float *gnn_last_grad(const Ctx &c) { return c.gnn->grad; }

}  // namespace tpe
