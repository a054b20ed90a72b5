// Jacobi-scaled circulant ("spectral") preconditioner for closed curves.  Not from the paper (which
// preconditions with geometric multigrid, App. B.3); this library's own choice for a dense GPU solver:
//
//   M^-1 r = D^-1/2 F^-1 diag(1 / lambda) F D^-1/2 r     on every closed curve, per component,
//
// D = diag(A) of the actual curve and lambda the eigenvalues of A = B + B0 for the regular n-gon
// (a circulant matrix) divided by its diagonal, lambda_0 := lambda_1.  On a regular polygon this is
// the exact inverse on the non-constant modes.
//
// lambda_k follows from the quadratic forms of Eq. 21 and Sec. 5.2.3 evaluated on the Fourier mode
// u_j = exp(i 2 pi k j / n), summed over the offset m = J - I of the edge pair (m = 2 .. n-2):
//   lambda_k = (16 sin^2(pi k/n) / l^2) sum_m w_m [sin^2(pi m/n) + cos(2 pi m/n) S_km]
//            + 2 cos^2(pi k/n) sum_m w0_m S_km,                      S_km = sin^2(pi (k m mod n) / n),
// with w_m = w_{0m} and w0_m = w0_{0m} + w0_{m0} of the regular n-gon (every term is >= 0, so no
// cancellation).  The transforms run in FP64: the symbol spans ~n^3.5 (1e17 at n = 2^18), and only
// an FFT that divides each frequency separately keeps that range; a dense circulant product would not.
//   n a power of two <= 8192 : radix-2 FFT in shared memory
//   other n <= 4096          : Bluestein (chirp-z) through a power-of-two FFT of size >= 2n - 1
//   n a power of two > 8192  : four-step FFT, n = N1 N2, batched shared-memory FFTs of N1 and N2
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <vector>

#include "tpe_internal.cuh"

namespace tpe {

#define TPE_CHECK(x)                      \
    do {                                  \
        cudaError_t e_ = (x);             \
        if (e_ != cudaSuccess) return e_; \
    } while (0)

constexpr int kMaxFFT = 8192;  // largest shared-memory FFT (8192 complex doubles = 128 KB)
constexpr int kFFTThreads = 512;

enum SpecKind { SK_POW2 = 0, SK_BLUESTEIN = 1, SK_FOURSTEP = 2 };

struct SpecCurve {
    int v0, n, M, logM;  // M: FFT size (pow2: n; Bluestein: pow2 >= 2n-1; four-step: N1)
    int kind, N2, logN2, nk;  // nk: number of sampled frequencies of the Rayleigh-quotient correction
    long long sym_off, chirp_off, bhat_off;  // offsets into the symbol / chirp / B-hat tables
};

constexpr int kMaxRQ = 24;  // sampled frequencies per curve for the Rayleigh-quotient symbol

}  // namespace tpe

struct tpe::SpecState {
    std::vector<SpecCurve> curves;
    SpecCurve *d_curves = nullptr;
    std::vector<int> small_idx, large_idx, cluster_idx;  // curve indices per path
    int *d_small_idx = nullptr;
    int *d_cluster_idx = nullptr;
    int max_small_M = 0;
    double *d_sym = nullptr;     // normalised symbols
    double2 *d_tw = nullptr;     // exp(-2 pi i k / kMaxFFT), k < kMaxFFT / 2
    double2 *d_chirp = nullptr;  // exp(i pi j^2 / n), j < n, per Bluestein size
    double2 *d_bhat = nullptr;   // FFT_M of the chirp filter, per Bluestein size
    double2 *d_buf0 = nullptr, *d_buf1 = nullptr;  // four-step workspace [3][n_large]
    double *d_dinv = nullptr;    // [nV] D^-1/2
    std::map<int, long long> sym_of_n;
    // Rayleigh-quotient corrected symbols (precond TP_PRECOND_SPECTRAL_RQ), one per curve at its vertex offset
    double *d_sym_rq = nullptr;  // [nV]
    int *d_klist = nullptr;      // [nCurves][kMaxRQ] sampled frequencies
    double *d_rq = nullptr;      // [nCurves][2 kMaxRQ] Rayleigh numerators (cos, sin)
    double *d_probe = nullptr;   // [2][batches][nV][3] the probe fields and their products (set-up scratch)
    int *d_vcurve = nullptr;     // [nV] curve of each vertex
    int max_nk = 0;
    int rq_ready = 0;
    // 1 / symbol in use, per curve at its vertex offset (the applies multiply; FP64 division is slow)
    double *d_ilam = nullptr;    // [nV]
    int ilam_src = -1;           // 0: regular-polygon symbols, 1: Rayleigh-quotient symbols, -1: stale
};

namespace tpe {

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

// In-place radix-2 FFT (decimation in time after a bit-reversal permutation) of G sequences of
// length M = 2^logM stored back to back in shared memory.  tw: exp(-2 pi i k / kMaxFFT).
__device__ void fft_batch(double2 *a, int G, int M, int logM, const double2 *__restrict__ tw, bool inv)
{
    const int total = G * M;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int g = idx >> logM, i = idx & (M - 1);
        int j = (int)(__brev((unsigned)i) >> (32 - logM));
        if (i < j) {
            double2 t = a[g * M + i];
            a[g * M + i] = a[g * M + j];
            a[g * M + j] = t;
        }
    }
    __syncthreads();
    const int tstride = kMaxFFT / M;
    for (int s = 1; s <= logM; ++s) {
        const int half = 1 << (s - 1), step = (M >> s) * tstride;
        for (int t = threadIdx.x; t < G * (M >> 1); t += blockDim.x) {
            int g = t >> (logM - 1), tt = t & ((M >> 1) - 1);
            int grp = tt >> (s - 1), pos = tt & (half - 1);
            int i = g * M + grp * (half << 1) + pos, j = i + half;
            double2 w = tw[pos * step];
            if (inv) w.y = -w.y;
            double2 u = a[i], v = cmul(a[j], w);
            a[i] = make_double2(u.x + v.x, u.y + v.y);
            a[j] = make_double2(u.x - v.x, u.y - v.y);
        }
        __syncthreads();
    }
}

// Bluestein DFT of length n (forward, X_k = sum_m x_m e^{-2 pi i k m / n}) of the n values in a[0, n)
// using the M-point FFT; result in a[0, n).
__device__ void bluestein(double2 *a, int n, int M, int logM, const double2 *__restrict__ chirp,
                          const double2 *__restrict__ bhat, const double2 *__restrict__ tw)
{
    for (int m = threadIdx.x; m < M; m += blockDim.x)
        a[m] = m < n ? cmul(a[m], cconj(chirp[m])) : make_double2(0.0, 0.0);
    __syncthreads();
    fft_batch(a, 1, M, logM, tw, false);
    for (int k = threadIdx.x; k < M; k += blockDim.x) a[k] = cmul(a[k], bhat[k]);
    __syncthreads();
    fft_batch(a, 1, M, logM, tw, true);
    const double s = 1.0 / M;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        double2 v = cmul(a[k], cconj(chirp[k]));
        a[k] = make_double2(v.x * s, v.y * s);
    }
    __syncthreads();
}

// ilam[v0 + k] = 1 / lam_c[k] for every curve c (lam: the regular-polygon table at sym_off, or the
// per-vertex-offset Rayleigh-quotient symbols when rq != NULL); one block per curve
__global__ void k_inv_symbol(const SpecCurve *__restrict__ curves, const double *__restrict__ sym,
                             const double *__restrict__ rq, double *__restrict__ ilam)
{
    const SpecCurve C = curves[blockIdx.x];
    const double *lam = rq ? rq + C.v0 : sym + C.sym_off;
    for (int k = threadIdx.x; k < C.n; k += blockDim.x) {
        const double l = lam[k];
        ilam[C.v0 + k] = l > 0.0 ? 1.0 / l : 0.0;
    }
}

// Small curves: one CTA per (curve, component).  z = D^-1/2 F^-1 (F (D^-1/2 r) / lambda).
__global__ void __launch_bounds__(kFFTThreads) k_spec_small(const SpecCurve *__restrict__ curves,
                                                            const int *__restrict__ idx, const double *__restrict__ r,
                                                            double *__restrict__ z, const double *__restrict__ dinv,
                                                            const double *__restrict__ sym,
                                                            const double2 *__restrict__ chirp,
                                                            const double2 *__restrict__ bhat,
                                                            const double2 *__restrict__ tw,
                                                            const double *__restrict__ ilam,
                                                            const int *__restrict__ skip, int indep)
{
    extern __shared__ double2 sa[];
    const int cidx = idx[blockIdx.x / 3];
    if (skip && skip[indep ? cidx : 0]) return;  // converged problem: its z is not used
    const SpecCurve C = curves[cidx];
    const int comp = blockIdx.x % 3, n = C.n;
    for (int m = threadIdx.x; m < n; m += blockDim.x)
        sa[m] = make_double2(r[3 * (C.v0 + m) + comp] * dinv[C.v0 + m], 0.0);
    __syncthreads();
    const double *il = ilam + C.v0;
    if (C.kind == SK_POW2) {
        fft_batch(sa, 1, n, C.logM, tw, false);
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const double f = il[k];
            sa[k] = make_double2(sa[k].x * f, sa[k].y * f);
        }
        __syncthreads();
        fft_batch(sa, 1, n, C.logM, tw, true);
        for (int m = threadIdx.x; m < n; m += blockDim.x) z[3 * (C.v0 + m) + comp] = sa[m].x / n * dinv[C.v0 + m];
    } else {
        const double2 *ch = chirp + C.chirp_off, *bh = bhat + C.bhat_off;
        bluestein(sa, n, C.M, C.logM, ch, bh, tw);
        // divide by lambda, then the inverse DFT as conj(DFT(conj(.))) / n
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const double f = il[k];
            sa[k] = make_double2(sa[k].x * f, -sa[k].y * f);
        }
        __syncthreads();
        bluestein(sa, n, C.M, C.logM, ch, bh, tw);
        for (int m = threadIdx.x; m < n; m += blockDim.x) z[3 * (C.v0 + m) + comp] = sa[m].x / n * dinv[C.v0 + m];
    }
}

// Powers of two 1024 <= n <= 8192: one transform per cluster of 8 CTAs (four-step with n = 8 N2 through
// distributed shared memory), so that the FP64 work of a few curves spreads over many SMs.
namespace cg = cooperative_groups;
constexpr int kClusterFFT = 8;                       // CTAs per transform (portable cluster size)
constexpr int kClusterMaxN2 = kMaxFFT / kClusterFFT;  // 1024
constexpr int kClusterThreads = 256;
constexpr int kClusterMinN = 1024;

// exp(-/+ 2 pi i j / kMaxFFT) for j in [0, kMaxFFT) from the half table
__device__ __forceinline__ double2 twiddle_full(const double2 *__restrict__ tw, int j, bool inv)
{
    double2 w = j < kMaxFFT / 2 ? tw[j] : make_double2(-tw[j - kMaxFFT / 2].x, -tw[j - kMaxFFT / 2].y);
    if (inv) w.y = -w.y;
    return w;
}

// z = D^-1/2 F^-1 diag(ilam) F D^-1/2 r for one (curve, component) per cluster.  Index m = m1 + 8 m2,
// k = k2 + N2 k1.  Rank m1 transforms its column over m2 and twists by W_n^{m1 k2}; rank q then owns
// rows k2 in [q N2/8, (q+1) N2/8): an 8-point DFT over m1 gathered from the cluster, the division by the
// symbol, the 8-point inverse DFT over k1 and the twist W_n^{-m1 k2}; finally rank m1 gathers row m1 of
// every k2 and transforms back over k2.
__global__ void __cluster_dims__(kClusterFFT, 1, 1) __launch_bounds__(kClusterThreads)
    k_spec_cluster(const SpecCurve *__restrict__ curves, const int *__restrict__ idx, const double *__restrict__ r,
                   double *__restrict__ z, const double *__restrict__ dinv, const double2 *__restrict__ tw,
                   const double *__restrict__ ilam, const int *__restrict__ skip, int indep)
{
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int tr = blockIdx.x / kClusterFFT;
    const int cidx = idx[tr / 3], comp = tr % 3;
    if (skip && skip[indep ? cidx : 0]) return;  // converged problem: the whole cluster leaves
    const SpecCurve C = curves[cidx];
    const int n = C.n, N2 = n / kClusterFFT, logN2 = C.logM - 3, per = N2 / kClusterFFT;
    const int sN = kMaxFFT / n, s8 = kMaxFFT / kClusterFFT;
    __shared__ double2 Y[kClusterMaxN2];
    __shared__ double2 V[kClusterMaxN2];
    for (int m2 = threadIdx.x; m2 < N2; m2 += blockDim.x) {
        const int v = C.v0 + rank + kClusterFFT * m2;
        Y[m2] = make_double2(r[3 * v + comp] * dinv[v], 0.0);
    }
    __syncthreads();
    fft_batch(Y, 1, N2, logN2, tw, false);
    for (int k2 = threadIdx.x; k2 < N2; k2 += blockDim.x)
        Y[k2] = cmul(Y[k2], twiddle_full(tw, ((rank * k2) % n) * sN, false));
    cl.sync();
    for (int t = threadIdx.x; t < per; t += blockDim.x) {
        const int k2 = rank * per + t;
        double2 a[kClusterFFT], X[kClusterFFT];
#pragma unroll
        for (int m1 = 0; m1 < kClusterFFT; ++m1) a[m1] = cl.map_shared_rank(Y, m1)[k2];
#pragma unroll
        for (int k1 = 0; k1 < kClusterFFT; ++k1) {
            double2 sacc = make_double2(0.0, 0.0);
#pragma unroll
            for (int m1 = 0; m1 < kClusterFFT; ++m1) {
                const double2 p = cmul(a[m1], twiddle_full(tw, ((m1 * k1) % kClusterFFT) * s8, false));
                sacc.x += p.x;
                sacc.y += p.y;
            }
            const double f = ilam[C.v0 + k2 + N2 * k1];
            X[k1] = make_double2(sacc.x * f, sacc.y * f);
        }
#pragma unroll
        for (int m1 = 0; m1 < kClusterFFT; ++m1) {
            double2 sacc = make_double2(0.0, 0.0);
#pragma unroll
            for (int k1 = 0; k1 < kClusterFFT; ++k1) {
                const double2 p = cmul(X[k1], twiddle_full(tw, ((m1 * k1) % kClusterFFT) * s8, true));
                sacc.x += p.x;
                sacc.y += p.y;
            }
            V[t * kClusterFFT + m1] = cmul(sacc, twiddle_full(tw, ((m1 * k2) % n) * sN, true));
        }
    }
    cl.sync();  // every rank's V is complete; nobody reads Y any more
    for (int k2 = threadIdx.x; k2 < N2; k2 += blockDim.x)
        Y[k2] = cl.map_shared_rank(V, k2 / per)[(k2 % per) * kClusterFFT + rank];
    __syncthreads();
    fft_batch(Y, 1, N2, logN2, tw, true);
    const double sc = 1.0 / n;
    for (int m2 = threadIdx.x; m2 < N2; m2 += blockDim.x) {
        const int v = C.v0 + rank + kClusterFFT * m2;
        z[3 * v + comp] = Y[m2].x * sc * dinv[v];
    }
    cl.sync();  // the other ranks may still read this rank's V
}

// Four-step pieces for n = N1 N2 (powers of two): index m = m1 + N1 m2, k = k2 + N2 k1.
// Pass A: for G consecutive m1, FFT over m2 of x[m1 + N1 m2], times exp(-/+ 2 pi i m1 k2 / n), in place.
__global__ void __launch_bounds__(kFFTThreads) k_four_a(double2 *__restrict__ buf, int n, int N1, int N2,
                                                        int logN2, int G, const double2 *__restrict__ tw, int inv)
{
    extern __shared__ double2 sa[];
    double2 *b = buf + (size_t)blockIdx.y * n;
    const int m1_0 = blockIdx.x * G;
    for (int t = threadIdx.x; t < G * N2; t += blockDim.x) {
        int m2 = t / G, g = t % G;  // consecutive threads read consecutive m1
        sa[g * N2 + m2] = b[(size_t)(m1_0 + g) + (size_t)N1 * m2];
    }
    __syncthreads();
    fft_batch(sa, G, N2, logN2, tw, inv != 0);
    for (int t = threadIdx.x; t < G * N2; t += blockDim.x) {
        int k2 = t / G, g = t % G;
        long long e = ((long long)(m1_0 + g) * k2) % n;
        double s, c;
        sincospi(2.0 * (double)e / (double)n, &s, &c);
        double2 w = make_double2(c, inv ? s : -s);
        b[(size_t)(m1_0 + g) + (size_t)N1 * k2] = cmul(sa[g * N2 + k2], w);
    }
}

// Pass C: for G consecutive k2, FFT over m1 of y[m1 + N1 k2] (contiguous), written to out[k2 + N2 k1].
__global__ void __launch_bounds__(kFFTThreads) k_four_c(const double2 *__restrict__ in, double2 *__restrict__ out,
                                                        int n, int N1, int N2, int logN1, int G,
                                                        const double2 *__restrict__ tw, int inv)
{
    extern __shared__ double2 sa[];
    const double2 *a = in + (size_t)blockIdx.y * n;
    double2 *o = out + (size_t)blockIdx.y * n;
    const int k2_0 = blockIdx.x * G;
    for (int t = threadIdx.x; t < G * N1; t += blockDim.x) {
        int g = t / N1, m1 = t % N1;
        sa[g * N1 + m1] = a[(size_t)m1 + (size_t)N1 * (k2_0 + g)];
    }
    __syncthreads();
    fft_batch(sa, G, N1, logN1, tw, inv != 0);
    for (int t = threadIdx.x; t < G * N1; t += blockDim.x) {
        int k1 = t / G, g = t % G;
        o[(size_t)(k2_0 + g) + (size_t)N2 * k1] = sa[g * N1 + k1];
    }
}

__global__ void k_four_prep(int v0, int n, const double *__restrict__ r, const double *__restrict__ dinv,
                            double2 *__restrict__ buf)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    double d = dinv[v0 + m];
    for (int c = 0; c < 3; ++c) buf[(size_t)c * n + m] = make_double2(r[3 * (v0 + m) + c] * d, 0.0);
}

__global__ void k_four_div(int n, const double *__restrict__ ilam, double2 *__restrict__ buf)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double f = ilam[k];
    for (int c = 0; c < 3; ++c) {
        double2 v = buf[(size_t)c * n + k];
        buf[(size_t)c * n + k] = make_double2(v.x * f, v.y * f);
    }
}

__global__ void k_four_out(int v0, int n, const double2 *__restrict__ buf, const double *__restrict__ dinv,
                           double *__restrict__ z)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    double d = dinv[v0 + m] / n;
    for (int c = 0; c < 3; ++c) z[3 * (v0 + m) + c] = buf[(size_t)c * n + m].x * d;
}

// dinv = exp(vlog) / sqrt(diag): the Jacobi scaling of the circulant, optionally rescaled per vertex
// (the learned preconditioner's log-scale; vlog may be NULL)
__global__ void k_dinv(int nV, const double *__restrict__ diag, const double *__restrict__ vlog,
                       double *__restrict__ dinv)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nV) dinv[i] = diag[i] > 0.0 ? (vlog ? exp(vlog[i]) : 1.0) / sqrt(diag[i]) : 0.0;
}

// ---------------------------------------------------------------------------------- set-up kernels

__global__ void k_twiddles(double2 *tw)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kMaxFFT / 2) return;
    double s, c;
    sincospi(-2.0 * k / (double)kMaxFFT, &s, &c);
    tw[k] = make_double2(c, s);
}

// Per-offset coefficients of the regular n-gon (unit circumradius, chord(j) = 2 sin(pi j / n)):
//   coef[m] = (w_m, w_m sin^2(pi m/n), w_m cos(2 pi m/n), w0_m),  m in [2, n-2]
__global__ void k_ngon_coef(int n, double p, double4 *coef)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    if (m < 2 || m > n - 2) {
        coef[m] = make_double4(0, 0, 0, 0);
        return;
    }
    double l = 2.0 * sinpi(1.0 / n);
    double w = 0.0, w0 = 0.0;
    for (int a = 0; a < 2; ++a)
        for (int b = m; b <= m + 1; ++b) {
            double ch = 2.0 * fabs(sinpi((double)(b - a) / n));
            double s0 = sinpi((double)(a + b - 1) / n), sm = sinpi((double)(a + b - 2 * m - 1) / n);
            w += pow(ch, -p);
            w0 += (s0 * s0 + sm * sm) * pow(ch, -(2.0 + p));
        }
    w *= 0.25 * l * l;
    w0 *= 0.25 * l * l;
    double sm2 = sinpi((double)m / n);
    coef[m] = make_double4(w, w * sm2 * sm2, w * cospi(2.0 * m / n), w0);
}

// Unnormalised lambda_k for k <= n/2 (lambda_{n-k} = lambda_k).  FP32 terms (all >= 0 in total),
// folded into FP64 every 64 terms.
__global__ void k_ngon_lambda(int n, const double4 *__restrict__ coef, double A0sum, double *__restrict__ lam)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > n / 2) return;
    double sk = sinpi((double)k / n), ck = cospi((double)k / n);
    double l = 2.0 * sinpi(1.0 / n);
    float fb = (float)(16.0 * sk * sk / (l * l)), fc = (float)(2.0 * ck * ck);
    double acc = 0.0;
    float part = 0.f;
    int r = (int)(((long long)k * 2) % n);  // k m mod n at m = 2
    const float inv_n = 1.0f / (float)n;
    for (int m = 2; m <= n - 2; ++m) {
        double4 cm = coef[m];
        float s = sinpif((float)r * inv_n);
        float S = s * s;
        part += fb * ((float)cm.y + (float)cm.z * S) + fc * (float)cm.w * S;
        r += k;
        if (r >= n) r -= n;
        if ((m & 63) == 63) {
            acc += (double)part;
            part = 0.f;
        }
    }
    acc += (double)part;
    lam[k] = acc;
    if (k > 0 && k < n - k) lam[n - k] = acc;
    (void)A0sum;
}

// Normalise by the diagonal (mean eigenvalue) and set lambda_0 := lambda_1.
__global__ void k_ngon_normalise(int n, double *lam)
{
    __shared__ double sh[256];
    double s = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) s += lam[k];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    double mean = sh[0] / n;
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) lam[k] /= mean;
    __syncthreads();
    if (threadIdx.x == 0) lam[0] = lam[1];
}

__global__ void k_chirp(int n, int M, double2 *__restrict__ chirp, double2 *__restrict__ b)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    if (j < n) {
        long long e = ((long long)j * j) % (2LL * n);
        double s, c;
        sincospi((double)e / n, &s, &c);
        chirp[j] = make_double2(c, s);
    }
    // circular filter b: b[j] = w_j for j < n, b[M - j] = w_j for 0 < j < n
    int jj = j < n ? j : (j > M - n ? M - j : -1);
    if (jj < 0) {
        b[j] = make_double2(0.0, 0.0);
    } else {
        long long e = ((long long)jj * jj) % (2LL * n);
        double s, c;
        sincospi((double)e / n, &s, &c);
        b[j] = make_double2(c, s);
    }
}

__global__ void __launch_bounds__(kFFTThreads) k_fft_inplace_global(double2 *data, int M, int logM,
                                                                    const double2 *__restrict__ tw)
{
    extern __shared__ double2 sa[];
    for (int i = threadIdx.x; i < M; i += blockDim.x) sa[i] = data[i];
    __syncthreads();
    fft_batch(sa, 1, M, logM, tw, false);
    for (int i = threadIdx.x; i < M; i += blockDim.x) data[i] = sa[i];
}

static int ilog2(int x)
{
    int l = 0;
    while ((1 << l) < x) ++l;
    return l;
}

static cudaError_t compute_symbol(Ctx &c, int n, double *dst, cudaStream_t s)
{
    double4 *coef = nullptr;
    TPE_CHECK(cudaMalloc(&coef, sizeof(double4) * n));
    k_ngon_coef<<<(n + 255) / 256, 256, 0, s>>>(n, c.kp.p, coef);
    k_ngon_lambda<<<(n / 2 + 1 + 127) / 128, 128, 0, s>>>(n, coef, 0.0, dst);
    k_ngon_normalise<<<1, 256, 0, s>>>(n, dst);
    c.launches += 3;
    TPE_CHECK(cudaGetLastError());
    TPE_CHECK(cudaStreamSynchronize(s));
    cudaFree(coef);
    return cudaSuccess;
}

cudaError_t spectral_setup(Ctx &c, cudaStream_t s)
{
    if (c.spec) return cudaSuccess;
    if (!c.spectral_ok) return cudaErrorNotSupported;
    c.spec = new SpecState();
    SpecState &S = *c.spec;
    // classify curves
    std::map<int, int> kinds;
    long long sym_total = 0, chirp_total = 0, bhat_total = 0;
    std::map<int, long long> chirp_of, bhat_of;
    size_t large_max = 0;
    std::vector<int> klist;
    for (int k = 0; k < c.nCurves; ++k) {
        int n = c.h_curve_n[k];
        SpecCurve C{};
        C.v0 = c.h_voff[k];
        C.n = n;
        bool pow2 = (n & (n - 1)) == 0;
        if (pow2 && n <= kMaxFFT) {
            C.kind = SK_POW2;
            C.M = n;
            C.logM = ilog2(n);
        } else if (!pow2 && 2 * n - 1 <= kMaxFFT) {
            C.kind = SK_BLUESTEIN;
            C.logM = ilog2(2 * n - 1);
            C.M = 1 << C.logM;
        } else if (pow2) {
            C.kind = SK_FOURSTEP;
            int lg = ilog2(n);
            C.logM = (lg + 1) / 2;
            C.M = 1 << C.logM;  // N1
            C.logN2 = lg - C.logM;
            C.N2 = 1 << C.logN2;
            large_max = std::max(large_max, (size_t)n);
        } else {
            delete c.spec;
            c.spec = nullptr;
            return cudaErrorNotSupported;  // non-power-of-two curves above 4096 vertices
        }
        if (!S.sym_of_n.count(n)) {
            S.sym_of_n[n] = sym_total;
            sym_total += n;
        }
        C.sym_off = S.sym_of_n[n];
        if (C.kind == SK_BLUESTEIN) {
            if (!chirp_of.count(n)) {
                chirp_of[n] = chirp_total;
                chirp_total += n;
                bhat_of[n] = bhat_total;
                bhat_total += C.M;
            }
            C.chirp_off = chirp_of[n];
            C.bhat_off = bhat_of[n];
        }
        // sampled frequencies of the Rayleigh-quotient correction: 1..8, then 14 log-spaced up to n/2
        {
            std::vector<int> ks;
            for (int k = 1; k <= 8; ++k) ks.push_back(k);
            for (int j = 0; j < 14; ++j) {
                double x = std::exp(std::log(9.0) + (std::log(std::max(9.0, n / 2.0)) - std::log(9.0)) * j / 13.0);
                ks.push_back((int)std::lround(x));
            }
            std::sort(ks.begin(), ks.end());
            ks.erase(std::unique(ks.begin(), ks.end()), ks.end());
            std::vector<int> kk;
            for (int k : ks)
                if (k >= 1 && k <= n / 2) kk.push_back(k);
            C.nk = (int)kk.size();
            S.max_nk = std::max(S.max_nk, C.nk);
            for (int j = 0; j < kMaxRQ; ++j) klist.push_back(j < C.nk ? kk[j] : 0);
        }
        S.curves.push_back(C);
        if (C.kind == SK_FOURSTEP)
            S.large_idx.push_back(k);
        else if (C.kind == SK_POW2 && n >= kClusterMinN)
            S.cluster_idx.push_back(k);
        else {
            S.small_idx.push_back(k);
            S.max_small_M = std::max(S.max_small_M, C.M);
        }
    }
    TPE_CHECK(cudaMalloc(&S.d_curves, sizeof(SpecCurve) * S.curves.size()));
    TPE_CHECK(cudaMemcpy(S.d_curves, S.curves.data(), sizeof(SpecCurve) * S.curves.size(), cudaMemcpyHostToDevice));
    TPE_CHECK(cudaMalloc(&S.d_cluster_idx, sizeof(int) * std::max<size_t>(1, S.cluster_idx.size())));
    if (!S.cluster_idx.empty())
        TPE_CHECK(cudaMemcpy(S.d_cluster_idx, S.cluster_idx.data(), sizeof(int) * S.cluster_idx.size(),
                             cudaMemcpyHostToDevice));
    TPE_CHECK(cudaMalloc(&S.d_small_idx, sizeof(int) * std::max<size_t>(1, S.small_idx.size())));
    if (!S.small_idx.empty())
        TPE_CHECK(cudaMemcpy(S.d_small_idx, S.small_idx.data(), sizeof(int) * S.small_idx.size(),
                             cudaMemcpyHostToDevice));
    TPE_CHECK(cudaMalloc(&S.d_sym, sizeof(double) * std::max<long long>(1, sym_total)));
    TPE_CHECK(cudaMalloc(&S.d_tw, sizeof(double2) * kMaxFFT / 2));
    TPE_CHECK(cudaMalloc(&S.d_chirp, sizeof(double2) * std::max<long long>(1, chirp_total)));
    TPE_CHECK(cudaMalloc(&S.d_bhat, sizeof(double2) * std::max<long long>(1, bhat_total)));
    TPE_CHECK(cudaMalloc(&S.d_dinv, sizeof(double) * c.nV));
    TPE_CHECK(cudaMalloc(&S.d_sym_rq, sizeof(double) * c.nV));
    TPE_CHECK(cudaMalloc(&S.d_ilam, sizeof(double) * c.nV));
    TPE_CHECK(cudaMalloc(&S.d_klist, sizeof(int) * klist.size()));
    TPE_CHECK(cudaMemcpy(S.d_klist, klist.data(), sizeof(int) * klist.size(), cudaMemcpyHostToDevice));
    TPE_CHECK(cudaMalloc(&S.d_rq, sizeof(double) * 2 * kMaxRQ * c.nCurves));
    {
        std::vector<int> vc(c.nV);
        for (int k = 0; k < c.nCurves; ++k)
            for (int v = c.h_voff[k]; v < c.h_voff[k + 1]; ++v) vc[v] = k;
        TPE_CHECK(cudaMalloc(&S.d_vcurve, sizeof(int) * c.nV));
        TPE_CHECK(cudaMemcpy(S.d_vcurve, vc.data(), sizeof(int) * c.nV, cudaMemcpyHostToDevice));
    }
    if (large_max) {
        TPE_CHECK(cudaMalloc(&S.d_buf0, sizeof(double2) * 3 * large_max));
        TPE_CHECK(cudaMalloc(&S.d_buf1, sizeof(double2) * 3 * large_max));
    }
    const size_t smem = sizeof(double2) * kMaxFFT;
    TPE_CHECK(cudaFuncSetAttribute(k_spec_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    TPE_CHECK(cudaFuncSetAttribute(k_four_a, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    TPE_CHECK(cudaFuncSetAttribute(k_four_c, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    TPE_CHECK(cudaFuncSetAttribute(k_fft_inplace_global, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_twiddles<<<(kMaxFFT / 2 + 255) / 256, 256, 0, s>>>(S.d_tw);
    c.launches++;
    for (auto &kv : S.sym_of_n) TPE_CHECK(compute_symbol(c, kv.first, S.d_sym + kv.second, s));
    for (auto &kv : chirp_of) {
        int n = kv.first, lg = ilog2(2 * n - 1), M = 1 << lg;
        k_chirp<<<(M + 255) / 256, 256, 0, s>>>(n, M, S.d_chirp + kv.second, S.d_bhat + bhat_of[n]);
        k_fft_inplace_global<<<1, kFFTThreads, sizeof(double2) * M, s>>>(S.d_bhat + bhat_of[n], M, lg, S.d_tw);
        c.launches += 2;
    }
    TPE_CHECK(cudaGetLastError());
    return cudaStreamSynchronize(s);
}

void spectral_free(Ctx &c)
{
    if (!c.spec) return;
    SpecState &S = *c.spec;
    void *p[] = {S.d_curves, S.d_small_idx, S.d_sym, S.d_tw, S.d_chirp, S.d_bhat, S.d_buf0, S.d_buf1, S.d_dinv,
                 S.d_sym_rq, S.d_klist, S.d_rq, S.d_vcurve, S.d_ilam, S.d_cluster_idx, S.d_probe};
    for (void *q : p)
        if (q) cudaFree(q);
    delete c.spec;
    c.spec = nullptr;
}

// The inverse symbols the applies currently divide by (refreshed after a Rayleigh-quotient set-up).
const double *spectral_ilam(Ctx &c, cudaStream_t s)
{
    if (!c.spec) return nullptr;
    SpecState &S = *c.spec;
    const double *rq = (c.prm.precond >= TP_PRECOND_SPECTRAL_RQ && S.rq_ready) ? S.d_sym_rq : nullptr;
    const int src = rq ? 1 : 0;
    if (S.ilam_src != src) {
        k_inv_symbol<<<c.nCurves, 256, 0, s>>>(S.d_curves, S.d_sym, rq, S.d_ilam);
        c.launches++;
        S.ilam_src = src;
    }
    return S.d_ilam;
}

cudaError_t spectral_apply(Ctx &c, const double *r, double *z, cudaStream_t s, const int *skip)
{
    if (!c.spec) return cudaErrorNotSupported;
    const double *il = spectral_ilam(c, s);
    return spectral_apply_ex(c, r, z, s, skip, c.d_diag, il, nullptr);
}

// z = W F^-1 diag(ilam) F W r per closed curve and component, W = diag(exp(vlog) / sqrt(diag)).
cudaError_t spectral_apply_ex(Ctx &c, const double *r, double *z, cudaStream_t s, const int *skip,
                              const double *diag, const double *ilam, const double *vlog)
{
    if (!c.spec) return cudaErrorNotSupported;
    SpecState &S = *c.spec;
    k_dinv<<<(c.nV + 255) / 256, 256, 0, s>>>(c.nV, diag, vlog, S.d_dinv);
    c.launches++;
    if (!S.cluster_idx.empty()) {
        k_spec_cluster<<<(int)S.cluster_idx.size() * 3 * kClusterFFT, kClusterThreads, 0, s>>>(
            S.d_curves, S.d_cluster_idx, r, z, S.d_dinv, S.d_tw, ilam, skip, c.independent);
        c.launches++;
    }
    if (!S.small_idx.empty()) {
        int M = S.max_small_M;
        k_spec_small<<<(int)S.small_idx.size() * 3, kFFTThreads, sizeof(double2) * M, s>>>(
            S.d_curves, S.d_small_idx, r, z, S.d_dinv, S.d_sym, S.d_chirp, S.d_bhat, S.d_tw, ilam, skip,
            c.independent);
        c.launches++;
    }
    for (int k : S.large_idx) {
        const SpecCurve &C = S.curves[k];
        int n = C.n, N1 = C.M, N2 = C.N2;
        int nb = (n + 255) / 256;
        int GA = std::max(1, kMaxFFT / N2), GC = std::max(1, kMaxFFT / N1);
        GA = std::min(GA, N1);
        GC = std::min(GC, N2);
        size_t smA = sizeof(double2) * GA * N2, smC = sizeof(double2) * GC * N1;
        k_four_prep<<<nb, 256, 0, s>>>(C.v0, n, r, S.d_dinv, S.d_buf0);
        k_four_a<<<dim3(N1 / GA, 3), kFFTThreads, smA, s>>>(S.d_buf0, n, N1, N2, C.logN2, GA, S.d_tw, 0);
        k_four_c<<<dim3(N2 / GC, 3), kFFTThreads, smC, s>>>(S.d_buf0, S.d_buf1, n, N1, N2, C.logM, GC, S.d_tw, 0);
        k_four_div<<<nb, 256, 0, s>>>(n, ilam + C.v0, S.d_buf1);
        k_four_a<<<dim3(N1 / GA, 3), kFFTThreads, smA, s>>>(S.d_buf1, n, N1, N2, C.logN2, GA, S.d_tw, 1);
        k_four_c<<<dim3(N2 / GC, 3), kFFTThreads, smC, s>>>(S.d_buf1, S.d_buf0, n, N1, N2, C.logM, GC, S.d_tw, 1);
        k_four_out<<<nb, 256, 0, s>>>(C.v0, n, S.d_buf0, S.d_dinv, z);
        c.launches += 7;
    }
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------------- Rayleigh-quotient symbol
//
// T. Chan's optimal circulant approximation of S = D^-1/2 A D^-1/2 has the eigenvalues
// lambda_opt(k) = f_k^H S f_k / n (the Rayleigh quotients of S on the Fourier modes).  They are
// sampled at <= 24 frequencies per curve with the multi-field apply (cos and sin probes scaled by
// D^-1/2), the ratio rho(k) = lambda_opt(k) / lambda_ngon(k) is interpolated linearly in
// (log k, log rho), and the preconditioner divides by lambda_ngon(k) rho(k).  On a regular polygon
// rho = 1.  On knotted curves the low modes are far stiffer than the polygon's (rho up to ~1e4 at
// k = 1), which is what the polygon symbol misses.

// probe batch b: component q of vertex v holds vector t = 3 b + q = (frequency index t/2, cos or sin)
__global__ void k_rq_probe(int nV, int b, const SpecCurve *__restrict__ curves, const int *__restrict__ vcurve,
                           const int *__restrict__ klist, const double *__restrict__ diag, double *__restrict__ y)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nV) return;
    int c = vcurve[v];
    const SpecCurve C = curves[c];
    int i = v - C.v0;
    double dv = diag[v] > 0.0 ? 1.0 / sqrt(diag[v]) : 0.0;
    for (int q = 0; q < 3; ++q) {
        int t = 3 * b + q, kk = t >> 1;
        double val = 0.0;
        if (kk < C.nk) {
            long long e = ((long long)klist[c * kMaxRQ + kk] * i) % C.n;
            double sn, cs;
            sincospi(2.0 * (double)e / C.n, &sn, &cs);
            val = ((t & 1) ? sn : cs) * dv;
        }
        y[3 * v + q] = val;
    }
}

// rq[c][t] = sum over the curve of y . Ay for the three probes of batch b (one block per curve)
__global__ void k_rq_reduce(int b, const SpecCurve *__restrict__ curves, const double *__restrict__ y,
                            const double *__restrict__ Ay, double *__restrict__ rq)
{
    const SpecCurve C = curves[blockIdx.x];
    __shared__ double sh[3][256];
    double s[3] = {0, 0, 0};
    for (int i = threadIdx.x; i < C.n; i += blockDim.x) {
        int v = C.v0 + i;
        for (int q = 0; q < 3; ++q) s[q] += y[3 * v + q] * Ay[3 * v + q];
    }
    for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] = s[q];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 3; ++q) {
            int t = 3 * b + q;
            if (t < 2 * kMaxRQ) rq[blockIdx.x * 2 * kMaxRQ + t] = sh[q][0];
        }
}

// corrected symbol of every curve (one block per curve)
__global__ void k_rq_symbol(const SpecCurve *__restrict__ curves, const int *__restrict__ klist,
                            const double *__restrict__ rq, const double *__restrict__ sym,
                            double *__restrict__ sym_rq)
{
    const SpecCurve C = curves[blockIdx.x];
    const double *lam = sym + C.sym_off;
    __shared__ double lk[kMaxRQ], lr[kMaxRQ];
    if (threadIdx.x < C.nk) {
        int k = klist[blockIdx.x * kMaxRQ + threadIdx.x];
        double q = (rq[blockIdx.x * 2 * kMaxRQ + 2 * threadIdx.x] + rq[blockIdx.x * 2 * kMaxRQ + 2 * threadIdx.x + 1]) / C.n;
        double rho = (q > 0.0 && lam[k] > 0.0) ? q / lam[k] : 1.0;
        lk[threadIdx.x] = log((double)k);
        lr[threadIdx.x] = log(rho);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < C.n; k += blockDim.x) {
        int kf = k <= C.n / 2 ? k : C.n - k;  // lambda_{n-k} = lambda_k
        double r;
        if (C.nk == 0) {
            r = 0.0;
        } else if (kf <= 1) {
            r = lr[0];
        } else {
            double x = log((double)kf);
            int j = 0;
            while (j + 1 < C.nk && lk[j + 1] < x) ++j;
            if (j + 1 >= C.nk)
                r = lr[C.nk - 1];
            else {
                double f = (x - lk[j]) / (lk[j + 1] - lk[j]);
                r = lr[j] + f * (lr[j + 1] - lr[j]);
            }
        }
        int kl = (k == 0) ? 1 : k;  // lambda_0 := corrected lambda_1
        sym_rq[C.v0 + k] = lam[kl] * exp(r);
    }
}

// Builds the corrected symbols of the curve `gamma_geom` (geometry slot `which`); needs diag(A) in
// c.d_diag.  The probe fields and their products live in a scratch of 2 x batches x 3 nV doubles.
cudaError_t spectral_rq_setup(Ctx &c, const double *gamma_geom, int which, cudaStream_t s)
{
    if (!c.spec) return cudaErrorNotSupported;
    SpecState &S = *c.spec;
    const int nb = (c.nV + 255) / 256;
    const int nbatch = (2 * S.max_nk + 2) / 3;
    // every batch of three probes is one vector field: one multi-field apply serves all of them
    const size_t nv3 = 3 * (size_t)c.nV;
    if (!S.d_probe) TPE_CHECK(cudaMalloc(&S.d_probe, sizeof(double) * 2 * std::max(1, nbatch) * nv3));
    double *Y = S.d_probe, *AY = S.d_probe + (size_t)nbatch * nv3;
    for (int b = 0; b < nbatch; ++b) {
        k_rq_probe<<<nb, 256, 0, s>>>(c.nV, b, S.d_curves, S.d_vcurve, S.d_klist, c.d_diag, Y + b * nv3);
        c.launches++;
    }
    TPE_CHECK(pair_apply_multi(c, gamma_geom, which, Y, AY, nbatch, s));
    for (int b = 0; b < nbatch; ++b) {
        k_rq_reduce<<<c.nCurves, 256, 0, s>>>(b, S.d_curves, Y + b * nv3, AY + b * nv3, S.d_rq);
        c.launches++;
    }
    k_rq_symbol<<<c.nCurves, 256, 0, s>>>(S.d_curves, S.d_klist, S.d_rq, S.d_sym, S.d_sym_rq);
    c.launches++;
    S.rq_ready = 1;
    S.ilam_src = -1;  // the next apply refreshes 1 / symbol
    return cudaGetLastError();
}

cudaError_t spectral_symbol_copy(Ctx &c, int rq, double *out, cudaStream_t s)
{
    if (!c.spec) return cudaErrorNotSupported;
    SpecState &S = *c.spec;
    if (rq) return cudaMemcpyAsync(out, S.d_sym_rq, sizeof(double) * c.nV, cudaMemcpyDeviceToDevice, s);
    for (int k = 0; k < c.nCurves; ++k) {
        const SpecCurve &C = S.curves[k];
        TPE_CHECK(cudaMemcpyAsync(out + C.v0, S.d_sym + C.sym_off, sizeof(double) * C.n, cudaMemcpyDeviceToDevice, s));
    }
    return cudaSuccess;
}

cudaError_t spectral_symbol_of(Ctx &c, int n, double *lam, cudaStream_t s)
{
    return compute_symbol(c, n, lam, s);
}

}  // namespace tpe

extern "C" TPE_API tp_status tp_spectral_symbol(tp_ctx *ctx, int n, double *lam, tp_stream stream)
{
    if (!ctx || !lam || n < 4) return TP_ERR_INVALID_ARG;
    cudaError_t e = tpe::spectral_symbol_of(ctx->c, n, lam, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        ctx->c.err = std::string("tp_spectral_symbol: ") + cudaGetErrorString(e);
        return TP_ERR_CUDA;
    }
    return TP_OK;
}
