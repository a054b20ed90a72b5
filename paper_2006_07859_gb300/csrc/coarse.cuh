// Coarse-space state shared by the coarse-space set-up and application (coarse.cu) and the pair pass
// that assembles the coarse columns A Z (coarse_az.cu).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "tpe_internal.cuh"

namespace tpe {

constexpr int kMaxCoarse = 8192;
constexpr int kSmemCoarse = 128;  // coarse spaces up to this size factor in shared memory, larger ones in global
constexpr int kFactorSmem = (kSmemCoarse - 1) * (kSmemCoarse - 1) * (int)sizeof(double);  // 127^2 doubles
constexpr int kMinPassCoarse = 8;  // coarse spaces from this size on are assembled by the A Z pass

struct CoarseCurve {
    int v0, n, m;  // hats j = 0 .. m-2 are the basis
    int e0;        // first edge: edge e0 + i joins local vertices i and (i + 1) mod n
    long long aoff, woff;  // offsets of the factor [(m-1)^2] and of the coarse vectors [(m-1) x 3]
    long long zoff;        // offset of the curve's A Z columns [(m-1)][n]
};

}  // namespace tpe

struct tpe::CoarseState {
    std::vector<CoarseCurve> curves;
    CoarseCurve *d_curves = nullptr;
    int *d_vcurve = nullptr;
    double *d_L = nullptr;   // per curve: (Z^T A Z)^-1, row-major (m-1) x (m-1)
    double *d_Li = nullptr;  // set-up scratch: L^-1 of the Cholesky factor, same layout
    double *d_W = nullptr;   // set-up scratch: tiled Cholesky work array (coarse spaces above 128 hats)
    double *d_w = nullptr;  // coarse vectors: restriction Z^T r
    double *d_w2 = nullptr; // coarse vectors: (Z^T A Z)^-1 Z^T r
    double *d_w3 = nullptr, *d_w4 = nullptr;  // balancing form: (A Z)^T y and its coarse solve
    double *d_AZ = nullptr;  // per curve the columns A z_j, [(m-1)][n] (column-major): kept for the
                             // balancing form, assembled by the A Z pass
    double *d_r2 = nullptr;  // balancing form: r - A Q r, [nV][3]
    int max_m = 0;
    int ready = 0;
    int balanced = 0;        // the AZ columns are kept (every problem is one curve)
    // A Z pass (every curve's coarse space has at least kMinPassCoarse hats)
    int az_pass = 0;
    int2 *d_items = nullptr;  // (curve, first local edge) of each block of 128 target rows
    int n_items = 0;
    int *d_hbase = nullptr;   // [nE] first hat touching each edge (unwrapped: 0 .. m-1)
    URecF *d_hatF = nullptr;  // [nE] hat slopes and means of each edge's three hats (FP32 contexts)
    URecD *d_hatD = nullptr;  // [nE] the same in FP64 (FP64 contexts)
};

namespace tpe {

// hat j of a curve with n vertices and m hats at local vertex i (periodic)
__device__ __forceinline__ double hat(int i, int j, int n, int m)
{
    double t = (double)i * m / n;
    double d = fabs(t - j);
    d = fmin(d, m - d);
    return fmax(0.0, 1.0 - d);
}

// local index range [lo, lo + len) (mod n) covering the support of hat j
__device__ __forceinline__ void hat_support(int j, int n, int m, int &lo, int &len)
{
    lo = (int)floor((double)(j - 1) * n / m) - 1;
    len = (int)ceil(2.0 * n / m) + 3;
    if (len > n) {
        lo = 0;
        len = n;
    }
}

cudaError_t coarse_az_pass(Ctx &c, int which, cudaStream_t s);
cudaError_t coarse_factor_tiled(Ctx &c, int mm, double *E, double *W, double *Y, cudaStream_t s);

}  // namespace tpe
