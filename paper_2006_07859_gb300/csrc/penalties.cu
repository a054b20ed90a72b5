// Penalties of Sec. 8.1 added to the energy and differential of the descent step:
//   w_length      sum_I l_I                                   (total length)
//   w_length_diff sum over vertices of degree 2 of (l_I - l_J)^2 (I, J the vertex's two edges)
//   w_field       sum_I l_I |T_I x X(x_I)|^2,  X(x) = u / |u|, u = M x + b (X = 0 where u = 0)
// Chain rule: d l_I / d g_i2 = T_I = -d l_I / d g_i1, d x_I / d g_ia = Id / 2; with e = g_i2 - g_i1 the
// field term of an edge is l - (e.X)^2 / l, so d/de = T - 2 (T.X) X + (T.X)^2 T and
// d/dx = -2 (T.X) M^T (e - (e.X) X) / |u|.
// Three passes, all deterministic: per-vertex length-difference weights, per-edge gradient
// contributions at both endpoints (and per-edge energies), and a vertex gather over the incidence lists.
#include <cuda_runtime.h>

#include <algorithm>

#include "tpe_internal.cuh"

namespace tpe {

#define TPE_CHECK(x)                      \
    do {                                  \
        cudaError_t e_ = (x);             \
        if (e_ != cudaSuccess) return e_; \
    } while (0)

struct PenState {
    tp_penalties p{};
    double *d_wv = nullptr;  // [nV] 2 w_diff (l_first - l_second) at degree-2 vertices, else 0
    double *d_ev = nullptr;  // [nV] vertex energies
    double *d_ee = nullptr;  // [nE] edge energies
    double *d_ge = nullptr;  // [nE][6] gradient contributions at i1, i2
    double *d_E = nullptr;   // [nProb] scratch sums
};

// first / second incident edge of a degree-2 vertex, in incidence order
__global__ void k_pen_vertex(int nV, const int *__restrict__ inc_ptr, const int *__restrict__ inc,
                             const double *__restrict__ ell, double w_diff, double *__restrict__ wv,
                             double *__restrict__ ev)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nV) return;
    double w = 0.0, e = 0.0;
    if (inc_ptr[v + 1] - inc_ptr[v] == 2) {
        const double dl = ell[inc[inc_ptr[v]] >> 1] - ell[inc[inc_ptr[v] + 1] >> 1];
        w = 2.0 * w_diff * dl;
        e = w_diff * dl * dl;
    }
    wv[v] = w;
    ev[v] = e;
}

// dE / d l_I from the vertex weights of I's two endpoints (+ when I is the vertex's first incident edge)
__device__ __forceinline__ double dl_of_vertex(int v, int I, const int *inc_ptr, const int *inc, const double *wv)
{
    if (inc_ptr[v + 1] - inc_ptr[v] != 2) return 0.0;
    return (inc[inc_ptr[v]] >> 1) == I ? wv[v] : -wv[v];
}

__global__ void k_pen_edge(int nE, const int *__restrict__ edges, const int *__restrict__ inc_ptr,
                           const int *__restrict__ inc, const double *__restrict__ ell, const double *__restrict__ T,
                           const double *__restrict__ x, const double *__restrict__ wv, const tp_penalties p,
                           double *__restrict__ ee, double *__restrict__ ge)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nE) return;
    const int a = edges[2 * I], b = edges[2 * I + 1];
    const double l = ell[I];
    const double t[3] = {T[3 * I], T[3 * I + 1], T[3 * I + 2]};
    // a vertex shared by both ends (a one-edge loop) would count twice; edges have distinct ends
    const double dl = p.w_length + dl_of_vertex(a, I, inc_ptr, inc, wv) + dl_of_vertex(b, I, inc_ptr, inc, wv);
    double g1[3], g2[3];
    for (int k = 0; k < 3; ++k) {
        g1[k] = -dl * t[k];
        g2[k] = dl * t[k];
    }
    double e = p.w_length * l;
    if (p.w_field != 0.0) {
        const double xi[3] = {x[3 * I], x[3 * I + 1], x[3 * I + 2]};
        double u[3];
        for (int r = 0; r < 3; ++r) u[r] = p.field_M[3 * r] * xi[0] + p.field_M[3 * r + 1] * xi[1] + p.field_M[3 * r + 2] * xi[2] + p.field_b[r];
        const double nu = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        if (nu > 0.0) {
            const double X[3] = {u[0] / nu, u[1] / nu, u[2] / nu};
            const double tx = t[0] * X[0] + t[1] * X[1] + t[2] * X[2];
            e += p.w_field * l * (1.0 - tx * tx);
            double de[3], w[3], dx[3];
            for (int k = 0; k < 3; ++k) {
                de[k] = t[k] - 2.0 * tx * X[k] + tx * tx * t[k];
                w[k] = l * (t[k] - tx * X[k]);  // e - (e.X) X
            }
            for (int k = 0; k < 3; ++k)
                dx[k] = -2.0 * tx * (p.field_M[k] * w[0] + p.field_M[3 + k] * w[1] + p.field_M[6 + k] * w[2]) / nu;
            for (int k = 0; k < 3; ++k) {
                g1[k] += p.w_field * (-de[k] + 0.5 * dx[k]);
                g2[k] += p.w_field * (de[k] + 0.5 * dx[k]);
            }
        }
    }
    ee[I] = e;
    for (int k = 0; k < 3; ++k) {
        ge[6 * (size_t)I + k] = g1[k];
        ge[6 * (size_t)I + 3 + k] = g2[k];
    }
}

__global__ void k_pen_gather(int nV, const int *__restrict__ inc_ptr, const int *__restrict__ inc,
                             const double *__restrict__ ge, double *__restrict__ dE)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nV) return;
    double s[3] = {0.0, 0.0, 0.0};
    for (int k = inc_ptr[v]; k < inc_ptr[v + 1]; ++k) {
        const int I = inc[k] >> 1, slot = inc[k] & 1;  // slot 1: v is i2
        for (int c = 0; c < 3; ++c) s[c] += ge[6 * (size_t)I + 3 * slot + c];
    }
    for (int c = 0; c < 3; ++c) dE[3 * (size_t)v + c] += s[c];
}

void penalties_free(Ctx &c)
{
    if (!c.pen) return;
    PenState &P = *c.pen;
    void *ptrs[] = {P.d_wv, P.d_ev, P.d_ee, P.d_ge, P.d_E};
    for (void *q : ptrs) cudaFree(q);
    delete c.pen;
    c.pen = nullptr;
}

bool penalties_active(const Ctx &c)
{
    return c.pen && (c.pen->p.w_length != 0.0 || c.pen->p.w_length_diff != 0.0 || c.pen->p.w_field != 0.0);
}

cudaError_t penalties_set(Ctx &c, const tp_penalties *p)
{
    if (!p) {
        penalties_free(c);
        return cudaSuccess;
    }
    if (!c.pen) {
        c.pen = new PenState();
        PenState &P = *c.pen;
        TPE_CHECK(cudaMalloc(&P.d_wv, sizeof(double) * std::max(1, c.nV)));
        TPE_CHECK(cudaMalloc(&P.d_ev, sizeof(double) * std::max(1, c.nV)));
        TPE_CHECK(cudaMalloc(&P.d_ee, sizeof(double) * std::max(1, c.nE)));
        TPE_CHECK(cudaMalloc(&P.d_ge, sizeof(double) * 6 * std::max(1, c.nE)));
        TPE_CHECK(cudaMalloc(&P.d_E, sizeof(double) * std::max(1, c.nProb)));
    }
    c.pen->p = *p;
    return cudaSuccess;
}

// E[q] += penalty energy of problem q (E may be null), dE += penalty gradient (dE may be null), for the
// geometry `which` (its edge quantities must be current).
cudaError_t penalties_add(Ctx &c, int which, double *E, double *dE, cudaStream_t s)
{
    if (!penalties_active(c)) return cudaSuccess;
    PenState &P = *c.pen;
    k_pen_vertex<<<(c.nV + 255) / 256, 256, 0, s>>>(c.nV, c.d_inc_ptr, c.d_inc, c.d_ellw[which], P.p.w_length_diff,
                                                    P.d_wv, P.d_ev);
    k_pen_edge<<<(c.nE + 255) / 256, 256, 0, s>>>(c.nE, c.d_edges, c.d_inc_ptr, c.d_inc, c.d_ellw[which],
                                                  c.d_Tw[which], c.d_xw[which], P.d_wv, P.p, P.d_ee, P.d_ge);
    c.launches += 2;
    TPE_CHECK(cudaGetLastError());
    if (dE) {
        k_pen_gather<<<(c.nV + 255) / 256, 256, 0, s>>>(c.nV, c.d_inc_ptr, c.d_inc, P.d_ge, dE);
        c.launches++;
        TPE_CHECK(cudaGetLastError());
    }
    if (E) {
        TPE_CHECK(sum_problems(c, P.d_ee, 0, E, s, 1));
        TPE_CHECK(sum_problems(c, P.d_ev, 1, E, s, 1));
    }
    return cudaSuccess;
}

}  // namespace tpe
