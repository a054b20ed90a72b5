// The coarse columns A z_j of the two-level preconditioners in one pair pass (this library's design; the
// paper has no coarse space).
//
// Probing assembles A Z with (m - 1) / 3 applies of the pair kernel, one hat per component.  On a
// closed curve in chain order (edge e0 + i joins local vertices i and i + 1 mod n) the hats have a
// structure that a single pass can use.  Edge J = (j, j + 1) lies in at most three consecutive hats
// f_J, f_J + 1, f_J + 2 with f_J = floor(j m / n), because m <= n / 4, and f_J never decreases along
// the curve.  For hat z, write du_J = (z(j + 1) - z(j)) / l_J and ub_J = (z(j) + z(j + 1)) / 2; both are
// zero when J is outside the hat.  In the exact difference form of the apply (the Gram weights W, W0
// and the tangent gap 1 - t_IJ of the Sobolev inner product, Secs. 5.2.2-5.2.3), a pair (I, J)
// contributes, for every hat z:
//   A1 += W [(du_I - du_J) + (1 - t_IJ) du_J],   A2 += W0 (ub_I - ub_J).
// Only the row's own hats (f_I .. f_I + 2) and the source's hats get a non-zero term.  On the source's
// other hats it reduces to -W t_IJ du_J and -W0 ub_J.
//
// A block of 128 target rows streams every source edge of its curve in order.  The own-column sums
// stay in registers for the whole pass.  The other columns sit in a window of three that moves with
// f_J, and a column leaves the window once f_J has passed it.  Every (column, row) value is produced
// once and turned into vertex rows with the apply gather's scaling: -/+ A1 / 2 to the row's two
// endpoints and l_I A2 / 8 to both.  It is then added to A Z.  Each entry receives exactly two
// additions onto zero, one from each of its two edges, so the result does not depend on their order.
// The pass evaluates every ordered pair once.  That is twice the pairs of one symmetric apply, where
// probing needs (m - 1) / 3 applies; with hats of a few hundred edges the pass is over a hundred
// times cheaper.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "coarse.cuh"
#include "pair_device.cuh"

namespace tpe {

#define TPE_CHECK(x)                      \
    do {                                  \
        cudaError_t e_ = (x);             \
        if (e_ != cudaSuccess) return e_; \
    } while (0)

// Per edge: its first hat f (unwrapped, 0 .. m - 1) and du, ub of the hats f, f + 1, f + 2, in the
// layout of the apply's per-edge vector records (hat q in component q; double-float in URecF).
__global__ void k_hat_recs(int nE, const int *__restrict__ E, const double *__restrict__ ell,
                           const CoarseCurve *__restrict__ cc, const int *__restrict__ vcurve, int *__restrict__ hbase,
                           URecF *__restrict__ uf, URecD *__restrict__ ud)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nE) return;
    const CoarseCurve C = cc[vcurve[E[2 * I]]];
    const int j = I - C.e0, n = C.n, m = C.m;
    const int f = (int)(((long long)j * m) / n);
    const int a = j, b = (j + 1) % n;
    const double l = ell[I];
    double du[3], ub[3];
    for (int q = 0; q < 3; ++q) {
        const int k = (f + q) % m;
        const double za = hat(a, k, n, m), zb = hat(b, k, n, m);
        du[q] = (zb - za) / l;
        ub[q] = 0.5 * (za + zb);
    }
    hbase[I] = f;
    if (uf) {
        float dh[3], uh[3], dl[3], ul[3];
        for (int q = 0; q < 3; ++q) {
            dh[q] = (float)du[q];
            uh[q] = (float)ub[q];
            dl[q] = (float)(du[q] - (double)dh[q]);
            ul[q] = (float)(ub[q] - (double)uh[q]);
        }
        URecF r;
        r.a = make_float4(dh[0], dh[1], dh[2], uh[0]);
        r.b = make_float4(uh[1], uh[2], dl[0], dl[1]);
        r.c = make_float4(dl[2], ul[0], ul[1], ul[2]);
        uf[I] = r;
    }
    if (ud) {
        URecD r;
        r.du0 = make_double2(du[0], du[1]);
        r.du1 = make_double2(du[2], 0.0);
        r.ub0 = make_double2(ub[0], ub[1]);
        r.ub1 = make_double2(ub[2], 0.0);
        ud[I] = r;
    }
}

struct AzArgs {
    const int2 *items;
    const CoarseCurve *cc;
    const RecF *recF;
    const RecLo *recLo;
    const RecD *recD;
    const URecF *hatF;
    const URecD *hatD;
    const int *hbase;
    const double *ell;  // FP64 edge lengths
    double *AZ;
    KernelParams kp;
};

// component q of a V3 without dynamic indexing (q is a compile-time constant after unrolling)
template <class R>
__device__ __forceinline__ R comp(const V3<R> &v, int q)
{
    return q == 0 ? v.x : (q == 1 ? v.y : v.z);
}

// acc += x: compensated (Kahan) in FP32, plain in FP64
template <class R>
__device__ __forceinline__ void az_add(R &acc, R &c, R x)
{
    if constexpr (sizeof(R) == 4)
        kahan_add(acc, c, x);
    else
        acc += x;
}

template <bool D, bool FAST>
__global__ void __launch_bounds__(kThreads, 2) k_coarse_az(const AzArgs a)
{
    constexpr int PREC = D ? P64 : PMIX;
    using R = typename RealOf<PREC>::type;
    __shared__ Tile<PREC, false> tl;
    __shared__ typename std::conditional<D, URecD, URecF>::type th[kTile];
    __shared__ int tf[kTile];
    const int2 it = a.items[blockIdx.x];
    const CoarseCurve C = a.cc[it.x];
    const int n = C.n, m = C.m, e0 = C.e0;
    const int jl = it.y + threadIdx.x;
    const bool valid = jl < n;
    const int I = e0 + min(jl, n - 1);
    Tgt<R> t;
    load_target<PREC>(t, I, a.recF, a.recLo, a.recD);
    UVal<R> tu;  // the row's own hats f_I .. f_I + 2
    load_uval<PREC>(tu, a.hatF, a.hatD, I);
    const int fI = a.hbase[I];
    const R pp = (R)a.kp.p;
    // own columns: tile sums (compensated in FP32) folded into FP64 every 4 tiles
    R o1[3], o2[3], c1[3], c2[3];
    double O1[3] = {0, 0, 0}, O2[3] = {0, 0, 0};
    // window columns wbase .. wbase + 2 (slot q <-> the source's hat f_J + q)
    R w1[3], w2[3], d1[3], d2[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) o1[q] = o2[q] = c1[q] = c2[q] = w1[q] = w2[q] = d1[q] = d2[q] = (R)0;
    int wbase = 0;
    double st1 = 0.0, st2 = 0.0;  // column 0's sums from the start of the curve (it also takes the end)
    const double lI = a.ell[I];
    double *az = a.AZ + C.zoff;
    const int ia = min(jl, n - 1), ib = (ia + 1) % n;
    auto own_col = [&](int col) { return col == fI % m || col == (fI + 1) % m || col == (fI + 2) % m; };
    auto emit = [&](int col, double v1, double v2) {
        if (!valid) return;
        const double h = 0.5 * v1, u = 0.125 * lI * v2;
        atomicAdd(az + (long long)col * n + ia, u - h);
        atomicAdd(az + (long long)col * n + ib, u + h);
    };
    // unwrapped column c in [0, m + 1] leaves the window with sums (v1, v2)
    auto flush = [&](int c, double v1, double v2) {
        const int col = c % m;
        if (col == m - 1 || c > m || own_col(col)) return;  // dropped hat / no content / the own sums carry it
        if (c == 0) {
            st1 = v1;
            st2 = v2;
            return;
        }
        if (c == m) {
            v1 += st1;
            v2 += st2;
        }
        emit(col, v1, v2);
    };
    int tiles = 0;
    for (int s0 = 0; s0 < n; s0 += kTile) {
        const int cnt = min(kTile, n - s0);
        __syncthreads();
        if (threadIdx.x < cnt) {
            const int J = e0 + s0 + threadIdx.x;
            if constexpr (D) {
                tl.r[threadIdx.x] = a.recD[J];
                th[threadIdx.x] = a.hatD[J];
            } else {
                tl.r[threadIdx.x] = a.recF[J];
                tl.lo[threadIdx.x] = a.recLo[J];
                th[threadIdx.x] = a.hatF[J];
            }
            tf[threadIdx.x] = a.hbase[J];
        }
        __syncthreads();
        for (int j = 0; j < cnt; ++j) {
            const int fJ = tf[j];
            if (fJ != wbase) {  // the same for every thread: f_J advanced by one
                flush(wbase, (double)w1[0] - (double)d1[0], (double)w2[0] - (double)d2[0]);
                w1[0] = w1[1], w2[0] = w2[1], d1[0] = d1[1], d2[0] = d2[1];
                w1[1] = w1[2], w2[1] = w2[2], d1[1] = d1[2], d2[1] = d2[2];
                w1[2] = w2[2] = d1[2] = d2[2] = (R)0;
                wbase = fJ;
            }
            Src<PREC> s;
            load_source<PREC, false>(s, tl, j);
            UVal<R> su;
            if constexpr (D) {
                const URecD u = th[j];
                su.dh = {u.du0.x, u.du0.y, u.du1.x};
                su.uh = {u.ub0.x, u.ub0.y, u.ub1.x};
                su.dl = su.ul = {0, 0, 0};
            } else {
                const float4 x = th[j].a, y = th[j].b, z = th[j].c;
                su.dh = {x.x, x.y, x.z};
                su.uh = {x.w, y.x, y.y};
                su.dl = {y.z, y.w, z.x};
                su.ul = {z.y, z.z, z.w};
            }
            const bool keep = (s.j1 != t.i1) & (s.j1 != t.i2) & (s.j2 != t.i1) & (s.j2 != t.i2);
            R W, W0, d211;
            gram_weights<FAST, !D>(t, s, keep, pp, W, W0, d211);
            const R omt = tangent_gap<!D>(t, s);
            const R wt = W * (omt - (R)1);  // -W t_IJ
            int dl = fJ - fI;               // source hats relative to the row's, periodic
            if (2 * dl > m) dl -= m;
            else if (2 * dl < -m) dl += m;
            if (dl >= -2 && dl <= 2) {
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                    const int q = p - dl;
                    const bool in = q >= 0 && q <= 2;
                    const R jdh = in ? comp(su.dh, q) : (R)0, jdl = in ? comp(su.dl, q) : (R)0;
                    const R juh = in ? comp(su.uh, q) : (R)0, jul = in ? comp(su.ul, q) : (R)0;
                    const R dd = (comp(tu.dh, p) - jdh) + (comp(tu.dl, p) - jdl);
                    const R db = (comp(tu.uh, p) - juh) + (comp(tu.ul, p) - jul);
                    az_add(o1[p], c1[p], W * (dd + omt * jdh));
                    az_add(o2[p], c2[p], W0 * db);
                }
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const int p = q + dl;
                    if (p < 0 || p > 2) {
                        az_add(w1[q], d1[q], wt * comp(su.dh, q));
                        az_add(w2[q], d2[q], -W0 * comp(su.uh, q));
                    }
                }
            } else {
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                    az_add(o1[p], c1[p], W * comp(tu.dh, p));
                    az_add(o2[p], c2[p], W0 * comp(tu.uh, p));
                }
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    az_add(w1[q], d1[q], wt * comp(su.dh, q));
                    az_add(w2[q], d2[q], -W0 * comp(su.uh, q));
                }
            }
        }
        if (++tiles == 4 || s0 + kTile >= n) {
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                O1[p] += (double)o1[p] - (double)c1[p];
                O2[p] += (double)o2[p] - (double)c2[p];
                o1[p] = o2[p] = c1[p] = c2[p] = (R)0;
            }
            tiles = 0;
        }
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) flush(wbase + q, (double)w1[q] - (double)d1[q], (double)w2[q] - (double)d2[q]);
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const int col = (fI + p) % m;
        if (col != m - 1) emit(col, O1[p], O2[p]);
    }
}

// E[j][l] = z_j^T (A z_l) over the support of hat j: one block per (curve, j), one warp per column l
__global__ void k_coarse_gram_az(const CoarseCurve *__restrict__ cc, const double *__restrict__ AZ,
                                 double *__restrict__ L)
{
    const CoarseCurve C = cc[blockIdx.x];
    const int j = blockIdx.y, mm = C.m - 1;
    if (j >= mm) return;
    int lo, len;
    hat_support(j, C.n, C.m, lo, len);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int l = warp; l < mm; l += nw) {
        const double *col = AZ + C.zoff + (long long)l * C.n;
        double s = 0.0;
        for (int k = lane; k < len; k += 32) {
            const int i = ((lo + k) % C.n + C.n) % C.n;
            s += hat(i, j, C.n, C.m) * col[i];
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) L[C.aoff + (long long)j * mm + l] = s;
    }
}

// A Z of every curve (geometry slot `which`, records already built) into S.d_AZ and Z^T A Z into S.d_L.
cudaError_t coarse_az_pass(Ctx &c, int which, cudaStream_t s)
{
    CoarseState &S = *c.coarse;
    if (!S.az_pass || c.nE == 0) return cudaSuccess;
    const bool d = c.prm.precision == TP_FP64;
    const CoarseCurve &last = S.curves.back();
    TPE_CHECK(cudaMemsetAsync(S.d_AZ, 0, sizeof(double) * (size_t)(last.zoff + (long long)(last.m - 1) * last.n), s));
    k_hat_recs<<<(c.nE + 255) / 256, 256, 0, s>>>(c.nE, c.d_edges, c.d_ellw[which], S.d_curves, S.d_vcurve, S.d_hbase,
                                                  d ? nullptr : S.d_hatF, d ? S.d_hatD : nullptr);
    AzArgs a;
    a.items = S.d_items;
    a.cc = S.d_curves;
    a.recF = which ? c.d_recF2 : c.d_recF;
    a.recLo = which ? c.d_recLo2 : c.d_recLo;
    a.recD = which ? c.d_recD2 : c.d_recD;
    a.hatF = S.d_hatF;
    a.hatD = S.d_hatD;
    a.hbase = S.d_hbase;
    a.ell = c.d_ellw[which];
    a.AZ = S.d_AZ;
    a.kp = c.kp;
    const int slot = c.profile ? prof_begin(c, 6, s) : -1;
    const bool f = c.kp.fast != 0;
    if (d) {
        if (f) k_coarse_az<true, true><<<S.n_items, kThreads, 0, s>>>(a);
        else k_coarse_az<true, false><<<S.n_items, kThreads, 0, s>>>(a);
    } else {
        if (f) k_coarse_az<false, true><<<S.n_items, kThreads, 0, s>>>(a);
        else k_coarse_az<false, false><<<S.n_items, kThreads, 0, s>>>(a);
    }
    if (slot >= 0 || slot <= -2) prof_end(c, slot, s);
    k_coarse_gram_az<<<dim3(c.nCurves, S.max_m), 256, 0, s>>>(S.d_curves, S.d_AZ, S.d_L);
    c.launches += 3;
    return cudaGetLastError();
}

}  // namespace tpe
