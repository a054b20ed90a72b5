// Pair passes of the tangent-point library: the O(|E|^2) loops over ordered pairs of edges that
// share no vertex.  Every pass is a gather: one thread owns TPT target edges I and loops over all
// source edges J staged through shared memory, so each output row is written by exactly one thread
// (no atomics, deterministic).  A persistent grid pulls (target block, source chunk) items from a
// queue; chunk results land in partial slots that a second kernel sums per row and gathers to the
// vertices through the vertex->edge incidence lists.
//
//   energy  : E_I   = sum_J E_IJ,  E_IJ = (1/4) l_I l_J sum_{a,b} k(g_ia, g_jb, T_I)   (Eqs. 3, 17-18)
//   diff    : d/d(g_i1, g_i2) of sum_J (E_IJ + E_JI)                                 (Sec. 5.1)
//   apply   : h_I = sum_J 2 w_IJ (du_I - <T_I,T_J> du_J),  l_I = sum_J (w0_IJ + w0_JI)(ub_I - ub_J)
//             (A u)_{i1,i2} = -/+ h_I / l_I + l_I / 2                                 (Secs. 5.2.2-5.2.3)
//   diag    : diag(A)_v = sum_{I ni v} [2 sum_J w_IJ / l_I^2 + sum_J (w0_IJ + w0_JI) / 4]
//
// w_IJ = (1/4) l_I l_J sum_ab |d|^-p and w0_IJ = (1/4) l_I l_J sum_ab |T_I x d|^2 |d|^-(4+p) with
// d = g_ia - g_jb and p = 2 sigma + 1.  The quadratic forms of Eq. 21 and Sec. 5.2.3 reduce to these
// row sums because w_IJ is symmetric in (I, J) and only w0_IJ + w0_JI enters the low-order form.
//
// Precision (template PREC): P64 all FP64; P32 FP32 pair arithmetic with the partial sums of every
// tile folded into FP64 accumulators; PMIX as P32 but positions are double-float (hi + lo) so that
// d = g_ia - g_jb keeps full FP32 relative accuracy, and pairs with |g_i1 - g_j1| below the near
// cutoff are evaluated in FP64 from the FP64 inputs instead.
//
// |T x d|^2 is formed as |d - (T.d) T|^2 (never as |d|^2 - (T.d)^2, which cancels for the nearly
// parallel pairs along the curve).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "tpe_internal.cuh"

namespace tpe {

#define TPE_CHECK(x)                          \
    do {                                      \
        cudaError_t e_ = (x);                 \
        if (e_ != cudaSuccess) return e_;     \
    } while (0)

// ---------------------------------------------------------------------------------- K0: edge records

__global__ void k_records(int nE, const double *__restrict__ g, const int *__restrict__ E, RecF *__restrict__ recF,
                          RecLo *__restrict__ recLo, RecD *__restrict__ recD, double *__restrict__ ell,
                          double *__restrict__ T, double *__restrict__ x, int *__restrict__ err)
{
    int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nE) return;
    int i1 = E[2 * I], i2 = E[2 * I + 1];
    double p1[3], p2[3], e[3];
    for (int k = 0; k < 3; ++k) {
        p1[k] = g[3 * i1 + k];
        p2[k] = g[3 * i2 + k];
        e[k] = p2[k] - p1[k];
    }
    double l = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
    bool fin = isfinite(l) && isfinite(p1[0] + p1[1] + p1[2]) && isfinite(p2[0] + p2[1] + p2[2]);
    if (!fin) {
        atomicCAS(err, 0, (int)TP_ERR_NONFINITE);
        l = 1.0;
    } else if (!(l > 0.0)) {
        atomicCAS(err, 0, (int)TP_ERR_DEGENERATE_EDGE);
        l = 1.0;
    }
    double t[3] = {e[0] / l, e[1] / l, e[2] / l};
    ell[I] = l;
    for (int k = 0; k < 3; ++k) {
        T[3 * I + k] = t[k];
        x[3 * I + k] = 0.5 * (p1[k] + p2[k]);
    }
    if (recF) {
        float h1[3], h2[3];
        for (int k = 0; k < 3; ++k) {
            h1[k] = (float)p1[k];
            h2[k] = (float)p2[k];
        }
        RecF r;
        r.a = make_float4(h1[0], h1[1], h1[2], (float)l);
        r.b = make_float4(h2[0], h2[1], h2[2], (float)t[0]);
        r.c = make_float4((float)t[1], (float)t[2], __int_as_float(i1), __int_as_float(i2));
        recF[I] = r;
        if (recLo) {
            RecLo q;
            q.lo = make_float4((float)(p1[0] - (double)h1[0]), (float)(p1[1] - (double)h1[1]),
                               (float)(p1[2] - (double)h1[2]), (float)(p2[0] - (double)h2[0]));
            float th[3] = {(float)t[0], (float)t[1], (float)t[2]};
            q.lo2 = make_float4((float)(p2[1] - (double)h2[1]), (float)(p2[2] - (double)h2[2]),
                                (float)(t[0] - (double)th[0]), (float)(t[1] - (double)th[1]));
            q.lo3 = make_float4((float)(t[2] - (double)th[2]), 0.f, 0.f, 0.f);
            recLo[I] = q;
        }
    }
    if (recD) {
        RecD r;
        r.a0 = make_double2(p1[0], p1[1]);
        r.a1 = make_double2(p1[2], l);
        r.b0 = make_double2(p2[0], p2[1]);
        r.b1 = make_double2(p2[2], t[0]);
        r.c0 = make_double2(t[1], t[2]);
        r.i1 = i1;
        r.i2 = i2;
        r.pad0 = r.pad1 = 0;
        recD[I] = r;
    }
}

// Per-edge data of u for an apply: du = (u_j2 - u_j1)/l_J, ub = (u_j1 + u_j2)/2 (3 components).
__global__ void k_urecs(int nE, const double *__restrict__ u, const int *__restrict__ E,
                        const double *__restrict__ ell, URecF *__restrict__ uf, URecD *__restrict__ ud)
{
    int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nE) return;
    int i1 = E[2 * I], i2 = E[2 * I + 1];
    double l = ell[I], du[3], ub[3];
    for (int k = 0; k < 3; ++k) {
        double a = u[3 * i1 + k], b = u[3 * i2 + k];
        du[k] = (b - a) / l;
        ub[k] = 0.5 * (a + b);
    }
    if (uf) {
        float dh[3], uh[3], dl[3], ul[3];
        for (int k = 0; k < 3; ++k) {
            dh[k] = (float)du[k];
            uh[k] = (float)ub[k];
            dl[k] = (float)(du[k] - (double)dh[k]);
            ul[k] = (float)(ub[k] - (double)uh[k]);
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

// ---------------------------------------------------------------------------------- powers

// 1/d2 and |d|^-e from d2 = |d|^2.  Fast paths: e = 4.5 (energy, differential) and e = 2.5 (Gram
// weights) from r = d2^-1/2 as r^4 sqrt(r) and r^2 sqrt(r), sqrt(r) = r rsqrt(r).
template <class R, bool FAST, int WHICH>  // WHICH 0: beta (4.5 fast), 1: p (2.5 fast)
__device__ __forceinline__ R inv_pow(R d2, R e, R &r2)
{
    if constexpr (FAST) {
        if constexpr (sizeof(R) == 4) {
            float r = rsqrtf(d2);
            float sr = r * rsqrtf(r);
            r2 = r * r;
            return WHICH == 0 ? r2 * r2 * sr : r2 * sr;
        } else {
            double r = rsqrt(d2);
            double sr = sqrt(r);
            r2 = r * r;
            return WHICH == 0 ? r2 * r2 * sr : r2 * sr;
        }
    } else {
        if constexpr (sizeof(R) == 4) {
            r2 = __frcp_rn(d2);
            return exp2f(-0.5f * e * log2f(d2));
        } else {
            r2 = 1.0 / d2;
            return pow(d2, -0.5 * e);
        }
    }
}

// |c|^alpha with c2 = |c|^2 (alpha = 2 in the fast path).
template <class R, bool FAST>
__device__ __forceinline__ R pow_c(R c2, R alpha)
{
    if constexpr (FAST) {
        return c2;
    } else {
        if constexpr (sizeof(R) == 4)
            return c2 > 0.f ? exp2f(0.5f * alpha * log2f(c2)) : 0.f;
        else
            return c2 > 0.0 ? pow(c2, 0.5 * alpha) : 0.0;
    }
}

// ---------------------------------------------------------------------------------- target / source views

template <class R>
struct V3 {
    R x, y, z;
};

template <class R>
__device__ __forceinline__ R dot3(V3<R> a, V3<R> b)
{
    return a.x * b.x + a.y * b.y + a.z * b.z;
}

// Target edge data held in registers.
template <class R>
struct Tgt {
    V3<R> p1, p2, T;   // hi parts (PMIX) or the values
    V3<R> l1, l2, Tl;  // lo parts (PMIX only)
    R ell;
    int i1, i2;
};

template <int PREC>
struct RealOf {
    using type = float;
};
template <>
struct RealOf<P64> {
    using type = double;
};

// Shared-memory tile of source records.
template <int PREC, bool NEEDU>
struct Tile;
template <bool NEEDU>
struct Tile<P64, NEEDU> {
    RecD r[kTile];
    URecD u[NEEDU ? kTile : 1];
};
template <bool NEEDU>
struct Tile<P32, NEEDU> {
    RecF r[kTile];
    URecF u[NEEDU ? kTile : 1];
};
template <bool NEEDU>
struct Tile<PMIX, NEEDU> {
    RecF r[kTile];
    RecLo lo[kTile];
    URecF u[NEEDU ? kTile : 1];
};

template <int PREC>
__device__ __forceinline__ void load_target(Tgt<typename RealOf<PREC>::type> &t, int I, const RecF *recF,
                                            const RecLo *recLo, const RecD *recD)
{
    if constexpr (PREC == P64) {
        RecD r = recD[I];
        t.p1 = {r.a0.x, r.a0.y, r.a1.x};
        t.ell = r.a1.y;
        t.p2 = {r.b0.x, r.b0.y, r.b1.x};
        t.T = {r.b1.y, r.c0.x, r.c0.y};
        t.i1 = r.i1;
        t.i2 = r.i2;
        t.l1 = {0, 0, 0};
        t.l2 = {0, 0, 0};
        t.Tl = {0, 0, 0};
    } else {
        RecF r = recF[I];
        t.p1 = {r.a.x, r.a.y, r.a.z};
        t.ell = r.a.w;
        t.p2 = {r.b.x, r.b.y, r.b.z};
        t.T = {r.b.w, r.c.x, r.c.y};
        t.i1 = __float_as_int(r.c.z);
        t.i2 = __float_as_int(r.c.w);
        if constexpr (PREC == PMIX) {
            RecLo q = recLo[I];
            t.l1 = {q.lo.x, q.lo.y, q.lo.z};
            t.l2 = {q.lo.w, q.lo2.x, q.lo2.y};
            t.Tl = {q.lo2.z, q.lo2.w, q.lo3.x};
        } else {
            t.l1 = {0.f, 0.f, 0.f};
            t.l2 = {0.f, 0.f, 0.f};
            t.Tl = {0.f, 0.f, 0.f};
        }
    }
}

template <int PREC>
struct Src {
    using R = typename RealOf<PREC>::type;
    V3<R> q1, q2, T, m1, m2, Tm;  // m = lo parts
    R ell;
    int j1, j2;
};

template <int PREC, bool NEEDU>
__device__ __forceinline__ void load_source(Src<PREC> &s, const Tile<PREC, NEEDU> &tl, int j)
{
    if constexpr (PREC == P64) {
        const RecD &r = tl.r[j];
        const double2 a0 = r.a0, a1 = r.a1, b0 = r.b0, b1 = r.b1, c0 = r.c0;
        s.q1 = V3<double>{a0.x, a0.y, a1.x};
        s.ell = a1.y;
        s.q2 = V3<double>{b0.x, b0.y, b1.x};
        s.T = V3<double>{b1.y, c0.x, c0.y};
        s.j1 = r.i1;
        s.j2 = r.i2;
    } else {
        float4 a = tl.r[j].a, b = tl.r[j].b, c = tl.r[j].c;
        s.q1 = {a.x, a.y, a.z};
        s.ell = a.w;
        s.q2 = {b.x, b.y, b.z};
        s.T = {b.w, c.x, c.y};
        s.j1 = __float_as_int(c.z);
        s.j2 = __float_as_int(c.w);
        if constexpr (PREC == PMIX) {
            float4 l = tl.lo[j].lo, l2 = tl.lo[j].lo2;
            s.m1 = {l.x, l.y, l.z};
            s.m2 = {l.w, l2.x, l2.y};
            s.Tm = {l2.z, l2.w, tl.lo[j].lo3.x};
        }
    }
}

// d = p - q (double-float positions when DF: hi difference plus lo difference).
template <bool DF, class R>
__device__ __forceinline__ V3<R> diff3(V3<R> p, V3<R> pl, V3<R> q, V3<R> ql)
{
    V3<R> d = {p.x - q.x, p.y - q.y, p.z - q.z};
    if constexpr (DF) {
        d.x += pl.x - ql.x;
        d.y += pl.y - ql.y;
        d.z += pl.z - ql.z;
    }
    return d;
}

// |d - (T.d) T|^2 = |T x d|^2 for unit T; also returns t = T.d.
template <class R>
__device__ __forceinline__ R perp2(V3<R> d, V3<R> T, R &t, V3<R> &dp)
{
    t = dot3(T, d);
    dp = {d.x - t * T.x, d.y - t * T.y, d.z - t * T.z};
    return dot3(dp, dp);
}

// ---------------------------------------------------------------------------------- FP64 near-pair paths

struct NearArgs {
    const double *g;    // [nV][3]
    const int *E;       // [nE][2]
    const double *ell;  // [nE]
    const double *T;    // [nE][3]
    const double *u;    // [nV][3] (apply)
};

__device__ __forceinline__ V3<double> ld3(const double *a, int i) { return {a[3 * i], a[3 * i + 1], a[3 * i + 2]}; }

// Differential accumulators of one target against its sources (all scaled by l_J):
//   S  = sum (fI + fJ);  G1, G2 = sum d/dp (fI + fJ) at p = g_i1, g_i2;  GT = sum d fI / d T_I
struct DiffAcc64 {
    double S, G1[3], G2[3], GT[3];
};

// Apply accumulators (scaled by l_J), in the exact difference form
//   du_I - <T_I,T_J> du_J = (du_I - du_J) + (|T_I - T_J|^2 / 2) du_J:
//   A1 = sum W [(du_I - du_J) + (1 - t_IJ) du_J],  A2 = sum W0 (ub_I - ub_J),
// with W = l_J sum_ab |d|^-p and W0 = l_J sum_ab (|T_I x d|^2 + |T_J x d|^2) |d|^-(4+p).
// Sw, Sw0 are the u-independent row sums used for diag(A).
struct ApplyAcc64 {
    double Sw, A1[3], Sw0, A2[3];
};

// ---------------------------------------------------------------------------------- the pair kernel

struct PairArgs {
    const WorkItem *items;
    int n_items;
    int *counter;
    const RecF *recF;
    const RecLo *recLo;
    const RecD *recD;
    const URecF *urecF;
    const URecD *urecD;
    NearArgs na;
    double *part;  // [slot][nE][stride]
    int nE;
    KernelParams kp;
    const int *skip;  // per-problem flags: items of flagged problems are skipped (may be NULL)
};

template <int PREC, int OP>
struct Acc32;  // per-target tile accumulators in the pair precision

template <int PREC>
struct Acc32<PREC, OP_ENERGY> {
    static constexpr int op = OP_ENERGY;
    typename RealOf<PREC>::type s;
};
template <int PREC>
struct Acc32<PREC, OP_DIFF> {
    static constexpr int op = OP_DIFF;
    typename RealOf<PREC>::type S, G1[3], G2[3], GT[3];
    typename RealOf<PREC>::type cS, c1[3], c2[3], cT[3];  // Kahan compensations (mixed path)
};
template <int PREC>
struct Acc32<PREC, OP_APPLY> {
    static constexpr int op = OP_APPLY;
    typename RealOf<PREC>::type A1[3], A2[3], C1[3], C2[3];  // C: Kahan compensations
};

// Kahan-compensated accumulation acc += x (c carries the lost low-order part, to be subtracted).
template <class R>
__device__ __forceinline__ void kahan_add(R &acc, R &c, R x)
{
    R y = x - c;
    R t = acc + y;
    c = (t - acc) - y;
    acc = t;
}
template <int PREC>
struct Acc32<PREC, OP_DIAG> {
    static constexpr int op = OP_DIAG;
    typename RealOf<PREC>::type Sw, Sw0;
};

template <int OP>
struct Acc64;
template <>
struct Acc64<OP_ENERGY> {
    static constexpr int op = OP_ENERGY;
    double s;
};
template <>
struct Acc64<OP_DIFF> : DiffAcc64 {
    static constexpr int op = OP_DIFF;
};
template <>
struct Acc64<OP_APPLY> : ApplyAcc64 {
    static constexpr int op = OP_APPLY;
};
template <>
struct Acc64<OP_DIAG> : ApplyAcc64 {
    static constexpr int op = OP_DIAG;
};

// Per-edge values of u seen by one side of a pair (double-float in PMIX).
template <class R>
struct UVal {
    V3<R> dh, dl, uh, ul;  // du and ub, hi and lo parts
};

template <int PREC>
__device__ __forceinline__ void load_uval(UVal<typename RealOf<PREC>::type> &v, const URecF *uf, const URecD *ud,
                                          int I)
{
    if constexpr (PREC == P64) {
        URecD r = ud[I];
        v.dh = {r.du0.x, r.du0.y, r.du1.x};
        v.uh = {r.ub0.x, r.ub0.y, r.ub1.x};
        v.dl = {0, 0, 0};
        v.ul = {0, 0, 0};
    } else {
        URecF r = uf[I];
        v.dh = {r.a.x, r.a.y, r.a.z};
        v.uh = {r.a.w, r.b.x, r.b.y};
        v.dl = {r.b.z, r.b.w, r.c.x};
        v.ul = {r.c.y, r.c.z, r.c.w};
    }
}


// Differential of one near pair in FP64 from the double-float positions and tangents, accumulated
// straight into the FP64 accumulators: along the curve the near-pair gradient terms are large and
// cancel between neighbours, so they need FP64 both in the arithmetic and in the sum.
__device__ __noinline__ void near_diff_df(const Tgt<float> &t, const Src<PMIX> &s, double alpha, double beta,
                                          bool fast, DiffAcc64 &acc)
{
    double TI[3] = {(double)t.T.x + t.Tl.x, (double)t.T.y + t.Tl.y, (double)t.T.z + t.Tl.z};
    double TJ[3] = {(double)s.T.x + s.Tm.x, (double)s.T.y + s.Tm.y, (double)s.T.z + s.Tm.z};
    double L = s.ell;
    for (int ab = 0; ab < 4; ++ab) {
        V3<float> P = (ab < 2) ? t.p1 : t.p2, PL = (ab < 2) ? t.l1 : t.l2;
        V3<float> Q = (ab & 1) ? s.q2 : s.q1, QL = (ab & 1) ? s.m2 : s.m1;
        double d[3] = {(double)(P.x - Q.x) + (double)(PL.x - QL.x), (double)(P.y - Q.y) + (double)(PL.y - QL.y),
                       (double)(P.z - Q.z) + (double)(PL.z - QL.z)};
        double tI = TI[0] * d[0] + TI[1] * d[1] + TI[2] * d[2];
        double tJ = TJ[0] * d[0] + TJ[1] * d[1] + TJ[2] * d[2];
        double dpI[3], dpJ[3];
        for (int k = 0; k < 3; ++k) {
            dpI[k] = d[k] - tI * TI[k];
            dpJ[k] = d[k] - tJ * TJ[k];
        }
        double cI2 = dpI[0] * dpI[0] + dpI[1] * dpI[1] + dpI[2] * dpI[2];
        double cJ2 = dpJ[0] * dpJ[0] + dpJ[1] * dpJ[1] + dpJ[2] * dpJ[2];
        double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        double rb, fI, fJ, aI, aJ;
        if (fast) {
            double r = rsqrt(d2), r2 = r * r;
            rb = r2 * r2 * sqrt(r);
            fI = cI2 * rb;
            fJ = cJ2 * rb;
            aI = aJ = 2.0 * rb;
        } else {
            rb = pow(d2, -0.5 * beta);
            fI = (cI2 > 0.0 ? pow(cI2, 0.5 * alpha) : 0.0) * rb;
            fJ = (cJ2 > 0.0 ? pow(cJ2, 0.5 * alpha) : 0.0) * rb;
            aI = cI2 > 0.0 ? alpha * fI / cI2 : 0.0;
            aJ = cJ2 > 0.0 ? alpha * fJ / cJ2 : 0.0;
        }
        double cb = beta * (fI + fJ) / d2;
        double *G = ab < 2 ? acc.G1 : acc.G2;
        for (int k = 0; k < 3; ++k) {
            G[k] += L * (aI * dpI[k] + aJ * dpJ[k] - cb * d[k]);
            acc.GT[k] += -L * aI * tI * d[k];
        }
        acc.S += L * (fI + fJ);
    }
}

// One (target, source) pair: accumulate into the tile accumulator a.
// DF: use the low parts (double-float differences) and compensated accumulation; only the mixed
// path's MID and NEAR tiles set it.
// |T x d|^2 in FP64 from the double-float position differences and tangent of a near pair: the
// angle between T and the chord is small there, so FP32 would lose most of the digits of the
// perpendicular part.  Only this quantity goes to FP64; the rest of the pair stays in FP32.
__device__ __forceinline__ float perp2_near(V3<float> P, V3<float> PL, V3<float> Q, V3<float> QL, V3<float> T,
                                            V3<float> Tl)
{
    double dx = (double)(P.x - Q.x) + (double)(PL.x - QL.x);
    double dy = (double)(P.y - Q.y) + (double)(PL.y - QL.y);
    double dz = (double)(P.z - Q.z) + (double)(PL.z - QL.z);
    double tx = (double)T.x + (double)Tl.x, ty = (double)T.y + (double)Tl.y, tz = (double)T.z + (double)Tl.z;
    double t = tx * dx + ty * dy + tz * dz;
    double px = dx - t * tx, py = dy - t * ty, pz = dz - t * tz;
    return (float)(px * px + py * py + pz * pz);
}

// Target-side |T x d|^2 with the double-float tangent T + Tl: a rounding error of T_I is the same for
// every source J, so it does not average out, and the vertex gather of the differential amplifies it
// by ~1 / (kappa l).  The source-side tangent's rounding is shared by the two edges at a vertex and
// cancels there.
__device__ __forceinline__ float perp2_df(V3<float> d, V3<float> T, V3<float> Tl, float &t, V3<float> &dp)
{
    t = fmaf(T.x, d.x, fmaf(T.y, d.y, fmaf(T.z, d.z, dot3(Tl, d))));
    dp = {fmaf(-t, T.x, fmaf(-t, Tl.x, d.x)), fmaf(-t, T.y, fmaf(-t, Tl.y, d.y)), fmaf(-t, T.z, fmaf(-t, Tl.z, d.z))};
    return dot3(dp, dp);
}

template <int PREC, int OP, bool FAST, bool DF = (PREC == PMIX)>
__device__ __forceinline__ void pair_eval(const Tgt<typename RealOf<PREC>::type> &t, const Src<PREC> &s,
                                          Acc32<PREC, OP> &a, bool keep, const KernelParams &kp,
                                          typename RealOf<PREC>::type &d2_11,
                                          const UVal<typename RealOf<PREC>::type> *tu,
                                          const UVal<typename RealOf<PREC>::type> *su, bool near = false)
{
    using R = typename RealOf<PREC>::type;
    const R alpha = (R)kp.alpha, beta = (R)kp.beta, pp = (R)kp.p;
    if constexpr (OP == OP_ENERGY) {
        R f = 0;
#pragma unroll
        for (int ab = 0; ab < 4; ++ab) {
            V3<R> P = (ab < 2) ? t.p1 : t.p2, PL = (ab < 2) ? t.l1 : t.l2;
            V3<R> Q = (ab & 1) ? s.q2 : s.q1, QL = (ab & 1) ? s.m2 : s.m1;
            V3<R> d = diff3<DF>(P, PL, Q, QL), dp;
            R tt, c2 = perp2(d, t.T, tt, dp), d2 = dot3(d, d);
            if constexpr (DF && sizeof(R) == 4)
                if (near) c2 = perp2_near(P, PL, Q, QL, t.T, t.Tl);
            if (ab == 0) d2_11 = d2;
            R r2;
            f += pow_c<R, FAST>(c2, alpha) * inv_pow<R, FAST, 0>(d2, beta, r2);
        }
        R c = s.ell * f;
        a.s += keep ? c : (R)0;
    } else if constexpr (OP == OP_DIFF) {
        R S = 0, G1[3] = {0, 0, 0}, G2[3] = {0, 0, 0}, GT[3] = {0, 0, 0};
#pragma unroll
        for (int ab = 0; ab < 4; ++ab) {
            V3<R> P = (ab < 2) ? t.p1 : t.p2, PL = (ab < 2) ? t.l1 : t.l2;
            V3<R> Q = (ab & 1) ? s.q2 : s.q1, QL = (ab & 1) ? s.m2 : s.m1;
            V3<R> d = diff3<DF>(P, PL, Q, QL), dpI, dpJ;
            R tI, tJ;
            R cI2, cJ2 = perp2(d, s.T, tJ, dpJ), d2 = dot3(d, d);
            if constexpr (DF && sizeof(R) == 4)
                cI2 = perp2_df(d, t.T, t.Tl, tI, dpI);
            else
                cI2 = perp2(d, t.T, tI, dpI);
            if constexpr (DF && sizeof(R) == 4)
                if (near) {
                    cI2 = perp2_near(P, PL, Q, QL, t.T, t.Tl);
                    cJ2 = perp2_near(P, PL, Q, QL, s.T, s.Tm);
                }
            if (ab == 0) d2_11 = d2;
            R r2;
            R rb = inv_pow<R, FAST, 0>(d2, beta, r2);
            R fI, fJ, aI, aJ;
            if constexpr (FAST) {
                fI = cI2 * rb;
                fJ = cJ2 * rb;
                aI = aJ = (R)2 * rb;
            } else {
                fI = pow_c<R, false>(cI2, alpha) * rb;
                fJ = pow_c<R, false>(cJ2, alpha) * rb;
                aI = cI2 > (R)0 ? alpha * fI / cI2 : (R)0;
                aJ = cJ2 > (R)0 ? alpha * fJ / cJ2 : (R)0;
            }
            R fs = fI + fJ;
            R cb = beta * fs * r2;
            R *G = (ab < 2) ? G1 : G2;
            G[0] += aI * dpI.x + aJ * dpJ.x - cb * d.x;
            G[1] += aI * dpI.y + aJ * dpJ.y - cb * d.y;
            G[2] += aI * dpI.z + aJ * dpJ.z - cb * d.z;
            R m = -aI * tI;
            GT[0] += m * d.x;
            GT[1] += m * d.y;
            GT[2] += m * d.z;
            S += fs;
        }
        if (!keep) {  // neighbours produce Inf/NaN: never let them touch the accumulators
            S = 0;
            for (int k = 0; k < 3; ++k) G1[k] = G2[k] = GT[k] = 0;
        }
        R L = keep ? s.ell : (R)0;
        if constexpr (PREC == PMIX) {
            // compensated: the vertex gather takes differences of neighbouring edges' rows, which
            // cancel by ~1 / (kappa l), so the rows need more than FP32 summation accuracy
            kahan_add(a.S, a.cS, L * S);
            for (int k = 0; k < 3; ++k) {
                kahan_add(a.G1[k], a.c1[k], L * G1[k]);
                kahan_add(a.G2[k], a.c2[k], L * G2[k]);
                kahan_add(a.GT[k], a.cT[k], L * GT[k]);
            }
        } else {
            a.S += L * S;
            for (int k = 0; k < 3; ++k) {
                a.G1[k] += L * G1[k];
                a.G2[k] += L * G2[k];
                a.GT[k] += L * GT[k];
            }
        }
    } else {  // OP_APPLY / OP_DIAG
        // the four trapezoid terms are summed as (11 + 22) + (12 + 21), an order that is the same
        // from row I and from row J, so W_IJ and W_JI (and W0) are bitwise equal: the FP32 operator
        // stays exactly symmetric
        R tw[4], tw0[4];
#pragma unroll
        for (int ab = 0; ab < 4; ++ab) {
            V3<R> P = (ab < 2) ? t.p1 : t.p2, PL = (ab < 2) ? t.l1 : t.l2;
            V3<R> Q = (ab & 1) ? s.q2 : s.q1, QL = (ab & 1) ? s.m2 : s.m1;
            V3<R> d = diff3<DF>(P, PL, Q, QL), dpI, dpJ;
            R tI, tJ;
            R c2 = perp2(d, t.T, tI, dpI) + perp2(d, s.T, tJ, dpJ), d2 = dot3(d, d);
            if constexpr (DF && sizeof(R) == 4)
                if (near) c2 = perp2_near(P, PL, Q, QL, t.T, t.Tl) + perp2_near(P, PL, Q, QL, s.T, s.Tm);
            if (ab == 0) d2_11 = d2;
            R r2;
            R rp = inv_pow<R, FAST, 1>(d2, pp, r2);
            tw[ab] = rp;
            tw0[ab] = c2 * (rp * r2 * r2);
        }
        R sw = (tw[0] + tw[3]) + (tw[1] + tw[2]);
        R sw0 = (tw0[0] + tw0[3]) + (tw0[1] + tw0[2]);
        R W = keep ? s.ell * sw : (R)0;
        R W0 = keep ? s.ell * sw0 : (R)0;
        if constexpr (OP == OP_DIAG) {
            a.Sw += W;
            a.Sw0 += W0;
        } else {
            // (du_I - du_J) + (|T_I - T_J|^2 / 2) du_J  and  ub_I - ub_J, differences of double-floats
            V3<R> dT = {t.T.x - s.T.x, t.T.y - s.T.y, t.T.z - s.T.z};
            if constexpr (DF) {
                dT.x += t.Tl.x - s.Tm.x;
                dT.y += t.Tl.y - s.Tm.y;
                dT.z += t.Tl.z - s.Tm.z;
            }
            R omt = (R)0.5 * dot3(dT, dT);
            R ddx = (tu->dh.x - su->dh.x), ddy = (tu->dh.y - su->dh.y), ddz = (tu->dh.z - su->dh.z);
            R dbx = (tu->uh.x - su->uh.x), dby = (tu->uh.y - su->uh.y), dbz = (tu->uh.z - su->uh.z);
            // the differences of u always use the double-float parts in the mixed path: for smooth u
            // they are small second differences, and the operator's accuracy on them sets how far CG
            // can reduce the true residual
            if constexpr (PREC == PMIX) {
                ddx += tu->dl.x - su->dl.x;
                ddy += tu->dl.y - su->dl.y;
                ddz += tu->dl.z - su->dl.z;
                dbx += tu->ul.x - su->ul.x;
                dby += tu->ul.y - su->ul.y;
                dbz += tu->ul.z - su->ul.z;
            }
            if constexpr (PREC != P32) {
                kahan_add(a.A1[0], a.C1[0], W * (ddx + omt * su->dh.x));
                kahan_add(a.A1[1], a.C1[1], W * (ddy + omt * su->dh.y));
                kahan_add(a.A1[2], a.C1[2], W * (ddz + omt * su->dh.z));
                kahan_add(a.A2[0], a.C2[0], W0 * dbx);
                kahan_add(a.A2[1], a.C2[1], W0 * dby);
                kahan_add(a.A2[2], a.C2[2], W0 * dbz);
            } else {
                a.A1[0] += W * (ddx + omt * su->dh.x);
                a.A1[1] += W * (ddy + omt * su->dh.y);
                a.A1[2] += W * (ddz + omt * su->dh.z);
                a.A2[0] += W0 * dbx;
                a.A2[1] += W0 * dby;
                a.A2[2] += W0 * dbz;
            }
        }
    }
}

template <int PREC, int OP>
__device__ __forceinline__ void acc_zero(Acc32<PREC, OP> &a)
{
    if constexpr (OP == OP_ENERGY) {
        a.s = 0;
    } else if constexpr (OP == OP_DIFF) {
        a.S = a.cS = 0;
        for (int k = 0; k < 3; ++k) a.G1[k] = a.G2[k] = a.GT[k] = a.c1[k] = a.c2[k] = a.cT[k] = 0;
    } else if constexpr (OP == OP_APPLY) {
        for (int k = 0; k < 3; ++k) a.A1[k] = a.A2[k] = a.C1[k] = a.C2[k] = 0;
    } else {
        a.Sw = a.Sw0 = 0;
    }
}

template <int OP>
__device__ __forceinline__ void acc64_zero(Acc64<OP> &a)
{
    if constexpr (OP == OP_ENERGY) {
        a.s = 0;
    } else if constexpr (OP == OP_DIFF) {
        a.S = 0;
        for (int k = 0; k < 3; ++k) a.G1[k] = a.G2[k] = a.GT[k] = 0;
    } else {
        a.Sw = a.Sw0 = 0;
        for (int k = 0; k < 3; ++k) a.A1[k] = a.A2[k] = 0;
    }
}

template <class X, class Y>
__device__ __forceinline__ void acc_add(X &A, const Y &a)
{
    constexpr int OPX = X::op;
    if constexpr (OPX == OP_ENERGY) {
        A.s += a.s;
    } else if constexpr (OPX == OP_DIFF) {
        // tile fold into FP64: value minus its compensation
        A.S += (double)a.S - (double)a.cS;
        for (int k = 0; k < 3; ++k) {
            A.G1[k] += (double)a.G1[k] - (double)a.c1[k];
            A.G2[k] += (double)a.G2[k] - (double)a.c2[k];
            A.GT[k] += (double)a.GT[k] - (double)a.cT[k];
        }
    } else if constexpr (OPX == OP_APPLY) {
        if constexpr (std::is_same_v<X, Acc64<OP_APPLY>>) {
            // tile fold into FP64: value minus its compensation
            for (int k = 0; k < 3; ++k) {
                A.A1[k] += (double)a.A1[k] - (double)a.C1[k];
                A.A2[k] += (double)a.A2[k] - (double)a.C2[k];
            }
        } else {
            // one pair's accumulator into the tile accumulator (mixed path), compensated
            for (int k = 0; k < 3; ++k) {
                kahan_add(A.A1[k], A.C1[k], a.A1[k] - a.C1[k]);
                kahan_add(A.A2[k], A.C2[k], a.A2[k] - a.C2[k]);
            }
        }
    } else {
        A.Sw += a.Sw;
        A.Sw0 += a.Sw0;
    }
}

template <int OP>
__host__ __device__ constexpr int part_stride()
{
    return (OP == OP_ENERGY || OP == OP_DIAG) ? 1 : 6;
}

template <int PREC, int OP, int TPT, bool FAST, bool CHECK, int MODE = 2>
__device__ __forceinline__ void tile_loop(const Tgt<typename RealOf<PREC>::type> (&tg)[TPT], const int (&tI)[TPT],
                                          const UVal<typename RealOf<PREC>::type> (&tu)[TPT],
                                          const Tile<PREC, OP == OP_APPLY> &tl, int cnt, int s0,
                                          Acc32<PREC, OP> (&a)[TPT], Acc64<OP> (&A)[TPT], const PairArgs &pa)
{
    using R = typename RealOf<PREC>::type;
#pragma unroll 2
    for (int j = 0; j < cnt; ++j) {
        Src<PREC> s;
        load_source<PREC, OP == OP_APPLY>(s, tl, j);
        UVal<R> su;
        if constexpr (OP == OP_APPLY) {
            if constexpr (PREC == P64) {
                URecD u = tl.u[j];
                su.dh = {u.du0.x, u.du0.y, u.du1.x};
                su.uh = {u.ub0.x, u.ub0.y, u.ub1.x};
            } else {
                float4 x = tl.u[j].a, y = tl.u[j].b, z = tl.u[j].c;
                su.dh = {x.x, x.y, x.z};
                su.uh = {x.w, y.x, y.y};
                su.dl = {y.z, y.w, z.x};
                su.ul = {z.y, z.z, z.w};
            }
        }
#pragma unroll
        for (int k = 0; k < TPT; ++k) {
            bool keep = true;
            if constexpr (CHECK)
                keep = (s.j1 != tg[k].i1) & (s.j1 != tg[k].i2) & (s.j2 != tg[k].i1) & (s.j2 != tg[k].i2);
            R d2_11;
            if constexpr (PREC == PMIX && MODE < 2) {
                pair_eval<PREC, OP, FAST, MODE == 1>(tg[k], s, a[k], keep, pa.kp, d2_11, &tu[k], &su);
            } else if constexpr (PREC == PMIX) {
                // near pairs (|g_i1 - g_j1| below the cutoff) take |T x d|^2 in FP64; the differential
                // evaluates and accumulates the whole near pair in FP64
                V3<float> e = diff3<true>(tg[k].p1, tg[k].l1, s.q1, s.m1);
                bool near = keep && (dot3(e, e) < (OP == OP_DIFF ? pa.kp.near2f_diff : pa.kp.near2f));
                if constexpr (OP == OP_DIFF) {
                    if (near)
                        near_diff_df(tg[k], s, pa.kp.alpha, pa.kp.beta, FAST, A[k]);
                    else
                        pair_eval<PREC, OP, FAST, true>(tg[k], s, a[k], keep, pa.kp, d2_11, &tu[k], &su, false);
                } else {
                    pair_eval<PREC, OP, FAST, true>(tg[k], s, a[k], keep, pa.kp, d2_11, &tu[k], &su, near);
                }
            } else {
                pair_eval<PREC, OP, FAST>(tg[k], s, a[k], keep, pa.kp, d2_11, &tu[k], &su);
            }
        }
    }
}

__device__ __forceinline__ void box_add(float (&b)[6], V3<float> p, V3<float> q)
{
    b[0] = fminf(b[0], fminf(p.x, q.x));
    b[1] = fminf(b[1], fminf(p.y, q.y));
    b[2] = fminf(b[2], fminf(p.z, q.z));
    b[3] = fmaxf(b[3], fmaxf(p.x, q.x));
    b[4] = fmaxf(b[4], fmaxf(p.y, q.y));
    b[5] = fmaxf(b[5], fmaxf(p.z, q.z));
}

// Block-wide bounding box: every thread ends with the box of all threads' boxes.  Contains one
// __syncthreads (the caller's tile barrier).
__device__ __forceinline__ void block_box(float (&b)[6], float (*sh)[6])
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        for (int q = 0; q < 6; ++q) {
            float v = __shfl_xor_sync(0xffffffffu, b[q], o);
            b[q] = q < 3 ? fminf(b[q], v) : fmaxf(b[q], v);
        }
    if ((threadIdx.x & 31) == 0)
        for (int q = 0; q < 6; ++q) sh[threadIdx.x >> 5][q] = b[q];
    __syncthreads();
    for (int wv = 0; wv < kThreads / 32; ++wv)
        for (int q = 0; q < 6; ++q) b[q] = q < 3 ? fminf(b[q], sh[wv][q]) : fmaxf(b[q], sh[wv][q]);
}

template <int PREC, int OP, int TPT, bool FAST>
__global__ void __launch_bounds__(kThreads, PREC == P64 ? 1 : 3) k_pairs(const PairArgs pa)
{
    using R = typename RealOf<PREC>::type;
    constexpr bool NEEDU = (OP == OP_APPLY);
    __shared__ Tile<PREC, NEEDU> tl;
    __shared__ int s_item;
    __shared__ float s_box[2][kThreads / 32][6];
    constexpr int S = part_stride<OP>();
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(pa.counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= pa.n_items) break;
        const WorkItem w = pa.items[it];
        if (pa.skip && pa.skip[w.pad]) continue;  // problem already converged: its output is not used
        Tgt<R> tg[TPT];
        UVal<R> tu[TPT];
        int tI[TPT];
#pragma unroll
        for (int k = 0; k < TPT; ++k) {
            int loc = threadIdx.x + k * kThreads;
            tI[k] = w.tgt0 + min(loc, w.ntgt - 1);
            load_target<PREC>(tg[k], tI[k], pa.recF, pa.recLo, pa.recD);
            if constexpr (NEEDU) load_uval<PREC>(tu[k], pa.urecF, pa.urecD, tI[k]);
        }
        Acc64<OP> A[TPT];
        Acc32<PREC, OP> a[TPT];
#pragma unroll
        for (int k = 0; k < TPT; ++k) acc64_zero<OP>(A[k]);
        float tbox[6];  // bounding box of this warp's targets (mixed path): min xyz, max xyz
        if constexpr (PREC == PMIX) {
            float b[6] = {1e30f, 1e30f, 1e30f, -1e30f, -1e30f, -1e30f};
#pragma unroll
            for (int k = 0; k < TPT; ++k) box_add(b, tg[k].p1, tg[k].p2);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                for (int q = 0; q < 6; ++q) {
                    float v = __shfl_xor_sync(0xffffffffu, b[q], o);
                    b[q] = q < 3 ? fminf(b[q], v) : fmaxf(b[q], v);
                }
            for (int q = 0; q < 6; ++q) tbox[q] = b[q];
        }
        int tiles_since_fold = 0;
        for (int s0 = w.src0; s0 < w.src1; s0 += kTile) {
            const int cnt = min(kTile, w.src1 - s0);
            __syncthreads();
            float sb[6] = {1e30f, 1e30f, 1e30f, -1e30f, -1e30f, -1e30f};
            if (threadIdx.x < cnt) {
                int J = s0 + threadIdx.x;
                if constexpr (PREC == P64) {
                    tl.r[threadIdx.x] = pa.recD[J];
                    if constexpr (NEEDU) tl.u[threadIdx.x] = pa.urecD[J];
                } else {
                    RecF r = pa.recF[J];
                    tl.r[threadIdx.x] = r;
                    if constexpr (PREC == PMIX) {
                        tl.lo[threadIdx.x] = pa.recLo[J];
                        box_add(sb, V3<float>{r.a.x, r.a.y, r.a.z}, V3<float>{r.b.x, r.b.y, r.b.z});
                    }
                    if constexpr (NEEDU) tl.u[threadIdx.x] = pa.urecF[J];
                }
            }
            if constexpr (PREC == PMIX) block_box(sb, s_box[1]);  // contains the barriers
            else __syncthreads();
            if (tiles_since_fold == 0) {
#pragma unroll
                for (int k = 0; k < TPT; ++k) acc_zero<PREC, OP>(a[k]);
            }
            const bool check = !(s0 + cnt - 1 < w.nb_lo || s0 > w.nb_hi);
            int mode = 2;
            if constexpr (PREC == PMIX) {
                // squared distance between the two boxes decides the arithmetic of the whole tile
                float g2 = 0.f;
                for (int q = 0; q < 3; ++q) {
                    float gap = fmaxf(fmaxf(sb[q] - tbox[3 + q], tbox[q] - sb[3 + q]), 0.f);
                    g2 += gap * gap;
                }
                const float nr2 = (OP == OP_DIFF) ? pa.kp.near2f_diff : pa.kp.near2f;
                mode = (g2 < nr2) ? 2 : (g2 < pa.kp.mid2f ? 1 : 0);
                // In the Gram weights |T x d|^2 enters only the low-order weight w0, whose near-pair
                // entries are ~(kappa l)^2 / 4 of the high-order ones, so FP32 double-float accuracy
                // suffices there: no FP64 near path for apply / diag.
                if constexpr (OP == OP_APPLY || OP == OP_DIAG) mode = min(mode, 1);
            }
            if (check || mode == 2) {
                if (check && (OP == OP_APPLY || OP == OP_DIAG) && PREC == PMIX)
                    tile_loop<PREC, OP, TPT, FAST, true, 1>(tg, tI, tu, tl, cnt, s0, a, A, pa);
                else if (check)
                    tile_loop<PREC, OP, TPT, FAST, true, 2>(tg, tI, tu, tl, cnt, s0, a, A, pa);
                else
                    tile_loop<PREC, OP, TPT, FAST, false, 2>(tg, tI, tu, tl, cnt, s0, a, A, pa);
            } else if (mode == 1) {
                tile_loop<PREC, OP, TPT, FAST, false, 1>(tg, tI, tu, tl, cnt, s0, a, A, pa);
            } else {
                tile_loop<PREC, OP, TPT, FAST, false, 0>(tg, tI, tu, tl, cnt, s0, a, A, pa);
            }
            // fold the tile accumulators into FP64 every 4 tiles and at the end of the item
            if (++tiles_since_fold == 4 || s0 + kTile >= w.src1) {
#pragma unroll
                for (int k = 0; k < TPT; ++k) acc_add(A[k], a[k]);
                tiles_since_fold = 0;
            }
        }
        // write this item's partial results for the valid targets
#pragma unroll
        for (int k = 0; k < TPT; ++k) {
            int loc = threadIdx.x + k * kThreads;
            if (loc >= w.ntgt) continue;
            int I = w.tgt0 + loc;
            double *o = pa.part + ((size_t)w.slot * pa.nE + I) * S;
            if constexpr (OP == OP_ENERGY) {
                o[0] = A[k].s;
            } else if constexpr (OP == OP_DIFF) {
                // G_i1 = (1/4)[-T S + l_I G1 - (Id - T T^t) GT],  G_i2 = (1/4)[T S + l_I G2 + (Id - T T^t) GT]
                const double *T = pa.na.T + 3 * I;
                double l = pa.na.ell[I];
                double tg3[3] = {T[0], T[1], T[2]};
                double gt = tg3[0] * A[k].GT[0] + tg3[1] * A[k].GT[1] + tg3[2] * A[k].GT[2];
                for (int c = 0; c < 3; ++c) {
                    double pgt = A[k].GT[c] - gt * tg3[c];
                    o[c] = 0.25 * (-tg3[c] * A[k].S + l * A[k].G1[c] - pgt);
                    o[3 + c] = 0.25 * (tg3[c] * A[k].S + l * A[k].G2[c] + pgt);
                }
            } else if constexpr (OP == OP_APPLY) {
                // h_I / l_I = A1 / 2 (to +i2, -i1) and l_I / 2 = l_I A2 / 8 (to both endpoints)
                double l = pa.na.ell[I];
                for (int c = 0; c < 3; ++c) {
                    o[c] = 0.5 * A[k].A1[c];
                    o[3 + c] = 0.125 * l * A[k].A2[c];
                }
            } else {
                double l = pa.na.ell[I];
                o[0] = A[k].Sw / (2.0 * l) + l * A[k].Sw0 / 16.0;
            }
        }
    }
}

// ---------------------------------------------------------------------------------- reductions / gathers

// rows[I] = (l_I / 4) sum_slots part[slot][I]
__global__ void k_energy_rows(int nE, int nslots_max, const int *__restrict__ eslots, const double *__restrict__ part,
                              const double *__restrict__ ell, double *__restrict__ rows)
{
    int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nE) return;
    double s = 0.0;
    int ns = eslots[I];
    for (int k = 0; k < ns; ++k) s += part[(size_t)k * nE + I];
    rows[I] = 0.25 * ell[I] * s;
}

// Per-problem sums of a per-edge array (deterministic: one block per problem, fixed order).
__global__ void k_segment_sum(const int *__restrict__ off, const double *__restrict__ x, double *__restrict__ out)
{
    int q = blockIdx.x;
    int b = off[q], e = off[q + 1];
    double s = 0.0;
    for (int i = b + threadIdx.x; i < e; i += blockDim.x) s += x[i];
    __shared__ double sh[256];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = sh[0];
}

// out_v = sum_{(I, slot) in inc(v)} sum_k part[k][I][slot*3 + c] (diff: slot selects G_i1 / G_i2;
// apply: -/+ first triple plus the second triple).
template <int OP>
__global__ void k_vertex_gather(int nV, int nE, const int *__restrict__ inc_ptr, const int *__restrict__ inc,
                                const int *__restrict__ eslots, const double *__restrict__ part,
                                double *__restrict__ out)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nV) return;
    double o[3] = {0, 0, 0};
    for (int k = inc_ptr[v]; k < inc_ptr[v + 1]; ++k) {
        int I = inc[k] >> 1, sl = inc[k] & 1;
        int ns = eslots[I];
        for (int q = 0; q < ns; ++q) {
            const double *p = part + ((size_t)q * nE + I) * (OP == OP_DIAG ? 1 : 6);
            if constexpr (OP == OP_DIFF) {
                for (int c = 0; c < 3; ++c) o[c] += p[3 * sl + c];
            } else if constexpr (OP == OP_APPLY) {
                double sg = sl ? 1.0 : -1.0;
                for (int c = 0; c < 3; ++c) o[c] += sg * p[c] + p[3 + c];
            } else {
                o[0] += p[0];
            }
        }
    }
    if constexpr (OP == OP_DIAG) {
        out[v] = o[0];
    } else {
        for (int c = 0; c < 3; ++c) out[3 * v + c] = o[c];
    }
}

// ---------------------------------------------------------------------------------- planning

// Build the (target block, source chunk) queue of one pass.  Items of big problems come first
// so the persistent grid ends with the small ones.
static void plan_pass(Ctx &c, Ctx::Plan &pl, int tpt, int occupancy)
{
    const int tb = kThreads * tpt;
    std::vector<WorkItem> items;
    // neighbour spans per target block: min/max edge index sharing a vertex with the block
    std::vector<int> vmin(c.nV, INT32_MAX), vmax(c.nV, -1);
    for (int I = 0; I < c.nE; ++I)
        for (int s = 0; s < 2; ++s) {
            int v = c.h_edges[2 * I + s];
            vmin[v] = std::min(vmin[v], I);
            vmax[v] = std::max(vmax[v], I);
        }
    const int target_items = std::max(1, 3 * c.sm_count * std::max(1, occupancy));
    // total work estimate to size chunks
    double total = 0.0;
    for (int q = 0; q < c.nProb; ++q) {
        double n = c.h_prob_e[q + 1] - c.h_prob_e[q];
        total += n * n;
    }
    int max_slots = 1;
    std::vector<int> eslots(c.nE, 1);
    struct Tmp {
        WorkItem w;
        double cost;
    };
    std::vector<Tmp> tmp;
    for (int q = 0; q < c.nProb; ++q) {
        int e0 = c.h_prob_e[q], e1 = c.h_prob_e[q + 1], n = e1 - e0;
        if (n <= 0) continue;
        int nblk = (n + tb - 1) / tb;
        // chunks so that this problem gets its share of the target item count
        double share = total > 0 ? (double)n * n / total : 1.0;
        int want = (int)std::ceil(share * target_items / nblk);
        int max_chunks = std::max(1, n / (8 * kTile));  // at least 8 source tiles per item
        int nch = std::min(std::max(1, want), max_chunks);
        nch = std::min(nch, 64);
        int clen = ((n + nch - 1) / nch + kTile - 1) / kTile * kTile;
        nch = (n + clen - 1) / clen;
        max_slots = std::max(max_slots, nch);
        for (int b = 0; b < nblk; ++b) {
            int t0 = e0 + b * tb, nt = std::min(tb, e1 - t0);
            int lo = INT32_MAX, hi = -1;
            for (int I = t0; I < t0 + nt; ++I)
                for (int s = 0; s < 2; ++s) {
                    int v = c.h_edges[2 * I + s];
                    lo = std::min(lo, vmin[v]);
                    hi = std::max(hi, vmax[v]);
                }
            for (int k = 0; k < nch; ++k) {
                int s0 = e0 + k * clen, s1 = std::min(e1, s0 + clen);
                WorkItem w{t0, nt, s0, s1, k, lo, hi, q};
                tmp.push_back({w, (double)nt * (s1 - s0)});
            }
        }
        for (int I = e0; I < e1; ++I) eslots[I] = nch;
    }
    std::stable_sort(tmp.begin(), tmp.end(), [](const Tmp &a, const Tmp &b) { return a.cost > b.cost; });
    for (auto &t : tmp) items.push_back(t.w);
    pl.n_items = (int)items.size();
    pl.max_slots = max_slots;
    pl.tpt = tpt;
    pl.grid = std::max(1, std::min(pl.n_items, c.sm_count * std::max(1, occupancy)));
    cudaMalloc(&pl.d_items, sizeof(WorkItem) * std::max<size_t>(1, items.size()));
    cudaMemcpy(pl.d_items, items.data(), sizeof(WorkItem) * items.size(), cudaMemcpyHostToDevice);
    cudaMalloc(&pl.d_eslots, sizeof(int) * std::max(1, c.nE));
    cudaMemcpy(pl.d_eslots, eslots.data(), sizeof(int) * c.nE, cudaMemcpyHostToDevice);
}

template <int PREC, int OP, int TPT>
static int occupancy_of(const Ctx &c)
{
    int occ = 0;
    if (c.kp.fast)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pairs<PREC, OP, TPT, true>, kThreads, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pairs<PREC, OP, TPT, false>, kThreads, 0);
    return occ;
}

constexpr int kTptEnergy = 4, kTptDiff = 2, kTptApply = 2;
constexpr int kTptEnergy64 = 1, kTptDiff64 = 1, kTptApply64 = 1;

// ---------------------------------------------------------------------------------- profiling

constexpr int kProfSlots = 1024;

int prof_begin(Ctx &c, int op, cudaStream_t s)
{
    if (c.prof_pool.empty()) {
        c.prof_pool.resize(2 * kProfSlots);
        for (auto &e : c.prof_pool) cudaEventCreate(&e);
    }
    if ((int)c.prof_pending.size() == kProfSlots) prof_harvest(c);
    int slot = (int)c.prof_pending.size();
    c.prof_pending.push_back({op, slot});
    cudaEventRecord(c.prof_pool[2 * slot], s);
    return slot;
}

void prof_end(Ctx &c, int slot, cudaStream_t s) { cudaEventRecord(c.prof_pool[2 * slot + 1], s); }

void prof_harvest(Ctx &c)
{
    for (auto &pe : c.prof_pending) {
        cudaEventSynchronize(c.prof_pool[2 * pe.second + 1]);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c.prof_pool[2 * pe.second], c.prof_pool[2 * pe.second + 1]);
        c.prof_ms[pe.first] += ms;
        c.prof_n[pe.first] += 1;
    }
    c.prof_pending.clear();
}

void make_plans(Ctx &c)
{
    // The chunking must be identical across precisions of one op class; all slots share one layout,
    // so every pass of the context uses the same targets-per-thread within an op class.
    const bool p64 = c.prm.precision == TP_FP64;
    int oe, od, oa;
    if (p64) {
        oe = occupancy_of<P64, OP_ENERGY, kTptEnergy64>(c);
        od = occupancy_of<P64, OP_DIFF, kTptDiff64>(c);
        oa = occupancy_of<P64, OP_APPLY, kTptApply64>(c);
    } else if (c.prm.precision == TP_MIXED) {
        oe = occupancy_of<PMIX, OP_ENERGY, kTptEnergy>(c);
        od = occupancy_of<PMIX, OP_DIFF, kTptDiff>(c);
        oa = occupancy_of<PMIX, OP_APPLY, kTptApply>(c);
    } else {
        oe = occupancy_of<P32, OP_ENERGY, kTptEnergy>(c);
        od = occupancy_of<P32, OP_DIFF, kTptDiff>(c);
        oa = occupancy_of<P32, OP_APPLY, kTptApply>(c);
    }
    plan_pass(c, c.plan_energy, p64 ? kTptEnergy64 : kTptEnergy, oe);
    plan_pass(c, c.plan_diff, p64 ? kTptDiff64 : kTptDiff, od);
    plan_pass(c, c.plan_apply, p64 ? kTptApply64 : kTptApply, oa);
}

// ---------------------------------------------------------------------------------- no-allocation energy

// Items of one problem spanning all edges (target blocks x source chunks); every tile checks
// disjointness (the neighbour span is the whole range) because no incidence lists are built.
__global__ void k_static_items(int nE, int tb, int clen, int nch, WorkItem *items, int *eslots, int *off)
{
    int it = blockIdx.x * blockDim.x + threadIdx.x;
    int nblk = (nE + tb - 1) / tb;
    if (it < nblk * nch) {
        int b = it / nch, k = it % nch;
        int t0 = b * tb, s0 = k * clen;
        items[it] = WorkItem{t0, min(tb, nE - t0), s0, min(nE, s0 + clen), k, 0, nE - 1, 0};
    }
    if (it < nE) eslots[it] = nch;
    if (it == 0) {
        off[0] = 0;
        off[1] = nE;
    }
}

__global__ void k_static_stats(int nV, int nE, const double *__restrict__ g, const double *__restrict__ ell,
                               double *__restrict__ out)
{
    __shared__ double sh[7][256];
    double b[7] = {1e300, 1e300, 1e300, -1e300, -1e300, -1e300, 0.0};
    for (int i = threadIdx.x; i < nV; i += blockDim.x)
        for (int k = 0; k < 3; ++k) {
            b[k] = fmin(b[k], g[3 * i + k]);
            b[3 + k] = fmax(b[3 + k], g[3 * i + k]);
        }
    for (int I = threadIdx.x; I < nE; I += blockDim.x) b[6] += ell[I];
    for (int k = 0; k < 7; ++k) sh[k][threadIdx.x] = b[k];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int k = 0; k < 7; ++k)
                sh[k][threadIdx.x] = k < 3 ? fmin(sh[k][threadIdx.x], sh[k][threadIdx.x + w])
                                           : (k < 6 ? fmax(sh[k][threadIdx.x], sh[k][threadIdx.x + w])
                                                    : sh[k][threadIdx.x] + sh[k][threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < 3; ++k) s += (sh[3 + k][0] - sh[k][0]) * (sh[3 + k][0] - sh[k][0]);
        out[0] = sh[6][0] / (nE > 0 ? nE : 1);  // mean edge length
        out[1] = sqrt(s);                       // bounding-box diagonal
    }
}

cudaError_t static_energy_launch(const double *gamma, const int *edges, int nV, int nE, double alpha, double beta,
                                 double near_cutoff, RecF *recF, RecLo *recLo, double *ell, double *T, double *x,
                                 WorkItem *items, int *eslots, double *part, double *rows, int *counter, int *err,
                                 double *scal, int *off, int max_items, int max_slots, double *E, cudaStream_t s,
                                 int *status)
{
    *status = 0;
    if (nE == 0) return cudaMemsetAsync(E, 0, sizeof(double), s);
    TPE_CHECK(cudaMemsetAsync(err, 0, sizeof(int), s));
    k_records<<<(nE + 255) / 256, 256, 0, s>>>(nE, gamma, edges, recF, recLo, nullptr, ell, T, x, err);
    k_static_stats<<<1, 256, 0, s>>>(nV, nE, gamma, ell, scal);
    TPE_CHECK(cudaGetLastError());
    // the cutoffs are kernel arguments: read the two statistics and the error word (synchronises)
    double st[2] = {0.0, 0.0};
    int e = 0;
    TPE_CHECK(cudaMemcpyAsync(st, scal, sizeof(st), cudaMemcpyDeviceToHost, s));
    TPE_CHECK(cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    TPE_CHECK(cudaStreamSynchronize(s));
    if (e) {
        *status = e;
        return cudaSuccess;
    }
    KernelParams kp{};
    kp.alpha = alpha;
    kp.beta = beta;
    kp.p = 2.0 * ((beta - 1.0) / alpha - 1.0) + 1.0;
    kp.fast = (alpha == 2.0 && beta == 4.5) ? 1 : 0;
    double rn = near_cutoff * st[0];
    kp.near2 = rn * rn;
    kp.near2f = (float)(rn * rn);
    kp.near2f_diff = (float)(16.0 * rn * rn);
    kp.mid2f = 3.0e38f;  // double-float positions in every tile (the context's default)
    // blocking: targets per item = kThreads * kTptEnergy, at least 8 source tiles per item
    int dev = 0, sms = 0, occ = 0;
    TPE_CHECK(cudaGetDevice(&dev));
    TPE_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (kp.fast)
        TPE_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pairs<PMIX, OP_ENERGY, kTptEnergy, true>, kThreads, 0));
    else
        TPE_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pairs<PMIX, OP_ENERGY, kTptEnergy, false>, kThreads, 0));
    const int tb = kThreads * kTptEnergy;
    const int nblk = (nE + tb - 1) / tb;
    int want = (3 * sms * std::max(1, occ) + nblk - 1) / nblk;
    int nch = std::min(std::min(std::max(1, want), std::max(1, nE / (8 * kTile))), max_slots);
    int clen = ((nE + nch - 1) / nch + kTile - 1) / kTile * kTile;
    nch = (nE + clen - 1) / clen;
    if (nblk * nch > max_items || nch > max_slots) return cudaErrorInvalidValue;
    const int nit = nblk * nch;
    k_static_items<<<(std::max(nit, nE) + 255) / 256, 256, 0, s>>>(nE, tb, clen, nch, items, eslots, off);
    TPE_CHECK(cudaMemsetAsync(counter, 0, sizeof(int), s));
    PairArgs pa;
    pa.items = items;
    pa.n_items = nit;
    pa.counter = counter;
    pa.recF = recF;
    pa.recLo = recLo;
    pa.recD = nullptr;
    pa.urecF = nullptr;
    pa.urecD = nullptr;
    pa.na = NearArgs{gamma, edges, ell, T, nullptr};
    pa.part = part;
    pa.nE = nE;
    pa.kp = kp;
    pa.skip = nullptr;
    const int grid = std::max(1, std::min(nit, sms * std::max(1, occ)));
    if (kp.fast)
        k_pairs<PMIX, OP_ENERGY, kTptEnergy, true><<<grid, kThreads, 0, s>>>(pa);
    else
        k_pairs<PMIX, OP_ENERGY, kTptEnergy, false><<<grid, kThreads, 0, s>>>(pa);
    k_energy_rows<<<(nE + 255) / 256, 256, 0, s>>>(nE, nch, eslots, part, ell, rows);
    k_segment_sum<<<1, 256, 0, s>>>(off, rows, E);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------- launchers

cudaError_t build_records(Ctx &c, const double *gamma, int which, cudaStream_t s)
{
    int nb = (c.nE + 255) / 256;
    const bool p64 = c.prm.precision == TP_FP64, mix = c.prm.precision == TP_MIXED;
    RecF *rf = p64 ? nullptr : (which ? c.d_recF2 : c.d_recF);
    RecLo *rl = mix ? (which ? c.d_recLo2 : c.d_recLo) : nullptr;
    RecD *rd = p64 ? (which ? c.d_recD2 : c.d_recD) : nullptr;
    if (c.nE == 0) return cudaSuccess;
    k_records<<<nb, 256, 0, s>>>(c.nE, gamma, c.d_edges, rf, rl, rd, c.d_ellw[which], c.d_Tw[which], c.d_xw[which], c.d_err);
    c.launches++;
    return cudaGetLastError();
}

cudaError_t build_urecs(Ctx &c, const double *u, int which, cudaStream_t s)
{
    if (c.nE == 0) return cudaSuccess;
    int nb = (c.nE + 255) / 256;
    const bool p64 = c.prm.precision == TP_FP64;
    k_urecs<<<nb, 256, 0, s>>>(c.nE, u, c.d_edges, c.d_ellw[which], p64 ? nullptr : c.d_urecF, p64 ? c.d_urecD : nullptr);
    c.launches++;
    return cudaGetLastError();
}

template <int OP>
static cudaError_t run_pairs(Ctx &c, int which, const double *gamma, const double *u, cudaStream_t s)
{
    Ctx::Plan &pl = (OP == OP_ENERGY) ? c.plan_energy : (OP == OP_DIFF ? c.plan_diff : c.plan_apply);
    if (pl.n_items == 0) return cudaSuccess;
    constexpr int ctr = OP;
    TPE_CHECK(cudaMemsetAsync(c.d_counter + ctr, 0, sizeof(int), s));
    PairArgs pa;
    pa.items = pl.d_items;
    pa.n_items = pl.n_items;
    pa.counter = c.d_counter + ctr;
    pa.recF = which ? c.d_recF2 : c.d_recF;
    pa.recLo = which ? c.d_recLo2 : c.d_recLo;
    pa.recD = which ? c.d_recD2 : c.d_recD;
    pa.urecF = c.d_urecF;
    pa.urecD = c.d_urecD;
    pa.na = NearArgs{gamma, c.d_edges, c.d_ellw[which], c.d_Tw[which], u};
    pa.part = c.d_part;
    pa.nE = c.nE;
    pa.kp = c.kp;
    pa.skip = (OP == OP_APPLY) ? c.d_skip : nullptr;
    const int g = pl.grid;
    const bool f = c.kp.fast != 0;
    // profiling: applies that skip converged problems are recorded apart (op 4), so op 2 always
    // times full passes of pairs_per_pass pairs
    const int slot = c.profile ? prof_begin(c, (OP == OP_APPLY && c.d_skip) ? 4 : OP, s) : -1;
    switch (c.prm.precision) {
    case TP_FP64:
        if (f) k_pairs<P64, OP, (OP == OP_ENERGY ? kTptEnergy64 : OP == OP_DIFF ? kTptDiff64 : kTptApply64), true><<<g, kThreads, 0, s>>>(pa);
        else k_pairs<P64, OP, (OP == OP_ENERGY ? kTptEnergy64 : OP == OP_DIFF ? kTptDiff64 : kTptApply64), false><<<g, kThreads, 0, s>>>(pa);
        break;
    case TP_MIXED:
        if (f) k_pairs<PMIX, OP, (OP == OP_ENERGY ? kTptEnergy : OP == OP_DIFF ? kTptDiff : kTptApply), true><<<g, kThreads, 0, s>>>(pa);
        else k_pairs<PMIX, OP, (OP == OP_ENERGY ? kTptEnergy : OP == OP_DIFF ? kTptDiff : kTptApply), false><<<g, kThreads, 0, s>>>(pa);
        break;
    default:
        if (f) k_pairs<P32, OP, (OP == OP_ENERGY ? kTptEnergy : OP == OP_DIFF ? kTptDiff : kTptApply), true><<<g, kThreads, 0, s>>>(pa);
        else k_pairs<P32, OP, (OP == OP_ENERGY ? kTptEnergy : OP == OP_DIFF ? kTptDiff : kTptApply), false><<<g, kThreads, 0, s>>>(pa);
        break;
    }
    if (slot >= 0) prof_end(c, slot, s);
    c.launches++;
    return cudaGetLastError();
}

cudaError_t pair_energy(Ctx &c, const double *gamma, int which, double *rows_out, double *E_out, cudaStream_t s)
{
    TPE_CHECK(run_pairs<OP_ENERGY>(c, which, gamma, nullptr, s));
    double *rows = rows_out ? rows_out : c.d_rows;
    if (c.nE > 0) {
        k_energy_rows<<<(c.nE + 255) / 256, 256, 0, s>>>(c.nE, c.plan_energy.max_slots, c.plan_energy.d_eslots, c.d_part, c.d_ellw[which],
                                                         rows);
        c.launches++;
    }
    if (E_out) {
        k_segment_sum<<<c.nProb, 256, 0, s>>>(c.d_prob_e, rows, E_out);
        c.launches++;
    }
    return cudaGetLastError();
}

cudaError_t pair_diff(Ctx &c, const double *gamma, int which, double *dE, cudaStream_t s)
{
    TPE_CHECK(run_pairs<OP_DIFF>(c, which, gamma, nullptr, s));
    if (c.nV > 0) {
        k_vertex_gather<OP_DIFF><<<(c.nV + 255) / 256, 256, 0, s>>>(c.nV, c.nE, c.d_inc_ptr, c.d_inc, c.plan_diff.d_eslots,
                                                                    c.d_part, dE);
        c.launches++;
    }
    return cudaGetLastError();
}

cudaError_t pair_apply(Ctx &c, const double *gamma_geom, int which, const double *u, double *Au, cudaStream_t s)
{
    TPE_CHECK(build_urecs(c, u, which, s));
    TPE_CHECK(run_pairs<OP_APPLY>(c, which, gamma_geom, u, s));
    if (c.nV > 0) {
        k_vertex_gather<OP_APPLY><<<(c.nV + 255) / 256, 256, 0, s>>>(c.nV, c.nE, c.d_inc_ptr, c.d_inc, c.plan_apply.d_eslots,
                                                                     c.d_part, Au);
        c.launches++;
    }
    return cudaGetLastError();
}

cudaError_t pair_diag(Ctx &c, const double *gamma_geom, int which, double *diag, cudaStream_t s)
{
    TPE_CHECK(run_pairs<OP_DIAG>(c, which, gamma_geom, nullptr, s));
    if (c.nV > 0) {
        k_vertex_gather<OP_DIAG><<<(c.nV + 255) / 256, 256, 0, s>>>(c.nV, c.nE, c.d_inc_ptr, c.d_inc, c.plan_apply.d_eslots,
                                                                    c.d_part, diag);
        c.launches++;
    }
    return cudaGetLastError();
}

}  // namespace tpe
