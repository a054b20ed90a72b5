// Device-side machinery of the pair passes, shared by the gather kernels (pairs.cu) and the
// symmetric apply (pairs_sym.cu): powers, record views, chords and |T x d|^2, the per-pair
// evaluation of every op, tile accumulators and the tile loop.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "tpe_internal.cuh"

namespace tpe {

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
    V3<R> e;           // edge vector g_i2 - g_i1 (rounded once from FP64 in PMIX)
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
        t.e = {t.p2.x - t.p1.x, t.p2.y - t.p1.y, t.p2.z - t.p1.z};
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
            t.e = {q.lo3.y, q.lo3.z, q.lo3.w};
        } else {
            t.l1 = {0.f, 0.f, 0.f};
            t.l2 = {0.f, 0.f, 0.f};
            t.Tl = {0.f, 0.f, 0.f};
            t.e = {t.p2.x - t.p1.x, t.p2.y - t.p1.y, t.p2.z - t.p1.z};
        }
    }
}

template <int PREC>
struct Src {
    using R = typename RealOf<PREC>::type;
    V3<R> q1, q2, T, m1, m2, Tm;  // m = lo parts
    V3<R> e;                      // edge vector g_j2 - g_j1
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
        s.e = V3<double>{s.q2.x - s.q1.x, s.q2.y - s.q1.y, s.q2.z - s.q1.z};
    } else {
        float4 a = tl.r[j].a, b = tl.r[j].b, c = tl.r[j].c;
        s.q1 = {a.x, a.y, a.z};
        s.ell = a.w;
        s.q2 = {b.x, b.y, b.z};
        s.T = {b.w, c.x, c.y};
        s.j1 = __float_as_int(c.z);
        s.j2 = __float_as_int(c.w);
        if constexpr (PREC == PMIX) {
            float4 l = tl.lo[j].lo, l2 = tl.lo[j].lo2, l3 = tl.lo[j].lo3;
            s.m1 = {l.x, l.y, l.z};
            s.m2 = {l.w, l2.x, l2.y};
            s.Tm = {l2.z, l2.w, l3.x};
            s.e = {l3.y, l3.z, l3.w};
        } else {
            s.e = {s.q2.x - s.q1.x, s.q2.y - s.q1.y, s.q2.z - s.q1.z};
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
static __device__ __noinline__ void near_diff_df(const Tgt<float> &t, const Src<PMIX> &s, double alpha, double beta,
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

// The four chords d_ab = g_ia - g_jb of a pair (index ab = 2 (a - 1) + (b - 1)), formed from d11
// by increments that mirror exactly between row I and row J: d12 = d11 - e_J, d21 = d11 + e_I,
// d22 = d11 + (e_I - e_J).  Seen from row J every chord is bitwise the negated chord of row I.
template <bool DF, class R, class TG, class SR>
__device__ __forceinline__ void chords(const TG &t, const SR &s, V3<R> (&dd)[4])
{
    const V3<R> d11 = diff3<DF>(t.p1, t.l1, s.q1, s.m1);
    const V3<R> eIJ = {t.e.x - s.e.x, t.e.y - s.e.y, t.e.z - s.e.z};
    dd[0] = d11;
    dd[1] = {d11.x - s.e.x, d11.y - s.e.y, d11.z - s.e.z};
    dd[2] = {d11.x + t.e.x, d11.y + t.e.y, d11.z + t.e.z};
    dd[3] = {d11.x + eIJ.x, d11.y + eIJ.y, d11.z + eIJ.z};
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

// The Gram weights of one pair: W = l_J sum_ab |d_ab|^-p and
// W0 = l_J sum_ab (|T_I x d_ab|^2 + |T_J x d_ab|^2) |d_ab|^-(p+4), both zero when the edges share a vertex
// (keep false); d2_11 = |d_11|^2.
// Since g_i2 = g_i1 + l_I T_I, T_I x (g_ia - g_jb) does not depend on a and T_J x (g_ia - g_jb) does not
// depend on b: two |T x d|^2 per tangent instead of four.  The chords come from d11 by increments that
// mirror exactly between row I and row J (d12 = d11 - e_J, d21 = d11 + e_I, d22 = d11 + (e_I - e_J)), and
// the four trapezoid terms are summed as (11 + 22) + (12 + 21): every quantity of the pair is bitwise the
// same (up to sign) from row I and from row J, so W_IJ = W_JI and W0_IJ + W0_JI are exact and the FP32
// operator stays exactly symmetric.
template <bool FAST, bool DF, class R, class SR>
__device__ __forceinline__ void gram_weights(const Tgt<R> &t, const SR &s, bool keep, R pp, R &W, R &W0, R &d2_11)
{
    V3<R> dd[4];
    chords<DF>(t, s, dd);
    R tt;
    V3<R> dp;
    const R cI1 = perp2(dd[0], t.T, tt, dp), cI2 = perp2(dd[1], t.T, tt, dp);  // |T_I x d_1b|^2
    const R cJ1 = perp2(dd[0], s.T, tt, dp), cJ2 = perp2(dd[2], s.T, tt, dp);  // |T_J x d_a1|^2
    const R c2s[4] = {cI1 + cJ1, cI2 + cJ1, cI1 + cJ2, cI2 + cJ2};
    R tw[4], tw0[4];
#pragma unroll
    for (int ab = 0; ab < 4; ++ab) {
        const R d2 = dot3(dd[ab], dd[ab]);
        if (ab == 0) d2_11 = d2;
        R r2;
        R rp = inv_pow<R, FAST, 1>(d2, pp, r2);
        tw[ab] = rp;
        tw0[ab] = c2s[ab] * (rp * r2 * r2);
    }
    const R sw = (tw[0] + tw[3]) + (tw[1] + tw[2]);
    const R sw0 = (tw0[0] + tw0[3]) + (tw0[1] + tw0[2]);
    W = keep ? s.ell * sw : (R)0;
    W0 = keep ? s.ell * sw0 : (R)0;
}

// |T_I - T_J|^2 / 2 = 1 - <T_I, T_J> (with the tangents' low parts when DF)
template <bool DF, class R, class SR>
__device__ __forceinline__ R tangent_gap(const Tgt<R> &t, const SR &s)
{
    V3<R> dT = {t.T.x - s.T.x, t.T.y - s.T.y, t.T.z - s.T.z};
    if constexpr (DF) {
        dT.x += t.Tl.x - s.Tm.x;
        dT.y += t.Tl.y - s.Tm.y;
        dT.z += t.Tl.z - s.Tm.z;
    }
    return (R)0.5 * dot3(dT, dT);
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
        V3<R> dd[4];
        chords<DF>(t, s, dd);
        R tt;
        V3<R> dp;
        R cI[2] = {perp2(dd[0], t.T, tt, dp), perp2(dd[1], t.T, tt, dp)};  // |T_I x d_1b|^2 = |T_I x d_2b|^2
        if constexpr (DF && sizeof(R) == 4)
            if (near) {
                cI[0] = perp2_near(t.p1, t.l1, s.q1, s.m1, t.T, t.Tl);
                cI[1] = perp2_near(t.p1, t.l1, s.q2, s.m2, t.T, t.Tl);
            }
        R f = 0;
#pragma unroll
        for (int ab = 0; ab < 4; ++ab) {
            const R d2 = dot3(dd[ab], dd[ab]);
            if (ab == 0) d2_11 = d2;
            R r2;
            f += pow_c<R, FAST>(cI[ab & 1], alpha) * inv_pow<R, FAST, 0>(d2, beta, r2);
        }
        R c = s.ell * f;
        a.s += keep ? c : (R)0;
    } else if constexpr (OP == OP_DIFF) {
        // |T_I x d_ab|, its perpendicular d - (T_I.d) T_I depend on b only (T_I . d_2b = T_I . d_1b + l_I);
        // |T_J x d_ab| and its perpendicular on a only
        V3<R> dd[4];
        chords<DF>(t, s, dd);
        R tI[2], tJ[2], cI[2], cJ[2];
        V3<R> dpI[2], dpJ[2];
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            if constexpr (DF && sizeof(R) == 4)
                cI[b] = perp2_df(dd[b], t.T, t.Tl, tI[b], dpI[b]);
            else
                cI[b] = perp2(dd[b], t.T, tI[b], dpI[b]);
            cJ[b] = perp2(dd[2 * b], s.T, tJ[b], dpJ[b]);
        }
        R S = 0, G1[3] = {0, 0, 0}, G2[3] = {0, 0, 0}, GT[3] = {0, 0, 0};
#pragma unroll
        for (int ab = 0; ab < 4; ++ab) {
            const int ia = ab >> 1, jb = ab & 1;
            const V3<R> d = dd[ab];
            const R d2 = dot3(d, d);
            if (ab == 0) d2_11 = d2;
            R r2;
            R rb = inv_pow<R, FAST, 0>(d2, beta, r2);
            R fI, fJ, aI, aJ;
            if constexpr (FAST) {
                fI = cI[jb] * rb;
                fJ = cJ[ia] * rb;
                aI = aJ = (R)2 * rb;
            } else {
                fI = pow_c<R, false>(cI[jb], alpha) * rb;
                fJ = pow_c<R, false>(cJ[ia], alpha) * rb;
                aI = cI[jb] > (R)0 ? alpha * fI / cI[jb] : (R)0;
                aJ = cJ[ia] > (R)0 ? alpha * fJ / cJ[ia] : (R)0;
            }
            R fs = fI + fJ;
            R cb = beta * fs * r2;
            R *G = ia ? G2 : G1;
            G[0] += aI * dpI[jb].x + aJ * dpJ[ia].x - cb * d.x;
            G[1] += aI * dpI[jb].y + aJ * dpJ[ia].y - cb * d.y;
            G[2] += aI * dpI[jb].z + aJ * dpJ[ia].z - cb * d.z;
            R m = -aI * (ia ? tI[jb] + t.ell : tI[jb]);
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
        R W, W0;
        gram_weights<FAST, DF>(t, s, keep, pp, W, W0, d2_11);
        if constexpr (OP == OP_DIAG) {
            a.Sw += W;
            a.Sw0 += W0;
        } else {
            // (du_I - du_J) + (|T_I - T_J|^2 / 2) du_J  and  ub_I - ub_J, differences of double-floats
            const R omt = tangent_gap<DF>(t, s);
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

}  // namespace tpe
