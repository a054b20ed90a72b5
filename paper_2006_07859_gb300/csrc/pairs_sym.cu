// Symmetric Sobolev apply: every unordered pair of disjoint edges {I, J} evaluated once.
//
// The Gram weights are symmetric: w_IJ = w_JI and the low-order weight enters as w0_IJ + w0_JI
// (Secs. 5.2.2-5.2.3).  One evaluation of a pair therefore yields what row I receives from J and what
// row J receives from I:
//   row I: h += l_J sw ((du_I - du_J) + (|T_I - T_J|^2 / 2) du_J),   l += l_J sw0 (ub_I - ub_J)
//   row J: h += l_I sw ((du_J - du_I) + (|T_I - T_J|^2 / 2) du_I),   l += l_I sw0 (ub_J - ub_I)
// with sw = sum_ab |d_ab|^-p and sw0 = sum_ab (|T_I x d_ab|^2 + |T_J x d_ab|^2) |d_ab|^-(4+p).  The chords
// and weights are bitwise the same from either side (pair_device.cuh), so the result equals the
// gather pass's up to summation order.
//
// Work items are pairs of edge blocks (b, c >= b) of one problem (block = 128 x TPT edges).  For
// b < c the CTA owns the targets of block b in registers and streams block c through shared memory;
// lane l of each warp visits source (step + l) mod P at step `step`, so the 32 lanes of a warp always
// touch 32 distinct sources and add what those sources receive into the warp's own Kahan-compensated
// shared-memory accumulators (no atomics).  Target rows of block b write partial slot c, source rows of
// block c write slot b, and the diagonal item (b, b) is a plain gather over its own block writing slot
// b: every row receives exactly one write per slot m = 0 .. nblk - 1, and the vertex gather sums the
// slots in index order, so the pass is deterministic.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "pair_device.cuh"

namespace tpe {

#define TPE_CHECK(x)                      \
    do {                                  \
        cudaError_t e_ = (x);             \
        if (e_ != cudaSuccess) return e_; \
    } while (0)

constexpr int kSymWarps = kThreads / 32;

// One unordered pair in mixed precision: target-side terms Kahan-accumulated into `a`, source-side
// terms added to hs (high-order, 3) and ls (low-order, 3).
template <bool FAST, bool DF>
__device__ __forceinline__ void pair_apply_both(const Tgt<float> &t, const Src<PMIX> &s, const UVal<float> &tu,
                                                const UVal<float> &su, bool keep, const KernelParams &kp,
                                                Acc32<PMIX, OP_APPLY> &a, float (&hs)[3], float (&ls)[3])
{
    const float pp = (float)kp.p;
    V3<float> dd[4];
    chords<DF>(t, s, dd);
    float tt;
    V3<float> dp;
    const float cI1 = perp2(dd[0], t.T, tt, dp), cI2 = perp2(dd[1], t.T, tt, dp);
    const float cJ1 = perp2(dd[0], s.T, tt, dp), cJ2 = perp2(dd[2], s.T, tt, dp);
    const float c2s[4] = {cI1 + cJ1, cI2 + cJ1, cI1 + cJ2, cI2 + cJ2};
    float tw[4], tw0[4];
#pragma unroll
    for (int ab = 0; ab < 4; ++ab) {
        const float d2 = dot3(dd[ab], dd[ab]);
        float r2;
        const float rp = inv_pow<float, FAST, 1>(d2, pp, r2);
        tw[ab] = rp;
        tw0[ab] = c2s[ab] * (rp * r2 * r2);
    }
    const float sw = (tw[0] + tw[3]) + (tw[1] + tw[2]);
    const float sw0 = (tw0[0] + tw0[3]) + (tw0[1] + tw0[2]);
    const float Wt = keep ? s.ell * sw : 0.f, W0t = keep ? s.ell * sw0 : 0.f;
    const float Ws = keep ? t.ell * sw : 0.f, W0s = keep ? t.ell * sw0 : 0.f;
    V3<float> dT = {t.T.x - s.T.x, t.T.y - s.T.y, t.T.z - s.T.z};
    dT.x += t.Tl.x - s.Tm.x;
    dT.y += t.Tl.y - s.Tm.y;
    dT.z += t.Tl.z - s.Tm.z;
    const float omt = 0.5f * dot3(dT, dT);
    // differences of the double-float u records (exact difference form)
    const float ddv[3] = {(tu.dh.x - su.dh.x) + (tu.dl.x - su.dl.x), (tu.dh.y - su.dh.y) + (tu.dl.y - su.dl.y),
                          (tu.dh.z - su.dh.z) + (tu.dl.z - su.dl.z)};
    const float dbv[3] = {(tu.uh.x - su.uh.x) + (tu.ul.x - su.ul.x), (tu.uh.y - su.uh.y) + (tu.ul.y - su.ul.y),
                          (tu.uh.z - su.uh.z) + (tu.ul.z - su.ul.z)};
    const float sdh[3] = {su.dh.x, su.dh.y, su.dh.z}, tdh[3] = {tu.dh.x, tu.dh.y, tu.dh.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        kahan_add(a.A1[k], a.C1[k], Wt * (ddv[k] + omt * sdh[k]));
        kahan_add(a.A2[k], a.C2[k], W0t * dbv[k]);
        hs[k] += Ws * (omt * tdh[k] - ddv[k]);
        ls[k] -= W0s * dbv[k];
    }
}

// Staggered loop over one staged tile: lane l takes source (step + l) mod P, P = max(cnt, 32).
// CHECK: the tile overlaps the targets' neighbour span (test disjointness per pair); DF: double-float
// chords (every tile but the far ones); SRC: accumulate what the sources receive (off on the diagonal
// item, which is a plain gather).
template <int TPT, bool FAST, bool CHECK, bool DF, bool SRC>
__device__ __forceinline__ void sym_tile(const Tgt<float> (&tg)[TPT], const UVal<float> (&tu)[TPT],
                                         const bool (&valid)[TPT], const Tile<PMIX, true> &tl, int cnt,
                                         Acc32<PMIX, OP_APPLY> (&a)[TPT], float2 (*sac)[kTile],
                                         const KernelParams &kp)
{
    const int lane = threadIdx.x & 31;
    const int P = max(cnt, 32);
    for (int step = 0; step < P; ++step) {
        int j = step + lane;
        if (j >= P) j -= P;
        if (j < cnt) {
            Src<PMIX> s;
            load_source<PMIX, true>(s, tl, j);
            UVal<float> su;
            {
                const float4 x = tl.u[j].a, y = tl.u[j].b, z = tl.u[j].c;
                su.dh = {x.x, x.y, x.z};
                su.uh = {x.w, y.x, y.y};
                su.dl = {y.z, y.w, z.x};
                su.ul = {z.y, z.z, z.w};
            }
            float hs[3] = {0.f, 0.f, 0.f}, ls[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < TPT; ++k) {
                bool keep = valid[k];
                if constexpr (CHECK)
                    keep = keep & (s.j1 != tg[k].i1) & (s.j1 != tg[k].i2) & (s.j2 != tg[k].i1) & (s.j2 != tg[k].i2);
                pair_apply_both<FAST, DF>(tg[k], s, tu[k], su, keep, kp, a[k], hs, ls);
            }
            if constexpr (SRC) {
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    float2 h = sac[q][j], l = sac[3 + q][j];  // (sum, Kahan compensation)
                    kahan_add(h.x, h.y, hs[q]);
                    kahan_add(l.x, l.y, ls[q]);
                    sac[q][j] = h;
                    sac[3 + q][j] = l;
                }
            }
        }
        if constexpr (SRC) __syncwarp();  // the next step hands this lane's source to lane - 1
    }
}

template <int TPT, bool FAST>
__global__ void __launch_bounds__(kThreads, 2) k_pairs_sym(const PairArgs pa)
{
    __shared__ Tile<PMIX, true> tl;
    __shared__ float2 sac[kSymWarps][6][kTile];  // per warp and source: (sum, Kahan compensation)
    __shared__ int s_item;
    __shared__ float s_box[2][kThreads / 32][6];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(pa.counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= pa.n_items) break;
        const WorkItem w = pa.items[it];
        if (pa.skip && pa.skip[w.pad]) continue;  // problem already converged
        const int bslot = w.slot >> 16, cslot = w.slot & 0xffff;
        const bool diag = bslot == cslot;
        Tgt<float> tg[TPT];
        UVal<float> tu[TPT];
        bool valid[TPT];
#pragma unroll
        for (int k = 0; k < TPT; ++k) {
            const int loc = threadIdx.x + k * kThreads;
            valid[k] = loc < w.ntgt;  // clamped duplicates must not feed the source side
            const int I = w.tgt0 + min(loc, w.ntgt - 1);
            load_target<PMIX>(tg[k], I, pa.recF, pa.recLo, pa.recD);
            load_uval<PMIX>(tu[k], pa.urecF, pa.urecD, I);
        }
        Acc64<OP_APPLY> A[TPT];
        Acc32<PMIX, OP_APPLY> a[TPT];
#pragma unroll
        for (int k = 0; k < TPT; ++k) {
            acc64_zero<OP_APPLY>(A[k]);
            acc_zero<PMIX, OP_APPLY>(a[k]);
        }
        float tbox[6];
        {
            float b[6] = {1e30f, 1e30f, 1e30f, -1e30f, -1e30f, -1e30f};
#pragma unroll
            for (int k = 0; k < TPT; ++k) box_add(b, tg[k].p1, tg[k].p2);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                for (int q = 0; q < 6; ++q) {
                    const float v = __shfl_xor_sync(0xffffffffu, b[q], o);
                    b[q] = q < 3 ? fminf(b[q], v) : fmaxf(b[q], v);
                }
            for (int q = 0; q < 6; ++q) tbox[q] = b[q];
        }
        for (int s0 = w.src0; s0 < w.src1; s0 += kTile) {
            const int cnt = min(kTile, w.src1 - s0);
            __syncthreads();  // the previous tile's readers are done
            float sb[6] = {1e30f, 1e30f, 1e30f, -1e30f, -1e30f, -1e30f};
            if (threadIdx.x < cnt) {
                const int J = s0 + threadIdx.x;
                const RecF r = pa.recF[J];
                tl.r[threadIdx.x] = r;
                tl.lo[threadIdx.x] = pa.recLo[J];
                tl.u[threadIdx.x] = pa.urecF[J];
                box_add(sb, V3<float>{r.a.x, r.a.y, r.a.z}, V3<float>{r.b.x, r.b.y, r.b.z});
            }
            for (int t = lane; t < kTile; t += 32)
                for (int q = 0; q < 6; ++q) sac[wid][q][t] = make_float2(0.f, 0.f);
            block_box(sb, s_box[1]);  // contains the barrier that publishes the tile
            const bool check = !(s0 + cnt - 1 < w.nb_lo || s0 > w.nb_hi);
            float g2 = 0.f;
            for (int q = 0; q < 3; ++q) {
                const float gap = fmaxf(fmaxf(sb[q] - tbox[3 + q], tbox[q] - sb[3 + q]), 0.f);
                g2 += gap * gap;
            }
            const bool far = g2 >= pa.kp.mid2f;
            if (diag) {
                sym_tile<TPT, FAST, true, true, false>(tg, tu, valid, tl, cnt, a, sac[wid], pa.kp);
            } else if (check) {
                sym_tile<TPT, FAST, true, true, true>(tg, tu, valid, tl, cnt, a, sac[wid], pa.kp);
            } else if (!far) {
                sym_tile<TPT, FAST, false, true, true>(tg, tu, valid, tl, cnt, a, sac[wid], pa.kp);
            } else {
                sym_tile<TPT, FAST, false, false, true>(tg, tu, valid, tl, cnt, a, sac[wid], pa.kp);
            }
            // fold the target tile accumulators into FP64
#pragma unroll
            for (int k = 0; k < TPT; ++k) {
                acc_add(A[k], a[k]);
                acc_zero<PMIX, OP_APPLY>(a[k]);
            }
            if (!diag) {
                __syncthreads();  // every warp's source accumulators are complete
                if (threadIdx.x < cnt) {
                    const int J = s0 + threadIdx.x;
                    double v[6];
                    for (int q = 0; q < 6; ++q) {
                        double x = 0.0;
                        for (int wv = 0; wv < kSymWarps; ++wv)
                            x += (double)sac[wv][q][threadIdx.x].x - (double)sac[wv][q][threadIdx.x].y;
                        v[q] = x;
                    }
                    const double l = pa.na.ell[J];
                    double *o = pa.part + ((size_t)bslot * pa.nE + J) * 6;
                    for (int q = 0; q < 3; ++q) {
                        o[q] = 0.5 * v[q];
                        o[3 + q] = 0.125 * l * v[3 + q];
                    }
                }
            }
        }
        // target rows of block b: slot c
#pragma unroll
        for (int k = 0; k < TPT; ++k) {
            if (!valid[k]) continue;
            const int I = w.tgt0 + threadIdx.x + k * kThreads;
            const double l = pa.na.ell[I];
            double *o = pa.part + ((size_t)cslot * pa.nE + I) * 6;
            for (int q = 0; q < 3; ++q) {
                o[q] = 0.5 * A[k].A1[q];
                o[3 + q] = 0.125 * l * A[k].A2[q];
            }
        }
    }
}

// ---------------------------------------------------------------------------------- symmetric energy

// One unordered pair of the energy: the target row receives l_J sum_ab |T_I x d_ab|^alpha |d_ab|^-beta,
// the source row l_I sum_ab |T_J x d_ab|^alpha |d_ab|^-beta (Eqs. 17-18; the factor l_I / 4 of a row
// is applied when the rows are summed).  Near pairs take both |T x d|^2 in FP64.
template <bool FAST, bool DF>
__device__ __forceinline__ void pair_energy_both(const Tgt<float> &t, const Src<PMIX> &s, bool keep, bool near,
                                                 const KernelParams &kp, float &at, float &as)
{
    const float alpha = (float)kp.alpha, beta = (float)kp.beta;
    V3<float> dd[4];
    chords<DF>(t, s, dd);
    float tt;
    V3<float> dp;
    float cI[2] = {perp2(dd[0], t.T, tt, dp), perp2(dd[1], t.T, tt, dp)};  // depends on b only
    float cJ[2] = {perp2(dd[0], s.T, tt, dp), perp2(dd[2], s.T, tt, dp)};  // depends on a only
    if constexpr (DF)
        if (near) {
            cI[0] = perp2_near(t.p1, t.l1, s.q1, s.m1, t.T, t.Tl);
            cI[1] = perp2_near(t.p1, t.l1, s.q2, s.m2, t.T, t.Tl);
            cJ[0] = perp2_near(t.p1, t.l1, s.q1, s.m1, s.T, s.Tm);
            cJ[1] = perp2_near(t.p2, t.l2, s.q1, s.m1, s.T, s.Tm);
        }
    const float pI[2] = {pow_c<float, FAST>(cI[0], alpha), pow_c<float, FAST>(cI[1], alpha)};
    const float pJ[2] = {pow_c<float, FAST>(cJ[0], alpha), pow_c<float, FAST>(cJ[1], alpha)};
    float fI = 0.f, fJ = 0.f;
#pragma unroll
    for (int ab = 0; ab < 4; ++ab) {
        const float d2 = dot3(dd[ab], dd[ab]);
        float r2;
        const float rb = inv_pow<float, FAST, 0>(d2, beta, r2);
        fI += pI[ab & 1] * rb;
        fJ += pJ[ab >> 1] * rb;
    }
    at += keep ? s.ell * fI : 0.f;
    as += keep ? t.ell * fJ : 0.f;
}

// MODE 2: near pairs possible (|g_i1 - g_j1|^2 < near cutoff^2 take FP64 cross products); 1: double-float
// chords; 0: single-float chords (far tiles).
template <int TPT, bool FAST, bool CHECK, int MODE, bool SRC>
__device__ __forceinline__ void sym_energy_tile(const Tgt<float> (&tg)[TPT], const bool (&valid)[TPT],
                                                const Tile<PMIX, false> &tl, int cnt, float (&at)[TPT],
                                                float2 *sac, const KernelParams &kp)
{
    const int lane = threadIdx.x & 31;
    const int P = max(cnt, 32);
    for (int step = 0; step < P; ++step) {
        int j = step + lane;
        if (j >= P) j -= P;
        if (j < cnt) {
            Src<PMIX> s;
            load_source<PMIX, false>(s, tl, j);
            float as = 0.f;
#pragma unroll
            for (int k = 0; k < TPT; ++k) {
                bool keep = valid[k];
                if constexpr (CHECK)
                    keep = keep & (s.j1 != tg[k].i1) & (s.j1 != tg[k].i2) & (s.j2 != tg[k].i1) & (s.j2 != tg[k].i2);
                bool near = false;
                if constexpr (MODE == 2) {
                    const V3<float> e = diff3<true>(tg[k].p1, tg[k].l1, s.q1, s.m1);
                    near = keep && dot3(e, e) < kp.near2f;
                }
                pair_energy_both<FAST, (MODE >= 1)>(tg[k], s, keep, near, kp, at[k], as);
            }
            if constexpr (SRC) {
                float2 ac = sac[j];  // (sum, Kahan compensation)
                kahan_add(ac.x, ac.y, as);
                sac[j] = ac;
            }
        }
        if constexpr (SRC) __syncwarp();
    }
}

template <int TPT, bool FAST>
__global__ void __launch_bounds__(kThreads, 3) k_energy_sym(const PairArgs pa)
{
    __shared__ Tile<PMIX, false> tl;
    __shared__ float2 sac[kSymWarps][kTile];  // per warp and source: (sum, Kahan compensation)
    __shared__ int s_item;
    __shared__ float s_box[2][kThreads / 32][6];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(pa.counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= pa.n_items) break;
        const WorkItem w = pa.items[it];
        const int bslot = w.slot >> 16, cslot = w.slot & 0xffff;
        const bool diag = bslot == cslot;
        Tgt<float> tg[TPT];
        bool valid[TPT];
#pragma unroll
        for (int k = 0; k < TPT; ++k) {
            const int loc = threadIdx.x + k * kThreads;
            valid[k] = loc < w.ntgt;
            load_target<PMIX>(tg[k], w.tgt0 + min(loc, w.ntgt - 1), pa.recF, pa.recLo, pa.recD);
        }
        double A[TPT];
        float at[TPT];
#pragma unroll
        for (int k = 0; k < TPT; ++k) A[k] = 0.0;
        float tbox[6];
        {
            float b[6] = {1e30f, 1e30f, 1e30f, -1e30f, -1e30f, -1e30f};
#pragma unroll
            for (int k = 0; k < TPT; ++k) box_add(b, tg[k].p1, tg[k].p2);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                for (int q = 0; q < 6; ++q) {
                    const float v = __shfl_xor_sync(0xffffffffu, b[q], o);
                    b[q] = q < 3 ? fminf(b[q], v) : fmaxf(b[q], v);
                }
            for (int q = 0; q < 6; ++q) tbox[q] = b[q];
        }
        for (int s0 = w.src0; s0 < w.src1; s0 += kTile) {
            const int cnt = min(kTile, w.src1 - s0);
            __syncthreads();
            float sb[6] = {1e30f, 1e30f, 1e30f, -1e30f, -1e30f, -1e30f};
            if (threadIdx.x < cnt) {
                const int J = s0 + threadIdx.x;
                const RecF r = pa.recF[J];
                tl.r[threadIdx.x] = r;
                tl.lo[threadIdx.x] = pa.recLo[J];
                box_add(sb, V3<float>{r.a.x, r.a.y, r.a.z}, V3<float>{r.b.x, r.b.y, r.b.z});
            }
            for (int t = lane; t < kTile; t += 32) sac[wid][t] = make_float2(0.f, 0.f);
            block_box(sb, s_box[1]);
            const bool check = !(s0 + cnt - 1 < w.nb_lo || s0 > w.nb_hi);
            float g2 = 0.f;
            for (int q = 0; q < 3; ++q) {
                const float gap = fmaxf(fmaxf(sb[q] - tbox[3 + q], tbox[q] - sb[3 + q]), 0.f);
                g2 += gap * gap;
            }
            const int mode = g2 < pa.kp.near2f ? 2 : (g2 < pa.kp.mid2f ? 1 : 0);
#pragma unroll
            for (int k = 0; k < TPT; ++k) at[k] = 0.f;
            if (diag)
                sym_energy_tile<TPT, FAST, true, 2, false>(tg, valid, tl, cnt, at, sac[wid], pa.kp);
            else if (check || mode == 2)
                sym_energy_tile<TPT, FAST, true, 2, true>(tg, valid, tl, cnt, at, sac[wid], pa.kp);
            else if (mode == 1)
                sym_energy_tile<TPT, FAST, false, 1, true>(tg, valid, tl, cnt, at, sac[wid], pa.kp);
            else
                sym_energy_tile<TPT, FAST, false, 0, true>(tg, valid, tl, cnt, at, sac[wid], pa.kp);
#pragma unroll
            for (int k = 0; k < TPT; ++k) A[k] += (double)at[k];
            if (!diag) {
                __syncthreads();
                if (threadIdx.x < cnt) {
                    double x = 0.0;
                    for (int wv = 0; wv < kSymWarps; ++wv) x += (double)sac[wv][threadIdx.x].x - (double)sac[wv][threadIdx.x].y;
                    pa.part[(size_t)bslot * pa.nE + s0 + threadIdx.x] = x;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < TPT; ++k)
            if (valid[k]) pa.part[(size_t)cslot * pa.nE + w.tgt0 + threadIdx.x + k * kThreads] = A[k];
    }
}

// ---------------------------------------------------------------------------------- symmetric differential
//
// Row I accumulates (scaled by l_J) S = sum (f_I + f_J), G_a += v_ab, GT += -a_I (T_I . d_ab) d_ab, with
// v_ab = d(f_I + f_J)/dd at d_ab = g_ia - g_jb.  Row J sees d' = -d and accumulates (scaled by l_I) the
// same S, G_b -= v_ab (its endpoint b) and GT += -a_J (T_J . d_ab) d_ab.  Both tangents are double-float
// in |T x d|^2 and T . d (each is the target tangent of one of the two rows).

// source-side accumulator slots: 0 S, 1-3 G1, 4-6 G2, 7-9 GT
constexpr int kDS = 10;

template <bool FAST, bool DF>
__device__ __forceinline__ void pair_diff_both(const Tgt<float> &t, const Src<PMIX> &s, bool keep,
                                               const KernelParams &kp, Acc32<PMIX, OP_DIFF> &a,
                                               float (&src)[kDS])
{
    const float alpha = (float)kp.alpha, beta = (float)kp.beta;
    V3<float> dd[4];
    chords<DF>(t, s, dd);
    float tI[2], tJ[2], cI[2], cJ[2];
    V3<float> dpI[2], dpJ[2];
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        cI[b] = perp2_df(dd[b], t.T, t.Tl, tI[b], dpI[b]);
        cJ[b] = perp2_df(dd[2 * b], s.T, s.Tm, tJ[b], dpJ[b]);
    }
    float S = 0.f, G1[3] = {0, 0, 0}, G2[3] = {0, 0, 0}, GT[3] = {0, 0, 0};
    float H1[3] = {0, 0, 0}, H2[3] = {0, 0, 0}, HT[3] = {0, 0, 0};
#pragma unroll
    for (int ab = 0; ab < 4; ++ab) {
        const int ia = ab >> 1, jb = ab & 1;
        const V3<float> d = dd[ab];
        const float d2 = dot3(d, d);
        float r2;
        const float rb = inv_pow<float, FAST, 0>(d2, beta, r2);
        float fI, fJ, aI, aJ;
        if constexpr (FAST) {
            fI = cI[jb] * rb;
            fJ = cJ[ia] * rb;
            aI = aJ = 2.f * rb;
        } else {
            fI = pow_c<float, false>(cI[jb], alpha) * rb;
            fJ = pow_c<float, false>(cJ[ia], alpha) * rb;
            aI = cI[jb] > 0.f ? alpha * fI / cI[jb] : 0.f;
            aJ = cJ[ia] > 0.f ? alpha * fJ / cJ[ia] : 0.f;
        }
        const float fs = fI + fJ, cb = beta * fs * r2;
        const float v[3] = {aI * dpI[jb].x + aJ * dpJ[ia].x - cb * d.x, aI * dpI[jb].y + aJ * dpJ[ia].y - cb * d.y,
                            aI * dpI[jb].z + aJ * dpJ[ia].z - cb * d.z};
        float *G = ia ? G2 : G1, *H = jb ? H2 : H1;
        const float mI = -aI * (ia ? tI[jb] + t.ell : tI[jb]);
        const float mJ = -aJ * (jb ? tJ[ia] - s.ell : tJ[ia]);
        const float dv[3] = {d.x, d.y, d.z};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            G[k] += v[k];
            H[k] -= v[k];
            GT[k] += mI * dv[k];
            HT[k] += mJ * dv[k];
        }
        S += fs;
    }
    const float L = keep ? s.ell : 0.f, Ls = keep ? t.ell : 0.f;
    kahan_add(a.S, a.cS, keep ? L * S : 0.f);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        kahan_add(a.G1[k], a.c1[k], keep ? L * G1[k] : 0.f);
        kahan_add(a.G2[k], a.c2[k], keep ? L * G2[k] : 0.f);
        kahan_add(a.GT[k], a.cT[k], keep ? L * GT[k] : 0.f);
    }
    if (keep) {
        src[0] += Ls * S;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            src[1 + k] += Ls * H1[k];
            src[4 + k] += Ls * H2[k];
            src[7 + k] += Ls * HT[k];
        }
    }
}

// A near pair entirely in FP64 from the double-float positions and tangents: row I's terms into tgt,
// row J's into src (both FP64).
static __device__ __noinline__ void near_diff_both_df(const Tgt<float> &t, const Src<PMIX> &s, double alpha,
                                                      double beta, bool fast, DiffAcc64 &tgt, double (&src)[kDS])
{
    const double TI[3] = {(double)t.T.x + t.Tl.x, (double)t.T.y + t.Tl.y, (double)t.T.z + t.Tl.z};
    const double TJ[3] = {(double)s.T.x + s.Tm.x, (double)s.T.y + s.Tm.y, (double)s.T.z + s.Tm.z};
    const double L = s.ell, Ls = t.ell;
    for (int ab = 0; ab < 4; ++ab) {
        const V3<float> P = (ab < 2) ? t.p1 : t.p2, PL = (ab < 2) ? t.l1 : t.l2;
        const V3<float> Q = (ab & 1) ? s.q2 : s.q1, QL = (ab & 1) ? s.m2 : s.m1;
        const double d[3] = {(double)(P.x - Q.x) + (double)(PL.x - QL.x), (double)(P.y - Q.y) + (double)(PL.y - QL.y),
                             (double)(P.z - Q.z) + (double)(PL.z - QL.z)};
        const double tI = TI[0] * d[0] + TI[1] * d[1] + TI[2] * d[2];
        const double tJ = TJ[0] * d[0] + TJ[1] * d[1] + TJ[2] * d[2];
        double dpI[3], dpJ[3];
        for (int k = 0; k < 3; ++k) {
            dpI[k] = d[k] - tI * TI[k];
            dpJ[k] = d[k] - tJ * TJ[k];
        }
        const double cI2 = dpI[0] * dpI[0] + dpI[1] * dpI[1] + dpI[2] * dpI[2];
        const double cJ2 = dpJ[0] * dpJ[0] + dpJ[1] * dpJ[1] + dpJ[2] * dpJ[2];
        const double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        double rb, fI, fJ, aI, aJ;
        if (fast) {
            const double r = rsqrt(d2), r2 = r * r;
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
        const double cb = beta * (fI + fJ) / d2;
        double *G = ab < 2 ? tgt.G1 : tgt.G2;
        const int hb = (ab & 1) ? 4 : 1;
        for (int k = 0; k < 3; ++k) {
            const double v = aI * dpI[k] + aJ * dpJ[k] - cb * d[k];
            G[k] += L * v;
            tgt.GT[k] += -L * aI * tI * d[k];
            src[hb + k] -= Ls * v;
            src[7 + k] += -Ls * aJ * tJ * d[k];
        }
        tgt.S += L * (fI + fJ);
        src[0] += Ls * (fI + fJ);
    }
}

// Row output of the differential from its accumulators (Sec. 5.1 by the chain rule through l_I and T_I):
// G_i1 = (1/4)[-T S + l G1 - (Id - T T^t) GT],  G_i2 = (1/4)[T S + l G2 + (Id - T T^t) GT]
__device__ __forceinline__ void diff_row_out(const double *T, double l, double S, const double *G1,
                                             const double *G2, const double *GT, double *o)
{
    const double gt = T[0] * GT[0] + T[1] * GT[1] + T[2] * GT[2];
    for (int c = 0; c < 3; ++c) {
        const double pgt = GT[c] - gt * T[c];
        o[c] = 0.25 * (-T[c] * S + l * G1[c] - pgt);
        o[3 + c] = 0.25 * (T[c] * S + l * G2[c] + pgt);
    }
}

// MODE 2: near pairs (|g_i1 - g_j1| inside the differential's FP64 band) possible; 1 / 0 as in the energy.
template <int TPT, bool FAST, bool CHECK, int MODE, bool SRC>
__device__ __forceinline__ void sym_diff_tile(const Tgt<float> (&tg)[TPT], const bool (&valid)[TPT],
                                              const Tile<PMIX, false> &tl, int cnt, Acc32<PMIX, OP_DIFF> (&a)[TPT],
                                              Acc64<OP_DIFF> (&A)[TPT], float2 *sac,
                                              const KernelParams &kp)
{
    const int lane = threadIdx.x & 31;
    const int P = max(cnt, 32);
    for (int step = 0; step < P; ++step) {
        int j = step + lane;
        if (j >= P) j -= P;
        if (j < cnt) {
            Src<PMIX> s;
            load_source<PMIX, false>(s, tl, j);
            float src[kDS];
#pragma unroll
            for (int q = 0; q < kDS; ++q) src[q] = 0.f;
            double srcd[kDS];
            bool anynear = false;
#pragma unroll
            for (int k = 0; k < TPT; ++k) {
                bool keep = valid[k];
                if constexpr (CHECK)
                    keep = keep & (s.j1 != tg[k].i1) & (s.j1 != tg[k].i2) & (s.j2 != tg[k].i1) & (s.j2 != tg[k].i2);
                bool near = false;
                if constexpr (MODE == 2) {
                    const V3<float> e = diff3<true>(tg[k].p1, tg[k].l1, s.q1, s.m1);
                    near = keep && dot3(e, e) < kp.near2f_diff;
                }
                if (near) {
                    if (!anynear) {
#pragma unroll
                        for (int q = 0; q < kDS; ++q) srcd[q] = 0.0;
                        anynear = true;
                    }
                    if constexpr (SRC)
                        near_diff_both_df(tg[k], s, kp.alpha, kp.beta, FAST, A[k], srcd);
                    else
                        near_diff_df(tg[k], s, kp.alpha, kp.beta, FAST, A[k]);
                } else {
                    pair_diff_both<FAST, (MODE >= 1)>(tg[k], s, keep, kp, a[k], src);
                }
            }
            if constexpr (SRC) {
#pragma unroll
                for (int q = 0; q < kDS; ++q) {
                    const float2 ac = sac[q * kTile + j];  // (sum, Kahan compensation)
                    float acc = ac.x, cmp = ac.y;
                    if (anynear) {
                        // FP64 near terms as hi + lo so the compensated sum keeps their digits
                        const double tot = (double)src[q] + srcd[q];
                        const float hi = (float)tot;
                        kahan_add(acc, cmp, hi);
                        kahan_add(acc, cmp, (float)(tot - (double)hi));
                    } else {
                        kahan_add(acc, cmp, src[q]);
                    }
                    sac[q * kTile + j] = make_float2(acc, cmp);
                }
            }
        }
        if constexpr (SRC) __syncwarp();
    }
}

constexpr size_t kDiffSymDynSmem = sizeof(float) * 2 * kSymWarps * kDS * kTile;

// MB: resident CTAs per SM the register allocation is held to (2 needs no spills at either TPT; the
// variants with 3 / 4 trade a few spilled registers for more warps to hide latency).
template <int TPT, bool FAST, int MB>
__global__ void __launch_bounds__(kThreads, MB) k_diff_sym(const PairArgs pa)
{
    __shared__ Tile<PMIX, false> tl;
    __shared__ int s_item;
    __shared__ float s_box[2][kThreads / 32][6];
    extern __shared__ float dyn[];  // [kSymWarps][kDS][kTile] float2 (sum, Kahan compensation) per source
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2 *sac = reinterpret_cast<float2 *>(dyn) + (size_t)wid * kDS * kTile;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(pa.counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= pa.n_items) break;
        const WorkItem w = pa.items[it];
        const int bslot = w.slot >> 16, cslot = w.slot & 0xffff;
        const bool diag = bslot == cslot;
        Tgt<float> tg[TPT];
        bool valid[TPT];
#pragma unroll
        for (int k = 0; k < TPT; ++k) {
            const int loc = threadIdx.x + k * kThreads;
            valid[k] = loc < w.ntgt;
            load_target<PMIX>(tg[k], w.tgt0 + min(loc, w.ntgt - 1), pa.recF, pa.recLo, pa.recD);
        }
        Acc64<OP_DIFF> A[TPT];
        Acc32<PMIX, OP_DIFF> a[TPT];
#pragma unroll
        for (int k = 0; k < TPT; ++k) {
            acc64_zero<OP_DIFF>(A[k]);
            acc_zero<PMIX, OP_DIFF>(a[k]);
        }
        float tbox[6];
        {
            float b[6] = {1e30f, 1e30f, 1e30f, -1e30f, -1e30f, -1e30f};
#pragma unroll
            for (int k = 0; k < TPT; ++k) box_add(b, tg[k].p1, tg[k].p2);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                for (int q = 0; q < 6; ++q) {
                    const float v = __shfl_xor_sync(0xffffffffu, b[q], o);
                    b[q] = q < 3 ? fminf(b[q], v) : fmaxf(b[q], v);
                }
            for (int q = 0; q < 6; ++q) tbox[q] = b[q];
        }
        for (int s0 = w.src0; s0 < w.src1; s0 += kTile) {
            const int cnt = min(kTile, w.src1 - s0);
            __syncthreads();
            float sb[6] = {1e30f, 1e30f, 1e30f, -1e30f, -1e30f, -1e30f};
            if (threadIdx.x < cnt) {
                const int J = s0 + threadIdx.x;
                const RecF r = pa.recF[J];
                tl.r[threadIdx.x] = r;
                tl.lo[threadIdx.x] = pa.recLo[J];
                box_add(sb, V3<float>{r.a.x, r.a.y, r.a.z}, V3<float>{r.b.x, r.b.y, r.b.z});
            }
            for (int t = lane; t < kDS * kTile; t += 32) sac[t] = make_float2(0.f, 0.f);
            block_box(sb, s_box[1]);
            const bool check = !(s0 + cnt - 1 < w.nb_lo || s0 > w.nb_hi);
            float g2 = 0.f;
            for (int q = 0; q < 3; ++q) {
                const float gap = fmaxf(fmaxf(sb[q] - tbox[3 + q], tbox[q] - sb[3 + q]), 0.f);
                g2 += gap * gap;
            }
            const int mode = g2 < pa.kp.near2f_diff ? 2 : (g2 < pa.kp.mid2f ? 1 : 0);
            if (diag)
                sym_diff_tile<TPT, FAST, true, 2, false>(tg, valid, tl, cnt, a, A, sac, pa.kp);
            else if (check || mode == 2)
                sym_diff_tile<TPT, FAST, true, 2, true>(tg, valid, tl, cnt, a, A, sac, pa.kp);
            else if (mode == 1)
                sym_diff_tile<TPT, FAST, false, 1, true>(tg, valid, tl, cnt, a, A, sac, pa.kp);
            else
                sym_diff_tile<TPT, FAST, false, 0, true>(tg, valid, tl, cnt, a, A, sac, pa.kp);
#pragma unroll
            for (int k = 0; k < TPT; ++k) {
                acc_add(A[k], a[k]);
                acc_zero<PMIX, OP_DIFF>(a[k]);
            }
            if (!diag) {
                __syncthreads();
                if (threadIdx.x < cnt) {
                    const int J = s0 + threadIdx.x;
                    double v[kDS];
                    for (int q = 0; q < kDS; ++q) {
                        double x = 0.0;
                        for (int wv = 0; wv < kSymWarps; ++wv) {
                            const float2 ac = reinterpret_cast<const float2 *>(dyn)[((size_t)wv * kDS + q) * kTile + threadIdx.x];
                            x += (double)ac.x - (double)ac.y;
                        }
                        v[q] = x;
                    }
                    diff_row_out(pa.na.T + 3 * J, pa.na.ell[J], v[0], v + 1, v + 4, v + 7,
                                 pa.part + ((size_t)bslot * pa.nE + J) * 6);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < TPT; ++k) {
            if (!valid[k]) continue;
            const int I = w.tgt0 + threadIdx.x + k * kThreads;
            diff_row_out(pa.na.T + 3 * I, pa.na.ell[I], A[k].S, A[k].G1, A[k].G2, A[k].GT,
                         pa.part + ((size_t)cslot * pa.nE + I) * 6);
        }
    }
}

// ---------------------------------------------------------------------------------- host side

static int sym_occupancy(int tpt)
{
    int occ = 0;
    if (tpt == 1)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pairs_sym<1, true>, kThreads, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pairs_sym<2, true>, kThreads, 0);
    return occ;
}

// Edge blocks of 128 x tpt per problem; items (b, c >= b) sorted by problem size (large first).
void sym_plan_items(Ctx &c, Ctx::Plan &pl, int tpt, int occupancy)
{
    const int tb = kThreads * tpt;
    std::vector<int> vmin(c.nV, INT32_MAX), vmax(c.nV, -1);
    for (int I = 0; I < c.nE; ++I)
        for (int s = 0; s < 2; ++s) {
            const int v = c.h_edges[2 * I + s];
            vmin[v] = std::min(vmin[v], I);
            vmax[v] = std::max(vmax[v], I);
        }
    std::vector<std::pair<long long, WorkItem>> tmp;
    std::vector<int> eslots(std::max(1, c.nE), 1);
    int max_slots = 1;
    for (int q = 0; q < c.nProb; ++q) {
        const int e0 = c.h_prob_e[q], e1 = c.h_prob_e[q + 1], n = e1 - e0;
        if (n <= 0) continue;
        const int nblk = (n + tb - 1) / tb;
        max_slots = std::max(max_slots, nblk);
        for (int b = 0; b < nblk; ++b) {
            const int t0 = e0 + b * tb, nt = std::min(tb, e1 - t0);
            int lo = INT32_MAX, hi = -1;
            for (int I = t0; I < t0 + nt; ++I)
                for (int s = 0; s < 2; ++s) {
                    const int v = c.h_edges[2 * I + s];
                    lo = std::min(lo, vmin[v]);
                    hi = std::max(hi, vmax[v]);
                }
            for (int cb = b; cb < nblk; ++cb) {
                const int s0 = e0 + cb * tb, s1 = std::min(e1, s0 + tb);
                tmp.push_back({(long long)n, WorkItem{t0, nt, s0, s1, (b << 16) | cb, lo, hi, q}});
            }
        }
        for (int I = e0; I < e1; ++I) eslots[I] = nblk;
    }
    std::stable_sort(tmp.begin(), tmp.end(), [](const auto &a, const auto &b) { return a.first > b.first; });
    std::vector<WorkItem> items;
    items.reserve(tmp.size());
    for (auto &t : tmp) items.push_back(t.second);
    pl.n_items = (int)items.size();
    pl.max_slots = max_slots;
    pl.tpt = tpt;
    pl.grid = std::max(1, std::min(pl.n_items, c.sm_count * std::max(1, occupancy)));
    cudaMalloc(&pl.d_items, sizeof(WorkItem) * std::max<size_t>(1, items.size()));
    cudaMemcpy(pl.d_items, items.data(), sizeof(WorkItem) * items.size(), cudaMemcpyHostToDevice);
    cudaMalloc(&pl.d_eslots, sizeof(int) * std::max(1, c.nE));
    cudaMemcpy(pl.d_eslots, eslots.data(), sizeof(int) * std::max(1, c.nE), cudaMemcpyHostToDevice);
}

// Slots the symmetric pass needs per row (the largest problem's block count) at tpt targets per thread.
size_t sym_slots(const Ctx &c, int tpt)
{
    const int tb = kThreads * tpt;
    int m = 1;
    for (int q = 0; q < c.nProb; ++q) m = std::max(m, (c.h_prob_e[q + 1] - c.h_prob_e[q] + tb - 1) / tb);
    return (size_t)m;
}

// Switch the apply to the symmetric pass with tpt targets per thread (1 or 2), or back to the gather
// pass (tpt = 0).  Mixed precision with the specialised powers only; grows the partial buffer if needed.
cudaError_t sym_select(Ctx &c, int tpt)
{
    graphs_reset(c);
    Ctx::Plan &pl = c.plan_sym;
    if (pl.d_items) TPE_CHECK(cudaFree(pl.d_items));
    if (pl.d_eslots) TPE_CHECK(cudaFree(pl.d_eslots));
    pl = Ctx::Plan{};
    c.apply_sym = 0;
    if (tpt <= 0) return cudaSuccess;
    if (c.prm.precision != TP_MIXED || !c.kp.fast || (tpt != 1 && tpt != 2)) return cudaErrorInvalidValue;
    sym_plan_items(c, pl, tpt, sym_occupancy(tpt));
    const size_t need = (size_t)pl.max_slots * std::max(1, c.nE) * 6;
    if (need > c.part_elems) {
        TPE_CHECK(cudaFree(c.d_part));
        TPE_CHECK(cudaMalloc(&c.d_part, sizeof(double) * need));
        c.part_elems = need;
    }
    c.apply_sym = tpt;
    return cudaGetLastError();
}

static int sym_energy_occupancy(int tpt)
{
    int occ = 0;
    if (tpt == 1)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_energy_sym<1, true>, kThreads, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_energy_sym<2, true>, kThreads, 0);
    return occ;
}

// The energy's symmetric pass on (tpt 1, 2) or off (0); same conditions as sym_select.
cudaError_t sym_select_energy(Ctx &c, int tpt)
{
    Ctx::Plan &pl = c.plan_sym_e;
    if (pl.d_items) TPE_CHECK(cudaFree(pl.d_items));
    if (pl.d_eslots) TPE_CHECK(cudaFree(pl.d_eslots));
    pl = Ctx::Plan{};
    c.energy_sym = 0;
    if (tpt <= 0) return cudaSuccess;
    if (c.prm.precision != TP_MIXED || !c.kp.fast || (tpt != 1 && tpt != 2)) return cudaErrorInvalidValue;
    sym_plan_items(c, pl, tpt, sym_energy_occupancy(tpt));
    const size_t need = (size_t)pl.max_slots * std::max(1, c.nE);
    if (need > c.part_elems) {
        TPE_CHECK(cudaFree(c.d_part));
        TPE_CHECK(cudaMalloc(&c.d_part, sizeof(double) * need));
        c.part_elems = need;
    }
    c.energy_sym = tpt;
    return cudaGetLastError();
}

cudaError_t sym_energy_pass(Ctx &c, int which, const double *gamma, cudaStream_t s)
{
    Ctx::Plan &pl = c.plan_sym_e;
    if (pl.n_items == 0) return cudaSuccess;
    TPE_CHECK(cudaMemsetAsync(c.d_counter + 5, 0, sizeof(int), s));
    PairArgs pa;
    pa.items = pl.d_items;
    pa.n_items = pl.n_items;
    pa.counter = c.d_counter + 5;
    pa.recF = which ? c.d_recF2 : c.d_recF;
    pa.recLo = which ? c.d_recLo2 : c.d_recLo;
    pa.recD = nullptr;
    pa.urecF = nullptr;
    pa.urecD = nullptr;
    pa.na = NearArgs{gamma, c.d_edges, c.d_ellw[which], c.d_Tw[which], nullptr};
    pa.part = c.d_part;
    pa.nE = c.nE;
    pa.kp = c.kp;
    pa.skip = nullptr;
    const int slot = c.profile ? prof_begin(c, OP_ENERGY, s) : -1;
    if (pl.tpt == 1)
        k_energy_sym<1, true><<<pl.grid, kThreads, 0, s>>>(pa);
    else
        k_energy_sym<2, true><<<pl.grid, kThreads, 0, s>>>(pa);
    if (slot >= 0 || slot <= -2) prof_end(c, slot, s);
    c.launches++;
    return cudaGetLastError();
}

// Symmetric differential variants: 1 / 2 targets per thread at 2 CTAs per SM, 3: one target at 4 CTAs
// per SM, 4: two targets at 3 CTAs per SM.
static int diff_variant_tpt(int v)
{
    return (v == 2 || v == 4) ? 2 : 1;
}

template <class F>
static void with_diff_kernel(int v, F f)
{
    switch (v) {
        case 1: f(k_diff_sym<1, true, 2>); break;
        case 2: f(k_diff_sym<2, true, 2>); break;
        case 3: f(k_diff_sym<1, true, 4>); break;
        default: f(k_diff_sym<2, true, 3>); break;
    }
}

static int sym_diff_occupancy(int v)
{
    int occ = 0;
    with_diff_kernel(v, [&](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDiffSymDynSmem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, kDiffSymDynSmem);
    });
    return occ;
}

// The differential's symmetric pass on (tpt 1, 2) or off (0); same conditions as sym_select.
cudaError_t sym_select_diff(Ctx &c, int tpt)
{
    Ctx::Plan &pl = c.plan_sym_d;
    if (pl.d_items) TPE_CHECK(cudaFree(pl.d_items));
    if (pl.d_eslots) TPE_CHECK(cudaFree(pl.d_eslots));
    pl = Ctx::Plan{};
    c.diff_sym = 0;
    if (tpt <= 0) return cudaSuccess;
    if (c.prm.precision != TP_MIXED || !c.kp.fast || tpt > 4) return cudaErrorInvalidValue;
    sym_plan_items(c, pl, diff_variant_tpt(tpt), sym_diff_occupancy(tpt));
    pl.tpt = tpt;  // the variant (the plan's blocking follows its targets per thread)
    const size_t need = (size_t)pl.max_slots * std::max(1, c.nE) * 6;
    if (need > c.part_elems) {
        TPE_CHECK(cudaFree(c.d_part));
        TPE_CHECK(cudaMalloc(&c.d_part, sizeof(double) * need));
        c.part_elems = need;
    }
    c.diff_sym = tpt;
    return cudaGetLastError();
}

cudaError_t sym_diff_pass(Ctx &c, int which, const double *gamma, cudaStream_t s)
{
    Ctx::Plan &pl = c.plan_sym_d;
    if (pl.n_items == 0) return cudaSuccess;
    TPE_CHECK(cudaMemsetAsync(c.d_counter + 6, 0, sizeof(int), s));
    PairArgs pa;
    pa.items = pl.d_items;
    pa.n_items = pl.n_items;
    pa.counter = c.d_counter + 6;
    pa.recF = which ? c.d_recF2 : c.d_recF;
    pa.recLo = which ? c.d_recLo2 : c.d_recLo;
    pa.recD = nullptr;
    pa.urecF = nullptr;
    pa.urecD = nullptr;
    pa.na = NearArgs{gamma, c.d_edges, c.d_ellw[which], c.d_Tw[which], nullptr};
    pa.part = c.d_part;
    pa.nE = c.nE;
    pa.kp = c.kp;
    pa.skip = nullptr;
    const int slot = c.profile ? prof_begin(c, OP_DIFF, s) : -1;
    with_diff_kernel(pl.tpt, [&](auto kern) { kern<<<pl.grid, kThreads, kDiffSymDynSmem, s>>>(pa); });
    if (slot >= 0 || slot <= -2) prof_end(c, slot, s);
    c.launches++;
    return cudaGetLastError();
}

cudaError_t sym_apply_pass(Ctx &c, int which, const double *gamma, const double *u, cudaStream_t s)
{
    Ctx::Plan &pl = c.plan_sym;
    if (pl.n_items == 0) return cudaSuccess;
    TPE_CHECK(cudaMemsetAsync(c.d_counter + 4, 0, sizeof(int), s));
    PairArgs pa;
    pa.items = pl.d_items;
    pa.n_items = pl.n_items;
    pa.counter = c.d_counter + 4;
    pa.recF = which ? c.d_recF2 : c.d_recF;
    pa.recLo = which ? c.d_recLo2 : c.d_recLo;
    pa.recD = nullptr;
    pa.urecF = c.d_urecF;
    pa.urecD = nullptr;
    pa.na = NearArgs{gamma, c.d_edges, c.d_ellw[which], c.d_Tw[which], u};
    pa.part = c.d_part;
    pa.nE = c.nE;
    pa.kp = c.kp;
    pa.skip = c.d_skip;
    const int slot = c.profile ? prof_begin(c, c.d_skip ? 4 : 2, s) : -1;
    if (pl.tpt == 1)
        k_pairs_sym<1, true><<<pl.grid, kThreads, 0, s>>>(pa);
    else
        k_pairs_sym<2, true><<<pl.grid, kThreads, 0, s>>>(pa);
    if (slot >= 0 || slot <= -2) prof_end(c, slot, s);
    c.launches++;
    return cudaGetLastError();
}

}  // namespace tpe
