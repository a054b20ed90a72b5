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
                          double *__restrict__ T, double *__restrict__ x, int *__restrict__ err,
                          float *__restrict__ ell_lo)
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
    if (ell_lo) ell_lo[I] = (float)(l - (double)(float)l);
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
            q.lo3 = make_float4((float)(t[2] - (double)th[2]), (float)e[0], (float)e[1], (float)e[2]);
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

}  // namespace tpe

#include "pair_device.cuh"

namespace tpe {

// Resident CTAs per SM the register allocation is sized for: the differential and the 4-target
// apply / diag need more than the 170 registers per thread that 3 CTAs allow, so they get 2.
template <int PREC, int OP, int TPT>
__host__ __device__ constexpr int pair_min_blocks()
{
    return PREC == P64 ? 1 : ((OP == OP_DIFF || (TPT >= 4 && OP != OP_ENERGY)) ? 2 : 3);
}

template <int PREC, int OP, int TPT, bool FAST>
__global__ void __launch_bounds__(kThreads, (pair_min_blocks<PREC, OP, TPT>())) k_pairs(const PairArgs pa)
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

// Two-stage gather for many slots: each edge's slots are summed once (k_edge_slots), then every vertex
// combines its edges' sums (k_vertex_from_edges).  The one-stage gather reads an edge's slots once per
// endpoint, twice the traffic when an edge has tens of slots (the symmetric passes on long curves).
template <int OP>
__global__ void k_edge_slots(int nE, const int *__restrict__ eslots, const double *__restrict__ part,
                             double *__restrict__ esum)
{
    constexpr int W = OP == OP_DIAG ? 1 : 6;
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nE) return;
    double o[W];
    for (int c = 0; c < W; ++c) o[c] = 0.0;
    for (int q = 0; q < eslots[I]; ++q) {
        const double *p = part + ((size_t)q * nE + I) * W;
        for (int c = 0; c < W; ++c) o[c] += p[c];
    }
    for (int c = 0; c < W; ++c) esum[(size_t)I * W + c] = o[c];
}

template <int OP>
__global__ void k_vertex_from_edges(int nV, const int *__restrict__ inc_ptr, const int *__restrict__ inc,
                                    const double *__restrict__ esum, double *__restrict__ out)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nV) return;
    double o[3] = {0, 0, 0};
    for (int k = inc_ptr[v]; k < inc_ptr[v + 1]; ++k) {
        const int I = inc[k] >> 1, sl = inc[k] & 1;
        if constexpr (OP == OP_DIAG) {
            o[0] += esum[I];
        } else {
            const double *p = esum + 6 * (size_t)I;
            if constexpr (OP == OP_DIFF) {
                for (int c = 0; c < 3; ++c) o[c] += p[3 * sl + c];
            } else {
                const double sg = sl ? 1.0 : -1.0;
                for (int c = 0; c < 3; ++c) o[c] += sg * p[c] + p[3 + c];
            }
        }
    }
    if constexpr (OP == OP_DIAG) {
        out[v] = o[0];
    } else {
        for (int c = 0; c < 3; ++c) out[3 * v + c] = o[c];
    }
}

// Sum the partial slots of a pass into the per-vertex output, in one or two stages by slot count.
template <int OP>
static cudaError_t gather_slots(Ctx &c, const Ctx::Plan &pl, double *out, cudaStream_t s)
{
    if (c.nV == 0) return cudaSuccess;
    if (pl.max_slots > 2 && c.d_esum) {
        k_edge_slots<OP><<<(c.nE + 255) / 256, 256, 0, s>>>(c.nE, pl.d_eslots, c.d_part, c.d_esum);
        k_vertex_from_edges<OP><<<(c.nV + 255) / 256, 256, 0, s>>>(c.nV, c.d_inc_ptr, c.d_inc, c.d_esum, out);
        c.launches += 2;
    } else {
        k_vertex_gather<OP><<<(c.nV + 255) / 256, 256, 0, s>>>(c.nV, c.nE, c.d_inc_ptr, c.d_inc, pl.d_eslots, c.d_part,
                                                              out);
        c.launches++;
    }
    return cudaGetLastError();
}

cudaError_t gather_apply(Ctx &c, const Ctx::Plan &pl, double *Au, cudaStream_t s)
{
    return gather_slots<OP_APPLY>(c, pl, Au, s);
}

// ---------------------------------------------------------------------------------- planning

// Build the (target block, source chunk) queue of one pass.  Items of big problems come first
// so the persistent grid ends with the small ones.
void plan_pass(Ctx &c, Ctx::Plan &pl, int tpt, int occupancy)
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

constexpr int kTptEnergy = 4, kTptDiff = 2, kTptApply = 2;
constexpr int kTptEnergy64 = 1, kTptDiff64 = 1, kTptApply64 = 1;

template <int PREC, int OP, int TPT>
static int occupancy_of(const Ctx &c)
{
    int occ = 0;
    if constexpr (PREC == PMIX && !((OP == OP_ENERGY && TPT == kTptEnergy) || (OP == OP_DIFF && TPT == kTptDiff) ||
                                    ((OP == OP_APPLY || OP == OP_DIAG) && TPT == kTptApply))) {
        // candidate-only targets-per-thread values exist for the specialised powers alone
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pairs<PREC, OP, TPT, true>, kThreads, 0);
    } else if (c.kp.fast) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pairs<PREC, OP, TPT, true>, kThreads, 0);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pairs<PREC, OP, TPT, false>, kThreads, 0);
    }
    return occ;
}


// Targets per thread: the default of each op class, and the values the autotuner may choose for the
// mixed-precision passes with the specialised powers ((alpha, beta) = (2, 4.5)), the only kernels
// instantiated for every candidate.
static int op_class(int op) { return op == OP_ENERGY ? 0 : (op == OP_DIFF ? 1 : 2); }

int tpt_default(const Ctx &c, int cls)
{
    if (c.prm.precision == TP_FP64) return 1;
    return cls == 0 ? kTptEnergy : (cls == 1 ? kTptDiff : kTptApply);
}

static bool tunable(const Ctx &c) { return c.prm.precision == TP_MIXED && c.kp.fast; }

int tpt_candidates(const Ctx &c, int cls, int *out)
{
    if (!tunable(c)) {
        out[0] = tpt_default(c, cls);
        return 1;
    }
    if (cls == 1) {
        out[0] = 1;
        out[1] = 2;
        return 2;
    }
    out[0] = 1;
    out[1] = 2;
    out[2] = 4;
    return 3;
}

static int tpt_for(const Ctx &c, int cls) { return (tunable(c) && c.tpt[cls]) ? c.tpt[cls] : tpt_default(c, cls); }

template <int OP>
static int occupancy_fast_mixed(const Ctx &c, int tpt)
{
    if constexpr (OP == OP_DIFF) {
        return tpt == 1 ? occupancy_of<PMIX, OP, 1>(c) : occupancy_of<PMIX, OP, 2>(c);
    } else {
        return tpt == 1 ? occupancy_of<PMIX, OP, 1>(c)
                        : (tpt == 4 ? occupancy_of<PMIX, OP, 4>(c) : occupancy_of<PMIX, OP, 2>(c));
    }
}

// Launch the pair kernel of the mixed / specialised-power path with `tpt` targets per thread.
template <int OP>
static void launch_fast_mixed(int tpt, int g, cudaStream_t s, const PairArgs &pa)
{
    if constexpr (OP == OP_DIFF) {
        if (tpt == 1)
            k_pairs<PMIX, OP, 1, true><<<g, kThreads, 0, s>>>(pa);
        else
            k_pairs<PMIX, OP, 2, true><<<g, kThreads, 0, s>>>(pa);
    } else {
        if (tpt == 1)
            k_pairs<PMIX, OP, 1, true><<<g, kThreads, 0, s>>>(pa);
        else if (tpt == 4)
            k_pairs<PMIX, OP, 4, true><<<g, kThreads, 0, s>>>(pa);
        else
            k_pairs<PMIX, OP, 2, true><<<g, kThreads, 0, s>>>(pa);
    }
}

// ---------------------------------------------------------------------------------- profiling

constexpr int kProfSlots = 1024;

int prof_begin(Ctx &c, int op, cudaStream_t s)
{
    if (c.capturing) {  // inside a captured CG block: external event nodes on events the graph owns
        CgGraph &g = *c.capturing;
        const int k = (int)g.prof_op.size();
        if (2 * k + 1 >= (int)g.ev.size()) return -1;  // events are created before the capture
        g.prof_op.push_back(op);
        cudaEventRecordWithFlags(g.ev[2 * k], s, cudaEventRecordExternal);
        return -2 - k;
    }
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

void prof_end(Ctx &c, int slot, cudaStream_t s)
{
    if (slot <= -2) {
        cudaEventRecordWithFlags(c.capturing->ev[2 * (-2 - slot) + 1], s, cudaEventRecordExternal);
        return;
    }
    cudaEventRecord(c.prof_pool[2 * slot + 1], s);
}

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

static int occupancy_cls(const Ctx &c, int cls, int tpt)
{
    if (c.prm.precision == TP_FP64)
        return cls == 0 ? occupancy_of<P64, OP_ENERGY, kTptEnergy64>(c)
                        : (cls == 1 ? occupancy_of<P64, OP_DIFF, kTptDiff64>(c) : occupancy_of<P64, OP_APPLY, kTptApply64>(c));
    if (c.prm.precision == TP_MIXED) {
        if (tunable(c))
            return cls == 0 ? occupancy_fast_mixed<OP_ENERGY>(c, tpt)
                            : (cls == 1 ? occupancy_fast_mixed<OP_DIFF>(c, tpt) : occupancy_fast_mixed<OP_APPLY>(c, tpt));
        return cls == 0 ? occupancy_of<PMIX, OP_ENERGY, kTptEnergy>(c)
                        : (cls == 1 ? occupancy_of<PMIX, OP_DIFF, kTptDiff>(c) : occupancy_of<PMIX, OP_APPLY, kTptApply>(c));
    }
    return cls == 0 ? occupancy_of<P32, OP_ENERGY, kTptEnergy>(c)
                    : (cls == 1 ? occupancy_of<P32, OP_DIFF, kTptDiff>(c) : occupancy_of<P32, OP_APPLY, kTptApply>(c));
}

static Ctx::Plan &plan_of(Ctx &c, int cls) { return cls == 0 ? c.plan_energy : (cls == 1 ? c.plan_diff : c.plan_apply); }

void make_plans(Ctx &c)
{
    // Every slot of an op class shares one layout, so all passes of an op class use the same
    // targets-per-thread (the plan records it and the launch follows the plan).
    for (int cls = 0; cls < 3; ++cls) {
        const int t = tpt_for(c, cls);
        plan_pass(c, plan_of(c, cls), t, occupancy_cls(c, cls, t));
    }
}

cudaError_t replan(Ctx &c, int cls)
{
    graphs_reset(c);
    Ctx::Plan &pl = plan_of(c, cls);
    if (pl.d_items) TPE_CHECK(cudaFree(pl.d_items));
    if (pl.d_eslots) TPE_CHECK(cudaFree(pl.d_eslots));
    pl = Ctx::Plan{};
    const int t = tpt_for(c, cls);
    plan_pass(c, pl, t, occupancy_cls(c, cls, t));
    const int ms = std::max(std::max(c.plan_energy.max_slots, c.plan_diff.max_slots), c.plan_apply.max_slots);
    const size_t need = (size_t)ms * std::max(1, c.nE) * 6;
    if (need > c.part_elems) {
        TPE_CHECK(cudaFree(c.d_part));
        TPE_CHECK(cudaMalloc(&c.d_part, sizeof(double) * need));
        c.part_elems = need;
    }
    return cudaGetLastError();
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
    k_records<<<(nE + 255) / 256, 256, 0, s>>>(nE, gamma, edges, recF, recLo, nullptr, ell, T, x, err, nullptr);
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
    const bool p64 = c.prm.precision == TP_FP64;
    RecF *rf = p64 ? nullptr : (which ? c.d_recF2 : c.d_recF);
    // the low parts serve the mixed pair passes and, in FP32 contexts too, the double-float apply
    RecLo *rl = p64 ? nullptr : (which ? c.d_recLo2 : c.d_recLo);
    RecD *rd = p64 ? (which ? c.d_recD2 : c.d_recD) : nullptr;
    if (c.nE == 0) return cudaSuccess;
    k_records<<<nb, 256, 0, s>>>(c.nE, gamma, c.d_edges, rf, rl, rd, c.d_ellw[which], c.d_Tw[which], c.d_xw[which], c.d_err,
                                 p64 ? nullptr : c.d_ell_lo[which]);
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

cudaError_t segment_sum(Ctx &c, const double *rows, double *E, cudaStream_t s)
{
    k_segment_sum<<<c.nProb, 256, 0, s>>>(c.d_prob_e, rows, E);
    c.launches++;
    return cudaGetLastError();
}

cudaError_t build_urecs_into(Ctx &c, const double *u, int which, URecF *uf, URecD *ud, cudaStream_t s)
{
    if (c.nE == 0) return cudaSuccess;
    k_urecs<<<(c.nE + 255) / 256, 256, 0, s>>>(c.nE, u, c.d_edges, c.d_ellw[which], uf, ud);
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
        if (f) {
            launch_fast_mixed<OP>(pl.tpt, g, s, pa);  // the plan's targets per thread (autotuned or default)
        } else {
            if (pl.tpt != tpt_default(c, op_class(OP))) return cudaErrorInvalidValue;  // plan / kernel mismatch
            k_pairs<PMIX, OP, (OP == OP_ENERGY ? kTptEnergy : OP == OP_DIFF ? kTptDiff : kTptApply), false><<<g, kThreads, 0, s>>>(pa);
        }
        break;
    default:
        if (f) k_pairs<P32, OP, (OP == OP_ENERGY ? kTptEnergy : OP == OP_DIFF ? kTptDiff : kTptApply), true><<<g, kThreads, 0, s>>>(pa);
        else k_pairs<P32, OP, (OP == OP_ENERGY ? kTptEnergy : OP == OP_DIFF ? kTptDiff : kTptApply), false><<<g, kThreads, 0, s>>>(pa);
        break;
    }
    if (slot >= 0 || slot <= -2) prof_end(c, slot, s);
    c.launches++;
    return cudaGetLastError();
}

cudaError_t pair_energy(Ctx &c, const double *gamma, int which, double *rows_out, double *E_out, cudaStream_t s)
{
    const bool sym = c.energy_sym > 0;
    if (sym)
        TPE_CHECK(sym_energy_pass(c, which, gamma, s));
    else
        TPE_CHECK(run_pairs<OP_ENERGY>(c, which, gamma, nullptr, s));
    const Ctx::Plan &pl = sym ? c.plan_sym_e : c.plan_energy;
    double *rows = rows_out ? rows_out : c.d_rows;
    if (c.nE > 0) {
        k_energy_rows<<<(c.nE + 255) / 256, 256, 0, s>>>(c.nE, pl.max_slots, pl.d_eslots, c.d_part, c.d_ellw[which],
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
    const bool sym = c.diff_sym > 0;
    if (sym)
        TPE_CHECK(sym_diff_pass(c, which, gamma, s));
    else
        TPE_CHECK(run_pairs<OP_DIFF>(c, which, gamma, nullptr, s));
    return gather_slots<OP_DIFF>(c, sym ? c.plan_sym_d : c.plan_diff, dE, s);
}

cudaError_t pair_apply(Ctx &c, const double *gamma_geom, int which, const double *u, double *Au, cudaStream_t s)
{
    TPE_CHECK(build_urecs(c, u, which, s));
    const bool sym = c.apply_sym > 0;
    if (sym)
        TPE_CHECK(sym_apply_pass(c, which, gamma_geom, u, s));
    else
        TPE_CHECK(run_pairs<OP_APPLY>(c, which, gamma_geom, u, s));
    return gather_slots<OP_APPLY>(c, sym ? c.plan_sym : c.plan_apply, Au, s);
}

cudaError_t pair_diag(Ctx &c, const double *gamma_geom, int which, double *diag, cudaStream_t s)
{
    TPE_CHECK(run_pairs<OP_DIAG>(c, which, gamma_geom, nullptr, s));
    return gather_slots<OP_DIAG>(c, c.plan_apply, diag, s);
}

}  // namespace tpe
