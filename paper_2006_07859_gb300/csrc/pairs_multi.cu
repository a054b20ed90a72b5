// Sobolev apply on several vector fields at once: AU_f = A-bar U_f for f = 0 .. m-1 (Secs. 5.2.2-5.2.3;
// the paper applies the Gram matrix to one vector at a time).
//
// Per pair the Gram weights W, W0 and the tangent gap 1 - t_IJ take about 220 of the single apply's 255
// canonical FLOP and do not depend on u.  This gather pass (one thread per target row, source tiles in
// shared memory, the apply's work items) evaluates them once per ordered pair and applies them to
// kMultiG vector fields (3 kMultiG scalar columns): each further column costs the difference-form
// terms alone, W ((du_I - du_J) + (1 - t_IJ) du_J) and W0 (ub_I - ub_J), about 6 FLOP.  The arithmetic
// per column is the single apply's: double-float differences of u and Kahan-compensated FP32 sums in
// the mixed path, plain FP32 or FP64 otherwise.
#include <cuda_runtime.h>

#include <algorithm>

#include "tpe_internal.cuh"
#include "pair_device.cuh"

namespace tpe {

#define TPE_CHECK(x)                      \
    do {                                  \
        cudaError_t e_ = (x);             \
        if (e_ != cudaSuccess) return e_; \
    } while (0)

struct MultiArgs {
    const WorkItem *items;
    int n_items;
    int *counter;
    const RecF *recF;
    const RecLo *recLo;
    const RecD *recD;
    const URecF *urecF;  // [kMultiG][nE]
    const URecD *urecD;  // [kMultiG][nE]
    const double *ell;   // FP64 edge lengths
    double *part;        // [slot][nE][6 kMultiG]
    int nE;
    KernelParams kp;
};

template <class R>
__device__ __forceinline__ void multi_add(R &acc, R &c, R x)
{
    if constexpr (sizeof(R) == 4)
        kahan_add(acc, c, x);
    else
        acc += x;
}

template <int PREC, bool FAST>
__global__ void __launch_bounds__(kThreads, 2) k_apply_multi(const MultiArgs a)
{
    using R = typename RealOf<PREC>::type;
    constexpr bool DF = PREC == PMIX;
    constexpr bool KAHAN = PREC == PMIX;  // as the single apply: compensated in the mixed path only
    constexpr int G = kMultiG;
    __shared__ Tile<PREC, false> tl;
    __shared__ typename std::conditional<PREC == P64, URecD, URecF>::type tu_s[G][kTile];
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= a.n_items) break;
        const WorkItem w = a.items[it];
        const int I = w.tgt0 + min((int)threadIdx.x, w.ntgt - 1);
        Tgt<R> t;
        load_target<PREC>(t, I, a.recF, a.recLo, a.recD);
        UVal<R> tu[G];
#pragma unroll
        for (int g = 0; g < G; ++g) load_uval<PREC>(tu[g], a.urecF + (size_t)g * a.nE, a.urecD + (size_t)g * a.nE, I);
        const R pp = (R)a.kp.p;
        R a1[G][3], a2[G][3], k1[G][3], k2[G][3];
        double A1[G][3], A2[G][3];
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                a1[g][q] = a2[g][q] = k1[g][q] = k2[g][q] = (R)0;
                A1[g][q] = A2[g][q] = 0.0;
            }
        int tiles = 0;
        for (int s0 = w.src0; s0 < w.src1; s0 += kTile) {
            const int cnt = min(kTile, w.src1 - s0);
            __syncthreads();
            if (threadIdx.x < cnt) {
                const int J = s0 + threadIdx.x;
                if constexpr (PREC == P64) {
                    tl.r[threadIdx.x] = a.recD[J];
#pragma unroll
                    for (int g = 0; g < G; ++g) tu_s[g][threadIdx.x] = a.urecD[(size_t)g * a.nE + J];
                } else {
                    tl.r[threadIdx.x] = a.recF[J];
                    if constexpr (PREC == PMIX) tl.lo[threadIdx.x] = a.recLo[J];
#pragma unroll
                    for (int g = 0; g < G; ++g) tu_s[g][threadIdx.x] = a.urecF[(size_t)g * a.nE + J];
                }
            }
            __syncthreads();
            const bool check = !(s0 + cnt - 1 < w.nb_lo || s0 > w.nb_hi);
            for (int j = 0; j < cnt; ++j) {
                Src<PREC> s;
                load_source<PREC, false>(s, tl, j);
                const bool keep =
                    !check || ((s.j1 != t.i1) & (s.j1 != t.i2) & (s.j2 != t.i1) & (s.j2 != t.i2));
                R W, W0, d211;
                gram_weights<FAST, DF>(t, s, keep, pp, W, W0, d211);
                const R omt = tangent_gap<DF>(t, s);
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    UVal<R> su;
                    if constexpr (PREC == P64) {
                        const URecD u = tu_s[g][j];
                        su.dh = {u.du0.x, u.du0.y, u.du1.x};
                        su.uh = {u.ub0.x, u.ub0.y, u.ub1.x};
                    } else {
                        const float4 x = tu_s[g][j].a, y = tu_s[g][j].b, z = tu_s[g][j].c;
                        su.dh = {x.x, x.y, x.z};
                        su.uh = {x.w, y.x, y.y};
                        su.dl = {y.z, y.w, z.x};
                        su.ul = {z.y, z.z, z.w};
                    }
                    R dd[3] = {tu[g].dh.x - su.dh.x, tu[g].dh.y - su.dh.y, tu[g].dh.z - su.dh.z};
                    R db[3] = {tu[g].uh.x - su.uh.x, tu[g].uh.y - su.uh.y, tu[g].uh.z - su.uh.z};
                    if constexpr (DF) {
                        dd[0] += tu[g].dl.x - su.dl.x;
                        dd[1] += tu[g].dl.y - su.dl.y;
                        dd[2] += tu[g].dl.z - su.dl.z;
                        db[0] += tu[g].ul.x - su.ul.x;
                        db[1] += tu[g].ul.y - su.ul.y;
                        db[2] += tu[g].ul.z - su.ul.z;
                    }
                    const R dj[3] = {su.dh.x, su.dh.y, su.dh.z};
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        if constexpr (KAHAN) {
                            multi_add(a1[g][q], k1[g][q], W * (dd[q] + omt * dj[q]));
                            multi_add(a2[g][q], k2[g][q], W0 * db[q]);
                        } else {
                            a1[g][q] += W * (dd[q] + omt * dj[q]);
                            a2[g][q] += W0 * db[q];
                        }
                    }
                }
            }
            // fold the tile sums into FP64 every 4 tiles and at the end of the item
            if (++tiles == 4 || s0 + kTile >= w.src1) {
#pragma unroll
                for (int g = 0; g < G; ++g)
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        A1[g][q] += (double)a1[g][q] - (double)k1[g][q];
                        A2[g][q] += (double)a2[g][q] - (double)k2[g][q];
                        a1[g][q] = a2[g][q] = k1[g][q] = k2[g][q] = (R)0;
                    }
                tiles = 0;
            }
        }
        if ((int)threadIdx.x < w.ntgt) {
            // h_I / l_I = A1 / 2 (to +i2, -i1) and l_I / 2 = l_I A2 / 8 (to both endpoints), per field
            const double l = a.ell[I];
            double *o = a.part + ((size_t)w.slot * a.nE + I) * (6 * G);
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    o[6 * g + q] = 0.5 * A1[g][q];
                    o[6 * g + 3 + q] = 0.125 * l * A2[g][q];
                }
        }
    }
}

// out[f0 + g][v] = sum over v's edges and their slots of (-/+ first triple + second triple) of field g
__global__ void k_multi_gather(int nV, int nE, int nf, const int *__restrict__ inc_ptr, const int *__restrict__ inc,
                               const int *__restrict__ eslots, const double *__restrict__ part, double *__restrict__ out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = t / kMultiG, g = t % kMultiG;
    if (v >= nV || g >= nf) return;
    double o[3] = {0, 0, 0};
    for (int k = inc_ptr[v]; k < inc_ptr[v + 1]; ++k) {
        const int I = inc[k] >> 1;
        const double sg = (inc[k] & 1) ? 1.0 : -1.0;
        for (int q = 0; q < eslots[I]; ++q) {
            const double *p = part + ((size_t)q * nE + I) * (6 * kMultiG) + 6 * g;
            for (int c = 0; c < 3; ++c) o[c] += sg * p[c] + p[3 + c];
        }
    }
    double *d = out + (size_t)g * 3 * nV + 3 * (size_t)v;
    for (int c = 0; c < 3; ++c) d[c] = o[c];
}

template <int PREC, bool FAST>
static int multi_occupancy()
{
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_apply_multi<PREC, FAST>, kThreads, 0);
    return std::max(1, occ);
}

// Work list, per-field vector records and partial sums of the multi-field apply, built at first use.
static cudaError_t multi_init(Ctx &c)
{
    if (c.multi_ready) return cudaSuccess;
    const bool f = c.kp.fast != 0;
    int occ;
    switch (c.prm.precision) {
    case TP_FP64: occ = f ? multi_occupancy<P64, true>() : multi_occupancy<P64, false>(); break;
    case TP_MIXED: occ = f ? multi_occupancy<PMIX, true>() : multi_occupancy<PMIX, false>(); break;
    default: occ = f ? multi_occupancy<P32, true>() : multi_occupancy<P32, false>(); break;
    }
    plan_pass(c, c.plan_multi, 1, occ);
    const size_t ne = (size_t)std::max(1, c.nE);
    if (c.prm.precision == TP_FP64)
        TPE_CHECK(cudaMalloc(&c.d_urecMD, sizeof(URecD) * kMultiG * ne));
    else
        TPE_CHECK(cudaMalloc(&c.d_urecMF, sizeof(URecF) * kMultiG * ne));
    TPE_CHECK(cudaMalloc(&c.d_partM, sizeof(double) * (size_t)c.plan_multi.max_slots * ne * 6 * kMultiG));
    c.multi_ready = 1;
    return cudaGetLastError();
}

cudaError_t pair_apply_multi(Ctx &c, const double *gamma_geom, int which, const double *U, double *AU, int m,
                             cudaStream_t s)
{
    (void)gamma_geom;
    if (c.nE == 0 || m <= 0) {
        if (m > 0 && c.nV > 0) TPE_CHECK(cudaMemsetAsync(AU, 0, sizeof(double) * 3 * c.nV * (size_t)m, s));
        return cudaSuccess;
    }
    TPE_CHECK(multi_init(c));
    const Ctx::Plan &pl = c.plan_multi;
    const bool p64 = c.prm.precision == TP_FP64;
    const size_t nv3 = 3 * (size_t)c.nV;
    for (int f0 = 0; f0 < m; f0 += kMultiG) {
        const int nf = std::min(kMultiG, m - f0);
        for (int g = 0; g < kMultiG; ++g) {
            // fields past m repeat the last one: their sums are computed and never gathered
            const double *u = U + (size_t)std::min(f0 + g, m - 1) * nv3;
            TPE_CHECK(build_urecs_into(c, u, which, p64 ? nullptr : c.d_urecMF + (size_t)g * c.nE,
                                       p64 ? c.d_urecMD + (size_t)g * c.nE : nullptr, s));
        }
        TPE_CHECK(cudaMemsetAsync(c.d_counter + 8, 0, sizeof(int), s));
        MultiArgs a;
        a.items = pl.d_items;
        a.n_items = pl.n_items;
        a.counter = c.d_counter + 8;
        a.recF = which ? c.d_recF2 : c.d_recF;
        a.recLo = which ? c.d_recLo2 : c.d_recLo;
        a.recD = which ? c.d_recD2 : c.d_recD;
        a.urecF = c.d_urecMF;
        a.urecD = c.d_urecMD;
        a.ell = c.d_ellw[which];
        a.part = c.d_partM;
        a.nE = c.nE;
        a.kp = c.kp;
        const bool f = c.kp.fast != 0;
        const int slot = c.profile ? prof_begin(c, 7, s) : -1;
        switch (c.prm.precision) {
        case TP_FP64:
            if (f) k_apply_multi<P64, true><<<pl.grid, kThreads, 0, s>>>(a);
            else k_apply_multi<P64, false><<<pl.grid, kThreads, 0, s>>>(a);
            break;
        case TP_MIXED:
            if (f) k_apply_multi<PMIX, true><<<pl.grid, kThreads, 0, s>>>(a);
            else k_apply_multi<PMIX, false><<<pl.grid, kThreads, 0, s>>>(a);
            break;
        default:
            if (f) k_apply_multi<P32, true><<<pl.grid, kThreads, 0, s>>>(a);
            else k_apply_multi<P32, false><<<pl.grid, kThreads, 0, s>>>(a);
            break;
        }
        if (slot >= 0 || slot <= -2) prof_end(c, slot, s);
        k_multi_gather<<<(c.nV * kMultiG + 255) / 256, 256, 0, s>>>(c.nV, c.nE, nf, c.d_inc_ptr, c.d_inc, pl.d_eslots,
                                                                     c.d_partM, AU + (size_t)f0 * nv3);
        c.launches += 2;
    }
    return cudaGetLastError();
}

void multi_free(Ctx &c)
{
    cudaFree(c.plan_multi.d_items);
    cudaFree(c.plan_multi.d_eslots);
    cudaFree(c.d_urecMF);
    cudaFree(c.d_urecMD);
    cudaFree(c.d_partM);
    c.plan_multi = Ctx::Plan{};
    c.d_urecMF = nullptr;
    c.d_urecMD = nullptr;
    c.d_partM = nullptr;
    c.multi_ready = 0;
}

}  // namespace tpe
