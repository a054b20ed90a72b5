// First collision time along a descent direction (Sec. 5.4: the isotopy-safe start of the line search).
//
// tau_max is the first tau in (0, T] at which two disjoint edges of gamma - tau d touch.  For a pair of
// segments moving linearly in tau, contact needs the four endpoints coplanar: with the edge vectors
// U = b - a, V = c - a, W = e - a (each linear in tau) the triple product U . (V x W) is a cubic in tau.
// At a root the segments must also touch (segment distance <= kTouchRel (l_I + l_J)).  If the cubic
// vanishes identically (coplanar motion), first contact is a vertex of one segment meeting the other:
// a quadratic in tau for each of the four vertex-segment choices, measured along the plane's normal.
//
// GPU layout: each problem's edges are cut into blocks of kCcdBlock; a first kernel computes every
// block's box swept over [0, T] (FP32, rounded outwards).  A persistent kernel walks the block pairs
// (b, c >= b) of each problem, skips pairs whose swept boxes are apart, stages the source block's
// endpoints and directions in shared memory, and tests each unordered edge pair whose own swept boxes
// meet, in FP64.  Roots are bracketed between the cubic's critical points and bisected; the earliest
// confirmed contact of each problem is kept with an atomic minimum on the (non-negative) double's bits,
// which is independent of the order of the updates.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "tpe_internal.cuh"

namespace tpe {

#define TPE_CHECK(x)                      \
    do {                                  \
        cudaError_t e_ = (x);             \
        if (e_ != cudaSuccess) return e_; \
    } while (0)

constexpr int kCcdBlock = 128;
constexpr double kTouchRel = 1e-8;

struct CcdItem {
    int tb, sb, prob, pad;  // target block, source block (sb >= tb), problem
};

struct CcdState {
    int nBlocks = 0, nItems = 0;
    int *d_block_e0 = nullptr, *d_block_n = nullptr;
    CcdItem *d_items = nullptr;
    float *d_box = nullptr;  // [nBlocks][6]
    int *d_counter = nullptr;
};

struct Seg {
    double a[3], b[3], da[3], db[3];
};

__device__ __forceinline__ void sub3(const double *x, const double *y, double *o)
{
    o[0] = x[0] - y[0];
    o[1] = x[1] - y[1];
    o[2] = x[2] - y[2];
}
__device__ __forceinline__ double dot3(const double *x, const double *y)
{
    return x[0] * y[0] + x[1] * y[1] + x[2] * y[2];
}
__device__ __forceinline__ void cross3(const double *x, const double *y, double *o)
{
    o[0] = x[1] * y[2] - x[2] * y[1];
    o[1] = x[2] * y[0] - x[0] * y[2];
    o[2] = x[0] * y[1] - x[1] * y[0];
}
__device__ __forceinline__ double det3(const double *u, const double *v, const double *w)
{
    double c[3];
    cross3(v, w, c);
    return dot3(u, c);
}
__device__ __forceinline__ double norm3(const double *x)
{
    return sqrt(dot3(x, x));
}

// Smallest |P(s) - Q(u)| over s, u in [0, 1]: the stationary point if inside the square, else the best
// clamped one-dimensional minimum along the square's four edges.
__device__ double seg_dist(const double *p1, const double *p2, const double *q1, const double *q2)
{
    double d1[3], d2[3], r[3];
    sub3(p2, p1, d1);
    sub3(q2, q1, d2);
    sub3(p1, q1, r);
    const double a = dot3(d1, d1), b = dot3(d1, d2), e = dot3(d2, d2), c = dot3(d1, r), f = dot3(d2, r);
    double best = 1e300;
    auto eval = [&](double s, double u) {
        double w[3];
        for (int k = 0; k < 3; ++k) w[k] = r[k] + s * d1[k] - u * d2[k];
        best = fmin(best, norm3(w));
    };
    const double den = a * e - b * b;
    if (den > 1e-14 * a * e) {
        const double s = (b * f - c * e) / den, u = (a * f - b * c) / den;
        if (s >= 0.0 && s <= 1.0 && u >= 0.0 && u <= 1.0) eval(s, u);
    }
    for (int k = 0; k < 2; ++k) {
        const double s = (double)k;
        eval(s, e > 0.0 ? fmin(1.0, fmax(0.0, (b * s + f) / e)) : 0.0);
        const double u = (double)k;
        eval(a > 0.0 ? fmin(1.0, fmax(0.0, (b * u - c) / a)) : 0.0, u);
    }
    return best;
}

__device__ __forceinline__ double seg_dist_at(const Seg &I, const Seg &J, double t)
{
    double p1[3], p2[3], q1[3], q2[3];
    for (int k = 0; k < 3; ++k) {
        p1[k] = I.a[k] - t * I.da[k];
        p2[k] = I.b[k] - t * I.db[k];
        q1[k] = J.a[k] - t * J.da[k];
        q2[k] = J.b[k] - t * J.db[k];
    }
    return seg_dist(p1, p2, q1, q2);
}

__device__ __forceinline__ double horner3(const double *c, double t)
{
    return ((c[3] * t + c[2]) * t + c[1]) * t + c[0];
}

// Real roots of c0 + c1 t + c2 t^2 in (0, T], ascending (n = count).
__device__ int quad_roots(double c0, double c1, double c2, double T, double *r)
{
    int n = 0;
    double x[2];
    if (c2 == 0.0) {
        if (c1 != 0.0) x[n++] = -c0 / c1;
    } else {
        const double disc = c1 * c1 - 4.0 * c2 * c0;
        if (disc >= 0.0) {
            const double q = -0.5 * (c1 + copysign(sqrt(disc), c1));
            x[n++] = q / c2;
            if (q != 0.0) x[n++] = c0 / q;
        }
    }
    int m = 0;
    for (int k = 0; k < n; ++k)
        if (x[k] > 0.0 && x[k] <= T) r[m++] = x[k];
    if (m == 2 && r[0] > r[1]) {
        const double t = r[0];
        r[0] = r[1];
        r[1] = t;
    }
    return m;
}

// First contact time of the pair in (0, T], or +inf.
__device__ double pair_ccd(const Seg &I, const Seg &J, double T)
{
    double U0[3], U1[3], V0[3], V1[3], W0[3], W1[3];
    for (int k = 0; k < 3; ++k) {
        U0[k] = I.b[k] - I.a[k];
        U1[k] = -(I.db[k] - I.da[k]);
        V0[k] = J.a[k] - I.a[k];
        V1[k] = -(J.da[k] - I.da[k]);
        W0[k] = J.b[k] - I.a[k];
        W1[k] = -(J.db[k] - I.da[k]);
    }
    const double tol = kTouchRel * (norm3(U0) + sqrt((J.b[0] - J.a[0]) * (J.b[0] - J.a[0]) +
                                                      (J.b[1] - J.a[1]) * (J.b[1] - J.a[1]) +
                                                      (J.b[2] - J.a[2]) * (J.b[2] - J.a[2])));
    const double c[4] = {det3(U0, V0, W0), det3(U1, V0, W0) + det3(U0, V1, W0) + det3(U0, V0, W1),
                         det3(U1, V1, W0) + det3(U1, V0, W1) + det3(U0, V1, W1), det3(U1, V1, W1)};
    const double sc = fmax(fmax(norm3(U0) + T * norm3(U1), norm3(V0) + T * norm3(V1)), norm3(W0) + T * norm3(W1));
    const double scale = sc * sc * sc;
    const double big = fmax(fmax(fabs(c[0]), fabs(c[1]) * T), fmax(fabs(c[2]) * T * T, fabs(c[3]) * T * T * T));
    if (big > 1e-13 * scale) {
        // critical points of the cubic split (0, T] into monotone pieces
        double cp[2];
        const int ncp = quad_roots(c[1], 2.0 * c[2], 3.0 * c[3], T, cp);
        double lo = 0.0, flo = c[0];
        for (int piece = 0; piece <= ncp; ++piece) {
            const double hi = piece < ncp ? cp[piece] : T;
            if (!(hi > lo)) continue;
            const double fhi = horner3(c, hi);
            double root = -1.0;
            if (fhi == 0.0) {
                root = hi;
            } else if ((flo < 0.0 && fhi > 0.0) || (flo > 0.0 && fhi < 0.0)) {
                double l = lo, h = hi, fl = flo;
                for (int it = 0; it < 80 && h - l > 1e-16 * T; ++it) {
                    const double m = 0.5 * (l + h), fm = horner3(c, m);
                    if ((fm < 0.0) == (fl < 0.0) && fm != 0.0) {
                        l = m;
                        fl = fm;
                    } else {
                        h = m;
                    }
                }
                root = 0.5 * (l + h);
            } else if (piece < ncp && fabs(fhi) <= 1e-12 * scale) {
                root = hi;  // a double root at the critical point: tangential touch
            }
            if (root > 0.0 && seg_dist_at(I, J, root) <= tol) return root;
            lo = hi;
            flo = fhi;
        }
        return INFINITY;
    }
    // coplanar motion: each vertex against the other segment, along the plane normal
    double n[3], u[3], v[3];
    for (int k = 0; k < 3; ++k) {
        u[k] = U0[k] + 0.5 * T * U1[k];
        v[k] = V0[k] + 0.5 * T * V1[k];
    }
    cross3(u, v, n);
    if (dot3(n, n) == 0.0) {
        for (int k = 0; k < 3; ++k) v[k] = W0[k] + 0.5 * T * W1[k];
        cross3(u, v, n);
        if (dot3(n, n) == 0.0) return INFINITY;
    }
    double best = INFINITY;
    for (int which = 0; which < 4; ++which) {
        const Seg &P = which < 2 ? I : J, &Q = which < 2 ? J : I;
        const double *p = (which & 1) ? P.b : P.a, *dp = (which & 1) ? P.db : P.da;
        double S0[3], S1[3], R0[3], R1[3], x[3], y[3];
        for (int k = 0; k < 3; ++k) {
            S0[k] = Q.b[k] - Q.a[k];
            S1[k] = -(Q.db[k] - Q.da[k]);
            R0[k] = p[k] - Q.a[k];
            R1[k] = -(dp[k] - Q.da[k]);
        }
        cross3(S0, R0, x);
        const double q0 = dot3(x, n);
        cross3(S1, R0, x);
        cross3(S0, R1, y);
        const double q1 = dot3(x, n) + dot3(y, n);
        cross3(S1, R1, x);
        const double q2 = dot3(x, n);
        double r[2];
        const int nr = quad_roots(q0, q1, q2, T, r);
        for (int k = 0; k < nr; ++k)
            if (seg_dist_at(I, J, r[k]) <= tol) {
                best = fmin(best, r[k]);
                break;
            }
    }
    return best;
}

__device__ __forceinline__ void load_seg(Seg &S, const double *g, const double *d, int i1, int i2)
{
    for (int k = 0; k < 3; ++k) {
        S.a[k] = g[3 * (size_t)i1 + k];
        S.b[k] = g[3 * (size_t)i2 + k];
        S.da[k] = d[3 * (size_t)i1 + k];
        S.db[k] = d[3 * (size_t)i2 + k];
    }
}

// swept box of a segment over [0, T] (FP32, rounded outwards)
__device__ __forceinline__ void seg_box(const Seg &S, double T, float *b)
{
    for (int k = 0; k < 3; ++k) {
        const double x0 = S.a[k], x1 = S.b[k], x2 = S.a[k] - T * S.da[k], x3 = S.b[k] - T * S.db[k];
        b[k] = __double2float_rd(fmin(fmin(x0, x1), fmin(x2, x3)));
        b[3 + k] = __double2float_ru(fmax(fmax(x0, x1), fmax(x2, x3)));
    }
}

__device__ __forceinline__ bool boxes_meet(const float *p, const float *q, float pad)
{
    return p[0] <= q[3] + pad && q[0] <= p[3] + pad && p[1] <= q[4] + pad && q[1] <= p[4] + pad &&
           p[2] <= q[5] + pad && q[2] <= p[5] + pad;
}

__global__ void __launch_bounds__(kCcdBlock) k_ccd_boxes(const int *__restrict__ block_e0, const int *__restrict__ block_n,
                                                         const int *__restrict__ edges, const double *__restrict__ g,
                                                         const double *__restrict__ d, double T, float *__restrict__ box)
{
    __shared__ float sh[6][kCcdBlock];
    const int blk = blockIdx.x, n = block_n[blk];
    float b[6] = {3e38f, 3e38f, 3e38f, -3e38f, -3e38f, -3e38f};
    if ((int)threadIdx.x < n) {
        const int I = block_e0[blk] + threadIdx.x;
        Seg S;
        load_seg(S, g, d, edges[2 * I], edges[2 * I + 1]);
        seg_box(S, T, b);
    }
    for (int k = 0; k < 6; ++k) sh[k][threadIdx.x] = b[k];
    __syncthreads();
    for (int o = kCcdBlock / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int k = 0; k < 6; ++k)
                sh[k][threadIdx.x] = k < 3 ? fminf(sh[k][threadIdx.x], sh[k][threadIdx.x + o])
                                           : fmaxf(sh[k][threadIdx.x], sh[k][threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x < 6) box[6 * blk + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(kCcdBlock) k_ccd(const CcdItem *__restrict__ items, int n_items,
                                                   int *__restrict__ counter, const int *__restrict__ block_e0,
                                                   const int *__restrict__ block_n, const float *__restrict__ box,
                                                   const int *__restrict__ edges, const double *__restrict__ g,
                                                   const double *__restrict__ d, double T, float pad,
                                                   unsigned long long *__restrict__ tmin)
{
    __shared__ Seg ss[kCcdBlock];
    __shared__ int sv[kCcdBlock][2];
    __shared__ float sb[kCcdBlock][6];
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= n_items) break;
        const CcdItem w = items[it];
        if (!boxes_meet(box + 6 * w.tb, box + 6 * w.sb, pad)) continue;  // uniform per CTA
        const int s0 = block_e0[w.sb], ns = block_n[w.sb], t0 = block_e0[w.tb], nt = block_n[w.tb];
        if ((int)threadIdx.x < ns) {
            const int J = s0 + threadIdx.x;
            const int j1 = edges[2 * J], j2 = edges[2 * J + 1];
            load_seg(ss[threadIdx.x], g, d, j1, j2);
            sv[threadIdx.x][0] = j1;
            sv[threadIdx.x][1] = j2;
            seg_box(ss[threadIdx.x], T, sb[threadIdx.x]);
        }
        __syncthreads();
        if ((int)threadIdx.x < nt) {
            const int I = t0 + threadIdx.x;
            const int i1 = edges[2 * I], i2 = edges[2 * I + 1];
            Seg S;
            load_seg(S, g, d, i1, i2);
            float tb[6];
            seg_box(S, T, tb);
            double best = INFINITY;
            const int sfirst = (w.tb == w.sb) ? (int)threadIdx.x + 1 : 0;  // unordered pairs once
            for (int s = sfirst; s < ns; ++s) {
                const int j1 = sv[s][0], j2 = sv[s][1];
                if (j1 == i1 || j1 == i2 || j2 == i1 || j2 == i2) continue;
                if (!boxes_meet(tb, sb[s], pad)) continue;
                best = fmin(best, pair_ccd(S, ss[s], T));
            }
            if (best < T) atomicMin(tmin + w.prob, (unsigned long long)__double_as_longlong(best));
        }
        __syncthreads();  // the source block is restaged by the next item
    }
}

__global__ void k_ccd_init(int n, double T, unsigned long long *tmin)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) tmin[i] = (unsigned long long)__double_as_longlong(T);
}

// ---------------------------------------------------------------------------------- host side

void ccd_free(Ctx &c)
{
    if (!c.ccd) return;
    CcdState &S = *c.ccd;
    void *ptrs[] = {S.d_block_e0, S.d_block_n, S.d_items, S.d_box, S.d_counter};
    for (void *p : ptrs) cudaFree(p);
    delete c.ccd;
    c.ccd = nullptr;
}

cudaError_t ccd_init(Ctx &c)
{
    if (c.ccd) return cudaSuccess;
    c.ccd = new CcdState();
    CcdState &S = *c.ccd;
    std::vector<int> be0, bn;
    std::vector<CcdItem> items;
    for (int q = 0; q < c.nProb; ++q) {
        const int e0 = c.h_prob_e[q], e1 = c.h_prob_e[q + 1];
        const int first = (int)be0.size();
        for (int x = e0; x < e1; x += kCcdBlock) {
            be0.push_back(x);
            bn.push_back(std::min(kCcdBlock, e1 - x));
        }
        const int last = (int)be0.size();
        for (int tb = first; tb < last; ++tb)
            for (int sb = tb; sb < last; ++sb) items.push_back(CcdItem{tb, sb, q, 0});
    }
    S.nBlocks = (int)be0.size();
    S.nItems = (int)items.size();
    TPE_CHECK(cudaMalloc(&S.d_block_e0, sizeof(int) * std::max(1, S.nBlocks)));
    TPE_CHECK(cudaMalloc(&S.d_block_n, sizeof(int) * std::max(1, S.nBlocks)));
    TPE_CHECK(cudaMalloc(&S.d_items, sizeof(CcdItem) * std::max(1, S.nItems)));
    TPE_CHECK(cudaMalloc(&S.d_box, sizeof(float) * 6 * std::max(1, S.nBlocks)));
    TPE_CHECK(cudaMalloc(&S.d_counter, sizeof(int)));
    if (S.nBlocks) {
        TPE_CHECK(cudaMemcpy(S.d_block_e0, be0.data(), sizeof(int) * S.nBlocks, cudaMemcpyHostToDevice));
        TPE_CHECK(cudaMemcpy(S.d_block_n, bn.data(), sizeof(int) * S.nBlocks, cudaMemcpyHostToDevice));
    }
    if (S.nItems) TPE_CHECK(cudaMemcpy(S.d_items, items.data(), sizeof(CcdItem) * S.nItems, cudaMemcpyHostToDevice));
    return cudaSuccess;
}

// tmin[q] = first collision time of problem q along gamma - tau d in (0, T], or T.  gamma, d: [nV][3].
cudaError_t ccd_time(Ctx &c, const double *gamma, const double *d, double T, double *tmin, cudaStream_t s)
{
    TPE_CHECK(ccd_init(c));
    CcdState &S = *c.ccd;
    unsigned long long *tm = reinterpret_cast<unsigned long long *>(tmin);
    k_ccd_init<<<(c.nProb + 127) / 128, 128, 0, s>>>(c.nProb, T, tm);
    c.launches++;
    if (S.nItems == 0) return cudaGetLastError();
    k_ccd_boxes<<<S.nBlocks, kCcdBlock, 0, s>>>(S.d_block_e0, S.d_block_n, c.d_edges, gamma, d, T, S.d_box);
    TPE_CHECK(cudaMemsetAsync(S.d_counter, 0, sizeof(int), s));
    // boxes may meet within the touch tolerance: pad by it (relative to the mean edge length)
    const float pad = (float)(4.0 * kTouchRel * c.mean_ell);
    const int grid = std::max(1, std::min(S.nItems, c.sm_count * 8));
    k_ccd<<<grid, kCcdBlock, 0, s>>>(S.d_items, S.nItems, S.d_counter, S.d_block_e0, S.d_block_n, S.d_box, c.d_edges,
                                     gamma, d, T, pad, tm);
    c.launches += 2;
    return cudaGetLastError();
}

}  // namespace tpe
