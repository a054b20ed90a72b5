// Barnes-Hut energy and differential over a bounding volume hierarchy of tangent-points (App. B.1): the
// paper's hierarchical comparator for the exact tiled passes, in FP64.
//
// Hierarchy (built on the host from the curve, once per call, one tree per problem):
//   * tangent-points p_I = (T_I, x_I) in R^6 (unit tangent, midpoint);
//   * a node with more than leaf_size edges is split at the median of the coordinate, among the six,
//     whose split minimises the sum of the squared diameters of the two children's 6-D boxes (left: the
//     first floor(n / 2) edges in that coordinate's order, equal values ordered by edge index; ties go
//     to the lower coordinate); the per-coordinate orders are sorted once and stably partitioned at
//     every split, so a level costs O(36 n) and the depth is about log2(n / leaf_size);
//   * per node: L = sum l_I, x_N = sum l_I x_I / L, T_N = sum l_I T_I / L, r_x = half the diagonal of
//     the box of the edges' endpoints, r_T = half the diagonal of the box of the tangents.
// Traversal (one thread per target edge, explicit stack):
//   * a node is admissible when r_x < eps |x_I - x_N| and r_T < eps (Eq. BarnesHutCondition) and it
//     holds neither the target nor an edge sharing a vertex with it;
//   * energy: an admissible node adds l_I L |T_I x (x_I - x_N)|^alpha / |x_I - x_N|^beta
//     (Eq. BVHNodeTPE); a leaf adds l_I l_J khat_IJ (Eq. 18) for its edges disjoint from I;
//   * differential: an admissible node adds L d/d gamma_{i_a} [l_I (k(x_I, x_N, T_I) + k(x_N, x_I, T_N))]
//     to the target's two endpoints, a leaf the target-side derivatives of l_I l_J (khat_IJ + khat_JI);
//     the per-edge rows are then summed per vertex.
// At eps = 0 nothing is admissible and both are the exact Eq. 17 sums; the work per target falls from
// O(n) to about O(log n / eps^2) as eps grows.  The multigrid V-cycle of the appendix is not built.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "tpe_internal.cuh"

namespace tpe {

#define TPE_CHECK(x)                      \
    do {                                  \
        cudaError_t e_ = (x);             \
        if (e_ != cudaSuccess) return e_; \
    } while (0)

constexpr int kBhMaxNear = 16;   // edges sharing a vertex with a target (itself included), at most
constexpr int kBhStack = 96;     // traversal stack depth

struct BhNode {
    double xbar[3], Tbar[3];
    double L, rx, rT;
    int b, e, left, right;
};

struct BhTree {
    std::vector<BhNode> nodes;
    std::vector<int> perm;                // edge ids in hierarchy order (global edge numbering)
    std::vector<int> root;                // per problem
};

// squared diagonal of a 6-D box, summed coordinate by coordinate in order
static double sq_diam6(const double *lo, const double *hi)
{
    double d = hi[0] - lo[0];
    double s = d * d;
    for (int c = 1; c < 6; ++c) {
        d = hi[c] - lo[c];
        s = s + d * d;
    }
    return s;
}

// The hierarchy of the edges [e0, e1) of one problem, appended to t.  P: [nE][6] tangent-points,
// x / T / ell / p1 / p2: per-edge midpoints, tangents, lengths and endpoints (global numbering).
static void bh_build_problem(BhTree &t, int e0, int e1, int leaf_size, const std::vector<double> &P,
                             const std::vector<double> &x, const std::vector<double> &T,
                             const std::vector<double> &ell, const std::vector<double> &p1,
                             const std::vector<double> &p2)
{
    const int n = e1 - e0;
    const int off = (int)t.perm.size();
    t.perm.resize(off + n);
    for (int i = 0; i < n; ++i) t.perm[off + i] = e0 + i;
    // per-coordinate orders (value, then edge index)
    std::vector<std::vector<int>> S(6, std::vector<int>(n));
    for (int c = 0; c < 6; ++c) {
        std::vector<int> &s = S[c];
        for (int i = 0; i < n; ++i) s[i] = e0 + i;
        std::sort(s.begin(), s.end(), [&](int a, int b) {
            const double va = P[6 * (size_t)a + c], vb = P[6 * (size_t)b + c];
            return va < vb || (va == vb && a < b);
        });
    }
    std::vector<char> left_flag(ell.size(), 0);
    std::vector<double> plo, phi, slo, shi;
    std::vector<int> tmp;
    struct Job {
        int b, e, parent, side;
    };
    std::vector<Job> stack{{0, n, -1, 0}};
    t.root.push_back((int)t.nodes.size());
    while (!stack.empty()) {
        const Job jb = stack.back();
        stack.pop_back();
        const int k = (int)t.nodes.size();
        BhNode blank{};
        blank.left = blank.right = -1;  // a leaf until its children are created
        t.nodes.push_back(blank);
        BhNode nd{};
        nd.b = off + jb.b;
        nd.e = off + jb.e;
        nd.left = nd.right = -1;
        if (jb.parent >= 0) (jb.side == 0 ? t.nodes[jb.parent].left : t.nodes[jb.parent].right) = k;
        const int cnt = jb.e - jb.b;
        if (cnt > leaf_size) {
            double best = INFINITY;
            int bc = 0, bk = 1;
            plo.assign(6 * (size_t)cnt, 0.0);
            phi.assign(6 * (size_t)cnt, 0.0);
            slo.assign(6 * (size_t)cnt, 0.0);
            shi.assign(6 * (size_t)cnt, 0.0);
            for (int c = 0; c < 6; ++c) {
                const int *s = S[c].data() + jb.b;
                for (int i = 0; i < cnt; ++i)
                    for (int q = 0; q < 6; ++q) {
                        const double v = P[6 * (size_t)s[i] + q];
                        plo[6 * i + q] = i ? std::min(plo[6 * (i - 1) + q], v) : v;
                        phi[6 * i + q] = i ? std::max(phi[6 * (i - 1) + q], v) : v;
                    }
                for (int i = cnt - 1; i >= 0; --i)
                    for (int q = 0; q < 6; ++q) {
                        const double v = P[6 * (size_t)s[i] + q];
                        slo[6 * i + q] = i < cnt - 1 ? std::min(slo[6 * (i + 1) + q], v) : v;
                        shi[6 * i + q] = i < cnt - 1 ? std::max(shi[6 * (i + 1) + q], v) : v;
                    }
                const int ks = cnt / 2;  // the median split
                const double cost = sq_diam6(&plo[6 * (ks - 1)], &phi[6 * (ks - 1)]) + sq_diam6(&slo[6 * ks], &shi[6 * ks]);
                if (cost < best) {
                    best = cost;
                    bc = c;
                    bk = ks;
                }
            }
            // left child = the first bk edges of the chosen order; every order is partitioned stably
            const int *sb = S[bc].data() + jb.b;
            for (int i = 0; i < cnt; ++i) left_flag[sb[i]] = i < bk;
            for (int i = 0; i < cnt; ++i) t.perm[off + jb.b + i] = sb[i];
            for (int c = 0; c < 6; ++c) {
                int *s = S[c].data() + jb.b;
                tmp.clear();
                for (int i = 0; i < cnt; ++i)
                    if (left_flag[s[i]]) tmp.push_back(s[i]);
                for (int i = 0; i < cnt; ++i)
                    if (!left_flag[s[i]]) tmp.push_back(s[i]);
                std::copy(tmp.begin(), tmp.end(), s);
            }
            stack.push_back({jb.b + bk, jb.e, k, 1});
            stack.push_back({jb.b, jb.b + bk, k, 0});
        }
        // node data over its edges (the set does not depend on the order inside the range)
        double L = 0.0, xs[3] = {0, 0, 0}, ts[3] = {0, 0, 0};
        double xl[3] = {INFINITY, INFINITY, INFINITY}, xh[3] = {-INFINITY, -INFINITY, -INFINITY};
        double tl[3] = {INFINITY, INFINITY, INFINITY}, th[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int i = jb.b; i < jb.e; ++i) {
            const int J = t.perm[off + i];
            L += ell[J];
            for (int q = 0; q < 3; ++q) {
                xs[q] += ell[J] * x[3 * (size_t)J + q];
                ts[q] += ell[J] * T[3 * (size_t)J + q];
                xl[q] = std::min(xl[q], std::min(p1[3 * (size_t)J + q], p2[3 * (size_t)J + q]));
                xh[q] = std::max(xh[q], std::max(p1[3 * (size_t)J + q], p2[3 * (size_t)J + q]));
                tl[q] = std::min(tl[q], T[3 * (size_t)J + q]);
                th[q] = std::max(th[q], T[3 * (size_t)J + q]);
            }
        }
        nd.L = L;
        double rx = 0.0, rt = 0.0;
        for (int q = 0; q < 3; ++q) {
            nd.xbar[q] = xs[q] / L;
            nd.Tbar[q] = ts[q] / L;
            rx += (xh[q] - xl[q]) * (xh[q] - xl[q]);
            rt += (th[q] - tl[q]) * (th[q] - tl[q]);
        }
        nd.rx = 0.5 * std::sqrt(rx);
        nd.rT = 0.5 * std::sqrt(rt);
        const int lft = t.nodes[k].left, rgt = t.nodes[k].right;
        t.nodes[k] = nd;
        t.nodes[k].left = lft;
        t.nodes[k].right = rgt;
    }
}

// ---------------------------------------------------------------------------------- device side

struct BhArgs {
    const BhNode *nodes;
    const int *perm;       // edge ids in hierarchy order
    const int *root;       // per problem
    const int *eprob;      // problem of each edge
    const int *near_ptr;   // [nE + 1] CSR of the hierarchy positions of each edge's vertex-sharing edges
    const int *near_pos;
    const int *E;          // [nE][2]
    const double *g;       // [nV][3]
    double alpha, beta, eps;
    int nE;
    double *rows;          // energy: [nE]; differential: [nE][6]
    unsigned long long *stats;  // [2]: admissible nodes, leaf pairs visited
};

__device__ __forceinline__ void bh_ld3(const double *a, int i, double (&v)[3])
{
    v[0] = a[3 * i];
    v[1] = a[3 * i + 1];
    v[2] = a[3 * i + 2];
}

__device__ __forceinline__ double bh_dot(const double (&a)[3], const double (&b)[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// f = |T x d|^alpha |d|^-beta and, when GRAD, its gradients in d and in T (T not assumed unit)
template <bool GRAD>
__device__ __forceinline__ double bh_kern(const double (&d)[3], const double (&T)[3], double alpha, double beta,
                                          double (&gd)[3], double (&gT)[3])
{
    const double dd = bh_dot(d, d), tt = bh_dot(T, T), td = bh_dot(T, d);
    const double cx = T[1] * d[2] - T[2] * d[1], cy = T[2] * d[0] - T[0] * d[2], cz = T[0] * d[1] - T[1] * d[0];
    const double c = cx * cx + cy * cy + cz * cz;  // |T x d|^2
    const double f = (alpha == 2.0 ? c : pow(c, 0.5 * alpha)) * pow(dd, -0.5 * beta);
    if constexpr (GRAD) {
        const double a = c > 0.0 ? 0.5 * alpha * f / c : 0.0;
        for (int q = 0; q < 3; ++q) {
            gd[q] = a * 2.0 * (tt * d[q] - td * T[q]) - beta * f * d[q] / dd;
            gT[q] = a * 2.0 * (dd * T[q] - td * d[q]);
        }
    }
    return f;
}

// one traversal per target edge: OP_ENERGY -> rows[I]; OP_DIFF -> rows[I][6] (gradients at i1, i2)
template <int OP>
__global__ void __launch_bounds__(128) k_bh(const BhArgs a)
{
    constexpr bool GRAD = OP == OP_DIFF;
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= a.nE) return;
    const int i1 = a.E[2 * I], i2 = a.E[2 * I + 1];
    double g1[3], g2[3], e[3], x[3], T[3];
    bh_ld3(a.g, i1, g1);
    bh_ld3(a.g, i2, g2);
    for (int q = 0; q < 3; ++q) e[q] = g2[q] - g1[q];
    const double l = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
    for (int q = 0; q < 3; ++q) {
        T[q] = e[q] / l;
        x[q] = 0.5 * (g1[q] + g2[q]);
    }
    int near[kBhMaxNear];
    const int n0 = a.near_ptr[I], nn = min(a.near_ptr[I + 1] - n0, kBhMaxNear);
    for (int k = 0; k < nn; ++k) near[k] = a.near_pos[n0 + k];
    double Esum = 0.0, o1[3] = {0, 0, 0}, o2[3] = {0, 0, 0};
    // diff: K (sum of kernel values times l_J, the l_I-derivative's factor), G1, G2 (point gradients),
    // GT (tangent gradient), each already multiplied by the partner's mass
    double K = 0.0, G1[3] = {0, 0, 0}, G2[3] = {0, 0, 0}, GT[3] = {0, 0, 0};
    unsigned long long n_adm = 0, n_pairs = 0;
    int stack[kBhStack];
    int sp = 0;
    stack[sp++] = a.root[a.eprob[I]];
    while (sp > 0) {
        const BhNode nd = a.nodes[stack[--sp]];
        double d[3] = {x[0] - nd.xbar[0], x[1] - nd.xbar[1], x[2] - nd.xbar[2]};
        const double dist = sqrt(bh_dot(d, d));
        bool holds = false;
        for (int k = 0; k < nn; ++k) holds |= (near[k] >= nd.b) & (near[k] < nd.e);
        if (!holds && nd.rx < a.eps * dist && nd.rT < a.eps) {
            ++n_adm;
            double gd1[3], gT1[3];
            const double f1 = bh_kern<GRAD>(d, T, a.alpha, a.beta, gd1, gT1);
            if constexpr (!GRAD) {
                Esum += l * nd.L * f1;
            } else {
                const double Tb[3] = {nd.Tbar[0], nd.Tbar[1], nd.Tbar[2]};
                double gd2[3], gT2[3];
                const double f2 = bh_kern<true>(d, Tb, a.alpha, a.beta, gd2, gT2);
                K += nd.L * (f1 + f2);
                for (int q = 0; q < 3; ++q) {
                    const double core = 0.5 * nd.L * (gd1[q] + gd2[q]);  // through the midpoint
                    G1[q] += core;
                    G2[q] += core;
                    GT[q] += nd.L * gT1[q];
                }
            }
        } else if (nd.left < 0) {
            for (int p = nd.b; p < nd.e; ++p) {
                const int J = a.perm[p];
                const int j1 = a.E[2 * J], j2 = a.E[2 * J + 1];
                if (j1 == i1 || j1 == i2 || j2 == i1 || j2 == i2) continue;
                ++n_pairs;
                double q1[3], q2[3];
                bh_ld3(a.g, j1, q1);
                bh_ld3(a.g, j2, q2);
                double f[3] = {q2[0] - q1[0], q2[1] - q1[1], q2[2] - q1[2]};
                const double lj = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
                const double TJ[3] = {f[0] / lj, f[1] / lj, f[2] / lj};
                for (int ia = 0; ia < 2; ++ia)
                    for (int jb = 0; jb < 2; ++jb) {
                        const double *ga = ia ? g2 : g1, *qb = jb ? q2 : q1;
                        double dd[3] = {ga[0] - qb[0], ga[1] - qb[1], ga[2] - qb[2]};
                        double gdI[3], gTI[3];
                        const double fI = bh_kern<GRAD>(dd, T, a.alpha, a.beta, gdI, gTI);
                        if constexpr (!GRAD) {
                            Esum += 0.25 * l * lj * fI;
                        } else {
                            double md[3] = {-dd[0], -dd[1], -dd[2]}, gdJ[3], gTJ[3];
                            const double fJ = bh_kern<true>(md, TJ, a.alpha, a.beta, gdJ, gTJ);
                            K += 0.25 * lj * (fI + fJ);
                            double *G = ia ? G2 : G1;
                            for (int q = 0; q < 3; ++q) {
                                G[q] += 0.25 * lj * (gdI[q] - gdJ[q]);
                                GT[q] += 0.25 * lj * gTI[q];
                            }
                        }
                    }
            }
        } else {  // the host bounds the tree depth so that the stack cannot overflow
            stack[sp++] = nd.right;
            stack[sp++] = nd.left;
        }
    }
    if constexpr (!GRAD) {
        a.rows[I] = Esum;
    } else {
        // F = l sum(mass x kernel terms):  dF/dg_a = K dl/dg_a + l (G_a +/- (Id - T T^t) GT / l)
        const double tg = bh_dot(T, GT);
        for (int q = 0; q < 3; ++q) {
            const double pgt = GT[q] - tg * T[q];
            o1[q] = -K * T[q] + l * G1[q] - pgt;
            o2[q] = K * T[q] + l * G2[q] + pgt;
            a.rows[6 * (size_t)I + q] = o1[q];
            a.rows[6 * (size_t)I + 3 + q] = o2[q];
        }
    }
    atomicAdd(a.stats, n_adm);
    atomicAdd(a.stats + 1, n_pairs);
}

// dE[v] = sum over v's edges of their row's gradient at v
__global__ void k_bh_gather(int nV, const int *__restrict__ inc_ptr, const int *__restrict__ inc,
                            const double *__restrict__ rows, double *__restrict__ dE)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nV) return;
    double o[3] = {0, 0, 0};
    for (int k = inc_ptr[v]; k < inc_ptr[v + 1]; ++k) {
        const int I = inc[k] >> 1, sl = inc[k] & 1;
        for (int q = 0; q < 3; ++q) o[q] += rows[6 * (size_t)I + 3 * sl + q];
    }
    for (int q = 0; q < 3; ++q) dE[3 * (size_t)v + q] = o[q];
}

// ---------------------------------------------------------------------------------- host side

}  // namespace tpe

struct tpe::BhState {
    BhNode *d_nodes = nullptr;
    int *d_perm = nullptr, *d_root = nullptr, *d_near_ptr = nullptr, *d_near_pos = nullptr;
    double *d_rows = nullptr;
    unsigned long long *d_stats = nullptr;
    size_t cap_nodes = 0;
    unsigned long long stats[2] = {0, 0};  // of the last pass
    int depth = 0;                          // of the last hierarchy
    double build_s = 0.0;                   // host time of the last hierarchy: copy-out, build, upload
};

namespace tpe {

// stack slots a depth-first traversal of `t` needs (children pushed in pairs); -1 if the links do not
// form a forest (a node reached twice)
static int bh_depth(const BhTree &t)
{
    int mx = 0;
    size_t visited = 0;
    std::vector<std::pair<int, int>> st;
    for (int r : t.root)
        if (r >= 0) st.push_back({r, 1});
    while (!st.empty()) {
        auto [k, d] = st.back();
        st.pop_back();
        if (++visited > t.nodes.size()) return -1;
        mx = std::max(mx, d);
        if (t.nodes[k].left >= 0) {
            st.push_back({t.nodes[k].left, d + 1});
            st.push_back({t.nodes[k].right, d + 1});
        }
    }
    return mx;
}

// Builds the hierarchy of the curve `gamma` (device) on the host and uploads it.
static cudaError_t bh_prepare(Ctx &c, const double *gamma, int leaf_size, cudaStream_t s, int &unsupported)
{
    unsupported = 0;
    if (!c.bh) c.bh = new BhState();
    BhState &B = *c.bh;
    const auto t0 = std::chrono::steady_clock::now();
    const int nV = c.nV, nE = c.nE;
    std::vector<double> g(3 * (size_t)nV);
    TPE_CHECK(cudaMemcpyAsync(g.data(), gamma, sizeof(double) * g.size(), cudaMemcpyDeviceToHost, s));
    TPE_CHECK(cudaStreamSynchronize(s));
    std::vector<double> x(3 * (size_t)nE), T(3 * (size_t)nE), ell(nE), p1(3 * (size_t)nE), p2(3 * (size_t)nE),
        P(6 * (size_t)nE);
    for (int I = 0; I < nE; ++I) {
        const int a = c.h_edges[2 * I], b = c.h_edges[2 * I + 1];
        double d[3];
        for (int q = 0; q < 3; ++q) {
            p1[3 * I + q] = g[3 * a + q];
            p2[3 * I + q] = g[3 * b + q];
            d[q] = g[3 * b + q] - g[3 * a + q];
        }
        const double l = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        ell[I] = l;
        for (int q = 0; q < 3; ++q) {
            T[3 * I + q] = d[q] / l;
            x[3 * I + q] = 0.5 * (g[3 * a + q] + g[3 * b + q]);
            P[6 * (size_t)I + q] = T[3 * I + q];
            P[6 * (size_t)I + 3 + q] = x[3 * I + q];
        }
    }
    BhTree t;
    for (int q = 0; q < c.nProb; ++q) {
        const int e0 = c.h_prob_e[q], e1 = c.h_prob_e[q + 1];
        if (e1 > e0)
            bh_build_problem(t, e0, e1, leaf_size, P, x, T, ell, p1, p2);
        else
            t.root.push_back(-1);
    }
    B.depth = bh_depth(t);
    // vertex-sharing edges of every edge, as hierarchy positions
    std::vector<int> pos(nE), vdeg(nV + 1, 0), vinc(2 * (size_t)nE);
    for (int i = 0; i < nE; ++i) pos[t.perm[i]] = i;
    for (int I = 0; I < nE; ++I) {
        vdeg[c.h_edges[2 * I] + 1]++;
        vdeg[c.h_edges[2 * I + 1] + 1]++;
    }
    for (int v = 0; v < nV; ++v) vdeg[v + 1] += vdeg[v];
    std::vector<int> fill(vdeg.begin(), vdeg.end() - 1);
    for (int I = 0; I < nE; ++I) {
        vinc[fill[c.h_edges[2 * I]]++] = I;
        vinc[fill[c.h_edges[2 * I + 1]]++] = I;
    }
    std::vector<int> near_ptr(nE + 1, 0), near_pos;
    for (int I = 0; I < nE; ++I) {
        std::vector<int> nb;
        for (int side = 0; side < 2; ++side) {
            const int v = c.h_edges[2 * I + side];
            for (int k = vdeg[v]; k < vdeg[v + 1]; ++k) nb.push_back(pos[vinc[k]]);
        }
        std::sort(nb.begin(), nb.end());
        nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
        if ((int)nb.size() > kBhMaxNear) unsupported = 1;
        near_pos.insert(near_pos.end(), nb.begin(), nb.end());
        near_ptr[I + 1] = (int)near_pos.size();
    }
    if (B.depth < 0) return cudaErrorUnknown;  // not reached: the build links every node once
    if (B.depth + 2 > kBhStack) unsupported = 1;
    if (unsupported) return cudaSuccess;
    if (t.nodes.size() > B.cap_nodes || !B.d_perm) {
        cudaFree(B.d_nodes);
        cudaFree(B.d_perm);
        cudaFree(B.d_root);
        cudaFree(B.d_near_ptr);
        cudaFree(B.d_near_pos);
        cudaFree(B.d_rows);
        cudaFree(B.d_stats);
        B.cap_nodes = std::max<size_t>(t.nodes.size(), 2 * (size_t)std::max(1, nE));
        TPE_CHECK(cudaMalloc(&B.d_nodes, sizeof(BhNode) * B.cap_nodes));
        TPE_CHECK(cudaMalloc(&B.d_perm, sizeof(int) * std::max(1, nE)));
        TPE_CHECK(cudaMalloc(&B.d_root, sizeof(int) * std::max(1, c.nProb)));
        TPE_CHECK(cudaMalloc(&B.d_near_ptr, sizeof(int) * (nE + 1)));
        TPE_CHECK(cudaMalloc(&B.d_near_pos, sizeof(int) * kBhMaxNear * (size_t)std::max(1, nE)));
        TPE_CHECK(cudaMalloc(&B.d_rows, sizeof(double) * 6 * (size_t)std::max(1, nE)));
        TPE_CHECK(cudaMalloc(&B.d_stats, sizeof(unsigned long long) * 2));
    }
    // synchronous copies: the host vectors end with this call
    TPE_CHECK(cudaMemcpy(B.d_nodes, t.nodes.data(), sizeof(BhNode) * t.nodes.size(), cudaMemcpyHostToDevice));
    TPE_CHECK(cudaMemcpy(B.d_perm, t.perm.data(), sizeof(int) * nE, cudaMemcpyHostToDevice));
    TPE_CHECK(cudaMemcpy(B.d_root, t.root.data(), sizeof(int) * c.nProb, cudaMemcpyHostToDevice));
    TPE_CHECK(cudaMemcpy(B.d_near_ptr, near_ptr.data(), sizeof(int) * (nE + 1), cudaMemcpyHostToDevice));
    if (!near_pos.empty())
        TPE_CHECK(cudaMemcpy(B.d_near_pos, near_pos.data(), sizeof(int) * near_pos.size(), cudaMemcpyHostToDevice));
    B.build_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return cudaSuccess;
}

// Barnes-Hut energy (op OP_ENERGY: per-edge rows and, if E, per-problem sums) or differential (OP_DIFF:
// dE [nV][3]) of the curve `gamma`.  unsupported = 1 when a vertex is shared by too many edges or the
// hierarchy is too deep for the traversal stack.
cudaError_t bh_pass(Ctx &c, const double *gamma, int op, double eps, int leaf_size, double *rows, double *E,
                    double *dE, cudaStream_t s, int &unsupported)
{
    TPE_CHECK(bh_prepare(c, gamma, leaf_size, s, unsupported));
    if (unsupported || c.nE == 0) return cudaSuccess;
    BhState &B = *c.bh;
    TPE_CHECK(cudaMemsetAsync(B.d_stats, 0, sizeof(unsigned long long) * 2, s));
    BhArgs a;
    a.nodes = B.d_nodes;
    a.perm = B.d_perm;
    a.root = B.d_root;
    a.eprob = c.d_eprob;
    a.near_ptr = B.d_near_ptr;
    a.near_pos = B.d_near_pos;
    a.E = c.d_edges;
    a.g = gamma;
    a.alpha = c.prm.alpha;
    a.beta = c.prm.beta;
    a.eps = eps;
    a.nE = c.nE;
    a.stats = B.d_stats;
    const int nb = (c.nE + 127) / 128;
    if (op == OP_ENERGY) {
        a.rows = rows ? rows : B.d_rows;
        k_bh<OP_ENERGY><<<nb, 128, 0, s>>>(a);
        c.launches++;
        if (E) TPE_CHECK(segment_sum(c, a.rows, E, s));
    } else {
        a.rows = B.d_rows;
        k_bh<OP_DIFF><<<nb, 128, 0, s>>>(a);
        k_bh_gather<<<(c.nV + 255) / 256, 256, 0, s>>>(c.nV, c.d_inc_ptr, c.d_inc, B.d_rows, dE);
        c.launches += 2;
    }
    TPE_CHECK(cudaMemcpyAsync(B.stats, B.d_stats, sizeof(B.stats), cudaMemcpyDeviceToHost, s));
    TPE_CHECK(cudaStreamSynchronize(s));
    return cudaGetLastError();
}

void bh_stats(const Ctx &c, unsigned long long *adm, unsigned long long *pairs, int *depth, double *build_s)
{
    *adm = c.bh ? c.bh->stats[0] : 0;
    *pairs = c.bh ? c.bh->stats[1] : 0;
    if (depth) *depth = c.bh ? c.bh->depth : 0;
    if (build_s) *build_s = c.bh ? c.bh->build_s : 0.0;
}

void bh_free(Ctx &c)
{
    if (!c.bh) return;
    BhState &B = *c.bh;
    cudaFree(B.d_nodes);
    cudaFree(B.d_perm);
    cudaFree(B.d_root);
    cudaFree(B.d_near_ptr);
    cudaFree(B.d_near_pos);
    cudaFree(B.d_rows);
    cudaFree(B.d_stats);
    delete c.bh;
    c.bh = nullptr;
}

}  // namespace tpe
