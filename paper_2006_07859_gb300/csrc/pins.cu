// Point constraints of Sec. 8.1 (TP_CONSTRAINTS_POINTS): pinned vertices gamma_v = p_v with the total
// length, and no barycenter row (a pin already fixes the translations).
//
// A-bar = I_3 (x) A is singular on the translations N, so the KKT system of Eq. 22 is solved by a Schur
// complement over mean-free solves (A^+ is the inverse of A on mean-free vectors):
//   g = A^+ (dE - C^T lambda) + N t,
// with rows C = [C_len; e_v (x) I_3 per pin].  A^+ (e_v (x) I_3) is the scalar field w_v = A^+ e_v in
// each component, so one three-column CG solve yields the fields of three pins (columns x, y, z carry
// different pins; A-bar never couples the components), and pins of different problems share a solve.
// With y0 = A^+ dE, y1 = A^+ C_len^T, S = C A^+ C^T and C N = [0; I_3 per pin], the conditions C g = 0
// and N^T (dE - C^T lambda) = 0 (dE - C^T lambda must lie in the range of A-bar) read
//   [S  CN; (CN)^T 0] [lambda; -t] = [C y0; N^T dE],   g = y0 - (lambda_len y1 + sum_v w_v lambda_v - t),
// and the constraint projection min x^T A-bar x / 2 s.t. C x = b (Sec. 5.3.2, Eq. 23) reads
//   [S  CN; (CN)^T 0] [nu; t] = [b; 0],                  x = nu_len y1 + sum_v w_v nu_v + t.
// S needs no extra reductions beyond <C_len, y1>: S_len,(v,i) = y1(v, i) and S_(u,i),(v,j) =
// delta_ij w_v(u) by the symmetry of A^+.  Each pin row takes its entries exactly as the final combination
// evaluates g (or x) at that vertex, so the pinned rows hold to rounding whatever the CG tolerance.  The
// small system (3 k + 4 unknowns for k pins) is solved per problem in shared memory by Gaussian
// elimination with partial pivoting in FP64.
#include <algorithm>
#include <cmath>
#include <vector>

#include "tpe_internal.cuh"

namespace tpe {

#define TPE_CHECK(x)                      \
    do {                                  \
        cudaError_t e_ = (x);             \
        if (e_ != cudaSuccess) return e_; \
    } while (0)

constexpr int kMaxPins = 24;                     // per problem
constexpr int kMaxUnknowns = 3 * kMaxPins + 4;   // 76: the augmented system takes 46.8 KB of shared memory
constexpr int kSysThreads = 128;

struct PinState {
    int n = 0;                   // pins of all problems
    int kmax = 0;                // pins of the most pinned problem
    int nsolve = 0;              // three-column solves per gradient: ceil(kmax / 3)
    int w_cap = 0;               // solves d_W has room for
    int warm = 0;                // d_W holds the fields of an earlier step for these pins
    int32_t *d_v = nullptr;      // [nProb * kMaxPins] pinned vertices, problem by problem
    int32_t *d_off = nullptr;    // [nProb + 1] first pin of each problem
    double *d_p = nullptr;       // [nProb * kMaxPins][3] targets
    double *d_W = nullptr;       // [w_cap][nV][3]: the field of local pin l is column l % 3 of solve l / 3
    double *d_red = nullptr;     // [nProb][5] (pin_reduce)
    double *d_coef = nullptr;    // [nProb][kMaxUnknowns] solution of the small system
};

cudaError_t pin_reduce(Ctx &c, const double *a, const double *b, const double *dE, double *out, cudaStream_t s);

bool pins_ready(const Ctx &c) { return c.pins && c.pins->n > 0; }

void pins_free(Ctx &c)
{
    if (!c.pins) return;
    PinState &p = *c.pins;
    cudaFree(p.d_v);
    cudaFree(p.d_off);
    cudaFree(p.d_p);
    cudaFree(p.d_W);
    cudaFree(p.d_red);
    cudaFree(p.d_coef);
    delete c.pins;
    c.pins = nullptr;
}

cudaError_t pins_set(Ctx &c, int n, const int32_t *v, const double *targets, std::string &why)
{
    if (n < 0) {
        why = "negative pin count";
        return cudaErrorInvalidValue;
    }
    if (n > 0 && (!v || !targets)) {
        why = "pins: null vertices or targets";
        return cudaErrorInvalidValue;
    }
    // validate on the host: range, distinct, finite targets, 1..kMaxPins per problem
    std::vector<std::vector<int>> per(c.nProb);
    std::vector<char> seen(c.nV, 0);
    for (int i = 0; i < n; ++i) {
        if (v[i] < 0 || v[i] >= c.nV) {
            why = "pinned vertex out of range";
            return cudaErrorInvalidValue;
        }
        if (seen[v[i]]) {
            why = "a vertex is pinned twice";
            return cudaErrorInvalidValue;
        }
        seen[v[i]] = 1;
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(targets[3 * i + k])) {
                why = "non-finite pin target";
                return cudaErrorInvalidValue;
            }
        int q = (int)(std::upper_bound(c.h_prob_v.begin(), c.h_prob_v.end(), v[i]) - c.h_prob_v.begin()) - 1;
        per[q].push_back(i);
    }
    int kmax = 0;
    if (n > 0)
        for (int q = 0; q < c.nProb; ++q) {
            int k = (int)per[q].size();
            if (k == 0) {
                why = "TP_CONSTRAINTS_POINTS: every problem needs at least one pinned vertex";
                return cudaErrorInvalidValue;
            }
            if (k > kMaxPins) {
                why = "more than 24 pinned vertices in one problem";
                return cudaErrorInvalidValue;
            }
            kmax = std::max(kmax, k);
        }
    if (!c.pins) {
        c.pins = new PinState();
        PinState &p = *c.pins;
        const size_t np = (size_t)c.nProb;
        TPE_CHECK(cudaMalloc(&p.d_v, sizeof(int32_t) * np * kMaxPins));
        TPE_CHECK(cudaMalloc(&p.d_off, sizeof(int32_t) * (np + 1)));
        TPE_CHECK(cudaMalloc(&p.d_p, sizeof(double) * 3 * np * kMaxPins));
        TPE_CHECK(cudaMalloc(&p.d_red, sizeof(double) * 5 * np));
        TPE_CHECK(cudaMalloc(&p.d_coef, sizeof(double) * kMaxUnknowns * np));
    }
    PinState &p = *c.pins;
    p.n = n;
    p.kmax = kmax;
    p.nsolve = (kmax + 2) / 3;
    p.warm = 0;
    if (n == 0) return cudaSuccess;
    if (p.nsolve > p.w_cap) {
        if (p.d_W) TPE_CHECK(cudaFree(p.d_W));
        p.d_W = nullptr;
        p.w_cap = 0;
        TPE_CHECK(cudaMalloc(&p.d_W, sizeof(double) * 3 * (size_t)c.nV * p.nsolve));
        p.w_cap = p.nsolve;
    }
    std::vector<int32_t> hv, hoff(c.nProb + 1, 0);
    std::vector<double> hp;
    for (int q = 0; q < c.nProb; ++q) {
        for (int i : per[q]) {
            hv.push_back(v[i]);
            for (int k = 0; k < 3; ++k) hp.push_back(targets[3 * i + k]);
        }
        hoff[q + 1] = (int32_t)hv.size();
    }
    TPE_CHECK(cudaMemcpy(p.d_v, hv.data(), sizeof(int32_t) * hv.size(), cudaMemcpyHostToDevice));
    TPE_CHECK(cudaMemcpy(p.d_off, hoff.data(), sizeof(int32_t) * hoff.size(), cudaMemcpyHostToDevice));
    TPE_CHECK(cudaMemcpy(p.d_p, hp.data(), sizeof(double) * hp.size(), cudaMemcpyHostToDevice));
    return cudaSuccess;
}

// Right-hand side of solve s: column j holds e_v for the problem's pin 3 s + j (one thread per problem;
// out was zeroed).
__global__ void k_pin_rhs(int nprob, int s, const int32_t *__restrict__ off, const int32_t *__restrict__ pv,
                          double *__restrict__ out)
{
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nprob) return;
    int k = off[q + 1] - off[q];
    for (int l = 3 * s; l < min(k, 3 * s + 3); ++l) out[3 * (size_t)pv[off[q] + l] + (l - 3 * s)] = 1.0;
}

// phi[4q + k] = max over the problem's pins of |gamma_v,k - p_v,k| (k < 3; row 4q + 3 is left alone).
__global__ void k_pin_phi(int nprob, const int32_t *__restrict__ off, const int32_t *__restrict__ pv,
                          const double *__restrict__ pt, const double *__restrict__ gamma, double *__restrict__ phi)
{
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nprob) return;
    double m[3] = {0.0, 0.0, 0.0};
    for (int i = off[q]; i < off[q + 1]; ++i)
        for (int k = 0; k < 3; ++k) {
            double d = fabs(gamma[3 * (size_t)pv[i] + k] - pt[3 * i + k]);
            m[k] = (d > m[k] || d != d) ? d : m[k];  // a NaN position propagates
        }
    for (int k = 0; k < 3; ++k) phi[4 * q + k] = m[k];
}

// One block per problem: assemble [S CN; (CN)^T 0 | rhs] and solve it.  Unknown order: 0 the length row,
// 1 + 3 l + i pin l component i, 3 k + 1 + j the translation component j.
//   mode 0 (gradient):   rhs = [<C_len, y0>; y0(v_l, i); sum dE_j]
//   mode 1 (projection): rhs = [-Phi_len; p_l,i - gamma(v_l, i); 0]
__global__ void __launch_bounds__(kSysThreads) k_pin_system(
    int mode, const int32_t *__restrict__ off, const int32_t *__restrict__ pv, const double *__restrict__ pt,
    const double *__restrict__ W, size_t wstride, const double *__restrict__ y0, const double *__restrict__ y1,
    const double *__restrict__ red, const double *__restrict__ gamma, const double *__restrict__ phi,
    double *__restrict__ coef, int *__restrict__ err)
{
    extern __shared__ double sm[];
    __shared__ int s_piv;
    __shared__ int s_bad;
    const int q = blockIdx.x;
    const int p0 = off[q], k = off[q + 1] - p0;
    const int m = 3 * k + 4, ld = m + 1;
    double *A = sm;          // [m][ld], last column the right-hand side
    double *f = sm + m * ld; // [m] elimination factors
    const double *r = red + 5 * q;
    if (threadIdx.x == 0) s_bad = 0;
    for (int e = threadIdx.x; e < m * ld; e += blockDim.x) {
        const int i = e / ld, j = e % ld;
        double a = 0.0;
        // classify row i and column j
        const int ti = 3 * k + 1;  // first translation unknown
        if (j == m) {  // right-hand side
            if (i == 0) {
                a = mode == 0 ? r[0] : -phi[4 * q + 3];
            } else if (i < ti) {
                const int l = (i - 1) / 3, c = (i - 1) % 3;
                const size_t v = (size_t)pv[p0 + l];
                a = mode == 0 ? y0[3 * v + c] : pt[3 * (p0 + l) + c] - gamma[3 * v + c];
            } else {
                a = mode == 0 ? r[2 + (i - ti)] : 0.0;
            }
        } else if (i == 0 || j == 0) {
            const int o = i == 0 ? j : i;  // the other index
            if (o == 0) a = r[1];
            else if (o < ti) a = y1[3 * (size_t)pv[p0 + (o - 1) / 3] + (o - 1) % 3];
        } else if (i < ti && j < ti) {
            const int l = (i - 1) / 3, c = (i - 1) % 3, mm = (j - 1) / 3, cj = (j - 1) % 3;
            if (c == cj) a = W[(size_t)(mm / 3) * wstride + 3 * (size_t)pv[p0 + l] + mm % 3];  // w_m(v_l)
        } else if (i < ti && j >= ti) {
            a = ((i - 1) % 3 == j - ti) ? 1.0 : 0.0;
        } else if (i >= ti && j < ti) {
            a = ((j - 1) % 3 == i - ti) ? 1.0 : 0.0;
        }
        A[e] = a;
    }
    __syncthreads();
    for (int col = 0; col < m; ++col) {
        if (threadIdx.x == 0) {
            int piv = col;
            double best = fabs(A[col * ld + col]);
            for (int i = col + 1; i < m; ++i) {
                double a = fabs(A[i * ld + col]);
                if (a > best) {
                    best = a;
                    piv = i;
                }
            }
            s_piv = piv;
            if (!(best > 1e-300) || !isfinite(best)) s_bad = 1;
        }
        __syncthreads();
        if (s_bad) break;
        const int piv = s_piv;
        if (piv != col)
            for (int j = threadIdx.x; j < ld; j += blockDim.x) {
                double t = A[col * ld + j];
                A[col * ld + j] = A[piv * ld + j];
                A[piv * ld + j] = t;
            }
        __syncthreads();
        for (int i = col + 1 + threadIdx.x; i < m; i += blockDim.x) f[i] = A[i * ld + col] / A[col * ld + col];
        __syncthreads();
        const int rows = m - col - 1, cols = ld - col;
        for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
            const int i = col + 1 + e / cols, j = col + e % cols;
            A[i * ld + j] -= f[i] * A[col * ld + j];
        }
        __syncthreads();
    }
    double *out = coef + (size_t)q * kMaxUnknowns;
    if (s_bad) {
        for (int i = threadIdx.x; i < m; i += blockDim.x) out[i] = 0.0;
        if (threadIdx.x == 0) atomicCAS(err, 0, (int)TP_ERR_BREAKDOWN);
        return;
    }
    if (threadIdx.x == 0) {
        for (int i = m - 1; i >= 0; --i) {
            double acc = A[i * ld + m];
            for (int j = i + 1; j < m; ++j) acc -= A[i * ld + j] * f[j];
            f[i] = acc / A[i * ld + i];  // f now holds the solution
        }
        bool fin = true;
        for (int i = 0; i < m; ++i) fin = fin && isfinite(f[i]);
        if (!fin) atomicCAS(err, 0, (int)TP_ERR_NONFINITE);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) out[i] = f[i];
}

// out(v) = base(v) - acc(v) (base given) or acc(v), acc = coef_len y1 + sum_l w_l coef_l + coef_t.
__global__ void k_pin_combine(int nV, const int32_t *__restrict__ vprob, const int32_t *__restrict__ off,
                              const double *__restrict__ W, size_t wstride, const double *__restrict__ y1,
                              const double *__restrict__ coef, const double *__restrict__ base,
                              double *__restrict__ out)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nV) return;
    const int q = vprob[v];
    const int k = off[q + 1] - off[q];
    const double *cf = coef + (size_t)q * kMaxUnknowns;
    double acc[3];
    for (int i = 0; i < 3; ++i) acc[i] = cf[0] * y1[3 * (size_t)v + i] + cf[3 * k + 1 + i];
    for (int l = 0; l < k; ++l) {
        const double w = W[(size_t)(l / 3) * wstride + 3 * (size_t)v + l % 3];
        for (int i = 0; i < 3; ++i) acc[i] += cf[1 + 3 * l + i] * w;
    }
    for (int i = 0; i < 3; ++i) out[3 * (size_t)v + i] = base ? base[3 * (size_t)v + i] - acc[i] : acc[i];
}

cudaError_t pins_phi(Ctx &c, const double *gamma, double *phi, cudaStream_t s)
{
    PinState &p = *c.pins;
    k_pin_phi<<<(c.nProb + 127) / 128, 128, 0, s>>>(c.nProb, p.d_off, p.d_v, p.d_p, gamma, phi);
    c.launches++;
    return cudaGetLastError();
}

static cudaError_t pin_system(Ctx &c, int mode, const double *y0, const double *y1, const double *gamma,
                              const double *phi, cudaStream_t s)
{
    PinState &p = *c.pins;
    const int m = 3 * p.kmax + 4;
    const size_t smem = sizeof(double) * ((size_t)m * (m + 1) + m);
    k_pin_system<<<c.nProb, kSysThreads, smem, s>>>(mode, p.d_off, p.d_v, p.d_p, p.d_W, 3 * (size_t)c.nV, y0, y1,
                                                    p.d_red, gamma, phi, p.d_coef, c.d_err);
    c.launches++;
    return cudaGetLastError();
}

static cudaError_t pin_combine(Ctx &c, const double *y1, const double *base, double *out, cudaStream_t s)
{
    PinState &p = *c.pins;
    k_pin_combine<<<(c.nV + 255) / 256, 256, 0, s>>>(c.nV, c.d_vprob, p.d_off, p.d_W, 3 * (size_t)c.nV, y1,
                                                     p.d_coef, base, out);
    c.launches++;
    return cudaGetLastError();
}

// The fields w_v = A^+ e_v of every pin (mean-free CG solves on the geometry in slot 0), warm-started from
// the previous step's fields.  rhs_scratch: [nV][3].
cudaError_t pins_fields(Ctx &c, const double *gamma, double *rhs_scratch, int *iters, double *rr, int *conv,
                        int *bd, int *flags, cudaStream_t s)
{
    PinState &p = *c.pins;
    const size_t vb = sizeof(double) * 3 * (size_t)c.nV;
    for (int sv = 0; sv < p.nsolve; ++sv) {
        TPE_CHECK(cudaMemsetAsync(rhs_scratch, 0, vb, s));
        k_pin_rhs<<<(c.nProb + 127) / 128, 128, 0, s>>>(c.nProb, sv, p.d_off, p.d_v, rhs_scratch);
        c.launches++;
        TPE_CHECK(cudaGetLastError());
        double *w = p.d_W + (size_t)sv * 3 * c.nV;
        int it = 0, cv = 0, b = 0;
        double r = 0.0;
        TPE_CHECK(cg_solve(c, gamma, 0, rhs_scratch, w, c.prm.cg_rtol, c.prm.cg_maxit, &it, &r, &cv, &b, s, 1, flags,
                           (p.warm && c.prm.warm_start) ? w : nullptr));
        *iters += it;
        *rr = std::max(*rr, r);
        *conv = *conv && cv;
        *bd = *bd || b;
    }
    p.warm = 1;
    return cudaSuccess;
}

// g = y0 - (lambda_len y1 + sum_v w_v lambda_v - t) from y0 = A^+ dE and y1 = A^+ C_len^T (the Jacobian in
// c.d_Cv, the fields in d_W).
cudaError_t pins_gradient(Ctx &c, const double *dE, const double *y0, const double *y1, double *g, cudaStream_t s)
{
    TPE_CHECK(pin_reduce(c, y0, y1, dE, c.pins->d_red, s));
    TPE_CHECK(pin_system(c, 0, y0, y1, nullptr, nullptr, s));
    return pin_combine(c, y1, y0, g, s);
}

// x = nu_len y1 + sum_v w_v nu_v + t with C x = -Phi at the trial curve gamma_t (y1 = A^+ C_len(gamma_t)^T,
// phi[4q + 3] = Phi_len of gamma_t).
cudaError_t pins_projection(Ctx &c, const double *y1, const double *gamma_t, const double *phi, double *x,
                            cudaStream_t s)
{
    TPE_CHECK(pin_reduce(c, nullptr, y1, nullptr, c.pins->d_red, s));
    TPE_CHECK(pin_system(c, 1, nullptr, y1, gamma_t, phi, s));
    return pin_combine(c, y1, nullptr, x, s);
}

}  // namespace tpe
