// Point, tangent and surface constraints of Sec. 8.1 (TP_CONSTRAINTS_POINTS): pinned vertices
// gamma_v = p_v, edges whose tangent is held at a unit vector X_I, vertices held on a quadric surface
// f(x) = x^T Q x + b^T x + c = 0, with the total length, and no barycenter row (a pin already fixes the
// translations).
//
// A-bar = I_3 (x) A is singular on the translations N, so the KKT system of Eq. 22 is solved by a Schur
// complement over mean-free solves (A^+ is the inverse of A on mean-free vectors):
//   g = A^+ (dE - C^T lambda) + N t.
// Every row here is a sparse combination of unit vectors e_u (x) e_j at a few vertices u ("fields"):
//   pin (v, i):          e_v (x) e_i
//   tangent (I, a):      sum_j r_j (e_i2 - e_i1) (x) e_j,  r = (b_a - (b_a . T_I) T_I) / l_I
//                        (the two rows b_a . T_I, b_1, b_2 an orthonormal basis across X_I: the printed
//                        three rows T_I - X_I have a Jacobian of rank 2)
//   surface v:           sum_j (grad f(gamma_v))_j e_v (x) e_j
// so A^+ C_r^T needs only the scalar fields w_u = A^+ e_u of those vertices.  One three-column CG solve
// yields three fields (columns x, y, z carry different vertices; A-bar never couples the components), and
// the fields of different problems share a solve.  With y0 = A^+ dE, y1 = A^+ C_len^T, S = C A^+ C^T and
// C N (I_3 per pin, 0 per tangent row, grad f per surface row), the conditions C g = 0 and
// N^T (dE - C^T lambda) = 0 (dE - C^T lambda must lie in the range of A-bar) read
//   [S  CN; (CN)^T 0] [lambda; -t] = [C y0; N^T dE],   g = y0 - (lambda_len y1 + sum_r lambda_r A^+ C_r^T - t),
// and the constraint projection min x^T A-bar x / 2 s.t. C x = b (Sec. 5.3.2, Eq. 23) reads
//   [S  CN; (CN)^T 0] [nu; t] = [b; 0],                  x = nu_len y1 + sum_r nu_r A^+ C_r^T + t.
// S needs only <C_len, y1> beyond values at the field vertices: S_len,r = the row's terms applied to y1
// and S_r,r' = the sum over term pairs of equal component of c c' w_u'(u), by the symmetry of A^+.  Each
// row takes its entries exactly as the final combination evaluates g (or x) at its vertices, so the
// linearised rows hold to rounding whatever the CG tolerance.  The small system (rows + 4 unknowns) is
// solved per problem in shared memory by Gaussian elimination with partial pivoting in FP64.
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

constexpr int kMaxFields = 24;               // distinct constrained vertices per problem
constexpr int kMaxRows = 96;                 // constraint rows per problem besides the length
constexpr int kMaxUnknowns = kMaxRows + 4;   // length, rows, translation
constexpr int kCoefStride = kMaxUnknowns;    // >= 3 kMaxFields + 4 (the combination's coefficients)
constexpr int kMaxTerms = 6;
constexpr int kSysThreads = 128;

enum RowType { ROW_PIN = 0, ROW_TANGENT = 1, ROW_SURFACE = 2 };

// One constraint row: ROW_PIN f0 = field, f1 = component, idx = pin (problem-major order);
// ROW_TANGENT f0 = field of i1, f1 = field of i2, idx = 2 * tangent + a (problem-major order);
// ROW_SURFACE f0 = field.
struct RowDesc {
    int type, f0, f1, idx;
};

struct PinState {
    // host lists as given (tangent targets normalised)
    std::vector<int32_t> pin_v, tan_e, surf_v;
    std::vector<double> pin_p, tan_X;
    double quad[13] = {0};  // Q (row-major), b, c
    // problem-major layout on the device
    int n_pin = 0, n_tan = 0, n_surf = 0;
    int fmax = 0, rmax = 0;  // most fields / rows of one problem
    int nsolve = 0;          // three-column solves per gradient: ceil(fmax / 3)
    int w_cap = 0;           // solves d_W has room for
    int warm = 0;            // d_W holds the fields of an earlier step for these vertices
    size_t smem = 0;         // dynamic shared memory of k_pin_system
    int32_t *d_fv = nullptr, *d_foff = nullptr;  // fields [nProb * kMaxFields], offsets [nProb + 1]
    RowDesc *d_rows = nullptr;                   // [nProb * kMaxRows]
    int32_t *d_roff = nullptr;
    int32_t *d_pv = nullptr, *d_poff = nullptr;  // pinned vertices [nProb * kMaxFields], offsets
    double *d_pt = nullptr;                      // their targets [.][3]
    int32_t *d_te = nullptr, *d_toff = nullptr;  // tangent edges [nProb * kMaxRows], offsets
    double *d_tX = nullptr;                      // targets [.][3]
    double *d_tB = nullptr;                      // bases across the targets [.][2][3]
    int32_t *d_sv = nullptr, *d_soff = nullptr;  // surface vertices [nProb * kMaxRows], offsets
    double *d_quad = nullptr;                    // [13]
    double *d_W = nullptr;       // [w_cap][nV][3]: field l of a problem is column l % 3 of solve l / 3
    double *d_red = nullptr;     // [nProb][5] (pin_reduce)
    double *d_coef = nullptr;    // [nProb][kCoefStride]
};

cudaError_t pin_reduce(Ctx &c, const double *a, const double *b, const double *dE, double *out, cudaStream_t s);

bool pins_ready(const Ctx &c) { return c.pins && c.pins->n_pin > 0; }

void pins_free(Ctx &c)
{
    if (!c.pins) return;
    PinState &p = *c.pins;
    void *ptrs[] = {p.d_fv, p.d_foff, p.d_rows, p.d_roff, p.d_pv, p.d_poff, p.d_pt, p.d_te, p.d_toff,
                    p.d_tX, p.d_tB, p.d_sv, p.d_soff, p.d_quad, p.d_W, p.d_red, p.d_coef};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    delete c.pins;
    c.pins = nullptr;
}

// Right-hand side of solve s: column j holds e_u for the problem's field 3 s + j (one thread per problem;
// out was zeroed).
__global__ void k_pin_rhs(int nprob, int s, const int32_t *__restrict__ off, const int32_t *__restrict__ fv,
                          double *__restrict__ out)
{
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nprob) return;
    int k = off[q + 1] - off[q];
    for (int l = 3 * s; l < min(k, 3 * s + 3); ++l) out[3 * (size_t)fv[off[q] + l] + (l - 3 * s)] = 1.0;
}

__device__ __forceinline__ double quad_f(const double *Q, const double *x)
{
    double f = Q[12];
    for (int i = 0; i < 3; ++i) {
        f += Q[9 + i] * x[i];
        for (int j = 0; j < 3; ++j) f += x[i] * Q[3 * i + j] * x[j];
    }
    return f;
}

__device__ __forceinline__ double nan_max(double m, double d) { return (d > m || d != d) ? d : m; }

// Per problem: phi[4q] = max over pins and components of |gamma_v,k - p_v,k|, phi[4q + 1] = max over
// tangent edges and components of |T_I,k - X_I,k|, phi[4q + 2] = max over surface vertices of |f(gamma_v)|
// (row 4q + 3, the length, is left alone).  A NaN propagates.
__global__ void k_pin_phi(int nprob, const int32_t *__restrict__ poff, const int32_t *__restrict__ pv,
                          const double *__restrict__ pt, const int32_t *__restrict__ toff,
                          const int32_t *__restrict__ te, const double *__restrict__ tX,
                          const int32_t *__restrict__ soff, const int32_t *__restrict__ sv,
                          const double *__restrict__ quad, const double *__restrict__ gamma,
                          const double *__restrict__ T, double *__restrict__ phi)
{
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nprob) return;
    double m0 = 0.0, m1 = 0.0, m2 = 0.0;
    for (int i = poff[q]; i < poff[q + 1]; ++i)
        for (int k = 0; k < 3; ++k) m0 = nan_max(m0, fabs(gamma[3 * (size_t)pv[i] + k] - pt[3 * i + k]));
    for (int i = toff[q]; i < toff[q + 1]; ++i)
        for (int k = 0; k < 3; ++k) m1 = nan_max(m1, fabs(T[3 * (size_t)te[i] + k] - tX[3 * i + k]));
    for (int i = soff[q]; i < soff[q + 1]; ++i) m2 = nan_max(m2, fabs(quad_f(quad, gamma + 3 * (size_t)sv[i])));
    phi[4 * q] = m0;
    phi[4 * q + 1] = m1;
    phi[4 * q + 2] = m2;
}

// One block per problem: the rows' terms (field, component, coefficient) at the given geometry, then
// [S CN; (CN)^T 0 | rhs], its solution, and the combination's coefficients
//   coef[0] = length multiplier, coef[1 + 3 f + j] = sum_r sol_r c_r(f, j), coef[3 nf + 1 + j] = t_j.
// Unknown order: 0 the length row, 1 + r the problem's row r, R + 1 + j the translation component j.
//   mode 0 (gradient):   rhs = [<C_len, y0>; C_r y0; sum dE_j]
//   mode 1 (projection): rhs = [-Phi_len; -Phi_r(gamma); 0]
__global__ void __launch_bounds__(kSysThreads) k_pin_system(
    int mode, const int32_t *__restrict__ foff, const int32_t *__restrict__ fv, const RowDesc *__restrict__ rows,
    const int32_t *__restrict__ roff, const double *__restrict__ pt, const int32_t *__restrict__ te,
    const double *__restrict__ tB, const double *__restrict__ quad, const double *__restrict__ T,
    const double *__restrict__ ell, const double *__restrict__ W, size_t wstride, const double *__restrict__ y0,
    const double *__restrict__ y1, const double *__restrict__ red, const double *__restrict__ gamma,
    const double *__restrict__ phi, double *__restrict__ coef, int *__restrict__ err)
{
    extern __shared__ double sm[];
    __shared__ int s_piv;
    __shared__ int s_bad;
    const int q = blockIdx.x;
    const int f0 = foff[q], nf = foff[q + 1] - f0;
    const int r0 = roff[q], R = roff[q + 1] - r0;
    const int m = R + 4, ld = m + 1;
    double *A = sm;                                // [m][ld], last column the right-hand side
    double *f = A + (size_t)m * ld;                // [m] elimination factors, then the solution
    double *tc = f + m;                            // [R][kMaxTerms] term coefficients
    double *rrhs = tc + (size_t)R * kMaxTerms;     // [R] the rows' right-hand sides
    int *tf = reinterpret_cast<int *>(rrhs + R);   // [R][kMaxTerms] term fields
    int *tj = tf + (size_t)R * kMaxTerms;          // [R][kMaxTerms] term components
    int *nt = tj + (size_t)R * kMaxTerms;          // [R] terms per row
    const double *r5 = red + 5 * q;
    if (threadIdx.x == 0) s_bad = 0;
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        const RowDesc d = rows[r0 + r];
        int n = 0;
        double rhs = 0.0;
        int *rf = tf + r * kMaxTerms, *rj = tj + r * kMaxTerms;
        double *rc = tc + r * kMaxTerms;
        if (d.type == ROW_PIN) {
            rf[0] = d.f0;
            rj[0] = d.f1;
            rc[0] = 1.0;
            n = 1;
            if (mode == 1) rhs = pt[3 * d.idx + d.f1] - gamma[3 * (size_t)fv[f0 + d.f0] + d.f1];
        } else if (d.type == ROW_TANGENT) {
            const int t = d.idx >> 1, a = d.idx & 1;
            const size_t I = (size_t)te[t];
            const double *b = tB + 6 * t + 3 * a;
            const double t0 = T[3 * I], t1 = T[3 * I + 1], t2 = T[3 * I + 2];
            const double bt = b[0] * t0 + b[1] * t1 + b[2] * t2;
            const double il = 1.0 / ell[I];
            const double rv[3] = {(b[0] - bt * t0) * il, (b[1] - bt * t1) * il, (b[2] - bt * t2) * il};
            for (int j = 0; j < 3; ++j) {
                rf[j] = d.f1;  // i2: +r
                rj[j] = j;
                rc[j] = rv[j];
                rf[3 + j] = d.f0;  // i1: -r
                rj[3 + j] = j;
                rc[3 + j] = -rv[j];
            }
            n = 6;
            if (mode == 1) rhs = -bt;
        } else {
            const double *x = gamma + 3 * (size_t)fv[f0 + d.f0];
            for (int j = 0; j < 3; ++j) {
                double gj = quad[9 + j];
                for (int k = 0; k < 3; ++k) gj += (quad[3 * j + k] + quad[3 * k + j]) * x[k];
                rf[j] = d.f0;
                rj[j] = j;
                rc[j] = gj;
            }
            n = 3;
            if (mode == 1) rhs = -quad_f(quad, x);
        }
        if (mode == 0)
            for (int k = 0; k < n; ++k) rhs += rc[k] * y0[3 * (size_t)fv[f0 + rf[k]] + rj[k]];
        nt[r] = n;
        rrhs[r] = rhs;
    }
    __syncthreads();
    const int ti = R + 1;  // first translation unknown
    for (int e = threadIdx.x; e < m * ld; e += blockDim.x) {
        const int i = e / ld, j = e % ld;
        double a = 0.0;
        if (j == m) {
            if (i == 0) a = mode == 0 ? r5[0] : -phi[4 * q + 3];
            else if (i < ti) a = rrhs[i - 1];
            else a = mode == 0 ? r5[2 + (i - ti)] : 0.0;
        } else if (i == 0 || j == 0) {
            const int o = i == 0 ? j : i;
            if (o == 0) {
                a = r5[1];
            } else if (o < ti) {  // the row's terms applied to y1
                const int r = o - 1;
                for (int k = 0; k < nt[r]; ++k)
                    a += tc[r * kMaxTerms + k] * y1[3 * (size_t)fv[f0 + tf[r * kMaxTerms + k]] + tj[r * kMaxTerms + k]];
            }
        } else if (i < ti && j < ti) {  // S_rr' = sum c c' w_f'(v_f) over terms of equal component
            const int r = i - 1, rr = j - 1;
            for (int k = 0; k < nt[r]; ++k) {
                const int comp = tj[r * kMaxTerms + k];
                const size_t v = (size_t)fv[f0 + tf[r * kMaxTerms + k]];
                for (int kk = 0; kk < nt[rr]; ++kk) {
                    if (tj[rr * kMaxTerms + kk] != comp) continue;
                    const int fl = tf[rr * kMaxTerms + kk];
                    a += tc[r * kMaxTerms + k] * tc[rr * kMaxTerms + kk] *
                         W[(size_t)(fl / 3) * wstride + 3 * v + fl % 3];
                }
            }
        } else if (i < ti || j < ti) {  // C N and its transpose
            const int r = (i < ti ? i : j) - 1, comp = (i < ti ? j : i) - ti;
            for (int k = 0; k < nt[r]; ++k)
                if (tj[r * kMaxTerms + k] == comp) a += tc[r * kMaxTerms + k];
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
        const int nr = m - col - 1, nc = ld - col;
        for (int e = threadIdx.x; e < nr * nc; e += blockDim.x) {
            const int i = col + 1 + e / nc, j = col + e % nc;
            A[i * ld + j] -= f[i] * A[col * ld + j];
        }
        __syncthreads();
    }
    double *out = coef + (size_t)q * kCoefStride;
    if (s_bad) {
        for (int i = threadIdx.x; i < 3 * nf + 4; i += blockDim.x) out[i] = 0.0;
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
        out[0] = f[0];
        for (int i = 0; i < 3 * nf; ++i) out[1 + i] = 0.0;
        for (int r = 0; r < R; ++r)
            for (int k = 0; k < nt[r]; ++k)
                out[1 + 3 * tf[r * kMaxTerms + k] + tj[r * kMaxTerms + k]] += f[1 + r] * tc[r * kMaxTerms + k];
        for (int j = 0; j < 3; ++j) out[3 * nf + 1 + j] = f[ti + j];
    }
}

// out(v) = base(v) - acc(v) (base given) or acc(v), acc = coef_len y1 + sum_f w_f coef_f + coef_t.
__global__ void k_pin_combine(int nV, const int32_t *__restrict__ vprob, const int32_t *__restrict__ foff,
                              const double *__restrict__ W, size_t wstride, const double *__restrict__ y1,
                              const double *__restrict__ coef, const double *__restrict__ base,
                              double *__restrict__ out)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nV) return;
    const int q = vprob[v];
    const int k = foff[q + 1] - foff[q];
    const double *cf = coef + (size_t)q * kCoefStride;
    double acc[3];
    for (int i = 0; i < 3; ++i) acc[i] = cf[0] * y1[3 * (size_t)v + i] + cf[3 * k + 1 + i];
    for (int l = 0; l < k; ++l) {
        const double w = W[(size_t)(l / 3) * wstride + 3 * (size_t)v + l % 3];
        for (int i = 0; i < 3; ++i) acc[i] += cf[1 + 3 * l + i] * w;
    }
    for (int i = 0; i < 3; ++i) out[3 * (size_t)v + i] = base ? base[3 * (size_t)v + i] - acc[i] : acc[i];
}

// ------------------------------------------------------------------------------------------ host side

static int problem_of(const std::vector<int32_t> &offsets, int i)
{
    return (int)(std::upper_bound(offsets.begin(), offsets.end(), i) - offsets.begin()) - 1;
}

// Two orthonormal vectors across the unit vector X: b1 = X x e_k / |.| with e_k the coordinate axis least
// aligned with X, b2 = X x b1.
static void perp_basis(const double *X, double *b1, double *b2)
{
    int k = 0;
    for (int j = 1; j < 3; ++j)
        if (std::fabs(X[j]) < std::fabs(X[k])) k = j;
    double e[3] = {0.0, 0.0, 0.0};
    e[k] = 1.0;
    b1[0] = X[1] * e[2] - X[2] * e[1];
    b1[1] = X[2] * e[0] - X[0] * e[2];
    b1[2] = X[0] * e[1] - X[1] * e[0];
    const double n = std::sqrt(b1[0] * b1[0] + b1[1] * b1[1] + b1[2] * b1[2]);
    for (int j = 0; j < 3; ++j) b1[j] /= n;
    b2[0] = X[1] * b1[2] - X[2] * b1[1];
    b2[1] = X[2] * b1[0] - X[0] * b1[2];
    b2[2] = X[0] * b1[1] - X[1] * b1[0];
}

// Lay the host lists out problem by problem (fields, rows, per-kind lists), check the per-problem limits
// and upload.  Returns cudaErrorInvalidValue with `why` set when the lists break a rule.
static cudaError_t rebuild(Ctx &c, std::string &why)
{
    PinState &p = *c.pins;
    const int P = c.nProb;
    std::vector<std::vector<int>> pins(P), tans(P), surfs(P);
    for (size_t i = 0; i < p.pin_v.size(); ++i) pins[problem_of(c.h_prob_v, p.pin_v[i])].push_back((int)i);
    for (size_t i = 0; i < p.tan_e.size(); ++i) tans[problem_of(c.h_prob_e, p.tan_e[i])].push_back((int)i);
    for (size_t i = 0; i < p.surf_v.size(); ++i) surfs[problem_of(c.h_prob_v, p.surf_v[i])].push_back((int)i);
    std::vector<int32_t> fv, foff(P + 1, 0), roff(P + 1, 0), pv, poff(P + 1, 0), te, toff(P + 1, 0), sv,
        soff(P + 1, 0);
    std::vector<RowDesc> rows;
    std::vector<double> pt, tX, tB;
    int fmax = 0, rmax = 0;
    std::vector<char> pinned(c.nV, 0);
    for (int v : p.pin_v) pinned[v] = 1;
    for (int q = 0; q < P; ++q) {
        std::vector<int> fl;  // this problem's field vertices
        auto field = [&](int v) {
            for (size_t k = 0; k < fl.size(); ++k)
                if (fl[k] == v) return (int)k;
            fl.push_back(v);
            return (int)fl.size() - 1;
        };
        const size_t r0 = rows.size();
        for (int i : pins[q]) {
            const int f = field(p.pin_v[i]);
            for (int k = 0; k < 3; ++k) rows.push_back({ROW_PIN, f, k, (int)pv.size()});
            pv.push_back(p.pin_v[i]);
            for (int k = 0; k < 3; ++k) pt.push_back(p.pin_p[3 * i + k]);
        }
        for (int i : tans[q]) {
            const int I = p.tan_e[i];
            const int i1 = c.h_edges[2 * I], i2 = c.h_edges[2 * I + 1];
            if (pinned[i1] && pinned[i2]) {
                why = "a tangent-constrained edge has both endpoints pinned";
                return cudaErrorInvalidValue;
            }
            const int fa = field(i1), fb = field(i2);
            const int t = (int)te.size();
            rows.push_back({ROW_TANGENT, fa, fb, 2 * t});
            rows.push_back({ROW_TANGENT, fa, fb, 2 * t + 1});
            te.push_back(I);
            double b1[3], b2[3];
            perp_basis(&p.tan_X[3 * i], b1, b2);
            for (int k = 0; k < 3; ++k) tX.push_back(p.tan_X[3 * i + k]);
            for (int k = 0; k < 3; ++k) tB.push_back(b1[k]);
            for (int k = 0; k < 3; ++k) tB.push_back(b2[k]);
        }
        for (int i : surfs[q]) {
            const int v = p.surf_v[i];
            if (pinned[v]) {
                why = "a vertex is both pinned and held on the surface";
                return cudaErrorInvalidValue;
            }
            rows.push_back({ROW_SURFACE, field(v), 0, (int)sv.size()});
            sv.push_back(v);
        }
        if ((int)fl.size() > kMaxFields) {
            why = "more than 24 constrained vertices in one problem";
            return cudaErrorInvalidValue;
        }
        if ((int)(rows.size() - r0) > kMaxRows) {
            why = "more than 96 point, tangent and surface rows in one problem";
            return cudaErrorInvalidValue;
        }
        fmax = std::max(fmax, (int)fl.size());
        rmax = std::max(rmax, (int)(rows.size() - r0));
        fv.insert(fv.end(), fl.begin(), fl.end());
        foff[q + 1] = (int32_t)fv.size();
        roff[q + 1] = (int32_t)rows.size();
        poff[q + 1] = (int32_t)pv.size();
        toff[q + 1] = (int32_t)te.size();
        soff[q + 1] = (int32_t)sv.size();
    }
    // buffers sized by the per-problem limits, allocated once
    if (!p.d_fv) {
        const size_t Pz = (size_t)P;
        TPE_CHECK(cudaMalloc(&p.d_fv, sizeof(int32_t) * Pz * kMaxFields));
        TPE_CHECK(cudaMalloc(&p.d_rows, sizeof(RowDesc) * Pz * kMaxRows));
        TPE_CHECK(cudaMalloc(&p.d_pv, sizeof(int32_t) * Pz * kMaxFields));
        TPE_CHECK(cudaMalloc(&p.d_pt, sizeof(double) * 3 * Pz * kMaxFields));
        TPE_CHECK(cudaMalloc(&p.d_te, sizeof(int32_t) * Pz * kMaxRows));
        TPE_CHECK(cudaMalloc(&p.d_tX, sizeof(double) * 3 * Pz * kMaxRows));
        TPE_CHECK(cudaMalloc(&p.d_tB, sizeof(double) * 6 * Pz * kMaxRows));
        TPE_CHECK(cudaMalloc(&p.d_sv, sizeof(int32_t) * Pz * kMaxRows));
        int32_t **offs[] = {&p.d_foff, &p.d_roff, &p.d_poff, &p.d_toff, &p.d_soff};
        for (int32_t **o : offs) TPE_CHECK(cudaMalloc(o, sizeof(int32_t) * (Pz + 1)));
        TPE_CHECK(cudaMalloc(&p.d_quad, sizeof(double) * 13));
        TPE_CHECK(cudaMalloc(&p.d_red, sizeof(double) * 5 * Pz));
        TPE_CHECK(cudaMalloc(&p.d_coef, sizeof(double) * kCoefStride * Pz));
    }
    const int nsolve = (fmax + 2) / 3;
    if (nsolve > p.w_cap) {
        if (p.d_W) TPE_CHECK(cudaFree(p.d_W));
        p.d_W = nullptr;
        p.w_cap = 0;
        TPE_CHECK(cudaMalloc(&p.d_W, sizeof(double) * 3 * (size_t)c.nV * nsolve));
        p.w_cap = nsolve;
    }
    const int m = rmax + 4;
    const size_t smem = sizeof(double) * ((size_t)m * (m + 1) + m + (size_t)rmax * (kMaxTerms + 1)) +
                        sizeof(int) * (size_t)rmax * (2 * kMaxTerms + 1);
    auto up = [](void *d, const void *h, size_t bytes) {
        return bytes ? cudaMemcpy(d, h, bytes, cudaMemcpyHostToDevice) : cudaSuccess;
    };
    TPE_CHECK(up(p.d_fv, fv.data(), sizeof(int32_t) * fv.size()));
    TPE_CHECK(up(p.d_foff, foff.data(), sizeof(int32_t) * foff.size()));
    TPE_CHECK(up(p.d_rows, rows.data(), sizeof(RowDesc) * rows.size()));
    TPE_CHECK(up(p.d_roff, roff.data(), sizeof(int32_t) * roff.size()));
    TPE_CHECK(up(p.d_pv, pv.data(), sizeof(int32_t) * pv.size()));
    TPE_CHECK(up(p.d_poff, poff.data(), sizeof(int32_t) * poff.size()));
    TPE_CHECK(up(p.d_pt, pt.data(), sizeof(double) * pt.size()));
    TPE_CHECK(up(p.d_te, te.data(), sizeof(int32_t) * te.size()));
    TPE_CHECK(up(p.d_toff, toff.data(), sizeof(int32_t) * toff.size()));
    TPE_CHECK(up(p.d_tX, tX.data(), sizeof(double) * tX.size()));
    TPE_CHECK(up(p.d_tB, tB.data(), sizeof(double) * tB.size()));
    TPE_CHECK(up(p.d_sv, sv.data(), sizeof(int32_t) * sv.size()));
    TPE_CHECK(up(p.d_soff, soff.data(), sizeof(int32_t) * soff.size()));
    TPE_CHECK(up(p.d_quad, p.quad, sizeof(double) * 13));
    p.n_pin = (int)pv.size();
    p.n_tan = (int)te.size();
    p.n_surf = (int)sv.size();
    p.fmax = fmax;
    p.rmax = rmax;
    p.nsolve = nsolve;
    p.smem = smem;
    p.warm = 0;
    return cudaSuccess;
}

// Validate a list of distinct indices in [0, bound).
static bool distinct_in_range(const int32_t *a, int n, int bound, const char *what, std::string &why)
{
    std::vector<char> seen(bound, 0);
    for (int i = 0; i < n; ++i) {
        if (a[i] < 0 || a[i] >= bound) {
            why = std::string(what) + " out of range";
            return false;
        }
        if (seen[a[i]]) {
            why = std::string(what) + " given twice";
            return false;
        }
        seen[a[i]] = 1;
    }
    return true;
}

// Apply a change to the host lists and rebuild; the old lists come back when the new ones break a rule.
template <typename F>
static cudaError_t change(Ctx &c, std::string &why, F &&mutate)
{
    if (!c.pins) c.pins = new PinState();
    PinState &p = *c.pins;
    const std::vector<int32_t> pin_v = p.pin_v, tan_e = p.tan_e, surf_v = p.surf_v;
    const std::vector<double> pin_p = p.pin_p, tan_X = p.tan_X;
    double quad[13];
    std::copy(p.quad, p.quad + 13, quad);
    mutate(p);
    cudaError_t e = rebuild(c, why);
    if (e == cudaErrorInvalidValue && !why.empty()) {
        p.pin_v = pin_v;
        p.pin_p = pin_p;
        p.tan_e = tan_e;
        p.tan_X = tan_X;
        p.surf_v = surf_v;
        std::copy(quad, quad + 13, p.quad);
        std::string ignore;
        TPE_CHECK(rebuild(c, ignore));
        return cudaErrorInvalidValue;
    }
    return e;
}

cudaError_t pins_set(Ctx &c, int n, const int32_t *v, const double *targets, std::string &why)
{
    if (n < 0 || (n > 0 && (!v || !targets))) {
        why = "pins: bad count or null arrays";
        return cudaErrorInvalidValue;
    }
    if (!distinct_in_range(v, n, c.nV, "pinned vertex", why)) return cudaErrorInvalidValue;
    for (int i = 0; i < 3 * n; ++i)
        if (!std::isfinite(targets[i])) {
            why = "non-finite pin target";
            return cudaErrorInvalidValue;
        }
    if (n > 0) {
        std::vector<int> cnt(c.nProb, 0);
        for (int i = 0; i < n; ++i) cnt[problem_of(c.h_prob_v, v[i])]++;
        for (int q = 0; q < c.nProb; ++q)
            if (cnt[q] == 0) {
                why = "TP_CONSTRAINTS_POINTS: every problem needs at least one pinned vertex";
                return cudaErrorInvalidValue;
            }
    }
    return change(c, why, [&](PinState &p) {
        p.pin_v.assign(v, v + n);
        p.pin_p.assign(targets, targets + 3 * (size_t)n);
    });
}

cudaError_t tangents_set(Ctx &c, int n, const int32_t *edges, const double *X, std::string &why)
{
    if (n < 0 || (n > 0 && (!edges || !X))) {
        why = "tangents: bad count or null arrays";
        return cudaErrorInvalidValue;
    }
    if (!distinct_in_range(edges, n, c.nE, "tangent edge", why)) return cudaErrorInvalidValue;
    std::vector<double> unit(3 * (size_t)n);
    for (int i = 0; i < n; ++i) {
        const double *x = X + 3 * i;
        const double r = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
        if (!std::isfinite(r) || !(r > 0.0)) {
            why = "tangent target must be finite and nonzero";
            return cudaErrorInvalidValue;
        }
        for (int k = 0; k < 3; ++k) unit[3 * i + k] = x[k] / r;
    }
    return change(c, why, [&](PinState &p) {
        p.tan_e.assign(edges, edges + n);
        p.tan_X = unit;
    });
}

cudaError_t surface_set(Ctx &c, const double *quadric, int n, const int32_t *v, std::string &why)
{
    if (n < 0 || (n > 0 && (!v || !quadric))) {
        why = "surface: bad count or null arrays";
        return cudaErrorInvalidValue;
    }
    if (!distinct_in_range(v, n, c.nV, "surface vertex", why)) return cudaErrorInvalidValue;
    if (n > 0)
        for (int k = 0; k < 13; ++k)
            if (!std::isfinite(quadric[k])) {
                why = "non-finite quadric coefficient";
                return cudaErrorInvalidValue;
            }
    return change(c, why, [&](PinState &p) {
        p.surf_v.assign(v, v + n);
        if (n > 0) std::copy(quadric, quadric + 13, p.quad);
    });
}

cudaError_t pins_phi(Ctx &c, const double *gamma, int which, double *phi, cudaStream_t s)
{
    PinState &p = *c.pins;
    k_pin_phi<<<(c.nProb + 127) / 128, 128, 0, s>>>(c.nProb, p.d_poff, p.d_pv, p.d_pt, p.d_toff, p.d_te, p.d_tX,
                                                    p.d_soff, p.d_sv, p.d_quad, gamma, c.d_Tw[which], phi);
    c.launches++;
    return cudaGetLastError();
}

static cudaError_t pin_system(Ctx &c, int mode, int which, const double *y0, const double *y1,
                              const double *gamma, const double *phi, cudaStream_t s)
{
    PinState &p = *c.pins;
    // the limit belongs to the kernel, not to this context: set it for this context's size every time
    TPE_CHECK(cudaFuncSetAttribute(k_pin_system, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem));
    k_pin_system<<<c.nProb, kSysThreads, p.smem, s>>>(mode, p.d_foff, p.d_fv, p.d_rows, p.d_roff, p.d_pt, p.d_te,
                                                      p.d_tB, p.d_quad, c.d_Tw[which], c.d_ellw[which], p.d_W,
                                                      3 * (size_t)c.nV, y0, y1, p.d_red, gamma, phi, p.d_coef,
                                                      c.d_err);
    c.launches++;
    return cudaGetLastError();
}

static cudaError_t pin_combine(Ctx &c, const double *y1, const double *base, double *out, cudaStream_t s)
{
    PinState &p = *c.pins;
    k_pin_combine<<<(c.nV + 255) / 256, 256, 0, s>>>(c.nV, c.d_vprob, p.d_foff, p.d_W, 3 * (size_t)c.nV, y1,
                                                     p.d_coef, base, out);
    c.launches++;
    return cudaGetLastError();
}

// The fields w_u = A^+ e_u of every constrained vertex (mean-free CG solves on the geometry in slot 0),
// warm-started from the previous step's fields.  rhs_scratch: [nV][3].
cudaError_t pins_fields(Ctx &c, const double *gamma, double *rhs_scratch, int *iters, double *rr, int *conv,
                        int *bd, int *flags, cudaStream_t s)
{
    PinState &p = *c.pins;
    const size_t vb = sizeof(double) * 3 * (size_t)c.nV;
    for (int sv = 0; sv < p.nsolve; ++sv) {
        TPE_CHECK(cudaMemsetAsync(rhs_scratch, 0, vb, s));
        k_pin_rhs<<<(c.nProb + 127) / 128, 128, 0, s>>>(c.nProb, sv, p.d_foff, p.d_fv, rhs_scratch);
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

// g = y0 - (lambda_len y1 + sum_r lambda_r A^+ C_r^T - t) from y0 = A^+ dE and y1 = A^+ C_len^T (gamma in
// geometry slot 0, its Jacobian in c.d_Cv, the fields in d_W).
cudaError_t pins_gradient(Ctx &c, const double *gamma, const double *dE, const double *y0, const double *y1,
                          double *g, cudaStream_t s)
{
    TPE_CHECK(pin_reduce(c, y0, y1, dE, c.pins->d_red, s));
    TPE_CHECK(pin_system(c, 0, 0, y0, y1, gamma, nullptr, s));
    return pin_combine(c, y1, y0, g, s);
}

// x = nu_len y1 + sum_r nu_r A^+ C_r^T + t with C x = -Phi at the trial curve gamma_t (geometry slot 1;
// y1 = A^+ C_len(gamma_t)^T, phi[4q + 3] = Phi_len of gamma_t).
cudaError_t pins_projection(Ctx &c, const double *y1, const double *gamma_t, const double *phi, double *x,
                            cudaStream_t s)
{
    TPE_CHECK(pin_reduce(c, nullptr, y1, nullptr, c.pins->d_red, s));
    TPE_CHECK(pin_system(c, 1, 1, nullptr, y1, gamma_t, phi, s));
    return pin_combine(c, y1, nullptr, x, s);
}

}  // namespace tpe
