"""Plain FP64 CPU oracle for the Repulsive Curves hot path (arXiv 2006.07859).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU-baseline
leg may import this module; the CUDA library never does, and this module never touches
the CUDA library.  The pair sums live in ``tpe_oracle.c`` (literal loops, FP64); this
file adds the linear algebra on top of them with numpy, one library primitive per step
(a dense solve, an FFT), in the order the paper states it:

  * constraints Phi and their Jacobian C ........... Sec. 8.1 (barycenter; total length or
                                                     every edge length; pinned points, tangents
                                                     and quadric surfaces)
  * gradient saddle-point problem .................. Sec. 5.3.1, Eq. 22 (dense solve)
  * projected system P^T A P y = P^T a, x = P y .... App. B.3.3 (solved by CG)
  * constraint projection via z = C^+ b, x = z - y . Sec. 5.3.2 Eq. 23, App. B.3.4
  * descent step: normalised gradient, backtracking
    from tau = 1 until Armijo holds and the
    constraint projection succeeds ................. Sec. 5.4

Readings taken where the paper is silent or garbled (each is listed with its reason in
the design notes of the repository):
  * P = I - C^T (C C^T)^{-1} C and C^+ = C^T (C C^T)^{-1} (the printed "P := C C^+" with
    C^+ = (C C^T)^{-1} C^T does not type-check; this is the Euclidean projector onto
    null(C)).
  * A-bar in the constraint projection is the one of the pre-step curve; C is evaluated
    at the current iterate.
  * The tangent constraint T_I = X keeps the two rows b_a . T_I across X (the printed three
    rows T_I - X have a Jacobian of rank 2); the surface constraint takes a quadric f.
  * Armijo constant 1e-4, halving, at most 30 halvings; projection tolerance on
    max|Phi| relative to max(1, L0).

The Jacobi-scaled circulant ("spectral") preconditioner at the end is not from the
paper; it is this library's preconditioner, and the oracle for it is written from its
definition (eigen-decomposition of the Gram matrix of a regular polygon) with numpy.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tpe_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle_tpe.so")
_lib = None


def build_library(force: bool = False) -> str:
    """Compile tpe_oracle.c with gcc (FP64, no fast-math, OpenMP over independent rows)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build_library()
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.POINTER
        d, i = ctypes.c_double, ctypes.c_int
        pd, pi = P(d), P(i)
        L.orc_energy.argtypes = [i, pd, i, pi, d, d, pd, pd]
        L.orc_energy_rows.argtypes = [i, pd, i, pi, d, d, i, pi, pd]
        L.orc_differential.argtypes = [i, pd, i, pi, d, d, pd]
        L.orc_differential_at.argtypes = [i, pd, i, pi, d, d, i, pi, pd]
        L.orc_gram_dense.argtypes = [i, pd, i, pi, d, pd, pd]
        L.orc_gram_apply.argtypes = [i, pd, i, pi, d, i, pd, pd]
        L.orc_gram_apply_at.argtypes = [i, pd, i, pi, d, i, pd, i, pi, pd]
        L.orc_bilinear.argtypes = [i, pd, i, pi, d, pd, pd, pd, pd]
        L.orc_edge_quantities.argtypes = [i, pd, i, pi, pd, pd, pd]
        L.orc_num_threads.argtypes = []
        _lib = L
    return _lib


def _pd(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _pi(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _geom(gamma, edges):
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    e = np.ascontiguousarray(edges, dtype=np.int32)
    return g, e


class OracleError(RuntimeError):
    pass


def _check(st):
    if st == 1:
        raise OracleError("edge of zero length: tangent undefined")
    if st != 0:
        raise OracleError(f"oracle status {st}")


def sigma_of(alpha: float, beta: float) -> float:
    """sigma = s - 1 with s = (beta - 1)/alpha (Sec. 4.2.2)."""
    return (beta - 1.0) / alpha - 1.0


def num_threads() -> int:
    return int(lib().orc_num_threads())


# ----------------------------------------------------------------------------- pair sums (C)

def edge_quantities(gamma, edges):
    g, e = _geom(gamma, edges)
    nE = e.shape[0]
    ell, T, x = np.empty(nE), np.empty((nE, 3)), np.empty((nE, 3))
    _check(lib().orc_edge_quantities(g.shape[0], _pd(g), nE, _pi(e), _pd(ell), _pd(T), _pd(x)))
    return ell, T, x


def energy(gamma, edges, alpha=2.0, beta=4.5, rows=False):
    """Discrete energy, Eq. 17 (and the per-target-edge row sums if rows=True)."""
    g, e = _geom(gamma, edges)
    r = np.empty(e.shape[0])
    tot = ctypes.c_double(0.0)
    _check(lib().orc_energy(g.shape[0], _pd(g), e.shape[0], _pi(e), alpha, beta, _pd(r), ctypes.byref(tot)))
    return (tot.value, r) if rows else tot.value


def energy_rows(gamma, edges, idx, alpha=2.0, beta=4.5):
    g, e = _geom(gamma, edges)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    out = np.empty(idx.shape[0])
    _check(lib().orc_energy_rows(g.shape[0], _pd(g), e.shape[0], _pi(e), alpha, beta, idx.shape[0], _pi(idx),
                                 _pd(out)))
    return out


def differential(gamma, edges, alpha=2.0, beta=4.5):
    """d hat-E / d gamma, vertex-major [nV, 3] (Sec. 5.1)."""
    g, e = _geom(gamma, edges)
    out = np.zeros((g.shape[0], 3))
    _check(lib().orc_differential(g.shape[0], _pd(g), e.shape[0], _pi(e), alpha, beta, _pd(out)))
    return out


def differential_at(gamma, edges, vidx, alpha=2.0, beta=4.5):
    g, e = _geom(gamma, edges)
    v = np.ascontiguousarray(vidx, dtype=np.int32)
    out = np.zeros((v.shape[0], 3))
    _check(lib().orc_differential_at(g.shape[0], _pd(g), e.shape[0], _pi(e), alpha, beta, v.shape[0], _pi(v),
                                     _pd(out)))
    return out


def gram_dense(gamma, edges, sigma):
    """(B, B0) built by the increment tables of Secs. 5.2.2-5.2.3 (row-major nV x nV)."""
    g, e = _geom(gamma, edges)
    n = g.shape[0]
    B, B0 = np.zeros((n, n)), np.zeros((n, n))
    _check(lib().orc_gram_dense(n, _pd(g), e.shape[0], _pi(e), sigma, _pd(B), _pd(B0)))
    return B, B0


def gram_apply(gamma, edges, sigma, u):
    """(B + B0) u, matrix-free with the same increments; u is [nV] or [nV, m]."""
    g, e = _geom(gamma, edges)
    u = np.asarray(u, dtype=np.float64)
    vec = u.ndim == 1
    U = np.ascontiguousarray(u.reshape(u.shape[0], -1))
    out = np.zeros_like(U)
    _check(lib().orc_gram_apply(g.shape[0], _pd(g), e.shape[0], _pi(e), sigma, U.shape[1], _pd(U), _pd(out)))
    return out[:, 0] if vec else out


def gram_apply_at(gamma, edges, sigma, u, vidx):
    g, e = _geom(gamma, edges)
    U = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(g.shape[0], -1))
    v = np.ascontiguousarray(vidx, dtype=np.int32)
    out = np.zeros((v.shape[0], U.shape[1]))
    _check(lib().orc_gram_apply_at(g.shape[0], _pd(g), e.shape[0], _pi(e), sigma, U.shape[1], _pd(U), v.shape[0],
                                   _pi(v), _pd(out)))
    return out


def bilinear(gamma, edges, sigma, u, v):
    """(u^T B v, u^T B0 v) evaluated from the bilinear forms of Eq. 21 and Sec. 5.2.3."""
    g, e = _geom(gamma, edges)
    u = np.ascontiguousarray(u, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    a, b = ctypes.c_double(0), ctypes.c_double(0)
    _check(lib().orc_bilinear(g.shape[0], _pd(g), e.shape[0], _pi(e), sigma, _pd(u), _pd(v), ctypes.byref(a),
                              ctypes.byref(b)))
    return a.value, b.value


# ----------------------------------------------------------------------------- constraints

def perp_basis(X):
    """Two orthonormal vectors spanning the plane orthogonal to the unit vector X: b1 = X x e_k / |.|
    with e_k the coordinate axis least aligned with X, and b2 = X x b1."""
    X = np.asarray(X, dtype=np.float64)
    k = int(np.argmin(np.abs(X)))
    e = np.zeros(3)
    e[k] = 1.0
    b1 = np.cross(X, e)
    b1 /= np.linalg.norm(b1)
    return b1, np.cross(X, b1)


def quadric(x, Q, b, c):
    """f(x) = x^T Q x + b^T x + c and its gradient (Q + Q^T) x + b (x: [..., 3])."""
    x = np.asarray(x)
    f = np.einsum("...i,ij,...j->...", x, Q, x) + x @ b + c
    return f, x @ (Q + Q.T).T + b


@dataclass
class ConstraintGroup:
    """Constraints of Sec. 8.1 over the edges [e0, e1), rows in this order: the barycenter (3 rows,
    unless bary is False); either the total length (1 row) or, when l0 is given, one edge-length row
    per edge (Phi_I = l0_I - l_I); then, when pins is given, three rows per pinned vertex v,
    Phi_v = gamma_v - p0_v (the point constraint); then two rows per tangent-constrained edge I,
    b_a . T_I with (b_1, b_2) = perp_basis(X_I) (the tangent constraint T_I = X_I; the printed three
    rows T_I - X_I have a Jacobian of rank 2, since |T_I| = 1, so the two rows across X_I are kept);
    then one row f(gamma_v) per vertex held on the quadric surface f = 0 (the surface constraint).
    The total-length row is the sum of the edge-length rows, so the two are never combined."""
    e0: int
    e1: int
    x0: np.ndarray
    L0: float
    l0: Optional[np.ndarray] = None
    bary: bool = True
    pins: Optional[np.ndarray] = None   # global vertex indices
    p0: Optional[np.ndarray] = None     # [len(pins), 3] target positions
    tangents: Optional[np.ndarray] = None   # global edge indices
    X: Optional[np.ndarray] = None          # [len(tangents), 3] unit target tangents
    surf: Optional[np.ndarray] = None       # global vertex indices held on the surface
    quad: Optional[tuple] = None            # (Q [3, 3], b [3], c) of f(x) = x^T Q x + b^T x + c

    @property
    def n_bary(self) -> int:
        return 3 if self.bary else 0

    @property
    def n_length(self) -> int:
        return 1 if self.l0 is None else self.e1 - self.e0

    @property
    def n_pin_rows(self) -> int:
        return 0 if self.pins is None else 3 * len(self.pins)

    @property
    def n_tangent_rows(self) -> int:
        return 0 if self.tangents is None else 2 * len(self.tangents)

    @property
    def n_rows(self) -> int:
        return (self.n_bary + self.n_length + self.n_pin_rows + self.n_tangent_rows +
                (0 if self.surf is None else len(self.surf)))


def constraint_groups(gamma, edges, edge_offsets=None, edge_lengths=False, pins=None, barycenter=True,
                      tangents=None, X=None, surf=None, quad=None):
    """x0, L0 (and, with edge_lengths, every l0_I) fixed at their values on the given curve; one
    group per curve if edge_offsets is given, else one group for the whole graph.  pins, tangents,
    surf (optional): one array of global vertex (edge) indices per group, or a single array when
    there is one group.  Each pinned vertex is held at its position on the given curve; X (same
    nesting as tangents) gives the unit target tangent of each tangent edge (default: its tangent on
    the given curve); quad = (Q, b, c) is the surface of every group's surf vertices."""
    gamma = np.asarray(gamma, dtype=np.float64)
    ell, T, x = edge_quantities(gamma, edges)
    offs = [0, len(edges)] if edge_offsets is None else list(edge_offsets)

    def per_group(a):
        if a is None:
            return [None] * (len(offs) - 1)
        if len(offs) == 2 and (len(a) == 0 or np.ndim(a[0]) == 0):
            return [a]
        return list(a)

    pins, tangents, surf = per_group(pins), per_group(tangents), per_group(surf)
    if X is not None and len(offs) == 2 and np.ndim(X) == 2:
        X = [X]
    groups = []
    for c in range(len(offs) - 1):
        e0, e1 = offs[c], offs[c + 1]
        L = ell[e0:e1].sum()
        x0 = (ell[e0:e1, None] * x[e0:e1]).sum(0) / L
        pv = None if pins[c] is None else np.asarray(pins[c], dtype=np.int64)
        tv = None if tangents[c] is None else np.asarray(tangents[c], dtype=np.int64)
        Xc = None
        if tv is not None:
            Xc = T[tv].copy() if X is None else np.asarray(X[c], dtype=np.float64).reshape(-1, 3)
            Xc = Xc / np.linalg.norm(Xc, axis=1, keepdims=True)
        sv = None if surf[c] is None else np.asarray(surf[c], dtype=np.int64)
        groups.append(ConstraintGroup(e0, e1, x0, L, ell[e0:e1].copy() if edge_lengths else None,
                                      bary=barycenter, pins=pv,
                                      p0=None if pv is None else gamma[pv].copy(),
                                      tangents=tv, X=Xc, surf=sv,
                                      quad=None if sv is None else tuple(np.asarray(q, dtype=np.float64)
                                                                        for q in quad)))
    return groups


def phi(gamma, edges, groups):
    """Per group: Phi_barycenter = sum_I l_I (x_I - x0) (3 rows, if present), then Phi_length =
    L0 - sum_I l_I (1 row) or Phi_length,I = l0_I - l_I (one row per edge, in edge order), then
    gamma_v - p0_v for each pinned vertex (3 rows each, in pin order)."""
    gamma = np.asarray(gamma, dtype=np.float64)
    ell, T, x = edge_quantities(gamma, edges)
    out = []
    for gr in groups:
        s = slice(gr.e0, gr.e1)
        if gr.bary:
            out.extend(list((ell[s, None] * (x[s] - gr.x0)).sum(0)))
        if gr.l0 is None:
            out.append(gr.L0 - ell[s].sum())
        else:
            out.extend(list(gr.l0 - ell[s]))
        if gr.pins is not None:
            out.extend(list((gamma[gr.pins] - gr.p0).reshape(-1)))
        if gr.tangents is not None:
            for I, X in zip(gr.tangents, gr.X):
                b1, b2 = perp_basis(X)
                out.extend([b1 @ T[I], b2 @ T[I]])
        if gr.surf is not None:
            out.extend(list(quadric(gamma[gr.surf], *gr.quad)[0]))
    return np.array(out)


def jacobian(gamma, edges, groups):
    """C = d Phi, shape [total rows, nV, 3] (vertex-major columns), rows in the order of phi.
    d l_I / d g_i2 = T_I = -d l_I / d g_i1, d x_I / d g_ia = Id / 2, d g_v / d g_v = Id."""
    g, e = _geom(gamma, edges)
    ell, T, x = edge_quantities(g, e)
    C = np.zeros((sum(gr.n_rows for gr in groups), g.shape[0], 3))
    r0 = 0
    for gr in groups:
        for I in range(gr.e0, gr.e1):
            i1, i2 = e[I]
            if gr.bary:
                for k in range(3):
                    r = r0 + k
                    C[r, i2] += T[I] * (x[I, k] - gr.x0[k])
                    C[r, i1] -= T[I] * (x[I, k] - gr.x0[k])
                    C[r, i1, k] += 0.5 * ell[I]
                    C[r, i2, k] += 0.5 * ell[I]
            r = r0 + gr.n_bary + (0 if gr.l0 is None else I - gr.e0)
            C[r, i2] -= T[I]
            C[r, i1] += T[I]
        rp = r0 + gr.n_bary + gr.n_length
        if gr.pins is not None:
            for a, v in enumerate(gr.pins):
                for k in range(3):
                    C[rp + 3 * a + k, v, k] = 1.0
        rp += gr.n_pin_rows
        if gr.tangents is not None:
            # d (b . T_I) / d g_i2 = (I - T T^T) b / l_I = -d (b . T_I) / d g_i1
            for a, (I, X) in enumerate(zip(gr.tangents, gr.X)):
                i1, i2 = e[I]
                for k, bk in enumerate(perp_basis(X)):
                    row = (bk - (bk @ T[I]) * T[I]) / ell[I]
                    C[rp + 2 * a + k, i2] += row
                    C[rp + 2 * a + k, i1] -= row
        rp += gr.n_tangent_rows
        if gr.surf is not None:
            grads = quadric(g[gr.surf], *gr.quad)[1]
            for a, v in enumerate(gr.surf):
                C[rp + a, v] = grads[a]
        r0 += gr.n_rows
    return C


# ----------------------------------------------------------------------------- saddle-point problems

def to_cm(v):
    """Vertex-major [nV, 3] -> component-major R^{3|V|} (all x, then y, then z), as in Eq. 19."""
    return np.asarray(v).T.reshape(-1)


def from_cm(v, nV):
    return np.asarray(v).reshape(3, nV).T.copy()


def abar_cm(A):
    """A-bar = diag(A, A, A) in component-major order, Eq. 19."""
    n = A.shape[0]
    Ab = np.zeros((3 * n, 3 * n))
    for k in range(3):
        Ab[k * n:(k + 1) * n, k * n:(k + 1) * n] = A
    return Ab


def kkt_solve(A, C, rhs_top, rhs_bottom):
    """Dense solve of [A-bar C^T; C 0][x; lambda] = [rhs_top; rhs_bottom] (Eqs. 22-23).
    A is the scalar nV x nV Gram matrix; C is [k, nV, 3]; rhs_top is [nV, 3]."""
    nV = A.shape[0]
    k = C.shape[0]
    Ab = abar_cm(A)
    Ccm = np.stack([to_cm(C[r]) for r in range(k)])
    K = np.zeros((3 * nV + k, 3 * nV + k))
    K[:3 * nV, :3 * nV] = Ab
    K[:3 * nV, 3 * nV:] = Ccm.T
    K[3 * nV:, :3 * nV] = Ccm
    rhs = np.concatenate([to_cm(rhs_top), np.asarray(rhs_bottom, dtype=np.float64)])
    sol = np.linalg.solve(K, rhs)
    return from_cm(sol[:3 * nV], nV), sol[3 * nV:]


class Projector:
    """P v = v - C^T (C C^T)^{-1} C v (App. B.3.3, read as the Euclidean projector onto null(C))."""

    def __init__(self, C):
        self.C = C.reshape(C.shape[0], -1)
        self.G = self.C @ self.C.T

    def __call__(self, v):
        s = v.shape
        f = v.reshape(-1)
        return (f - self.C.T @ np.linalg.solve(self.G, self.C @ f)).reshape(s)

    def pinv(self, b):
        """C^+ b = C^T (C C^T)^{-1} b."""
        return (self.C.T @ np.linalg.solve(self.G, b))


@dataclass
class CGResult:
    x: np.ndarray
    iters: int
    rel_res: float
    converged: bool
    history: list = field(default_factory=list)


def projected_cg(apply_abar, P, a, tol=1e-6, maxit=10000, precond=None, x0=None):
    """CG on P A-bar P y = P a, returning x = P y (App. B.3.3).  apply_abar maps [nV,3] -> [nV,3];
    precond (optional, SPD) maps [nV,3] -> [nV,3] and is used as P M^{-1} P."""
    Pa = P(a)
    nb = np.linalg.norm(Pa)
    y = np.zeros_like(a) if x0 is None else P(x0)
    r = Pa - P(apply_abar(P(y))) if x0 is not None else Pa.copy()
    if nb == 0.0:
        return CGResult(P(y), 0, 0.0, True)
    z = P(precond(r)) if precond else r.copy()
    p = z.copy()
    rz = float(np.vdot(r, z))
    hist = []
    for it in range(1, maxit + 1):
        q = P(apply_abar(P(p)))
        pq = float(np.vdot(p, q))
        if not pq > 0.0:
            return CGResult(P(y), it, np.linalg.norm(r) / nb, False, hist)
        al = rz / pq
        y = y + al * p
        r = r - al * q
        rel = np.linalg.norm(r) / nb
        hist.append(rel)
        if rel <= tol:
            return CGResult(P(y), it, rel, True, hist)
        z = P(precond(r)) if precond else r
        rz2 = float(np.vdot(r, z))
        p = z + (rz2 / rz) * p
        rz = rz2
    return CGResult(P(y), maxit, np.linalg.norm(r) / nb, False, hist)


# ----------------------------------------------------------------------------- penalties (Sec. 8.1)
#
# Soft terms added to the tangent-point energy: the total length sum_I l_I; the length difference
# sum over vertices of degree 2 of (l_I - l_J)^2 (I, J the two edges at the vertex); and the field
# potential sum_I l_I |T_I x X(x_I)|^2 for a unit vector field X, here X(x) = u / |u| with
# u = M x + b (a constant field when M = 0; X = 0 where u = 0).


@dataclass
class Penalties:
    w_length: float = 0.0
    w_length_diff: float = 0.0
    w_field: float = 0.0
    field_M: np.ndarray = field(default_factory=lambda: np.zeros((3, 3)))
    field_b: np.ndarray = field(default_factory=lambda: np.array([0.0, 0.0, 1.0]))


def _field(pen, x):
    u = pen.field_M @ x + pen.field_b
    nu = np.linalg.norm(u)
    return (u / nu, nu) if nu > 0 else (np.zeros(3), 0.0)


def penalty_energy(gamma, edges, pen: Penalties):
    """w_length sum l_I + w_length_diff sum_v (l_I - l_J)^2 + w_field sum_I l_I |T_I x X(x_I)|^2."""
    g, e = _geom(gamma, edges)
    ell, T, x = edge_quantities(g, e)
    E = pen.w_length * ell.sum()
    inc = [[] for _ in range(g.shape[0])]
    for I, (a, b) in enumerate(e):
        inc[a].append(I)
        inc[b].append(I)
    for v in range(g.shape[0]):
        if len(inc[v]) == 2:
            E += pen.w_length_diff * (ell[inc[v][0]] - ell[inc[v][1]]) ** 2
    for I in range(len(e)):
        X, _ = _field(pen, x[I])
        E += pen.w_field * ell[I] * float(np.cross(T[I], X) @ np.cross(T[I], X))
    return float(E)


def penalty_gradient(gamma, edges, pen: Penalties):
    """Gradient of penalty_energy with respect to the vertices ([nV, 3]), by the chain rule:
    d l_I / d g_i2 = T_I = -d l_I / d g_i1, d x_I / d g_ia = Id / 2 and, for the field term with
    e = g_i2 - g_i1, l (1 - (T.X)^2) = l - (e.X)^2 / l:
      d/de = T - 2 (T.X) X + (T.X)^2 T,   d/dx = -2 (T.X) M^T (e - (e.X) X) / |u|."""
    g, e = _geom(gamma, edges)
    ell, T, x = edge_quantities(g, e)
    G = np.zeros_like(g)
    dl = np.full(len(e), pen.w_length)      # dE / d l_I of the length terms
    inc = [[] for _ in range(g.shape[0])]
    for I, (a, b) in enumerate(e):
        inc[a].append(I)
        inc[b].append(I)
    for v in range(g.shape[0]):
        if len(inc[v]) == 2:
            I, J = inc[v]
            w = 2.0 * pen.w_length_diff * (ell[I] - ell[J])
            dl[I] += w
            dl[J] -= w
    for I, (a, b) in enumerate(e):
        G[b] += dl[I] * T[I]
        G[a] -= dl[I] * T[I]
        if pen.w_field != 0.0:
            X, nu = _field(pen, x[I])
            tx = float(T[I] @ X)
            de = T[I] - 2.0 * tx * X + tx * tx * T[I]
            dx = np.zeros(3)
            if nu > 0:
                ev = ell[I] * T[I]
                dx = -2.0 * tx * (pen.field_M.T @ (ev - (ev @ X) * X)) / nu
            G[b] += pen.w_field * (de + 0.5 * dx)
            G[a] += pen.w_field * (-de + 0.5 * dx)
    return G


# ----------------------------------------------------------------------------- collision time (Sec. 5.4)
#
# The isotopy-safe start of the line search: tau_max is the first tau > 0 at which the moving curve
# gamma - tau d brings two disjoint edges into contact; the backtracking starts at 2/3 tau_max.
# Contact of two segments moving linearly in time needs their four endpoints coplanar, a cubic in tau
# (the determinant of three edge vectors that are each linear in tau), and, at that root, the
# segments must actually touch (distance zero, up to TOUCH_REL times the two lengths).  When every
# coefficient of the cubic vanishes the motion is coplanar, and the first contact is a vertex of one
# segment meeting the other segment: a quadratic in tau for each of the four vertex-segment choices.

TOUCH_REL = 1e-8


def segment_distance(p1, p2, q1, q2):
    """Smallest |P(s) - Q(u)| over s, u in [0, 1]: the stationary point of the quadratic if it lies
    in the square, else the best of the four edges of the square (each a clamped 1-D minimum)."""
    d1, d2, r = p2 - p1, q2 - q1, p1 - q1
    a, b, e = d1 @ d1, d1 @ d2, d2 @ d2
    c, f = d1 @ r, d2 @ r
    cand = []
    den = a * e - b * b
    if den > 1e-14 * a * e:
        s, u = (b * f - c * e) / den, (a * f - b * c) / den
        if 0.0 <= s <= 1.0 and 0.0 <= u <= 1.0:
            cand.append((s, u))
    for s in (0.0, 1.0):
        cand.append((s, min(1.0, max(0.0, (b * s + f) / e)) if e > 0 else 0.0))
    for u in (0.0, 1.0):
        cand.append((min(1.0, max(0.0, (b * u - c) / a)) if a > 0 else 0.0, u))
    return min(float(np.linalg.norm(p1 + s * d1 - q1 - u * d2)) for s, u in cand)


def _det3(u, v, w):
    return float(np.dot(u, np.cross(v, w)))


def _real_roots(coef, T):
    """Real roots in (0, T] of sum_k coef[k] t^k (numpy.roots on the trimmed polynomial)."""
    c = list(coef)
    while c and c[-1] == 0.0:
        c.pop()
    if len(c) <= 1:
        return []
    r = np.roots(c[::-1])
    out = []
    for z in r:
        if abs(z.imag) <= 1e-9 * max(1.0, abs(z.real)) and 0.0 < z.real <= T:
            out.append(float(z.real))
    return sorted(out)


def pair_collision_time(a, b, da, db, c, e, dc, de, T):
    """First tau in (0, T] at which segment [a - tau da, b - tau db] touches [c - tau dc, e - tau de],
    or inf."""
    a, b, da, db, c, e, dc, de = (np.asarray(x, dtype=np.float64) for x in (a, b, da, db, c, e, dc, de))
    tol = TOUCH_REL * (np.linalg.norm(b - a) + np.linalg.norm(e - c))
    at = lambda p, dp, t: p - t * dp
    # edge vectors relative to a, each linear in tau: X(t) = X0 + t X1
    U0, U1 = b - a, -(db - da)
    V0, V1 = c - a, -(dc - da)
    W0, W1 = e - a, -(de - da)
    coef = [_det3(U0, V0, W0),
            _det3(U1, V0, W0) + _det3(U0, V1, W0) + _det3(U0, V0, W1),
            _det3(U1, V1, W0) + _det3(U1, V0, W1) + _det3(U0, V1, W1),
            _det3(U1, V1, W1)]
    scale = max(np.linalg.norm(U0) + T * np.linalg.norm(U1), np.linalg.norm(V0) + T * np.linalg.norm(V1),
                np.linalg.norm(W0) + T * np.linalg.norm(W1)) ** 3
    if max(abs(coef[k]) * T ** k for k in range(4)) > 1e-13 * scale:
        for t in _real_roots(coef, T):
            if segment_distance(at(a, da, t), at(b, db, t), at(c, dc, t), at(e, de, t)) <= tol:
                return t
        return np.inf
    # coplanar motion: vertex-segment contacts
    best = np.inf
    for p, dp, q1, dq1, q2, dq2 in ((a, da, c, dc, e, de), (b, db, c, dc, e, de),
                                    (c, dc, a, da, b, db), (e, de, a, da, b, db)):
        # (q2 - q1) x (p - q1) = 0 along the plane normal: a quadratic in tau
        S0, S1 = q2 - q1, -(dq2 - dq1)
        R0, R1 = p - q1, -(dp - dq1)
        nrm = np.cross(U0 + 0.5 * T * U1, V0 + 0.5 * T * V1)
        if np.linalg.norm(nrm) == 0.0:
            nrm = np.cross(U0 + 0.5 * T * U1, W0 + 0.5 * T * W1)
        if np.linalg.norm(nrm) == 0.0:
            continue
        q = [np.cross(S0, R0) @ nrm, (np.cross(S1, R0) + np.cross(S0, R1)) @ nrm, np.cross(S1, R1) @ nrm]
        for t in _real_roots(q, T):
            if segment_distance(at(a, da, t), at(b, db, t), at(c, dc, t), at(e, de, t)) <= tol:
                best = min(best, t)
                break
    return best


def first_collision_time(gamma, edges, d, T, edge_offsets=None):
    """Sec. 5.4: the first tau in (0, T] at which two disjoint edges of gamma - tau d touch, per group of
    edges (one per curve if edge_offsets is given, else the whole graph); T where none touch."""
    g, e = _geom(gamma, edges)
    d = np.asarray(d, dtype=np.float64).reshape(g.shape)
    offs = [0, len(e)] if edge_offsets is None else list(edge_offsets)
    out = []
    for k in range(len(offs) - 1):
        best = np.inf
        for I in range(offs[k], offs[k + 1]):
            a, b = e[I]
            for J in range(I + 1, offs[k + 1]):
                c, f = e[J]
                if len({a, b, c, f}) < 4:
                    continue
                t = pair_collision_time(g[a], g[b], d[a], d[b], g[c], g[f], d[c], d[f], T)
                best = min(best, t)
        out.append(min(best, T))
    return np.array(out)


# ----------------------------------------------------------------------------- descent

@dataclass
class Params:
    alpha: float = 2.0
    beta: float = 4.5
    cg_tol: float = 1e-6
    cg_maxit: int = 20000
    proj_cg_tol: float = 1e-6
    proj_tol: float = 1e-10
    proj_maxit: int = 5
    armijo_c: float = 1e-4
    shrink: float = 0.5
    max_halvings: int = 30
    isotopy_safe: bool = False   # Sec. 5.4's first strategy: start at 2/3 of the first collision time
    ccd_horizon: float = 1.5     # collision times are searched in (0, ccd_horizon]
    penalties: object = None     # Penalties (Sec. 8.1) added to the energy and its differential

    @property
    def sigma(self):
        return sigma_of(self.alpha, self.beta)


def make_apply(gamma, edges, sigma):
    """Matrix-free A-bar u for vertex-major u [nV, 3] (A-bar acts on each component, Eq. 19)."""
    return lambda u: gram_apply(gamma, edges, sigma, u)


def sobolev_gradient(gamma, edges, groups, dE, prm: Params, dense=False, precond=None):
    """Projected H^s gradient g~ (Eq. 22).  dense=True: direct dense KKT solve; otherwise projected CG."""
    C = jacobian(gamma, edges, groups)
    if dense:
        B, B0 = gram_dense(gamma, edges, prm.sigma)
        g, lam = kkt_solve(B + B0, C, dE, np.zeros(C.shape[0]))
        return g, None
    P = Projector(C)
    res = projected_cg(make_apply(gamma, edges, prm.sigma), P, dE, prm.cg_tol, prm.cg_maxit, precond)
    return res.x, res


def constraint_projection(gamma_t, edges, groups, apply_abar, prm: Params, precond=None, A_dense=None):
    """Sec. 5.3.2: repeat x = argmin x^T A-bar x / 2 subject to C x = -Phi(g~); g~ += x; until
    max|Phi| <= tol.  With A_dense (the Gram matrix of the pre-step curve) x is the dense solve of the
    saddle-point system of Eq. 23; otherwise App. B.3.4's route: z = C^+ b with b = -Phi, the
    projected solve P A P y = P A z by CG, x = z - y.  Returns (curve, iterations, success)."""
    g = gamma_t.copy()
    scale = max(1.0, max(gr.L0 for gr in groups))
    for it in range(prm.proj_maxit + 1):
        ph = phi(g, edges, groups)
        if np.max(np.abs(ph)) <= prm.proj_tol * scale:
            return g, it, True
        if it == prm.proj_maxit:
            break
        C = jacobian(g, edges, groups)
        if A_dense is not None:
            x, _ = kkt_solve(A_dense, C, np.zeros_like(g), -ph)
            g = g + x
            continue
        P = Projector(C)
        z = P.pinv(-ph).reshape(g.shape)
        res = projected_cg(apply_abar, P, apply_abar(z), prm.proj_cg_tol, prm.cg_maxit, precond)
        g = g + (z - res.x)
    return g, prm.proj_maxit, False


@dataclass
class StepInfo:
    E_before: float
    E_after: float
    tau: float
    gnorm: float
    halvings: int
    proj_iters: int
    cg_iters: int
    accepted: bool


def descent_step(gamma, edges, groups, prm: Params, dense=False, precond_factory=None):
    """One H^s descent step with normalised-gradient backtracking (Sec. 5.4) from tau = 1, or with
    prm.isotopy_safe from 2/3 of the first collision time along gamma - tau d (searched up to
    ccd_horizon; ccd_horizon itself when no collision comes first)."""
    pen = prm.penalties
    total = lambda gg: energy(gg, edges, prm.alpha, prm.beta) + (penalty_energy(gg, edges, pen) if pen else 0.0)
    E0 = total(gamma)
    dE = differential(gamma, edges, prm.alpha, prm.beta)
    if pen:
        dE = dE + penalty_gradient(gamma, edges, pen)
    pc = precond_factory(gamma) if precond_factory else None
    g, res = sobolev_gradient(gamma, edges, groups, dE, prm, dense=dense, precond=pc)
    gn = float(np.linalg.norm(g))
    if gn == 0.0:
        return gamma.copy(), StepInfo(E0, E0, 0.0, 0.0, 0, 0, res.iters if res else 0, False)
    d = g / gn
    slope = float(np.vdot(dE, d))
    apply_abar = make_apply(gamma, edges, prm.sigma)  # A-bar of the pre-step curve
    A_dense = None
    if dense:
        B, B0 = gram_dense(gamma, edges, prm.sigma)
        A_dense = B + B0
    tau = 1.0
    if prm.isotopy_safe:
        tau = 2.0 / 3.0 * float(first_collision_time(gamma, edges, d, prm.ccd_horizon)[0])
    for h in range(prm.max_halvings + 1):
        cand = gamma - tau * d
        cand, pit, ok = constraint_projection(cand, edges, groups, apply_abar, prm, pc, A_dense)
        if ok:
            E1 = total(cand)
            if E1 <= E0 - prm.armijo_c * tau * slope:
                return cand, StepInfo(E0, E1, tau, gn, h, pit, res.iters if res else 0, True)
        tau *= prm.shrink
    return gamma.copy(), StepInfo(E0, E0, 0.0, gn, prm.max_halvings, 0, res.iters if res else 0, False)


# ----------------------------------------------------------------------------- spectral preconditioner

def circle_symbol(n, sigma):
    """Eigenvalues of the Gram matrix A = B + B0 of a regular n-gon, normalised by its diagonal.
    The regular n-gon's A is circulant, so its eigenvalues are the DFT of its first column.
    lambda_0 (the constant mode, 0) is replaced by lambda_1."""
    g = np.stack([np.cos(2 * np.pi * np.arange(n) / n), np.sin(2 * np.pi * np.arange(n) / n), np.zeros(n)], 1)
    e = np.stack([np.arange(n), (np.arange(n) + 1) % n], 1).astype(np.int32)
    if n <= 1024:
        B, B0 = gram_dense(g, e, sigma)
        col = (B + B0)[:, 0]
    else:
        u = np.zeros(n)
        u[0] = 1.0
        col = gram_apply(g, e, sigma, u)
    lam = np.real(np.fft.fft(col)) / col[0]
    lam[0] = lam[1]
    return lam


def spectral_preconditioner(diagA, vertex_offsets, symbols):
    """M^{-1} r = D^{-1/2} F^{-1} diag(1/lambda) F D^{-1/2} r on every closed curve (per component),
    with D = diag(A) of the actual curve and lambda the normalised regular-polygon symbol."""
    ds = np.sqrt(diagA)

    def apply(r):
        out = np.empty_like(r)
        for c in range(len(vertex_offsets) - 1):
            v0, v1 = vertex_offsets[c], vertex_offsets[c + 1]
            s = r[v0:v1] / ds[v0:v1, None]
            lam = symbols[v1 - v0]
            y = np.real(np.fft.ifft(np.fft.fft(s, axis=0) / lam[:, None], axis=0))
            out[v0:v1] = y / ds[v0:v1, None]
        return out

    return apply


def gram_diagonal(gamma, edges, sigma):
    """diag(A) by applying A to unit vectors would be O(n^3); instead read it off the dense build
    for small n, or from rows of the matrix-free apply for selected vertices."""
    n = gamma.shape[0]
    B, B0 = gram_dense(gamma, edges, sigma)
    return np.diag(B + B0).copy()


def gram_diagonal_at(gamma, edges, sigma, vidx):
    n = gamma.shape[0]
    out = np.empty(len(vidx))
    for k, v in enumerate(vidx):
        u = np.zeros(n)
        u[v] = 1.0
        out[k] = gram_apply_at(gamma, edges, sigma, u, [v])[0, 0]
    return out


def ngon_symbol_closed_form(n, sigma, normalized=True):
    """Eigenvalues of A = B + B0 of the regular n-gon (unit circumradius) from the quadratic forms
    (Eq. 21, Sec. 5.2.3) evaluated on the Fourier modes u_j = exp(i 2 pi k j / n), summed over the
    offset m = J - I in [2, n - 2] of the edge pair:
        lambda_k = sum_m 2 w_m |e^{i th k} - 1|^2 / l^2 (1 - cos(th k m) <T_0, T_m>)
                 + sum_m (w0_m / 4) |1 + e^{i th k}|^2 (1 - cos(th k m)),      th = 2 pi / n,
    w_m = w_{0m}, w0_m = w0_{0m} + w0_{m0} from the vertex chords 2 sin(pi j / n).  Equal to the DFT
    of the first column of the dense circulant Gram matrix (pinned by a test), but every term is
    >= 0, so it stays accurate where that DFT cancels.  normalized: divide by the diagonal (the mean
    eigenvalue) and set lambda_0 := lambda_1, as the spectral preconditioner uses it."""
    p = 2.0 * sigma + 1.0
    m = np.arange(2, n - 1)
    l = 2.0 * np.sin(np.pi / n)
    w = np.zeros(m.shape)
    w0 = np.zeros(m.shape)
    for a in (0, 1):
        for b in (0, 1):
            off = m + b - a
            ch = 2.0 * np.abs(np.sin(np.pi * off / n))
            s0 = np.sin(np.pi * (a + m + b - 1) / n)
            sm = np.sin(np.pi * (a + m + b - 2 * m - 1) / n)
            w += ch ** -p
            w0 += (s0 ** 2 + sm ** 2) * ch ** (-(2.0 + p))
    w *= 0.25 * l * l
    w0 *= 0.25 * l * l
    t = np.cos(2 * np.pi * m / n)
    lam = np.zeros(n)
    for k0 in range(0, n, 256):
        k = np.arange(k0, min(n, k0 + 256))[:, None]
        r = (k * m[None, :]) % n
        one_m_cos = 2.0 * np.sin(np.pi * r / n) ** 2
        ek = 4.0 * np.sin(np.pi * k / n) ** 2
        pk = 4.0 * np.cos(np.pi * k / n) ** 2
        term = 2 * w * ek / l ** 2 * ((1 - t) + t * one_m_cos) + (w0 / 4) * pk * one_m_cos
        lam[k0:k0 + k.shape[0]] = term.sum(1)
    if normalized:
        lam = lam / lam.mean()
        lam[0] = lam[1]
    return lam


def rq_frequencies(n):
    """Sampled frequencies of the Rayleigh-quotient symbol correction: 1..8 and 14 values spaced
    evenly in log between 9 and n/2 (rounded), unique, at most n/2."""
    ks = list(range(1, 9))
    lo, hi = math.log(9.0), math.log(max(9.0, n / 2.0))
    ks += [int(round(math.exp(lo + (hi - lo) * j / 13.0))) for j in range(14)]
    return sorted(k for k in set(ks) if 1 <= k <= n // 2)


def spectral_rq_symbol(A, n, sigma):
    """Rayleigh-quotient corrected symbol of one closed curve with Gram matrix A (n x n): the
    eigenvalues of T. Chan's optimal circulant approximation of S = D^-1/2 A D^-1/2,
    lambda_opt(k) = (c_k^T S c_k + s_k^T S s_k) / n with c_k, s_k the cosine and sine modes, are taken
    at the sampled frequencies; rho = lambda_opt / lambda_ngon is interpolated linearly in
    (log k, log rho) and the symbol is lambda_ngon * rho (lambda_0 := the corrected lambda_1)."""
    d = np.diag(A)
    ds = np.sqrt(d)
    lam = ngon_symbol_closed_form(n, sigma)
    i = np.arange(n)
    ks = rq_frequencies(n)
    lk, lr = [], []
    for k in ks:
        c = np.cos(2 * np.pi * ((k * i) % n) / n) / ds
        s = np.sin(2 * np.pi * ((k * i) % n) / n) / ds
        q = (c @ A @ c + s @ A @ s) / n
        lk.append(math.log(k))
        lr.append(math.log(q / lam[k]))
    out = np.empty(n)
    for k in range(n):
        kf = k if k <= n // 2 else n - k
        if kf <= 1:
            r = lr[0]
        else:
            r = float(np.interp(math.log(kf), lk, lr))
        out[k] = lam[1 if k == 0 else k] * math.exp(r)
    return out


def coarse_hats(n, m):
    """The first m - 1 of m periodic hat functions on a closed curve of n vertices: hat j is
    max(0, 1 - |i m / n - j|) (distance taken modulo m).  Columns of an n x (m - 1) matrix."""
    t = np.arange(n) * m / n
    Z = np.zeros((n, m - 1))
    for j in range(m - 1):
        d = np.abs(t - j)
        d = np.minimum(d, m - d)
        Z[:, j] = np.maximum(0.0, 1.0 - d)
    return Z


def twolevel_apply(A, n, sigma, m, r):
    """Two-level preconditioner of one closed curve: the Rayleigh-quotient corrected spectral term
    plus the additive coarse term Z (Z^T A Z)^-1 Z^T r with m periodic hats (m <= n / 4).
    r: [n, 3]; returns [n, 3] (before the mean-free projection)."""
    ds = np.sqrt(np.diag(A))
    lam = spectral_rq_symbol(A, n, sigma)
    z = np.real(np.fft.ifft(np.fft.fft(r / ds[:, None], axis=0) / lam[:, None], axis=0)) / ds[:, None]
    Z = coarse_hats(n, m)
    Ac = Z.T @ A @ Z
    return z + Z @ np.linalg.solve(Ac, Z.T @ r)


def balanced_apply(A, Z, spectral, r):
    """Balancing two-level preconditioner (not from the paper; this library's design): with the
    Galerkin coarse operator E = Z^T A Z and Q = Z E^-1 Z^T,
        z = Q r + (I - Q A) S (I - A Q) r,
    S the one-level term (a callable on [n, 3]).  It is symmetric when S is, reproduces A^-1 exactly
    on range(A Z), and equals A^-1 when S does (on the complement of the null space).
    A: [n, n]; Z: [n, k]; r: [n, 3]."""
    E = Z.T @ A @ Z
    Q = lambda v: Z @ np.linalg.solve(E, Z.T @ v)
    y = spectral(r - A @ Q(r))
    return Q(r) + y - Q(A @ y)


def twolevel_balanced_apply(A, n, sigma, m, r):
    """The balancing form of the two-level preconditioner of one closed curve: the Rayleigh-quotient
    corrected spectral term of twolevel_apply as S, the m - 1 first of m periodic hats as Z.
    r: [n, 3]; returns [n, 3] (before the mean-free projection)."""
    ds = np.sqrt(np.diag(A))
    lam = spectral_rq_symbol(A, n, sigma)
    spec = lambda v: np.real(np.fft.ifft(np.fft.fft(v / ds[:, None], axis=0) / lam[:, None], axis=0)) / ds[:, None]
    return balanced_apply(A, coarse_hats(n, m), spec, r)
