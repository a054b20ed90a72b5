"""Thin ctypes binding of include/tpe.h.  Argument marshalling only: every computation runs in
libtpe.so.  Tensors must be CUDA float64 (vertex arrays [nV, 3], contiguous); the calls are enqueued
on torch's current CUDA stream.  There is no CPU fallback: a missing library raises."""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtpe.so")

TP_OK, TP_ERR_INVALID_ARG, TP_ERR_CUDA, TP_ERR_DEGENERATE_EDGE, TP_ERR_NONFINITE = 0, 1, 2, 3, 4
TP_ERR_NOT_CONVERGED, TP_ERR_BREAKDOWN, TP_ERR_LINESEARCH, TP_ERR_PROJECTION, TP_ERR_OOM = 5, 6, 7, 8, 9
TP_ERR_UNSUPPORTED = 10
TP_FP64, TP_FP32, TP_MIXED = 0, 1, 2
TP_PRECOND_NONE, TP_PRECOND_JACOBI, TP_PRECOND_SPECTRAL, TP_PRECOND_SPECTRAL_RQ, TP_PRECOND_TWOLEVEL = 0, 1, 2, 3, 4
TP_PRECOND_LEARNED = 5
TP_PRECOND_TWOLEVEL_BALANCED = 6
TP_PRECOND_LEARNED_BALANCED = 7
TP_GNN_HIDDEN, TP_GNN_FEATURES = 64, 8
TP_CONSTRAINTS_TOTAL_LENGTH, TP_CONSTRAINTS_EDGE_LENGTHS, TP_CONSTRAINTS_POINTS = 0, 1, 2
TP_LINESEARCH_UNIT, TP_LINESEARCH_ISOTOPY = 0, 1

STATUS_NAMES = {0: "TP_OK", 1: "TP_ERR_INVALID_ARG", 2: "TP_ERR_CUDA", 3: "TP_ERR_DEGENERATE_EDGE",
                4: "TP_ERR_NONFINITE", 5: "TP_ERR_NOT_CONVERGED", 6: "TP_ERR_BREAKDOWN", 7: "TP_ERR_LINESEARCH",
                8: "TP_ERR_PROJECTION", 9: "TP_ERR_OOM", 10: "TP_ERR_UNSUPPORTED"}

EXPORTED = ["tp_default_params", "tp_create", "tp_destroy", "tp_last_error", "tp_num_problems", "tp_set_params",
            "tp_energy", "tp_differential", "sobolev_apply", "sobolev_apply_accurate", "sobolev_apply_multi", "tp_gram_diagonal", "tp_precond_apply",
            "tp_spectral_symbol", "tp_set_constraints_from", "tp_constraints", "sobolev_gradient", "descent_step",
            "tp_launch_count", "tp_pairs_per_pass", "tp_profile", "tp_profile_read", "tp_measure_peaks", "tp_energy_static",
            "tp_spectral_symbols", "tp_gnn_num_params", "tp_gnn_set_params", "tp_gnn_get_params", "tp_gnn_bind",
            "tp_gnn_forward", "tp_gnn_backward", "tp_gnn_adam", "tp_gnn_g_apply", "tp_gnn_out_grad", "tp_cg_harvest",
            "tp_gnn_prepare_pairs", "tp_gnn_train_step", "tp_autotune", "tp_set_apply_variant",
            "tp_set_energy_variant", "tp_last_solve", "tp_set_diff_variant", "tp_collision_time",
            "tp_set_penalties", "tp_penalty", "tp_set_pins", "tp_bh_energy", "tp_bh_differential", "tp_bh_stats",
            "tp_set_tangents", "tp_set_surface"]


class TpParams(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("sigma", ctypes.c_double),
                ("precision", ctypes.c_int), ("near_cutoff", ctypes.c_double), ("cg_rtol", ctypes.c_double),
                ("cg_maxit", ctypes.c_int), ("cg_check_every", ctypes.c_int), ("proj_cg_rtol", ctypes.c_double),
                ("precond", ctypes.c_int), ("armijo_c", ctypes.c_double), ("shrink", ctypes.c_double),
                ("max_halvings", ctypes.c_int), ("proj_tol", ctypes.c_double), ("proj_maxit", ctypes.c_int),
                ("independent", ctypes.c_int), ("coarse_dim", ctypes.c_int), ("far_cutoff", ctypes.c_double),
                ("use_graphs", ctypes.c_int), ("precond_refresh", ctypes.c_int), ("constraint_set", ctypes.c_int),
                ("line_search", ctypes.c_int), ("ccd_horizon", ctypes.c_double), ("warm_start", ctypes.c_int)]


class TpPenalties(ctypes.Structure):
    _fields_ = [("w_length", ctypes.c_double), ("w_length_diff", ctypes.c_double), ("w_field", ctypes.c_double),
                ("field_M", ctypes.c_double * 9), ("field_b", ctypes.c_double * 3)]


class TpSolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("rel_res", ctypes.c_double), ("converged", ctypes.c_int),
                ("n_converged", ctypes.c_int)]


class TpStepInfo(ctypes.Structure):
    _fields_ = [("E_before", ctypes.c_double), ("E_after", ctypes.c_double), ("tau", ctypes.c_double),
                ("gnorm", ctypes.c_double), ("halvings", ctypes.c_int), ("proj_iters", ctypes.c_int),
                ("cg_iters", ctypes.c_int), ("proj_cg_iters", ctypes.c_int), ("accepted", ctypes.c_int),
                ("rel_res", ctypes.c_double), ("n_converged", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def library() -> ctypes.CDLL:
    """Load libtpe.so (built by paper_2006_07859_gb300.build); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run `python -m paper_2006_07859_gb300.build` first "
                               "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.tp_default_params.argtypes = [ctypes.POINTER(TpParams)]
        L.tp_create.argtypes = [ctypes.POINTER(vp), i, i, vp, i, vp, vp, ctypes.POINTER(TpParams)]
        L.tp_destroy.argtypes = [vp]
        L.tp_last_error.argtypes = [vp]
        L.tp_last_error.restype = ctypes.c_char_p
        L.tp_num_problems.argtypes = [vp]
        L.tp_set_params.argtypes = [vp, ctypes.POINTER(TpParams)]
        L.tp_energy.argtypes = [vp, vp, vp, vp, vp]
        L.tp_differential.argtypes = [vp, vp, vp, vp, vp]
        L.sobolev_apply.argtypes = [vp, vp, vp, vp, vp]
        L.sobolev_apply_accurate.argtypes = [vp, vp, vp, vp, vp]
        L.sobolev_apply_multi.argtypes = [vp, vp, vp, vp, i, vp]
        L.tp_bh_energy.argtypes = [vp, vp, d, i, vp, vp, vp]
        L.tp_bh_differential.argtypes = [vp, vp, d, i, vp, vp]
        L.tp_bh_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                  ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)]
        L.tp_gram_diagonal.argtypes = [vp, vp, vp, vp]
        L.tp_precond_apply.argtypes = [vp, vp, vp, vp, vp]
        L.tp_spectral_symbol.argtypes = [vp, i, vp, vp]
        L.tp_set_constraints_from.argtypes = [vp, vp, vp]
        L.tp_constraints.argtypes = [vp, vp, vp, vp]
        L.sobolev_gradient.argtypes = [vp, vp, vp, vp, ctypes.POINTER(TpSolveInfo), vp]
        L.tp_collision_time.argtypes = [vp, vp, vp, ctypes.c_double, vp, vp]
        L.tp_set_penalties.argtypes = [vp, ctypes.POINTER(TpPenalties)]
        L.tp_penalty.argtypes = [vp, vp, vp, vp, vp]
        L.tp_set_pins.argtypes = [vp, i, vp, vp]
        L.tp_set_tangents.argtypes = [vp, i, vp, vp]
        L.tp_set_surface.argtypes = [vp, vp, i, vp]
        L.descent_step.argtypes = [vp, vp, ctypes.POINTER(TpStepInfo), vp]
        L.tp_launch_count.argtypes = [vp]
        L.tp_launch_count.restype = ctypes.c_int64
        L.tp_pairs_per_pass.argtypes = [vp]
        L.tp_pairs_per_pass.restype = ctypes.c_int64
        L.tp_profile.argtypes = [vp, i]
        L.tp_profile_read.argtypes = [vp, i, ctypes.POINTER(d), ctypes.POINTER(ctypes.c_int64)]
        pdd = ctypes.POINTER(d)
        L.tp_measure_peaks.argtypes = [pdd, pdd, pdd]
        L.tp_energy_static.argtypes = [vp, vp, i, i, d, d, vp, vp]
        L.tp_spectral_symbols.argtypes = [vp, i, vp, vp]
        L.tp_gnn_num_params.argtypes = []
        L.tp_gnn_set_params.argtypes = [vp, vp, i, vp]
        L.tp_gnn_get_params.argtypes = [vp, vp, vp]
        L.tp_gnn_bind.argtypes = [vp, vp, vp]
        L.tp_gnn_forward.argtypes = [vp, vp, vp, vp]
        L.tp_gnn_backward.argtypes = [vp, vp, vp, vp]
        L.tp_gnn_adam.argtypes = [vp, vp, ctypes.c_float, vp]
        L.tp_gnn_g_apply.argtypes = [vp, vp, vp, i, vp]
        L.tp_gnn_out_grad.argtypes = [vp, vp, vp, vp, i, vp]
        L.tp_cg_harvest.argtypes = [vp, vp, vp, i, i, vp, vp, ctypes.POINTER(i), ctypes.POINTER(TpSolveInfo), vp]
        L.tp_gnn_prepare_pairs.argtypes = [vp, vp, i, vp, vp, vp, vp, vp, vp, vp, vp]
        L.tp_gnn_train_step.argtypes = [vp, vp, i, vp, vp, vp, vp, vp, vp, ctypes.c_float, pdd, vp, vp]
        L.tp_autotune.argtypes = [vp, vp, vp, vp, vp]
        L.tp_set_apply_variant.argtypes = [vp, i]
        L.tp_set_energy_variant.argtypes = [vp, i]
        L.tp_last_solve.argtypes = [vp, vp, vp]
        L.tp_set_diff_variant.argtypes = [vp, i]
        _lib = L
    return _lib


def default_params(**kw) -> TpParams:
    p = TpParams()
    library().tp_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _ptr(t):
    if t is None:
        return None
    import torch
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA float64 tensor")
    return ctypes.c_void_p(t.data_ptr())


def _fptr(t):
    if t is None:
        return None
    import torch
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA float32 tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Context:
    """Owns a tp_ctx for one fixed graph (edges and curve offsets given on the host)."""

    def __init__(self, edges, vertex_offsets, edge_offsets, n_vertices, params: TpParams | None = None, **kw):
        L = library()
        self._edges = np.ascontiguousarray(edges, dtype=np.int32)
        self._voff = np.ascontiguousarray(vertex_offsets, dtype=np.int32)
        self._eoff = np.ascontiguousarray(edge_offsets, dtype=np.int32)
        self.params = params if params is not None else default_params(**kw)
        self.n_vertices = int(n_vertices)
        self.n_edges = int(self._edges.shape[0])
        h = ctypes.c_void_p()
        st = L.tp_create(ctypes.byref(h), self.n_vertices, self.n_edges, self._edges.ctypes.data, len(self._voff) - 1,
                         self._voff.ctypes.data, self._eoff.ctypes.data, ctypes.byref(self.params))
        self.handle = h
        if st != TP_OK:
            msg = L.tp_last_error(h).decode() if h.value else ""
            if h.value:
                L.tp_destroy(h)
                self.handle = ctypes.c_void_p()
            raise TpError(st, msg)
        self.n_problems = L.tp_num_problems(h)

    @classmethod
    def from_curves(cls, curves, **kw):
        return cls(curves.edges, curves.vertex_offsets, curves.edge_offsets, curves.n_vertices, **kw)

    def close(self):
        if self.handle and self.handle.value:
            library().tp_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, allow=()):
        if st != TP_OK and st not in allow:
            raise TpError(st, library().tp_last_error(self.handle).decode())
        return st

    def launch_count(self) -> int:
        return int(library().tp_launch_count(self.handle))

    def pairs_per_pass(self) -> int:
        return int(library().tp_pairs_per_pass(self.handle))

    def profile(self, enable=True):
        self._check(library().tp_profile(self.handle, 1 if enable else 0))

    def profile_read(self, op: int):
        ms, n = ctypes.c_double(), ctypes.c_int64()
        self._check(library().tp_profile_read(self.handle, op, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def set_params(self, **kw):
        for k, v in kw.items():
            setattr(self.params, k, v)
        self._check(library().tp_set_params(self.handle, ctypes.byref(self.params)))


# ---------------------------------------------------------------- entry points (same names as the C ABI)

def _new(shape, like=None):
    import torch
    return torch.empty(shape, dtype=torch.float64, device="cuda")


def tp_energy(ctx: Context, gamma, E=None, rows=None):
    E = _new(ctx.n_problems) if E is None else E
    ctx._check(library().tp_energy(ctx.handle, _ptr(gamma), _ptr(E), _ptr(rows), _stream()))
    return E


def tp_differential(ctx: Context, gamma, dE=None, E=None):
    dE = _new((ctx.n_vertices, 3)) if dE is None else dE
    ctx._check(library().tp_differential(ctx.handle, _ptr(gamma), _ptr(dE), _ptr(E), _stream()))
    return dE


def sobolev_apply(ctx: Context, gamma, u, Au=None):
    Au = _new((ctx.n_vertices, 3)) if Au is None else Au
    ctx._check(library().sobolev_apply(ctx.handle, _ptr(gamma), _ptr(u), _ptr(Au), _stream()))
    return Au


def sobolev_apply_multi(ctx: Context, gamma, U, AU=None):
    """AU[f] = A-bar U[f] for the m vector fields of U, a CUDA float64 tensor [m, nV, 3]."""
    m = int(U.shape[0])
    AU = _new((m, ctx.n_vertices, 3)) if AU is None else AU
    ctx._check(library().sobolev_apply_multi(ctx.handle, _ptr(gamma), _ptr(U), _ptr(AU), m, _stream()))
    return AU


def tp_bh_energy(ctx: Context, gamma, eps, leaf_size=8, E=None, rows=None):
    """Barnes-Hut energy per problem (and optionally per edge); returns E."""
    E = _new(ctx.n_problems) if E is None else E
    ctx._check(library().tp_bh_energy(ctx.handle, _ptr(gamma), float(eps), int(leaf_size), _ptr(E), _ptr(rows),
                                      _stream()))
    return E


def tp_bh_differential(ctx: Context, gamma, eps, leaf_size=8, dE=None):
    dE = _new((ctx.n_vertices, 3)) if dE is None else dE
    ctx._check(library().tp_bh_differential(ctx.handle, _ptr(gamma), float(eps), int(leaf_size), _ptr(dE), _stream()))
    return dE


def tp_bh_stats(ctx: Context, with_build_time=False):
    """(admissible nodes, leaf pairs, tree depth) of the last Barnes-Hut pass, and with
    with_build_time the host seconds of its hierarchy."""
    a, p, dp, bs = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_double()
    ctx._check(library().tp_bh_stats(ctx.handle, ctypes.byref(a), ctypes.byref(p), ctypes.byref(dp), ctypes.byref(bs)))
    return (a.value, p.value, dp.value, bs.value) if with_build_time else (a.value, p.value, dp.value)


def sobolev_apply_accurate(ctx: Context, gamma, u, Au=None):
    Au = _new((ctx.n_vertices, 3)) if Au is None else Au
    ctx._check(library().sobolev_apply_accurate(ctx.handle, _ptr(gamma), _ptr(u), _ptr(Au), _stream()))
    return Au


def tp_gram_diagonal(ctx: Context, gamma, diag=None):
    diag = _new(ctx.n_vertices) if diag is None else diag
    ctx._check(library().tp_gram_diagonal(ctx.handle, _ptr(gamma), _ptr(diag), _stream()))
    return diag


def tp_precond_apply(ctx: Context, gamma, r, z=None):
    z = _new((ctx.n_vertices, 3)) if z is None else z
    ctx._check(library().tp_precond_apply(ctx.handle, _ptr(gamma), _ptr(r), _ptr(z), _stream()))
    return z


def tp_spectral_symbol(ctx: Context, n: int, lam=None):
    lam = _new(n) if lam is None else lam
    ctx._check(library().tp_spectral_symbol(ctx.handle, int(n), _ptr(lam), _stream()))
    return lam


def tp_set_constraints_from(ctx: Context, gamma):
    ctx._check(library().tp_set_constraints_from(ctx.handle, _ptr(gamma), _stream()))


def tp_constraints(ctx: Context, gamma, phi=None):
    phi = _new(4 * ctx.n_problems) if phi is None else phi
    ctx._check(library().tp_constraints(ctx.handle, _ptr(gamma), _ptr(phi), _stream()))
    return phi


def tp_collision_time(ctx: Context, gamma, d, horizon: float, t=None):
    """Per problem, the first tau in (0, horizon] at which two disjoint edges of gamma - tau d touch
    (horizon where none do); a device tensor [n_problems]."""
    t = _new(ctx.n_problems) if t is None else t
    ctx._check(library().tp_collision_time(ctx.handle, _ptr(gamma), _ptr(d), ctypes.c_double(horizon), _ptr(t),
                                           _stream()))
    return t


def tp_set_penalties(ctx: Context, w_length=0.0, w_length_diff=0.0, w_field=0.0, field_M=None, field_b=None,
                     clear=False):
    """Penalties of Sec. 8.1 that descent_step adds to the energy (clear=True removes them); the field is
    X(x) = (M x + b) / |M x + b| (M 3 x 3, b 3-vector; default a constant field along z)."""
    if clear:
        ctx._check(library().tp_set_penalties(ctx.handle, None))
        return
    p = TpPenalties()
    p.w_length, p.w_length_diff, p.w_field = w_length, w_length_diff, w_field
    M = np.zeros(9) if field_M is None else np.asarray(field_M, dtype=np.float64).reshape(9)
    b = np.array([0.0, 0.0, 1.0]) if field_b is None else np.asarray(field_b, dtype=np.float64).reshape(3)
    for k in range(9):
        p.field_M[k] = float(M[k])
    for k in range(3):
        p.field_b[k] = float(b[k])
    ctx._check(library().tp_set_penalties(ctx.handle, ctypes.byref(p)))


def tp_set_pins(ctx: Context, vertices, targets):
    """Pinned vertices of TP_CONSTRAINTS_POINTS (Sec. 8.1): vertex indices and their target positions
    [n, 3] (host arrays, copied); an empty list removes the pins."""
    v = np.ascontiguousarray(np.asarray(vertices, dtype=np.int32).reshape(-1))
    t = np.ascontiguousarray(np.asarray(targets, dtype=np.float64).reshape(-1, 3))
    if t.shape[0] != v.shape[0]:
        raise ValueError("one target per pinned vertex")
    ctx._check(library().tp_set_pins(ctx.handle, int(v.shape[0]), v.ctypes.data if v.size else None,
                                      t.ctypes.data if t.size else None))


def tp_set_tangents(ctx: Context, edges, X):
    """Tangent constraints T_I = X_I of TP_CONSTRAINTS_POINTS (Sec. 8.1): edge indices and target
    directions [n, 3] (normalised by the library); an empty list removes them."""
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
    x = np.ascontiguousarray(np.asarray(X, dtype=np.float64).reshape(-1, 3))
    if x.shape[0] != e.shape[0]:
        raise ValueError("one target per tangent edge")
    ctx._check(library().tp_set_tangents(ctx.handle, int(e.shape[0]), e.ctypes.data if e.size else None,
                                          x.ctypes.data if x.size else None))


def tp_set_surface(ctx: Context, vertices, Q=None, b=None, c=0.0):
    """Surface constraints f(gamma_v) = 0 of TP_CONSTRAINTS_POINTS (Sec. 8.1) for the quadric
    f(x) = x^T Q x + b^T x + c; an empty vertex list removes them."""
    v = np.ascontiguousarray(np.asarray(vertices, dtype=np.int32).reshape(-1))
    q = np.zeros(13)
    q[:9] = np.zeros(9) if Q is None else np.asarray(Q, dtype=np.float64).reshape(9)
    q[9:12] = np.zeros(3) if b is None else np.asarray(b, dtype=np.float64).reshape(3)
    q[12] = float(c)
    ctx._check(library().tp_set_surface(ctx.handle, q.ctypes.data, int(v.shape[0]), v.ctypes.data if v.size else None))


def tp_penalty(ctx: Context, gamma):
    """(E [n_problems], dE [nV, 3]) of the penalties alone at gamma (device tensors)."""
    E = _new(ctx.n_problems)
    dE = _new((ctx.n_vertices, 3))
    ctx._check(library().tp_penalty(ctx.handle, _ptr(gamma), _ptr(E), _ptr(dE), _stream()))
    return E, dE


def sobolev_gradient(ctx: Context, gamma, dE, g=None, allow_not_converged=False):
    g = _new((ctx.n_vertices, 3)) if g is None else g
    info = TpSolveInfo()
    allow = (TP_ERR_NOT_CONVERGED,) if allow_not_converged else ()
    st = ctx._check(library().sobolev_gradient(ctx.handle, _ptr(gamma), _ptr(dE), _ptr(g), ctypes.byref(info),
                                               _stream()), allow)
    return g, {"iters": info.iters, "rel_res": info.rel_res, "converged": info.converged,
               "n_converged": info.n_converged, "status": st}


def descent_step(ctx: Context, gamma, allow=()):
    info = TpStepInfo()
    st = ctx._check(library().descent_step(ctx.handle, _ptr(gamma), ctypes.byref(info), _stream()), allow)
    d = info.as_dict()
    d["status"] = st
    return d


def tp_measure_peaks():
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    st = library().tp_measure_peaks(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    if st != 0:
        raise TpError(TP_ERR_CUDA, "tp_measure_peaks failed")
    return {"fp32_flops": a.value, "mufu_ops": b.value, "fp64_flops": c.value}


def tp_energy_static(gamma, edges, alpha=2.0, beta=4.5, E=None):
    """Energy without device allocation inside the library (edges: CUDA int32 [nE, 2])."""
    import torch
    if not (edges.is_cuda and edges.dtype == torch.int32 and edges.is_contiguous()):
        raise ValueError("edges must be a contiguous CUDA int32 tensor")
    E = _new(1) if E is None else E
    st = library().tp_energy_static(_ptr(gamma), ctypes.c_void_p(edges.data_ptr()), int(gamma.shape[0]),
                                    int(edges.shape[0]), float(alpha), float(beta), _ptr(E), _stream())
    if st != TP_OK:
        raise TpError(st, "tp_energy_static failed")
    return E


def tp_spectral_symbols(ctx: Context, rq: int, out=None):
    out = _new(ctx.n_vertices) if out is None else out
    ctx._check(library().tp_spectral_symbols(ctx.handle, int(rq), _ptr(out), _stream()))
    return out


# ---------------------------------------------------------------- learned preconditioner

def tp_gnn_num_params() -> int:
    return int(library().tp_gnn_num_params())


def tp_gnn_set_params(ctx: Context, theta, reset_optimizer=True):
    ctx._check(library().tp_gnn_set_params(ctx.handle, _fptr(theta), 1 if reset_optimizer else 0, _stream()))


def tp_gnn_get_params(ctx: Context, theta=None):
    import torch
    theta = torch.empty(tp_gnn_num_params(), dtype=torch.float32, device="cuda") if theta is None else theta
    ctx._check(library().tp_gnn_get_params(ctx.handle, _fptr(theta), _stream()))
    return theta


def tp_gnn_bind(ctx: Context, gamma):
    ctx._check(library().tp_gnn_bind(ctx.handle, _ptr(gamma), _stream()))


def tp_gnn_forward(ctx: Context, features=None, out=None):
    """Returns (features [nE, 8], outputs [nE, 3]: a, b, c) as float32 CUDA tensors."""
    import torch
    features = torch.empty((ctx.n_edges, TP_GNN_FEATURES), dtype=torch.float32, device="cuda") \
        if features is None else features
    out = torch.empty((ctx.n_edges, 3), dtype=torch.float32, device="cuda") if out is None else out
    ctx._check(library().tp_gnn_forward(ctx.handle, _fptr(features), _fptr(out), _stream()))
    return features, out


def tp_gnn_backward(ctx: Context, dout, grad=None):
    import torch
    grad = torch.empty(tp_gnn_num_params(), dtype=torch.float32, device="cuda") if grad is None else grad
    ctx._check(library().tp_gnn_backward(ctx.handle, _fptr(dout), _fptr(grad), _stream()))
    return grad


def tp_gnn_adam(ctx: Context, grad, lr: float):
    ctx._check(library().tp_gnn_adam(ctx.handle, _fptr(grad), ctypes.c_float(lr), _stream()))


def tp_gnn_g_apply(ctx: Context, r, z=None, accumulate=False):
    z = _new((ctx.n_vertices, 3)) if z is None else z
    ctx._check(library().tp_gnn_g_apply(ctx.handle, _ptr(r), _ptr(z), 1 if accumulate else 0, _stream()))
    return z


def tp_gnn_out_grad(ctx: Context, r, gz, dout=None, accumulate=False):
    import torch
    dout = torch.empty((ctx.n_edges, 3), dtype=torch.float32, device="cuda") if dout is None else dout
    ctx._check(library().tp_gnn_out_grad(ctx.handle, _ptr(r), _ptr(gz), _fptr(dout), 1 if accumulate else 0,
                                         _stream()))
    return dout


def tp_cg_harvest(ctx: Context, gamma, rhs, every: int, R, E):
    """R, E: CUDA float64 [max_pairs, nV, 3].  Returns (n_pairs, solve info dict)."""
    n = ctypes.c_int()
    info = TpSolveInfo()
    ctx._check(library().tp_cg_harvest(ctx.handle, _ptr(gamma), _ptr(rhs), int(every), int(R.shape[0]), _ptr(R),
                                       _ptr(E), ctypes.byref(n), ctypes.byref(info), _stream()))
    return n.value, {"iters": info.iters, "rel_res": info.rel_res, "converged": info.converged}


def tp_gnn_prepare_pairs(ctx: Context, gamma, R, E, B, AB, ER, ILAM=None, R2=None):
    """ER: CUDA float64 [n, n_problems]; B may be E (in place); ILAM (CUDA float64 [nV] or None)
    receives the curve's inverse circulant symbols and leaves the circulant to training; R2 (like R)
    receives (I - A Q) r in a balancing-form context (required there)."""
    ctx._check(library().tp_gnn_prepare_pairs(ctx.handle, _ptr(gamma), int(R.shape[0]), _ptr(R), _ptr(E), _ptr(B),
                                              _ptr(AB), _ptr(ER), _ptr(ILAM), _ptr(R2), _stream()))


def tp_gnn_train_step(ctx: Context, gamma, R, B, AB, ER, lr: float, grad=None, ILAM=None, R2=None) -> float:
    loss = ctypes.c_double()
    ctx._check(library().tp_gnn_train_step(ctx.handle, _ptr(gamma), int(R.shape[0]), _ptr(R), _ptr(B), _ptr(AB),
                                           _ptr(ER), _ptr(ILAM), _ptr(R2), ctypes.c_float(lr), ctypes.byref(loss),
                                           _fptr(grad), _stream()))
    return loss.value


def tp_autotune(ctx: Context, gamma) -> dict:
    """Pick the fastest targets-per-thread of each pair pass on `gamma` (mixed precision, alpha = 2,
    beta = 4.5); returns the choices and the measured ms per pass."""
    t = (ctypes.c_int32 * 6)()
    ms = (ctypes.c_double * 17)()
    ctx._check(library().tp_autotune(ctx.handle, _ptr(gamma), t, ms, _stream()))
    names = ["energy", "diff", "apply"]
    out = {"tpt": {n: int(t[k]) for k, n in enumerate(names)},
           "ms": {n: {str(v): ms[3 * k + j] for j, v in enumerate((1, 2, 4)) if ms[3 * k + j] > 0}
                  for k, n in enumerate(names)}}
    out["tpt"]["apply_symmetric"] = int(t[3])
    out["tpt"]["energy_symmetric"] = int(t[4])
    out["ms"]["apply_symmetric"] = {str(v): ms[9 + j] for j, v in enumerate((1, 2)) if ms[9 + j] > 0}
    out["ms"]["energy_symmetric"] = {str(v): ms[11 + j] for j, v in enumerate((1, 2)) if ms[11 + j] > 0}
    out["tpt"]["diff_symmetric"] = int(t[5])
    out["ms"]["diff_symmetric"] = {str(v): ms[i] for v, i in ((1, 13), (2, 14), (3, 15), (4, 16)) if ms[i] > 0}
    return out


def tp_set_apply_variant(ctx: Context, symmetric_tpt: int):
    """0: gather apply (every ordered pair); 1 or 2: symmetric apply with that many targets per thread."""
    ctx._check(library().tp_set_apply_variant(ctx.handle, int(symmetric_tpt)))


def tp_set_energy_variant(ctx: Context, symmetric_tpt: int):
    """0: gather energy pass (every ordered pair); 1 or 2: symmetric pass with that many targets per thread."""
    ctx._check(library().tp_set_energy_variant(ctx.handle, int(symmetric_tpt)))


def tp_last_solve(ctx: Context):
    """(true relative residual, iterations) per problem of the context's last CG solve, as numpy arrays."""
    rr = np.zeros(ctx.n_problems)
    it = np.zeros(ctx.n_problems, dtype=np.int32)
    ctx._check(library().tp_last_solve(ctx.handle, rr.ctypes.data, it.ctypes.data))
    return rr, it


def tp_set_diff_variant(ctx: Context, symmetric_tpt: int):
    """0: gather differential (every ordered pair); 1 or 2: symmetric pass with that many targets per thread."""
    ctx._check(library().tp_set_diff_variant(ctx.handle, int(symmetric_tpt)))
