"""Point, tangent and surface constraints (Sec. 8.1, TP_CONSTRAINTS_POINTS: pinned vertices, edges with
a fixed tangent, vertices on a quadric, with the total length and no barycenter row) on the GPU against
the oracle: the projected gradient against the dense KKT solve of Eq. 22 (one pin, more constrained
vertices than one three-column solve holds, open curves pinned at both ends, an independent batch with
ragged counts, two curves in one problem), descent steps against the oracle's, a mixed-precision run on a
4,096-vertex knot with the two-level preconditioner, and the argument checks."""
import numpy as np
import pytest

import synth as S
from tests.gpu_util import dev, host, make_ctx, need_gpu, rel

pytestmark = pytest.mark.gpu
POINTS = 2  # TP_CONSTRAINTS_POINTS


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle as O
    O.build_library()
    return O


def _case(name):
    """(curves, independent, preconditioner, pins per problem in global vertex indices)."""
    if name == "closed_one":
        return S.single(S.trefoil(64, 0.01, 3)), 0, 1, [[7]]
    if name == "closed_seven":  # three solves, the last with one column
        return S.single(S.trefoil(64, 0.01, 3)), 0, 2, [[0, 5, 9, 20, 33, 34, 50]]
    if name == "open_ends":
        return S.single(S.fourier_knot(50, 4, 5), closed=False), 0, 1, [[0, 49]]
    if name == "batch":
        b = S.batch_of_knots([40, 57, 64], 4, 71)
        vo = b.vertex_offsets
        return b, 1, 1, [[vo[0] + 11], [vo[1] + 0, vo[1] + 3, vo[1] + 30, vo[1] + 56], [vo[2] + 8, vo[2] + 40]]
    if name == "scene":  # two curves, one problem, one pin on each
        return S.scene([S.fourier_knot(36, 3, 8), S.fourier_knot(45, 3, 9)]), 0, 1, [[3, 40]]
    raise KeyError(name)


def _set_pins(tpe, ctx, c, pins):
    allp = np.concatenate([np.asarray(p) for p in pins])
    tpe.tp_set_pins(ctx, allp, c.gamma[allp])
    return allp


@pytest.mark.parametrize("name", ["closed_one", "closed_seven", "open_ends", "batch", "scene"])
def test_pinned_gradient_matches_dense_kkt(torch, orc, name):
    from paper_2006_07859_gb300 import tpe
    c, indep, precond, pins = _case(name)
    ctx = make_ctx(c, precision=0, precond=precond, independent=indep, constraint_set=POINTS, cg_rtol=1e-11,
                   cg_maxit=20000)
    allp = _set_pins(tpe, ctx, c, pins)
    g = dev(c.gamma)
    dE = tpe.tp_differential(ctx, g)
    gt, info = tpe.sobolev_gradient(ctx, g, dE)
    assert info["converged"]
    gt = host(gt)
    assert np.abs(gt[allp]).max() <= 1e-12 * np.abs(gt).max()
    if indep:
        parts = []
        for k in range(c.n_curves):
            gk, ek = c.curve(k)
            v0 = c.vertex_offsets[k]
            grk = orc.constraint_groups(gk, ek, pins=np.asarray(pins[k]) - v0, barycenter=False)
            parts.append(orc.sobolev_gradient(gk, ek, grk, orc.differential(gk, ek), orc.Params(), dense=True)[0])
        ref = np.concatenate(parts)
    else:
        gr = orc.constraint_groups(c.gamma, c.edges, pins=np.asarray(pins[0]), barycenter=False)
        ref = orc.sobolev_gradient(c.gamma, c.edges, gr, orc.differential(c.gamma, c.edges), orc.Params(),
                                   dense=True)[0]
    assert rel(gt, ref) <= 1e-7


@pytest.mark.parametrize("closed", [True, False])
def test_pinned_descent_steps_match_oracle(torch, orc, closed):
    from paper_2006_07859_gb300 import tpe
    if closed:
        c, pins = S.single(S.trefoil(48, 0.01, 2)), np.array([0, 17, 30])
    else:
        c, pins = S.single(S.fourier_knot(40, 3, 8), closed=False), np.array([0, 39])
    ctx = make_ctx(c, precision=0, precond=1, constraint_set=POINTS, cg_rtol=1e-11, proj_cg_rtol=1e-11,
                   cg_maxit=20000)
    tpe.tp_set_pins(ctx, pins, c.gamma[pins])
    g = dev(c.gamma)
    gr = orc.constraint_groups(c.gamma, c.edges, pins=pins, barycenter=False)
    prm = orc.Params(cg_tol=1e-11, proj_cg_tol=1e-11)
    go = c.gamma.copy()
    for _ in range(2):
        info = tpe.descent_step(ctx, g)
        go, io = orc.descent_step(go, c.edges, gr, prm)
        assert info["accepted"] == 1 and io.accepted
        assert info["tau"] == io.tau
        assert abs(info["E_after"] - io.E_after) <= 1e-9 * io.E_after
        assert rel(host(g), go) <= 1e-7
        assert np.abs(host(g)[pins] - c.gamma[pins]).max() <= 1e-10
    phi = host(tpe.tp_constraints(ctx, g))
    assert np.abs(phi).max() <= 1e-10 * max(1.0, gr[0].L0)


def test_pins_on_a_large_knot_in_mixed_precision(torch):
    """4,096 vertices, five pins (two solves), mixed precision, two-level preconditioner: every step is
    accepted, the energy falls, the pins stay at their targets and the length at L0."""
    from paper_2006_07859_gb300 import tpe
    c = S.single(S.fourier_knot(4096, 8, 21))
    pins = np.array([0, 700, 1500, 2900, 4095])
    ctx = make_ctx(c, precision=2, precond=4, constraint_set=POINTS)
    tpe.tp_set_pins(ctx, pins, c.gamma[pins])
    g = dev(c.gamma)
    ell = np.linalg.norm(c.gamma[c.edges[:, 1]] - c.gamma[c.edges[:, 0]], axis=1)
    L0 = ell.sum()
    E = None
    for _ in range(3):
        info = tpe.descent_step(ctx, g)
        assert info["accepted"] == 1 and info["n_converged"] >= 1
        assert E is None or info["E_after"] < E
        E = info["E_after"]
        gh = host(g)
        assert np.abs(gh[pins] - c.gamma[pins]).max() <= 1e-9 * L0
        L = np.linalg.norm(gh[c.edges[:, 1]] - gh[c.edges[:, 0]], axis=1).sum()
        assert abs(L - L0) <= 1e-9 * L0


def test_pin_arguments_are_checked(torch):
    from paper_2006_07859_gb300 import tpe
    b = S.batch_of_knots([40, 50], 4, 90)
    ctx = make_ctx(b, precision=0, precond=1, independent=1, constraint_set=POINTS)
    g = dev(b.gamma)
    with pytest.raises(tpe.TpError):   # the points set without pins
        tpe.descent_step(ctx, g)
    for verts in ([0], [0, 0, 45], [0, 40, 90], [-1, 45], list(range(25)) + [45]):
        with pytest.raises(tpe.TpError):  # a problem without pins, a repeat, out of range, 25 in a problem
            tpe.tp_set_pins(ctx, verts, np.zeros((len(verts), 3)))
    with pytest.raises(tpe.TpError):
        tpe.tp_set_pins(ctx, [0, 45], np.array([[0.0, np.nan, 0.0], [0.0, 0.0, 0.0]]))
    tpe.tp_set_pins(ctx, [3, 45], b.gamma[[3, 45]])
    tpe.sobolev_gradient(ctx, g, tpe.tp_differential(ctx, g))
    # the barycenter slots of tp_constraints report the largest pin, tangent and surface residuals
    moved = b.gamma.copy()
    moved[45] += np.array([0.0, 2e-3, -5e-4])
    phi = host(tpe.tp_constraints(ctx, dev(moved))).reshape(2, 4)
    np.testing.assert_allclose(phi[0, :3], 0.0, atol=0.0)
    np.testing.assert_allclose(phi[1, :3], [2e-3, 0.0, 0.0], rtol=1e-12, atol=1e-15)
    tpe.tp_set_pins(ctx, [], np.zeros((0, 3)))
    with pytest.raises(tpe.TpError):
        tpe.sobolev_gradient(ctx, g, tpe.tp_differential(ctx, g))


def _sphere(center, radius):
    center = np.asarray(center, dtype=np.float64)
    return np.eye(3), -2.0 * center, float(center @ center - radius * radius)


def _rows_case(name):
    """(curves, independent, precond, pins, tangent edges, surface vertices) per problem, global indices."""
    if name == "closed":
        return S.single(S.trefoil(64, 0.01, 3)), 0, 2, [[2]], [[6, 30]], [[10, 40]]
    if name == "open":
        return S.single(S.fourier_knot(50, 4, 5), closed=False), 0, 1, [[0, 49]], [[0, 48]], [[25]]
    if name == "batch":
        b = S.batch_of_knots([40, 57, 64], 4, 71)
        vo, eo = b.vertex_offsets, b.edge_offsets
        return (b, 1, 1, [[vo[0] + 3], [vo[1] + 0, vo[1] + 30], [vo[2] + 8]],
                [[eo[0] + 20], [eo[1] + 10, eo[1] + 40], [eo[2] + 1]], [[vo[0] + 30], [], [vo[2] + 50, vo[2] + 20]])
    raise KeyError(name)


@pytest.mark.parametrize("name", ["closed", "open", "batch"])
def test_tangent_and_surface_gradient_matches_dense_kkt(torch, orc, name):
    from paper_2006_07859_gb300 import tpe
    c, indep, precond, pins, tans, surf = _rows_case(name)
    ctx = make_ctx(c, precision=0, precond=precond, independent=indep, constraint_set=POINTS, cg_rtol=1e-11,
                   cg_maxit=20000)
    allp = np.concatenate([np.asarray(p, dtype=np.int64) for p in pins])
    allt = np.concatenate([np.asarray(t, dtype=np.int64) for t in tans])
    alls = np.concatenate([np.asarray(v, dtype=np.int64) for v in surf])
    T = orc.edge_quantities(c.gamma, c.edges)[1]
    quad = _sphere(c.gamma[alls].mean(0) + np.array([0.1, -0.2, 0.05]), 0.9)
    tpe.tp_set_tangents(ctx, allt, T[allt])
    tpe.tp_set_surface(ctx, alls, *quad)
    tpe.tp_set_pins(ctx, allp, c.gamma[allp])
    g = dev(c.gamma)
    dE = tpe.tp_differential(ctx, g)
    gt, info = tpe.sobolev_gradient(ctx, g, dE)
    assert info["converged"]
    gt = host(gt)
    assert np.abs(gt[allp]).max() <= 1e-12 * np.abs(gt).max()
    if indep:
        parts = []
        for k in range(c.n_curves):
            gk, ek = c.curve(k)
            v0, e0 = c.vertex_offsets[k], c.edge_offsets[k]
            grk = orc.constraint_groups(gk, ek, pins=np.asarray(pins[k]) - v0, barycenter=False,
                                        tangents=np.asarray(tans[k], dtype=np.int64) - e0,
                                        surf=np.asarray(surf[k], dtype=np.int64) - v0, quad=quad)
            parts.append(orc.sobolev_gradient(gk, ek, grk, orc.differential(gk, ek), orc.Params(), dense=True)[0])
        ref = np.concatenate(parts)
    else:
        gr = orc.constraint_groups(c.gamma, c.edges, pins=allp, barycenter=False, tangents=allt, surf=alls, quad=quad)
        ref = orc.sobolev_gradient(c.gamma, c.edges, gr, orc.differential(c.gamma, c.edges), orc.Params(),
                                   dense=True)[0]
    assert rel(gt, ref) <= 1e-7


def test_tangent_and_surface_descent_steps_match_oracle(torch, orc):
    """An open curve pinned at both ends with its end edges' tangents held and its middle vertex on a
    sphere through it: every trial is projected back onto all of them."""
    from paper_2006_07859_gb300 import tpe
    c = S.single(S.fourier_knot(40, 3, 8), closed=False)
    pins, tans, surf = np.array([0, 39]), np.array([0, 38]), np.array([20])
    X = orc.edge_quantities(c.gamma, c.edges)[1][tans]
    quad = _sphere(np.zeros(3), float(np.linalg.norm(c.gamma[20])))
    ctx = make_ctx(c, precision=0, precond=1, constraint_set=POINTS, cg_rtol=1e-11, proj_cg_rtol=1e-11,
                   cg_maxit=20000)
    tpe.tp_set_pins(ctx, pins, c.gamma[pins])
    tpe.tp_set_tangents(ctx, tans, X)
    tpe.tp_set_surface(ctx, surf, *quad)
    g = dev(c.gamma)
    gr = orc.constraint_groups(c.gamma, c.edges, pins=pins, barycenter=False, tangents=tans, X=X, surf=surf,
                               quad=quad)
    prm = orc.Params(cg_tol=1e-11, proj_cg_tol=1e-11)
    go = c.gamma.copy()
    for _ in range(2):
        info = tpe.descent_step(ctx, g)
        go, io = orc.descent_step(go, c.edges, gr, prm)
        assert info["accepted"] == 1 and io.accepted
        assert info["tau"] == io.tau
        assert abs(info["E_after"] - io.E_after) <= 1e-9 * io.E_after
        assert rel(host(g), go) <= 1e-7
    gh = host(g)
    Tn = orc.edge_quantities(gh, c.edges)[1]
    tol = 1e-10 * max(1.0, gr[0].L0)   # the projection's stopping rule, max|Phi| <= proj_tol max(1, L0)
    assert np.abs(Tn[tans] - X).max() <= tol
    assert abs(orc.quadric(gh[surf], *quad)[0]).max() <= tol
    phi = host(tpe.tp_constraints(ctx, g))
    assert np.abs(phi).max() <= 1e-10 * max(1.0, gr[0].L0)


def test_tangent_and_surface_arguments_are_checked(torch):
    from paper_2006_07859_gb300 import tpe
    c = S.single(S.fourier_knot(60, 3, 9), closed=False)
    ctx = make_ctx(c, precision=0, precond=1, constraint_set=POINTS, cg_rtol=1e-11, cg_maxit=20000)
    tpe.tp_set_pins(ctx, [0, 59], c.gamma[[0, 59]])
    bad = [lambda: tpe.tp_set_tangents(ctx, [60], [[1.0, 0, 0]]),            # edge out of range (59 edges)
           lambda: tpe.tp_set_tangents(ctx, [3, 3], [[1.0, 0, 0]] * 2),      # repeated edge
           lambda: tpe.tp_set_tangents(ctx, [3], [[0.0, 0, 0]]),             # zero target
           lambda: tpe.tp_set_surface(ctx, [0], np.eye(3)),                  # a pinned vertex on the surface
           lambda: tpe.tp_set_surface(ctx, list(range(1, 24)), np.eye(3)),   # 25 constrained vertices
           lambda: tpe.tp_set_surface(ctx, [5], np.eye(3), [np.inf, 0, 0])]  # non-finite quadric
    for call in bad:
        with pytest.raises(tpe.TpError):
            call()
    two = make_ctx(S.single(S.fourier_knot(12, 2, 3), closed=False), precision=0, precond=1, constraint_set=POINTS)
    tpe.tp_set_pins(two, [0, 1], np.zeros((2, 3)))
    with pytest.raises(tpe.TpError):   # both ends of edge 0 pinned
        tpe.tp_set_tangents(two, [0], [[1.0, 0, 0]])
    # a rejected call leaves the lists as they were: the gradient matches the one before it
    g = dev(c.gamma)
    dE = tpe.tp_differential(ctx, g)
    tpe.tp_set_tangents(ctx, [10], [c.gamma[11] - c.gamma[10]])
    g1 = host(tpe.sobolev_gradient(ctx, g, dE)[0])
    with pytest.raises(tpe.TpError):   # 25 constrained vertices: rejected after the lists were laid out
        tpe.tp_set_surface(ctx, list(range(1, 24)), np.eye(3))
    g2 = host(tpe.sobolev_gradient(ctx, g, dE)[0])
    assert rel(g2, g1) <= 1e-8


def test_contexts_with_different_row_counts_interleave(torch, orc):
    """24 pins (72 rows: the small system takes more than 48 KB of shared memory) in one context, one pin
    in another set up after it: the first context's gradient still matches the dense KKT solve."""
    from paper_2006_07859_gb300 import tpe
    c = S.single(S.trefoil(64, 0.01, 3))
    big = make_ctx(c, precision=0, precond=2, constraint_set=POINTS, cg_rtol=1e-11, cg_maxit=20000)
    pins = np.arange(0, 64, 64 // 24)[:24]
    tpe.tp_set_pins(big, pins, c.gamma[pins])
    small = make_ctx(c, precision=0, precond=2, constraint_set=POINTS, cg_rtol=1e-11, cg_maxit=20000)
    tpe.tp_set_pins(small, [5], c.gamma[[5]])
    g = dev(c.gamma)
    tpe.sobolev_gradient(small, g, tpe.tp_differential(small, g))
    gt = host(tpe.sobolev_gradient(big, g, tpe.tp_differential(big, g))[0])
    gr = orc.constraint_groups(c.gamma, c.edges, pins=pins, barycenter=False)
    ref = orc.sobolev_gradient(c.gamma, c.edges, gr, orc.differential(c.gamma, c.edges), orc.Params(), dense=True)[0]
    assert rel(gt, ref) <= 1e-7
