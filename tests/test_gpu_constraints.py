"""Edge-length constraints (Sec. 8.1, TP_CONSTRAINTS_EDGE_LENGTHS) on the GPU against the oracle: the
projected gradient against the dense KKT solve of Eq. 22 with the barycenter + edge-length rows, the
descent step (projection of App. B.3.4 with those rows) against the oracle's, and the projector's
defining properties on a chain long enough for the global-memory reduction."""
import numpy as np
import pytest

import synth as S
from tests.gpu_util import dev, host, make_ctx, need_gpu, rel

pytestmark = pytest.mark.gpu
EDGE = 1  # TP_CONSTRAINTS_EDGE_LENGTHS


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle as O
    O.build_library()
    return O


def edge_rows(gamma, edges, v):
    """R v: T_I . (v_i2 - v_i1) per edge (the edge-length rows of the Jacobian up to sign)."""
    e = gamma[edges[:, 1]] - gamma[edges[:, 0]]
    T = e / np.linalg.norm(e, axis=1, keepdims=True)
    return np.einsum("ij,ij->i", T, v[edges[:, 1]] - v[edges[:, 0]])


def _case(name):
    if name == "closed":
        return S.single(S.trefoil(64, 0.01, 3)), 0, 4
    if name == "open":
        return S.single(S.fourier_knot(50, 4, 5), closed=False), 0, 1
    if name == "batch":
        return S.batch_of_knots([40, 57, 64], 4, 71), 1, 1
    if name == "scene":  # two curves, one problem: two chains share one barycenter row
        return S.scene([S.fourier_knot(36, 3, 8), S.fourier_knot(45, 3, 9)]), 0, 1
    raise KeyError(name)


@pytest.mark.parametrize("name", ["closed", "open", "batch", "scene"])
def test_edge_gradient_matches_dense_kkt(torch, orc, name):
    from paper_2006_07859_gb300 import tpe
    c, indep, precond = _case(name)
    ctx = make_ctx(c, precision=0, precond=precond, independent=indep, constraint_set=EDGE, cg_rtol=1e-11,
                   cg_maxit=20000)
    g = dev(c.gamma)
    dE = tpe.tp_differential(ctx, g)
    gt, info = tpe.sobolev_gradient(ctx, g, dE)
    assert info["converged"]
    gt = host(gt)
    dEh = host(dE)
    # rows of every edge and the barycenter vanish on the gradient
    assert np.abs(edge_rows(c.gamma, c.edges, gt)).max() <= 1e-10 * np.abs(gt).max()
    if indep:
        groups = orc.constraint_groups(c.gamma, c.edges, c.edge_offsets, edge_lengths=True)
        parts = []
        for k in range(c.n_curves):
            gk, ek = c.curve(k)
            grk = orc.constraint_groups(gk, ek, edge_lengths=True)
            dk = orc.differential(gk, ek)
            parts.append(orc.sobolev_gradient(gk, ek, grk, dk, orc.Params(), dense=True)[0])
            v0, v1 = c.vertex_offsets[k], c.vertex_offsets[k + 1]
            assert rel(dEh[v0:v1], dk) <= 1e-10   # independent curves: no cross-curve pairs
        gk_all = np.concatenate(parts)
        assert len(groups) == c.n_curves
    else:
        gr = orc.constraint_groups(c.gamma, c.edges, edge_lengths=True)
        gk_all = orc.sobolev_gradient(c.gamma, c.edges, gr, orc.differential(c.gamma, c.edges), orc.Params(),
                                      dense=True)[0]
        C = orc.jacobian(c.gamma, c.edges, gr).reshape(gr[0].n_rows, -1)
        assert np.abs(C @ gt.reshape(-1)).max() <= 1e-10 * np.abs(gt).max()
        assert rel(dEh, orc.differential(c.gamma, c.edges)) <= 1e-10
    assert rel(gt, gk_all) <= 1e-7


def test_edge_descent_steps_match_oracle(torch, orc):
    from paper_2006_07859_gb300 import tpe
    c = S.single(S.trefoil(48, 0.01, 2))
    ctx = make_ctx(c, precision=0, precond=1, constraint_set=EDGE, cg_rtol=1e-11, proj_cg_rtol=1e-11,
                   cg_maxit=20000)
    g = dev(c.gamma)
    gr = orc.constraint_groups(c.gamma, c.edges, edge_lengths=True)
    prm = orc.Params(cg_tol=1e-11, proj_cg_tol=1e-11)
    go = c.gamma.copy()
    ell0 = orc.edge_quantities(c.gamma, c.edges)[0]
    for step in range(3):
        info = tpe.descent_step(ctx, g)
        go, io = orc.descent_step(go, c.edges, gr, prm)
        assert info["accepted"] == 1 and io.accepted
        assert info["tau"] == io.tau
        assert abs(info["E_after"] - io.E_after) <= 1e-9 * io.E_after
        assert rel(host(g), go) <= 1e-7
        ell = orc.edge_quantities(host(g), c.edges)[0]
        assert np.abs(ell - ell0).max() <= 1e-10 * max(1.0, ell0.sum())
    phi = host(tpe.tp_constraints(ctx, g))
    assert np.abs(phi).max() <= 1e-10 * max(1.0, ell0.sum())


@pytest.mark.parametrize("closed", [True, False])
def test_edge_projector_on_a_long_chain(torch, orc, closed):
    """12,289 edges: above the shared-memory size, so the reduction runs through global memory; a
    ragged length (not a power of two).  P y lies in null(R) whatever the CG iterate is, so a few
    iterations suffice to check the projector: R g = 0, the barycenter row vanishes, and g is
    mean-free up to the barycenter translation."""
    from paper_2006_07859_gb300 import tpe
    n = 12289
    c = S.single(S.fourier_knot(n, 8, 12), closed=closed)
    ctx = make_ctx(c, precision=2, precond=1, constraint_set=EDGE, cg_maxit=16, cg_rtol=1e-12)
    g = dev(c.gamma)
    dE = tpe.tp_differential(ctx, g)
    gt, info = tpe.sobolev_gradient(ctx, g, dE, allow_not_converged=True)
    gt = host(gt)
    assert np.isfinite(gt).all() and np.abs(gt).max() > 0
    assert np.abs(edge_rows(c.gamma, c.edges, gt)).max() <= 1e-8 * np.abs(gt).max()
    gr = orc.constraint_groups(c.gamma, c.edges, edge_lengths=False)
    ell, T, x = orc.edge_quantities(c.gamma, c.edges)
    # barycenter row: sum_I l_I (d x_I) + (d l_I)(x_I - x0) = 0 along g
    dx = 0.5 * (gt[c.edges[:, 0]] + gt[c.edges[:, 1]])
    dl = edge_rows(c.gamma, c.edges, gt)
    row = (ell[:, None] * dx + dl[:, None] * (x - gr[0].x0)).sum(0)
    assert np.abs(row).max() <= 1e-9 * np.abs(gt).max() * ell.sum()


def test_edge_constraints_reject_a_branching_graph(torch):
    from paper_2006_07859_gb300 import tpe
    # a "Y": vertex 0 starts two edges
    gam = np.array([[0.0, 0, 0], [1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]])
    edges = np.array([[0, 1], [0, 2], [0, 3]], dtype=np.int32)
    with pytest.raises(tpe.TpError):
        tpe.Context(edges, [0, 4], [0, 3], 4, precision=0, precond=1, constraint_set=EDGE)
    ctx = tpe.Context(edges, [0, 4], [0, 3], 4, precision=0, precond=1)
    with pytest.raises(tpe.TpError):
        ctx.set_params(constraint_set=EDGE)
