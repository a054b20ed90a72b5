"""Penalties of Sec. 8.1 on the GPU against the oracle: energies and gradients of the total length,
length difference and field potential (closed and open curves, independent batches), and a descent
step on the energy plus penalties."""
import numpy as np
import pytest

import synth as S
from tests.gpu_util import dev, host, make_ctx, need_gpu, rel

pytestmark = pytest.mark.gpu
M = np.array([[0.0, -1.0, 0.2], [1.0, 0.0, 0.0], [0.3, 0.0, 0.1]])
B = np.array([0.1, 0.2, 0.5])
W = dict(w_length=0.4, w_length_diff=1.7, w_field=2.2)


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle as O
    O.build_library()
    return O


def opens(orc):
    return orc.Penalties(field_M=M, field_b=B, **W)


@pytest.mark.parametrize("closed", [True, False])
def test_penalty_energy_and_gradient(torch, orc, closed):
    from paper_2006_07859_gb300 import tpe
    c = S.single(S.fourier_knot(200, 6, 21), closed=closed)
    ctx = make_ctx(c, precision=0, precond=1)
    tpe.tp_set_penalties(ctx, field_M=M, field_b=B, **W)
    E, dE = tpe.tp_penalty(ctx, dev(c.gamma))
    pen = opens(orc)
    assert host(E)[0] == pytest.approx(orc.penalty_energy(c.gamma, c.edges, pen), rel=1e-12)
    assert rel(host(dE), orc.penalty_gradient(c.gamma, c.edges, pen)) <= 1e-12
    tpe.tp_set_penalties(ctx, clear=True)
    E0, dE0 = tpe.tp_penalty(ctx, dev(c.gamma))
    assert np.all(host(E0) == 0.0) and np.all(host(dE0) == 0.0)


def test_penalties_per_problem_in_a_batch(torch, orc):
    from paper_2006_07859_gb300 import tpe
    b = S.batch_of_knots([60, 130, 77], 4, 333)
    ctx = make_ctx(b, precision=0, precond=1, independent=1)
    tpe.tp_set_penalties(ctx, field_M=M, field_b=B, **W)
    E, dE = tpe.tp_penalty(ctx, dev(b.gamma))
    E, dE = host(E), host(dE)
    pen = opens(orc)
    for k in range(3):
        gk, ek = b.curve(k)
        v0, v1 = b.vertex_offsets[k], b.vertex_offsets[k + 1]
        assert E[k] == pytest.approx(orc.penalty_energy(gk, ek, pen), rel=1e-12)
        assert rel(dE[v0:v1], orc.penalty_gradient(gk, ek, pen)) <= 1e-12


def test_descent_steps_with_penalties_match_oracle(torch, orc):
    from paper_2006_07859_gb300 import tpe
    c = S.single(S.trefoil(64, 0.01, 4))
    ctx = make_ctx(c, precision=0, precond=1, cg_rtol=1e-10, proj_cg_rtol=1e-10)
    w = dict(w_length=0.05, w_length_diff=0.5, w_field=0.3)
    tpe.tp_set_penalties(ctx, field_b=np.array([0.0, 0.0, 1.0]), **w)
    g = dev(c.gamma)
    gr = orc.constraint_groups(c.gamma, c.edges)
    prm = orc.Params(cg_tol=1e-10, proj_cg_tol=1e-10,
                     penalties=orc.Penalties(field_b=np.array([0.0, 0.0, 1.0]), **w))
    go = c.gamma.copy()
    for _ in range(2):
        info = tpe.descent_step(ctx, g)
        go, io = orc.descent_step(go, c.edges, gr, prm)
        assert info["accepted"] == 1 and io.accepted
        assert info["tau"] == io.tau
        assert abs(info["E_before"] - io.E_before) <= 1e-10 * io.E_before
        assert abs(info["E_after"] - io.E_after) <= 1e-9 * io.E_after
        assert rel(host(g), go) <= 1e-7


@pytest.mark.parametrize("cset", [0, 1, 2])
def test_gradient_with_a_swirling_field_matches_dense_kkt(torch, orc, cset):
    """A non-constant field makes the differential translation-dependent (N^T dE != 0), so the
    barycenter multiplier of Eq. 22 is no longer zero (sets 0 and 1), and with pins, tangents and a
    surface (set 2) the translation rows of the Schur system carry N^T dE; the GPU route must still give
    the KKT solution."""
    from paper_2006_07859_gb300 import tpe
    c = S.single(S.trefoil(60, 0.01, 6))
    ctx = make_ctx(c, precision=0, precond=1, cg_rtol=1e-11, cg_maxit=20000, constraint_set=cset)
    tpe.tp_set_penalties(ctx, field_M=M, field_b=B, **W)
    rows = {}
    if cset == 2:
        pins, tans, surf = np.array([4, 33]), np.array([10]), np.array([50])
        quad = (np.eye(3), np.zeros(3), -float(c.gamma[50] @ c.gamma[50]))
        tpe.tp_set_pins(ctx, pins, c.gamma[pins])
        tpe.tp_set_tangents(ctx, tans, orc.edge_quantities(c.gamma, c.edges)[1][tans])
        tpe.tp_set_surface(ctx, surf, *quad)
        rows = dict(pins=pins, barycenter=False, tangents=tans, surf=surf, quad=quad)
    g = dev(c.gamma)
    dE = tpe.tp_differential(ctx, g)
    _, dP = tpe.tp_penalty(ctx, g)
    tot = dE + dP
    gt, info = tpe.sobolev_gradient(ctx, g, tot)
    assert info["converged"]
    pen = opens(orc)
    dEo = orc.differential(c.gamma, c.edges) + orc.penalty_gradient(c.gamma, c.edges, pen)
    assert np.abs(dEo.sum(0)).max() > 1e-3 * np.abs(dEo).max()   # really not translation invariant
    gr = orc.constraint_groups(c.gamma, c.edges, edge_lengths=cset == 1, **rows)
    gk, _ = orc.sobolev_gradient(c.gamma, c.edges, gr, dEo, orc.Params(), dense=True)
    assert rel(host(gt), gk) <= 1e-7
