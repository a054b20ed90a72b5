"""GPU projected CG and descent step against the oracle (dense KKT / oracle descent step)."""
import numpy as np
import pytest

import synth as S
from tests.gpu_util import dev, host, make_ctx, need_gpu, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle as O
    O.build_library()
    return O


def _kkt_residual(orc, c, g_gpu, dE):
    B, B0 = orc.gram_dense(c.gamma, c.edges, 0.75)
    gr = orc.constraint_groups(c.gamma, c.edges)
    C = orc.jacobian(c.gamma, c.edges, gr).reshape(4 * len(gr), -1)
    P = np.eye(C.shape[1]) - C.T @ np.linalg.solve(C @ C.T, C)
    Ab = np.kron(B + B0, np.eye(3))
    b = P @ dE.reshape(-1)
    r = P @ (dE.reshape(-1) - Ab @ g_gpu.reshape(-1))
    return np.linalg.norm(r) / np.linalg.norm(b), np.abs(C @ g_gpu.reshape(-1)).max()


@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("precond", [0, 1])
def test_gradient_matches_dense_kkt(torch, orc, prec, precond):
    from paper_2006_07859_gb300 import tpe
    c = S.trefoil_256()
    # FP64 solves to 1e-8; the mixed operator's rounding floor at n = 256 is ~1e-7, so it solves to 1e-6
    rtol = 1e-8 if prec == 0 else 1e-6
    ctx = make_ctx(c, precision=prec, precond=precond, cg_rtol=rtol, cg_maxit=5000)
    g = dev(c.gamma)
    dE = tpe.tp_differential(ctx, g)
    gt, info = tpe.sobolev_gradient(ctx, g, dE)
    assert info["converged"] and info["rel_res"] <= 2 * rtol
    res, cg = _kkt_residual(orc, c, host(gt), host(dE))   # judged by the dense FP64 operator
    assert res <= (1e-7 if prec == 0 else 5e-6)
    assert cg <= 1e-10 * np.abs(host(gt)).max()
    gr = orc.constraint_groups(c.gamma, c.edges)
    gk, _ = orc.sobolev_gradient(c.gamma, c.edges, gr, orc.differential(c.gamma, c.edges), orc.Params(), dense=True)
    assert rel(host(gt), gk) <= (1e-6 if prec == 0 else 1e-3)


def test_descent_step_matches_oracle(torch, orc):
    from paper_2006_07859_gb300 import tpe
    c = S.single(S.trefoil(96, 0.01, 0))
    ctx = make_ctx(c, precision=0, precond=1, cg_rtol=1e-10, proj_cg_rtol=1e-10)
    g = dev(c.gamma)
    gr = orc.constraint_groups(c.gamma, c.edges)
    prm = orc.Params(cg_tol=1e-10, proj_cg_tol=1e-10)
    go = c.gamma.copy()
    for step in range(3):
        info = tpe.descent_step(ctx, g)
        go, io = orc.descent_step(go, c.edges, gr, prm)
        assert info["accepted"] == 1 and io.accepted
        assert info["tau"] == io.tau
        assert abs(info["E_after"] - io.E_after) <= 1e-9 * io.E_after
        assert rel(host(g), go) <= 1e-7
        assert np.abs(orc.phi(host(g), c.edges, gr)).max() <= 1e-9


def test_independent_batch_equals_single_curves(torch):
    from paper_2006_07859_gb300 import tpe
    sizes = [64, 97, 130, 255]
    b = S.batch_of_knots(sizes, 6, 500)
    ctx = make_ctx(b, precision=2, precond=1, independent=1)
    E = host(tpe.tp_energy(ctx, dev(b.gamma)))
    dE = host(tpe.tp_differential(ctx, dev(b.gamma)))
    for k in range(len(sizes)):
        gk, ek = b.curve(k)
        cs = S.single(gk)
        c1 = make_ctx(cs, precision=2, precond=1)
        # equal up to the order in which FP32 tile partials are summed (the chunking differs)
        assert abs(host(tpe.tp_energy(c1, dev(gk)))[0] - E[k]) <= 1e-7 * E[k]
        v0, v1 = b.vertex_offsets[k], b.vertex_offsets[k + 1]
        assert rel(host(tpe.tp_differential(c1, dev(gk))), dE[v0:v1]) <= 1e-6
