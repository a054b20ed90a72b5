"""The accurate (double-float) Sobolev apply and the residual refinement of the mixed solves.

sobolev_apply_accurate forms every pair term of Secs. 5.2.2-5.2.3 as a double-float (~48 bits), so it
must agree with the FP64 oracle's apply to ~1e-12 relative, also on smooth vectors where |A u| << |A||u|
(the case that sets the FP32 pass's rounding floor).  The solves of TP_MIXED contexts judge their true
residual with it and refine until it is within cg_rtol: the gradient solve's reported rel_res must then
be confirmed by the oracle's FP64 operator."""
import numpy as np
import pytest

import synth as S
from tests.gpu_util import dev, host, make_ctx, need_gpu, rel

pytestmark = pytest.mark.gpu

SIG = 0.75


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle as O
    O.build_library()
    return O


def _cases():
    return {
        "trefoil256": S.trefoil_256(),
        "knot1500": S.single(S.fourier_knot(1500, 8, 5)),
        "scene3": S.scene([S.fourier_knot(70, 3, 1), S.fourier_knot(150, 4, 2), S.fourier_knot(201, 5, 3)]),
        "open": S.single(S.fourier_knot(130, 3, 9), closed=False),
    }


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("name", ["trefoil256", "knot1500", "scene3", "open"])
def test_accurate_apply_matches_fp64_oracle(torch, orc, name, prec):
    from paper_2006_07859_gb300 import tpe
    c = _cases()[name]
    ctx = make_ctx(c, precision=prec, precond=1)
    g = dev(c.gamma)
    U = np.random.default_rng(5).normal(size=(c.n_vertices, 3))
    Auo = orc.gram_apply(c.gamma, c.edges, SIG, U)
    Au = host(tpe.sobolev_apply_accurate(ctx, g, dev(U)))
    assert rel(Au, Auo) <= 1e-11, rel(Au, Auo)
    # smooth vector: the result is a small second difference of large terms
    n = c.n_vertices
    t = np.linspace(0, 2 * np.pi, n, endpoint=False)
    V = np.stack([np.cos(t), np.sin(2 * t), np.cos(3 * t)], 1)
    Avo = orc.gram_apply(c.gamma, c.edges, SIG, V)
    Av = host(tpe.sobolev_apply_accurate(ctx, g, dev(V)))
    assert rel(Av, Avo) <= 1e-10, rel(Av, Avo)


@pytest.mark.parametrize("alpha,beta", [(3.0, 6.0)])
def test_accurate_apply_general_exponents(torch, orc, alpha, beta):
    from paper_2006_07859_gb300 import tpe
    c = S.single(S.fourier_knot(400, 5, 12))
    ctx = make_ctx(c, precision=2, precond=1, alpha=alpha, beta=beta)
    U = np.random.default_rng(8).normal(size=(c.n_vertices, 3))
    Auo = orc.gram_apply(c.gamma, c.edges, orc.sigma_of(alpha, beta), U)
    Au = host(tpe.sobolev_apply_accurate(ctx, dev(c.gamma), dev(U)))
    assert rel(Au, Auo) <= 1e-11


def test_refined_mixed_solve_reaches_true_tolerance(torch, orc):
    """A-bar y = P dE on two 4,096-vertex knots (mixed, two-level, 1e-6): the reported relative residual
    is the accurate operator's, and the FP64 oracle confirms it."""
    from paper_2006_07859_gb300 import tpe
    b = S.batch_of_knots([4096, 4096], 8, 0)
    ctx = make_ctx(b, precision=2, precond=tpe.TP_PRECOND_TWOLEVEL, independent=1, cg_rtol=1e-6, warm_start=0)
    g = dev(b.gamma)
    dE = tpe.tp_differential(ctx, g)
    gt, info = tpe.sobolev_gradient(ctx, g, dE)
    assert info["converged"], info
    assert info["rel_res"] <= 1e-6
    rr, it = tpe.tp_last_solve(ctx)
    assert max(rr) <= 1e-6
    # the KKT residual of Eq. 22 under the FP64 oracle operator: dE - A-bar g~ must lie in range(C^T)
    # up to the two solves' tolerance (g~ combines A^+ dE and A^+ C_len^T)
    dEh, gth = host(dE), host(gt)
    for k in range(2):
        v0, v1 = b.vertex_offsets[k], b.vertex_offsets[k + 1]
        gk, ek = b.curve(k)
        gr = orc.constraint_groups(gk, ek)
        C = orc.jacobian(gk, ek, gr).reshape(4, -1)
        res = dEh[v0:v1].reshape(-1) - orc.gram_apply(gk, ek, SIG, gth[v0:v1]).reshape(-1)
        lam, *_ = np.linalg.lstsq(C.T, res, rcond=None)
        res -= C.T @ lam
        ratio = np.linalg.norm(res) / np.linalg.norm(dEh[v0:v1])
        assert ratio <= 3e-6, ratio
        assert np.abs(C @ gth[v0:v1].reshape(-1)).max() <= 1e-9 * np.abs(gth[v0:v1]).max()
