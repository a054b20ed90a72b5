"""The balancing form of the two-level preconditioner (TP_PRECOND_TWOLEVEL_BALANCED; this library's
design, not the paper's): M^-1 r = Q r + (I - Q A) S (I - A Q) r with the spectral term S and the Galerkin
coarse term Q.  The GPU preconditioner is compared with the oracle's twolevel_balanced_apply (built
from the dense Gram matrix, pinned in tests/test_oracle_twolevel.py), and its CG iterations with those
of the additive form."""
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


# Coarse spaces of 8 hats and more are assembled by the A Z pass, smaller ones by probing (m = 4, 6);
# in FP64 both agree with the oracle to ~1e-8.  In mixed precision the pass and the pair kernel work in
# FP32 with double-float differences, and the coarse solve E^-1 amplifies the operator's rounding with
# the coarse space's condition: measured 5e-6 (128 hats) and 3e-5 (256 hats) of the norm.  A wrong
# index or sign anywhere in the pass moves the result by O(1).
@pytest.mark.parametrize("name,m,prec,tol", [("trefoil256", 32, 0, 1e-6), ("knot600", 128, 0, 1e-6),
                                             ("batch3", 32, 0, 1e-6), ("knot1200", 256, 0, 1e-6),
                                             ("knot1200", 300, 0, 1e-6),
                                             ("trefoil256", 4, 0, 1e-6), ("batch3", 6, 0, 1e-6),
                                             ("knot600", 128, 2, 1e-4), ("knot1200", 256, 2, 1e-4),
                                             ("batch3", 32, 2, 1e-4)])
def test_balanced_apply_matches_oracle(torch, orc, name, m, prec, tol):
    from paper_2006_07859_gb300 import tpe
    if name == "trefoil256":
        c, indep = S.trefoil_256(), 0
    elif name == "knot600":
        c, indep = S.single(S.fourier_knot(600, 6, 4)), 0
    elif name == "knot1200":
        c, indep = S.single(S.fourier_knot(1200, 8, 5)), 0
    else:
        c, indep = S.batch_of_knots([64, 129, 256], 5, 700), 1
    ctx = make_ctx(c, precision=prec, precond=tpe.TP_PRECOND_TWOLEVEL_BALANCED, independent=indep, coarse_dim=m)
    r = np.random.default_rng(6).normal(size=(c.n_vertices, 3))
    for k in range(c.n_curves):
        v0, v1 = c.vertex_offsets[k], c.vertex_offsets[k + 1]
        r[v0:v1] -= r[v0:v1].mean(0)
    z = host(tpe.tp_precond_apply(ctx, dev(c.gamma), dev(r)))
    for k in range(c.n_curves):
        gk, ek = c.curve(k)
        n = gk.shape[0]
        B, B0 = orc.gram_dense(gk, ek, SIG)
        v0, v1 = c.vertex_offsets[k], c.vertex_offsets[k + 1]
        zo = orc.twolevel_balanced_apply(B + B0, n, SIG, min(m, n // 4), r[v0:v1])
        a, b = z[v0:v1] - z[v0:v1].mean(0), zo - zo.mean(0)
        print(name, m, prec, k, rel(a, b))
        assert rel(a, b) <= tol, k


def test_balanced_cuts_iterations(torch):
    """FP64 and mixed solves to 1e-6 on Fourier knots: fewer CG iterations than the additive form."""
    from paper_2006_07859_gb300 import tpe
    b = S.batch_of_knots([2048, 2048], 8, 40)
    g = dev(b.gamma)
    for prec in (0, 2):
        its = {}
        for pc in (tpe.TP_PRECOND_TWOLEVEL, tpe.TP_PRECOND_TWOLEVEL_BALANCED):
            ctx = make_ctx(b, precision=prec, precond=pc, independent=1, coarse_dim=64, cg_rtol=1e-6, warm_start=0)
            dE = tpe.tp_differential(ctx, g)
            _, info = tpe.sobolev_gradient(ctx, g, dE)
            assert info["converged"] and info["rel_res"] <= 1e-6
            its[pc] = info["iters"]
        print(prec, its)
        assert its[tpe.TP_PRECOND_TWOLEVEL_BALANCED] < 0.75 * its[tpe.TP_PRECOND_TWOLEVEL], its


def test_balanced_needs_single_curve_problems(torch):
    from paper_2006_07859_gb300 import tpe
    c = S.scene([S.fourier_knot(100, 3, 1), S.fourier_knot(120, 4, 2)])
    with pytest.raises(tpe.TpError) as ei:
        make_ctx(c, precision=2, precond=tpe.TP_PRECOND_TWOLEVEL_BALANCED)
    assert ei.value.status == tpe.TP_ERR_UNSUPPORTED
    ctx = make_ctx(c, precision=2, precond=tpe.TP_PRECOND_TWOLEVEL)
    with pytest.raises(tpe.TpError):
        ctx.set_params(precond=tpe.TP_PRECOND_TWOLEVEL_BALANCED)
