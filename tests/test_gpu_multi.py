"""Multi-field Sobolev apply (sobolev_apply_multi): AU_f = A-bar U_f for m vector fields in one call
(Secs. 5.2.2-5.2.3 per field).  Every field is checked against the FP64 oracle's gram_apply, which
takes the 3 m scalar columns at once, and against the single-field sobolev_apply of the same context.
The field counts cover one partial group (m = 1), one full group of four (m = 4) and a full group
plus a partial one (m = 6); the graphs are those of the single-apply parity tests plus a batch of
independent knots long enough to split sources into several chunks (partial-sum slots)."""
import numpy as np
import pytest

import synth as S
from tests.gpu_util import cosine, dev, host, make_ctx, need_gpu, rel

pytestmark = pytest.mark.gpu

SIG = 0.75
PRECS = [(0, 1e-10), (1, 1e-4), (2, 1e-4)]   # TP_FP64, TP_FP32, TP_MIXED: the single apply's bars
AGREE = {0: 1e-12, 1: 1e-4, 2: 1e-6}          # against the single-field apply of the same context


def cases():
    return {
        "square": S.single(S.unit_square()),
        "trefoil256": S.trefoil_256(),
        "ragged300": S.single(S.fourier_knot(300, 5, 3)),
        "scene3": S.scene([S.fourier_knot(70, 3, 1), S.fourier_knot(150, 4, 2), S.fourier_knot(201, 5, 3)]),
        "open": S.single(S.fourier_knot(130, 3, 9), closed=False),
    }


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle as O
    O.build_library()
    return O


def oracle_fields(orc, gamma, edges, U):
    """The oracle's product on the fields of U [m, nV, 3] as 3 m scalar columns."""
    m, nv = U.shape[0], U.shape[1]
    cols = np.ascontiguousarray(U.transpose(1, 0, 2).reshape(nv, 3 * m))
    return orc.gram_apply(gamma, edges, SIG, cols).reshape(nv, m, 3).transpose(1, 0, 2)


@pytest.mark.parametrize("m", [1, 4, 6])
@pytest.mark.parametrize("prec,tol", PRECS)
@pytest.mark.parametrize("name", ["square", "trefoil256", "ragged300", "scene3", "open"])
def test_multi_apply_matches_oracle(torch, orc, name, prec, tol, m):
    from paper_2006_07859_gb300 import tpe
    c = cases()[name]
    ctx = make_ctx(c, precision=prec, precond=1)
    g = dev(c.gamma)
    U = np.random.default_rng(11 + m).normal(size=(m, c.n_vertices, 3))
    AU = host(tpe.sobolev_apply_multi(ctx, g, dev(U)))
    AUo = oracle_fields(orc, c.gamma, c.edges, U)
    for f in range(m):
        if prec == 0:
            assert rel(AU[f], AUo[f]) <= tol, f
        else:
            assert cosine(AU[f], AUo[f]) >= 0.9999, f
            assert rel(AU[f], AUo[f]) <= tol, f
        single = host(tpe.sobolev_apply(ctx, g, dev(U[f])))
        assert rel(AU[f], single) <= AGREE[prec], f


@pytest.mark.parametrize("prec", [0, 2])
def test_multi_apply_on_independent_batch(torch, orc, prec):
    """Independent knots of 1,500 to 2,600 vertices: several source chunks per target block, ragged
    tails, and no pair across curves."""
    from paper_2006_07859_gb300 import tpe
    b = S.batch_of_knots([1500, 2600, 2049], 6, 300)
    ctx = make_ctx(b, precision=prec, precond=1, independent=1)
    U = np.random.default_rng(5).normal(size=(5, b.n_vertices, 3))
    AU = host(tpe.sobolev_apply_multi(ctx, dev(b.gamma), dev(U)))
    for k in range(b.n_curves):
        gk, ek = b.curve(k)
        v0, v1 = b.vertex_offsets[k], b.vertex_offsets[k + 1]
        AUo = oracle_fields(orc, gk, ek, U[:, v0:v1])
        for f in range(U.shape[0]):
            assert rel(AU[f, v0:v1], AUo[f]) <= (1e-10 if prec == 0 else 1e-4), (k, f)


def test_multi_apply_zero_fields(torch):
    from paper_2006_07859_gb300 import tpe
    c = S.trefoil_256()
    ctx = make_ctx(c, precision=2, precond=1)
    U = torch.empty((0, c.n_vertices, 3), dtype=torch.float64, device="cuda")
    AU = tpe.sobolev_apply_multi(ctx, dev(c.gamma), U)
    assert tuple(AU.shape) == (0, c.n_vertices, 3)
