"""First collision time along a direction (Sec. 5.4, TP_LINESEARCH_ISOTOPY) on the GPU against the
oracle: closed-form crossings, random knots and motions (one block and several, ragged), coplanar
motion, independent batches, and the isotopy-safe descent step."""
import numpy as np
import pytest

import synth as S
from tests.gpu_util import dev, host, make_ctx, need_gpu

pytestmark = pytest.mark.gpu
H = 1.5


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle as O
    O.build_library()
    return O


def two_segments(torch, c, e, dc, de):
    """Segment I on the x axis at rest, segment J = (c, e) moving with (dc, de): one problem."""
    from paper_2006_07859_gb300 import tpe
    g = np.array([[-1.0, 0, 0], [1.0, 0, 0], c, e])
    d = np.array([[0.0, 0, 0], [0, 0, 0], dc, de])
    ctx = tpe.Context(np.array([[0, 1], [2, 3]], dtype=np.int32), [0, 4], [0, 2], 4, precision=0, precond=1)
    return float(host(tpe.tp_collision_time(ctx, dev(g), dev(d), H))[0])


def test_closed_form_crossings(torch):
    c, e = [0.0, -1, 1], [0.0, 1, 1]
    assert two_segments(torch, c, e, [0, 0, 1.0], [0, 0, 1.0]) == pytest.approx(1.0, rel=1e-12)
    assert two_segments(torch, c, e, [0, 0, 2.5], [0, 0, 2.5]) == pytest.approx(0.4, rel=1e-12)
    assert two_segments(torch, c, e, [0, 0, 0], [0, 0, 2.0]) == pytest.approx(1.0, rel=1e-12)   # swinging end
    assert two_segments(torch, c, e, [0, 0, 0.5], [0, 0, 0.5]) == H                              # beyond the horizon
    assert two_segments(torch, [3.0, -1, 1], [3.0, 1, 1], [0, 0, 1.0], [0, 0, 1.0]) == H          # passes beside
    # coplanar motion: a parallel segment above I lands on it at 1 / v
    assert two_segments(torch, [0.25, 1, 0], [0.75, 1, 0], [0, 2.0, 0], [0, 2.0, 0]) == pytest.approx(0.5, rel=1e-12)


@pytest.mark.parametrize("n,scale,seed", [(40, 1.0, 0), (100, 0.6, 1), (300, 0.3, 2), (300, 0.01, 3)])
def test_knot_collision_time_matches_oracle(torch, orc, n, scale, seed):
    """Fourier knots with a random motion: one block (40), a ragged block (100) and three blocks (300);
    the last case moves too little to collide within the horizon."""
    from paper_2006_07859_gb300 import tpe
    c = S.single(S.fourier_knot(n, 4, 60 + seed))
    d = np.random.default_rng(seed).normal(0, scale, (n, 3))
    ctx = make_ctx(c, precision=0, precond=1)
    t = float(host(tpe.tp_collision_time(ctx, dev(c.gamma), dev(d), H))[0])
    to = float(orc.first_collision_time(c.gamma, c.edges, d, H)[0])
    if seed == 3:
        assert to == H
    else:
        assert to < H
    assert t == pytest.approx(to, rel=1e-10)


def test_coplanar_motion_matches_oracle(torch, orc):
    from paper_2006_07859_gb300 import tpe
    n = 24
    c = S.single(S.regular_polygon(n, 1.0))
    rng = np.random.default_rng(5)
    d = rng.normal(0, 1.5, (n, 3))
    d[:, 2] = 0.0   # in-plane motion of a planar polygon
    ctx = make_ctx(c, precision=0, precond=1)
    t = float(host(tpe.tp_collision_time(ctx, dev(c.gamma), dev(d), H))[0])
    to = float(orc.first_collision_time(c.gamma, c.edges, d, H)[0])
    assert to < H
    assert t == pytest.approx(to, rel=1e-10)


def test_independent_batch_per_curve(torch, orc):
    from paper_2006_07859_gb300 import tpe
    b = S.batch_of_knots([50, 130, 77], 4, 300)
    d = np.random.default_rng(9).normal(0, 0.8, (b.n_vertices, 3))
    ctx = make_ctx(b, precision=0, precond=1, independent=1)
    t = host(tpe.tp_collision_time(ctx, dev(b.gamma), dev(d), H))
    for k in range(3):
        gk, ek = b.curve(k)
        v0, v1 = b.vertex_offsets[k], b.vertex_offsets[k + 1]
        assert t[k] == pytest.approx(orc.first_collision_time(gk, ek, d[v0:v1], H)[0], rel=1e-10)


def test_isotopy_safe_descent_step_matches_oracle(torch, orc):
    from paper_2006_07859_gb300 import tpe
    c = S.single(S.trefoil(64, 0.01, 3))
    ctx = make_ctx(c, precision=0, precond=1, cg_rtol=1e-10, proj_cg_rtol=1e-10,
                   line_search=tpe.TP_LINESEARCH_ISOTOPY)
    g = dev(c.gamma)
    gr = orc.constraint_groups(c.gamma, c.edges)
    prm = orc.Params(cg_tol=1e-10, proj_cg_tol=1e-10, isotopy_safe=True)
    go = c.gamma.copy()
    for _ in range(2):
        info = tpe.descent_step(ctx, g)
        go, io = orc.descent_step(go, c.edges, gr, prm)
        assert info["accepted"] == 1 and io.accepted
        assert info["tau"] == pytest.approx(io.tau, rel=1e-9)
        assert abs(info["E_after"] - io.E_after) <= 1e-9 * io.E_after
