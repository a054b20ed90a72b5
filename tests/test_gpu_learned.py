"""GPU learned preconditioner (TP_PRECOND_LEARNED) against its FP64 oracle (oracle/gnn.py):
features, BF16-weight forward, backward, the G term and its output gradient, the full training-step
gradient, and what a trained network gains over the two-level preconditioner alone."""
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


@pytest.fixture(scope="module")
def G():
    from oracle import gnn
    return gnn


def bf16_round(x):
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def knots(sizes, seed0):
    return [S.fourier_knot(n, 8, seed0 + i) for i, n in enumerate(sizes)]


def theta0(G, seed=3):
    th = G.init_params(seed, out_bias=-1.0).astype(np.float32)
    rng = np.random.default_rng(seed + 100)
    # non-zero hidden biases so that every ReLU layer has both signs
    o = 0
    for name, s in G.SHAPES:
        k = int(np.prod(s))
        if name in ("b1", "b2", "b3"):
            th[o:o + k] = rng.normal(0, 0.3, size=k)
        o += k
    return th


def setup(torch, orc, sizes, seed0=11, precision=0, precond=None, **kw):
    from paper_2006_07859_gb300 import tpe
    cs = knots(sizes, seed0)
    gam = np.concatenate(cs, axis=0)
    voff = np.concatenate([[0], np.cumsum([len(x) for x in cs])]).astype(np.int32)
    edges = np.concatenate([S.closed_edges(len(x)) + voff[i] for i, x in enumerate(cs)]).astype(np.int32)
    ctx = tpe.Context(edges, voff, voff, gam.shape[0], precision=precision,
                      precond=tpe.TP_PRECOND_LEARNED if precond is None else precond, independent=1, **kw)
    return ctx, cs, gam, voff


def test_features_forward_backward(torch, orc, G):
    from paper_2006_07859_gb300 import tpe
    ctx, cs, gam, voff = setup(torch, orc, [96, 130])
    th = theta0(G)
    tpe.tp_gnn_set_params(ctx, torch.as_tensor(th).cuda())
    g = dev(gam)
    tpe.tp_gnn_bind(ctx, g)
    feat, out = tpe.tp_gnn_forward(ctx)
    feat, out = host(feat), host(out)
    thb = bf16_round(th)
    rng = np.random.default_rng(5)
    dout = rng.normal(size=out.shape).astype(np.float32)
    grad = host(tpe.tp_gnn_backward(ctx, torch.as_tensor(dout).cuda()))
    gref = np.zeros_like(thb)
    for k, x in enumerate(cs):
        v0, v1 = voff[k], voff[k + 1]
        e = S.closed_edges(len(x))
        diag = orc.gram_diagonal(x, e, SIG)
        f_o = G.features(x, diag)
        assert rel(feat[v0:v1], f_o) <= 1e-6
        o_o, cache = G.forward(thb, f_o)
        assert rel(out[v0:v1], o_o) <= 1e-4
        gref += G.backward(thb, cache, dout[v0:v1].astype(np.float64))
    assert rel(grad, gref) <= 1e-4


def test_g_apply_and_output_gradient(torch, orc, G):
    from paper_2006_07859_gb300 import tpe
    ctx, cs, gam, voff = setup(torch, orc, [64, 100])
    tpe.tp_gnn_set_params(ctx, torch.as_tensor(theta0(G)).cuda())
    g = dev(gam)
    tpe.tp_gnn_bind(ctx, g)
    _, out = tpe.tp_gnn_forward(ctx)
    out = host(out).astype(np.float64)
    rng = np.random.default_rng(7)
    r = rng.normal(size=gam.shape)
    gz = rng.normal(size=gam.shape)
    Gr = host(tpe.tp_gnn_g_apply(ctx, dev(r)))
    dout = host(tpe.tp_gnn_out_grad(ctx, dev(r), dev(gz)))
    for k, x in enumerate(cs):
        v0, v1 = voff[k], voff[k + 1]
        diag = orc.gram_diagonal(x, S.closed_edges(len(x)), SIG)
        assert rel(Gr[v0:v1], G.g_apply(out[v0:v1], diag, r[v0:v1])) <= 1e-11
        assert rel(dout[v0:v1], G.g_out_grad(out[v0:v1], diag, r[v0:v1], gz[v0:v1])) <= 1e-6
    # SPD: r . G r > 0
    assert float((r * Gr).sum()) > 0


def test_training_step_gradient_matches_oracle(torch, orc, G):
    """Loss and parameter gradient of one training step (one harvested pair, FP64 pair kernels)
    against the oracle's loss_and_grad with the dense Gram matrix: the learned rescaling of the
    circulant (with the symbol the GPU set up), the G term and the prepared coarse term."""
    from paper_2006_07859_gb300 import tpe
    ctx, cs, gam, voff = setup(torch, orc, [120])
    x = cs[0]
    e = S.closed_edges(len(x))
    th = theta0(G, seed=8)
    g = dev(gam)
    ctx.set_params(precond=tpe.TP_PRECOND_TWOLEVEL)
    dE = tpe.tp_differential(ctx, g)
    R = torch.empty((4, gam.shape[0], 3), dtype=torch.float64, device="cuda")
    E = torch.empty_like(R)
    n, _ = tpe.tp_cg_harvest(ctx, g, dE, 3, R, E)
    assert n >= 2
    R, E = R[:n].contiguous(), E[:n].contiguous()
    Ecopy = E.clone()
    B, AB = torch.empty_like(R), torch.empty_like(R)
    ER = torch.empty((n, 1), dtype=torch.float64, device="cuda")
    ILAM = torch.empty(gam.shape[0], dtype=torch.float64, device="cuda")
    tpe.tp_gnn_prepare_pairs(ctx, g, R, E, B, AB, ER, ILAM)
    ctx.set_params(precond=tpe.TP_PRECOND_LEARNED)
    tpe.tp_gnn_set_params(ctx, torch.as_tensor(th).cuda())
    tpe.tp_gnn_bind(ctx, g)
    grad = torch.empty(tpe.tp_gnn_num_params(), dtype=torch.float32, device="cuda")
    k = 1
    loss = tpe.tp_gnn_train_step(ctx, g, R[k:k + 1], B[k:k + 1], AB[k:k + 1], ER[k:k + 1], 0.0, grad=grad,
                                 ILAM=ILAM)
    Bm, B0m = orc.gram_dense(x, e, SIG)
    A = Bm + B0m
    diag = np.diag(A).copy()
    f = G.features(x, diag)
    r, ee, bz = host(R[k]), host(Ecopy[k]), host(B[k])
    # prepared pairs are exactly consistent: r = A e, so e . r = ||e||_A^2 > 0 and the loss is >= 0
    assert rel(r, A @ ee) <= 1e-9
    assert abs(float((ee * r).sum()) - float(host(ER[k])[0])) <= 1e-12 * abs(float((ee * r).sum()))
    lam = 1.0 / host(ILAM)      # the circulant symbol the GPU set up for this curve
    L, gref = G.loss_and_grad(bf16_round(th), f, diag, A, r, ee, bz, lam)
    assert L >= 0.0
    assert abs(loss - L) <= 1e-6 * max(1.0, abs(L))
    assert rel(host(grad), gref) <= 1e-3


def test_balanced_training_step_gradient_matches_oracle(torch, orc, G):
    """The training step of the learned smoother inside the balancing form (z = Q r + (I - Q A) y,
    y = W S W r2 + G r2, r2 = (I - A Q) r) against the oracle's loss_and_grad_balanced with the dense
    Gram matrix and the same 16 hats."""
    from paper_2006_07859_gb300 import tpe
    ctx, cs, gam, voff = setup(torch, orc, [120], precond=tpe.TP_PRECOND_LEARNED_BALANCED, coarse_dim=16)
    x = cs[0]
    e = S.closed_edges(len(x))
    th = theta0(G, seed=9)
    g = dev(gam)
    ctx.set_params(precond=tpe.TP_PRECOND_TWOLEVEL_BALANCED)
    dE = tpe.tp_differential(ctx, g)
    R = torch.empty((4, gam.shape[0], 3), dtype=torch.float64, device="cuda")
    E = torch.empty_like(R)
    n, _ = tpe.tp_cg_harvest(ctx, g, dE, 2, R, E)
    assert n >= 2
    R, E = R[:n].contiguous(), E[:n].contiguous()
    Ecopy = E.clone()
    B, AB, R2 = torch.empty_like(R), torch.empty_like(R), torch.empty_like(R)
    ER = torch.empty((n, 1), dtype=torch.float64, device="cuda")
    ILAM = torch.empty(gam.shape[0], dtype=torch.float64, device="cuda")
    tpe.tp_gnn_prepare_pairs(ctx, g, R, E, B, AB, ER, ILAM, R2)
    tpe.tp_gnn_set_params(ctx, torch.as_tensor(th).cuda())
    tpe.tp_gnn_bind(ctx, g)
    grad = torch.empty(tpe.tp_gnn_num_params(), dtype=torch.float32, device="cuda")
    k = 1
    loss = tpe.tp_gnn_train_step(ctx, g, R[k:k + 1], B[k:k + 1], AB[k:k + 1], ER[k:k + 1], 0.0, grad=grad,
                                 ILAM=ILAM, R2=R2[k:k + 1])
    Bm, B0m = orc.gram_dense(x, e, SIG)
    A = Bm + B0m
    diag = np.diag(A).copy()
    f = G.features(x, diag)
    r, ee = host(R[k]), host(Ecopy[k])
    Z = orc.coarse_hats(len(x), 16)
    # the prepared pieces: B = Q r and R2 = (I - A Q) r
    Qr = Z @ np.linalg.solve(Z.T @ A @ Z, Z.T @ r)
    assert rel(host(R2[k]), r - A @ Qr) <= 1e-8
    bz = host(B[k])
    assert rel(bz - bz.mean(0), Qr - Qr.mean(0)) <= 1e-8
    lam = 1.0 / host(ILAM)
    L, gref = G.loss_and_grad_balanced(bf16_round(th), f, diag, A, Z, r, ee, lam)
    assert L >= 0.0
    assert abs(loss - L) <= 1e-6 * max(1.0, abs(L))
    assert rel(host(grad), gref) <= 1e-3


def test_learned_training_lowers_loss_and_keeps_the_solve_within_15pct(torch, orc, record_property):
    """Train on pairs harvested from the descent of 4 knots, then compare CG iterations to 1e-3 on
    4 unseen knots: the trained G term on top of the two-level preconditioner versus the two-level
    preconditioner alone (and the loss before and after training).

    What this shows on these curves: training lowers the loss (0.317 -> 0.180 in the last measured
    run), but with the default coarse space of 128 hats the learned term does not save iterations on
    unseen knots (56 against 55): the two-level preconditioner already covers what a per-vertex
    rescaling and a two-point stencil can express.  So the test checks what must hold (the loss
    decreases; the learned PCG converges and its true residual under the exact operator stays small;
    the iteration count stays within 15% of the two-level count) and records the numbers."""
    from paper_2006_07859_gb300 import learned, tpe
    sizes = [512, 700, 900, 1200]
    ctx, cs, gam, voff = setup(torch, orc, sizes, seed0=40, precision=2)
    ctx.set_params(precond=tpe.TP_PRECOND_TWOLEVEL, cg_rtol=1e-6)
    g = dev(gam)
    sets = learned.harvest_descent(ctx, g, steps=3, every=2, max_pairs=24)
    assert sum(s.n for s in sets) >= 24
    th0 = learned.init_params(0)
    loss0 = learned.evaluate_loss(ctx, sets, torch.as_tensor(th0).cuda())
    res = learned.train(ctx, sets, steps=150, lr=3e-3, batch=4, seed=0)
    loss1 = learned.evaluate_loss(ctx, sets, res["theta"])
    print(f"training loss {loss0:.4f} -> {loss1:.4f}")
    assert 0.0 <= loss1 < loss0
    # unseen curves
    ctx2, cs2, gam2, _ = setup(torch, orc, [600, 800, 1000, 1400], seed0=90, precision=2)
    g2 = dev(gam2)
    dE2 = tpe.tp_differential(ctx2, g2)
    # both solves from zero: a warm start from the first would make the second look cheap.  The
    # comparison is of the preconditioned CG itself, at 1e-3 (no residual refinement rounds, whose count
    # depends on how far the mixed operator's true residual drifts from the recursive one)
    ctx2.set_params(precond=tpe.TP_PRECOND_TWOLEVEL, cg_rtol=1e-3, warm_start=0)
    _, i2l = tpe.sobolev_gradient(ctx2, g2, dE2)
    tpe.tp_gnn_set_params(ctx2, res["theta"])
    ctx2.set_params(precond=tpe.TP_PRECOND_LEARNED)
    _, ilr = tpe.sobolev_gradient(ctx2, g2, dE2)
    print(f"CG iterations to 1e-3: two-level {i2l['iters']}, learned {ilr['iters']}")
    record_property("loss", [loss0, loss1])
    record_property("cg_iters_twolevel_vs_learned", [i2l["iters"], ilr["iters"]])
    record_property("true_rel_res_twolevel_vs_learned", [i2l["rel_res"], ilr["rel_res"]])
    assert ilr["converged"] and i2l["converged"]
    assert ilr["rel_res"] <= 1.5e-3
    assert ilr["iters"] <= 1.15 * i2l["iters"]
