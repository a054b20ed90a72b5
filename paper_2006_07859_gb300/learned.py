"""Training loop of the learned preconditioner term (TP_PRECOND_LEARNED; not part of the paper).

Orchestration only: every computation (CG solves, pair passes, network forward / backward, Adam)
runs in libtpe.so through the tp_gnn_* / tp_cg_harvest entry points.  Pairs are harvested from the
gradient solves of the method itself: at each descent step of the training curves, the CG solve of
A-bar y = P dE is run once more with capture, and its residuals r_k with the exact corrections
e_k = y* - y_k become training pairs bound to that step's geometry.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import tpe

HIDDEN, FEATURES = tpe.TP_GNN_HIDDEN, tpe.TP_GNN_FEATURES
# parameter blocks in the order of the C ABI (row-major matrices)
SHAPES = [("W1", (HIDDEN, FEATURES)), ("b1", (HIDDEN,)), ("W2s", (HIDDEN, HIDDEN)), ("W2n", (HIDDEN, HIDDEN)),
          ("b2", (HIDDEN,)), ("W3s", (HIDDEN, HIDDEN)), ("W3n", (HIDDEN, HIDDEN)), ("b3", (HIDDEN,)),
          ("W4", (3, HIDDEN)), ("b4", (3,))]


def init_params(seed: int = 0, out_bias: float = -2.0) -> np.ndarray:
    """He-style initial parameters (float32): weights N(0, 1 / fan_in), read-out weights scaled by 0.1,
    hidden biases 0, read-out biases `out_bias` for (a, b) (so G starts as a small multiple of the
    Jacobi-scaled stencils, e^{2 out_bias}) and 0 for c (the circulant starts unscaled)."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, s in SHAPES:
        if name.startswith("W"):
            w = rng.normal(0.0, 1.0 / np.sqrt(s[1]), size=s)
            parts.append((0.1 * w if name == "W4" else w).ravel())
        elif name == "b4":
            parts.append(np.array([out_bias, out_bias, 0.0]))
        else:
            parts.append(np.zeros(s))
    theta = np.concatenate(parts).astype(np.float32)
    assert theta.size == tpe.tp_gnn_num_params()
    return theta


@dataclasses.dataclass
class PairSet:
    """Prepared training pairs of one geometry: R = A-bar e (the residuals exactly consistent with the
    harvested corrections e), B = the coarse term of R, AB = A-bar B (all [n, nV, 3] float64 on the GPU),
    ER = e . r per problem ([n, n_problems]) and ILAM, the geometry's inverse circulant symbols ([nV])."""
    gamma: object
    R: object
    B: object
    AB: object
    ER: object
    ILAM: object = None
    R2: object = None     # balancing form: (I - A Q) r, what the learned smoother acts on

    @property
    def n(self) -> int:
        return int(self.R.shape[0])


def harvest(ctx: tpe.Context, gamma, rhs, every: int = 1, max_pairs: int = 32) -> PairSet:
    """Run the gradient-type CG solve A-bar y = P rhs on `gamma` with capture and prepare its pairs.
    The context's preconditioner should be the base the learned term shapes: TP_PRECOND_TWOLEVEL (for
    TP_PRECOND_LEARNED) or TP_PRECOND_TWOLEVEL_BALANCED (for TP_PRECOND_LEARNED_BALANCED)."""
    import torch
    nV = ctx.n_vertices
    R = torch.empty((max_pairs, nV, 3), dtype=torch.float64, device="cuda")
    E = torch.empty((max_pairs, nV, 3), dtype=torch.float64, device="cuda")
    n, _ = tpe.tp_cg_harvest(ctx, gamma, rhs, every, R, E)
    R, E = R[:n].contiguous(), E[:n].contiguous()
    AB = torch.empty_like(R)
    ER = torch.empty((n, ctx.n_problems), dtype=torch.float64, device="cuda")
    ILAM = torch.empty(nV, dtype=torch.float64, device="cuda")
    balanced = ctx.params.precond in (tpe.TP_PRECOND_TWOLEVEL_BALANCED, tpe.TP_PRECOND_LEARNED_BALANCED)
    R2 = torch.empty_like(R) if balanced else None
    if n:
        tpe.tp_gnn_prepare_pairs(ctx, gamma, R, E, E, AB, ER, ILAM, R2)  # R := A-bar E; B overwrites E in place
    return PairSet(gamma.clone(), R, E, AB, ER, ILAM, R2)


def harvest_descent(ctx: tpe.Context, gamma, steps: int, every: int = 1, max_pairs: int = 32) -> list[PairSet]:
    """Pairs from the gradient solves of `steps` descent steps starting at gamma (gamma is advanced in
    place): before each step, the solve for dE is repeated with capture."""
    sets = []
    for _ in range(steps):
        dE = tpe.tp_differential(ctx, gamma)
        sets.append(harvest(ctx, gamma, dE, every, max_pairs))
        tpe.descent_step(ctx, gamma)
    return sets


def train(ctx: tpe.Context, sets: list[PairSet], steps: int = 200, lr: float = 3e-3, batch: int = 4,
          seed: int = 0, theta0=None, log_every: int = 0) -> dict:
    """Adam on the mean loss (A-norm error of the best multiple of the preconditioned correction, in
    [0, 1]) over minibatches of `batch` consecutive pairs of one geometry
    (geometries and windows drawn in a seeded random order; each switch of geometry re-binds the
    curve).  Returns the loss history and the trained parameters (float32 CUDA tensor)."""
    import torch
    rng = np.random.default_rng(seed)
    theta = torch.as_tensor(init_params(seed) if theta0 is None else theta0, device="cuda").float().contiguous()
    tpe.tp_gnn_set_params(ctx, theta, reset_optimizer=True)
    sets = [s for s in sets if s.n > 0]
    if not sets:
        raise ValueError("no training pairs")
    losses = []
    bound = -1
    for it in range(steps):
        k = int(rng.integers(len(sets)))
        ps = sets[k]
        if k != bound:
            tpe.tp_gnn_bind(ctx, ps.gamma)
            bound = k
        b = min(batch, ps.n)
        j = int(rng.integers(ps.n - b + 1))          # a contiguous window of pairs: views, no copies
        loss = tpe.tp_gnn_train_step(ctx, ps.gamma, ps.R[j:j + b], ps.B[j:j + b], ps.AB[j:j + b],
                                     ps.ER[j:j + b], lr, ILAM=ps.ILAM,
                                     R2=None if ps.R2 is None else ps.R2[j:j + b])
        losses.append(loss)
        if log_every and (it % log_every == 0 or it == steps - 1):
            print(f"step {it:5d}  loss {loss:.6f}", flush=True)
    return {"losses": losses, "theta": tpe.tp_gnn_get_params(ctx)}


def evaluate_loss(ctx: tpe.Context, sets: list[PairSet], theta) -> float:
    """Mean training loss of `theta` over every pair of `sets` (no parameter update)."""
    tpe.tp_gnn_set_params(ctx, theta, reset_optimizer=False)
    tot, cnt = 0.0, 0
    for ps in sets:
        if ps.n == 0:
            continue
        tpe.tp_gnn_bind(ctx, ps.gamma)
        tot += tpe.tp_gnn_train_step(ctx, ps.gamma, ps.R, ps.B, ps.AB, ps.ER, 0.0, ILAM=ps.ILAM, R2=ps.R2) * ps.n
        cnt += ps.n
    return tot / max(1, cnt)
