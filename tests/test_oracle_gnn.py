"""Pins of the learned-preconditioner oracle (oracle/gnn.py): finite differences of the loss
with respect to the parameters, symmetry and positivity of the learned term.  CPU only."""
import numpy as np
import pytest

import synth as S
from oracle import gnn


@pytest.fixture(scope="module")
def setup(orc):
    n = 24
    c = S.single(S.fourier_knot(n, 3, 5))
    B, B0 = orc.gram_dense(c.gamma, c.edges, 0.75)
    A = B + B0
    diag = np.diag(A).copy()
    rng = np.random.default_rng(0)
    e = rng.normal(size=(n, 3))
    e -= e.mean(0)
    r = A @ e
    base_z = r / diag[:, None]
    return c, A, diag, r, e, base_z


def test_g_term_is_symmetric_positive(setup):
    c, A, diag, r, e, base_z = setup
    theta = gnn.init_params(3, out_bias=-0.5)
    out, _ = gnn.forward(theta, gnn.features(c.gamma, diag))
    n = c.n_vertices
    G = np.zeros((n, n))
    for k in range(n):
        u = np.zeros((n, 3))
        u[k, 0] = 1.0
        G[:, k] = gnn.g_apply(out, diag, u)[:, 0]
    assert np.abs(G - G.T).max() <= 1e-12 * np.abs(G).max()
    assert np.linalg.eigvalsh(G).min() >= -1e-12 * np.abs(G).max()


def test_loss_gradient_matches_central_differences(setup):
    c, A, diag, r, e, base_z = setup
    theta = gnn.init_params(1, out_bias=-0.5)
    f = gnn.features(c.gamma, diag)
    L, g = gnn.loss_and_grad(theta, f, diag, A, r, e, base_z)
    rng = np.random.default_rng(2)
    idx = rng.choice(theta.size, 40, replace=False)
    h = 1e-6
    for k in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (gnn.loss_and_grad(tp, f, diag, A, r, e, base_z)[0] - gnn.loss_and_grad(tm, f, diag, A, r, e, base_z)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g).max()), (k, fd, g[k])


def test_loss_is_the_best_scaled_a_norm_error(setup):
    """L = min over a of ||a z - e||_A^2 / ||e||_A^2 (A e = r), found here by a brute-force scan of a:
    the loss ignores the preconditioner's scale, as preconditioned CG does."""
    c, A, diag, r, e, base_z = setup
    theta = gnn.init_params(4, out_bias=-1.0)
    f = gnn.features(c.gamma, diag)
    out, _ = gnn.forward(theta, f)
    z = base_z + gnn.g_apply(out, diag, r)
    L, _ = gnn.loss_and_grad(theta, f, diag, A, r, e, base_z)
    ee = (e * (A @ e)).sum()

    def err(a):
        d = a * z - e
        return (d * (A @ d)).sum() / ee

    a_scale = np.sqrt(ee / (z * (A @ z)).sum())
    grid = np.linspace(0.0, 4.0 * a_scale, 40001)
    vals = np.array([err(a) for a in grid])
    assert 0.0 <= L <= 1.0
    assert vals.min() >= L - 1e-12
    assert vals.min() - L <= 1e-6


def test_rescaled_spectral_gradient_matches_central_differences(setup, orc):
    """The full learned preconditioner (rescaled circulant + G term + a fixed part): parameter gradient
    of the loss against central differences, with the regular-polygon symbol as the circulant."""
    c, A, diag, r, e, base_z = setup
    n = c.n_vertices
    lam = orc.ngon_symbol_closed_form(n, 0.75)
    theta = gnn.init_params(6, out_bias=-1.0)
    f = gnn.features(c.gamma, diag)
    zc = 0.3 * base_z
    L, g = gnn.loss_and_grad(theta, f, diag, A, r, e, zc, lam)
    rng = np.random.default_rng(9)
    o = sum(int(np.prod(s)) for name, s in gnn.SHAPES[:-2])   # start of W4
    idx = np.concatenate([rng.choice(theta.size, 30, replace=False), o + 2 * gnn.H + np.arange(0, gnn.H, 8),
                          [theta.size - 1]])                  # include the c row of W4 and its bias
    h = 1e-6
    for k in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (gnn.loss_and_grad(tp, f, diag, A, r, e, zc, lam)[0]
              - gnn.loss_and_grad(tm, f, diag, A, r, e, zc, lam)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g).max()), (k, fd, g[k])


def test_zero_log_scale_is_the_jacobi_scaled_circulant(setup, orc):
    """With c = 0 the rescaled circulant is the plain D^-1/2 F^-1 diag(1/lambda) F D^-1/2 of the
    spectral preconditioner (computed by the oracle's own routine)."""
    c, A, diag, r, e, base_z = setup
    n = c.n_vertices
    lam = orc.ngon_symbol_closed_form(n, 0.75)
    z = gnn.scaled_spectral(diag, np.zeros(n), lam, r)
    ref = orc.spectral_preconditioner(diag, [0, n], {n: lam})(r)
    assert np.abs(z - ref).max() <= 1e-12 * np.abs(ref).max()
