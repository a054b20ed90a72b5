"""Pins of the oracle's two-level preconditioners (this library's design, not the paper's).

The coarse term of twolevel_apply is the Galerkin correction Z (Z^T A Z)^-1 Z^T r: it is pinned by the
identities that define a Galerkin projection (Z^T A z_c = Z^T r, exactness on A Z, the A-orthogonal
projector Pi = Z E^-1 Z^T A with Pi^2 = Pi), which a transposed operand, a dropped factor or a wrong
hat would break.  The spectral part is pinned apart (exact on the regular polygon).  The balancing form
is pinned by its reduction to A^+ when the one-level term is A^+, its exactness on range(A Z) and
its symmetry."""
import numpy as np
import pytest

import synth as S

N, M = 192, 16


@pytest.fixture(scope="module")
def setup(orc):
    g = S.fourier_knot(N, 6, 21)
    e = S.closed_edges(N)
    sig = orc.sigma_of(2.0, 4.5)
    B, B0 = orc.gram_dense(g, e, sig)
    return orc, B + B0, sig


def test_hats_partition_unity_and_support():
    from oracle import oracle as O
    Z = O.coarse_hats(N, M)
    assert Z.shape == (N, M - 1)
    full = np.concatenate([Z, 1.0 - Z.sum(1, keepdims=True)], 1)   # the dropped m-th hat
    assert np.all(full >= -1e-15)
    i = np.arange(N)
    for j in range(M - 1):
        c = j * N // M
        assert Z[c, j] == pytest.approx(1.0)
        assert np.count_nonzero(Z[:, j] > 1e-15) == 2 * N // M - 1
    # the dropped hat is the periodic hat centred at (m - 1) n / m
    c = (M - 1) * N // M
    assert full[c, M - 1] == pytest.approx(1.0)
    assert np.count_nonzero(full[:, M - 1] > 1e-15) == 2 * N // M - 1


def _coarse_term(orc, A, sig, r):
    """twolevel_apply minus its spectral part (the spectral part by the separately pinned
    spectral_preconditioner with the Rayleigh-quotient symbol)."""
    z = orc.twolevel_apply(A, N, sig, M, r)
    sp = orc.spectral_preconditioner(np.diag(A), [0, N], {N: orc.spectral_rq_symbol(A, N, sig)})
    return z - sp(r)


def test_coarse_term_is_galerkin_projection(setup):
    orc, A, sig = setup
    Z = orc.coarse_hats(N, M)
    r = np.random.default_rng(3).normal(size=(N, 3))
    zc = _coarse_term(orc, A, sig, r)
    # z_c lies in range(Z) and satisfies the Galerkin condition Z^T A z_c = Z^T r
    c, *_ = np.linalg.lstsq(Z, zc, rcond=None)
    assert np.abs(Z @ c - zc).max() <= 1e-10 * np.abs(zc).max()
    assert np.abs(Z.T @ A @ zc - Z.T @ r).max() <= 1e-9 * np.abs(Z.T @ r).max()
    # exact on the coarse space: r = A Z c gives z_c = Z c
    cc = np.random.default_rng(4).normal(size=(M - 1, 3))
    zc2 = _coarse_term(orc, A, sig, A @ Z @ cc)
    assert np.abs(zc2 - Z @ cc).max() <= 1e-8 * np.abs(Z @ cc).max()


def test_coarse_projector_is_a_orthogonal(setup):
    orc, A, sig = setup
    Z = orc.coarse_hats(N, M)
    # columns of Pi = (coarse term applied to A e_i)
    Pi = np.stack([_coarse_term(orc, A, sig, np.repeat(A[:, [i]], 3, 1))[:, 0] for i in range(N)], 1)
    assert np.abs(Pi @ Pi - Pi).max() <= 1e-8 * np.abs(Pi).max()
    APi = A @ Pi
    assert np.abs(APi - APi.T).max() <= 1e-8 * np.abs(APi).max()
    x = np.random.default_rng(5).normal(size=N)
    x -= x.mean()
    assert (x - Pi @ x) @ A @ (x - Pi @ x) <= x @ A @ x * (1 + 1e-12)


def test_balanced_reduces_to_pseudoinverse(setup):
    orc, A, sig = setup
    Z = orc.coarse_hats(N, M)
    Ap = np.linalg.pinv(A, rcond=1e-13)
    r = np.random.default_rng(6).normal(size=(N, 3))
    r -= r.mean(0)
    z = orc.balanced_apply(A, Z, lambda v: Ap @ v, r)
    z -= z.mean(0)
    assert np.abs(z - Ap @ r).max() <= 1e-8 * np.abs(Ap @ r).max()


def test_balanced_is_symmetric_exact_on_coarse_space_and_positive(setup):
    orc, A, sig = setup
    Z = orc.coarse_hats(N, M)
    cc = np.random.default_rng(7).normal(size=(M - 1, 3))
    z = orc.twolevel_balanced_apply(A, N, sig, M, A @ Z @ cc)
    assert np.abs(z - Z @ cc).max() <= 1e-8 * np.abs(Z @ cc).max()
    # operator matrix on one component: symmetric, positive on the mean-free subspace
    Mb = np.stack([orc.twolevel_balanced_apply(A, N, sig, M, np.repeat(np.eye(N)[:, [i]], 3, 1))[:, 0]
                   for i in range(N)], 1)
    assert np.abs(Mb - Mb.T).max() <= 1e-9 * np.abs(Mb).max()
    P = np.eye(N) - 1.0 / N
    ev = np.linalg.eigvalsh(P @ Mb @ P)
    assert ev[0] >= -1e-10 * ev[-1] and np.sum(ev > 1e-10 * ev[-1]) == N - 1
