"""Pins of the oracle's discrete inner product A = B + B0 (Secs. 5.2.1-5.2.3, Eq. 21) and of the
solves built on it (Secs. 5.3-5.4, App. B.3.3-B.3.4).  CPU only."""
import numpy as np
import pytest

import synth as S

SIG = (4.5 - 1.0) / 2.0 - 1.0   # sigma for (alpha, beta) = (2, 4.5)


def test_dense_apply_and_bilinear_agree(orc):
    c = S.single(S.trefoil(40, 0.01, 5))
    g, e = c.gamma, c.edges
    B, B0 = orc.gram_dense(g, e, SIG)
    A = B + B0
    U = np.random.default_rng(0).normal(size=(40, 3))
    np.testing.assert_allclose(orc.gram_apply(g, e, SIG, U), A @ U, rtol=0, atol=1e-13 * np.abs(A).max() * 40)
    # the bilinear forms evaluated from their definitions agree with the increment tables
    for a, b in [(0, 1), (1, 2), (2, 2)]:
        uBv, uB0v = orc.bilinear(g, e, SIG, U[:, a], U[:, b])
        assert abs(uBv - U[:, a] @ B @ U[:, b]) <= 1e-12 * abs(uBv) + 1e-12
        assert abs(uB0v - U[:, a] @ B0 @ U[:, b]) <= 1e-12 * abs(uB0v) + 1e-12


def test_entrywise_bilinear(orc):
    # entry (a, b) of each Gram matrix is the bilinear form on unit vectors e_a, e_b
    c = S.single(S.fourier_knot(9, 2, 4))
    g, e = c.gamma, c.edges
    B, B0 = orc.gram_dense(g, e, SIG)
    I = np.eye(9)
    for a in range(9):
        for b in range(9):
            x, y = orc.bilinear(g, e, SIG, I[a], I[b])
            assert abs(x - B[a, b]) <= 1e-12 * np.abs(B).max()
            assert abs(y - B0[a, b]) <= 1e-12 * np.abs(B0).max()


def test_symmetric_psd_nullspace(orc):
    sc = S.scene([S.fourier_knot(24, 3, 1), S.fourier_knot(30, 3, 2)], spacing=2.5)
    B, B0 = orc.gram_dense(sc.gamma, sc.edges, SIG)
    A = B + B0
    assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()
    assert np.abs(A @ np.ones(54)).max() <= 1e-12 * np.abs(A).max()
    ev = np.linalg.eigvalsh(A)
    tol = 1e-11 * ev[-1]
    assert ev[0] >= -tol
    assert np.sum(np.abs(ev) <= tol) == 1            # only global constants (Sec. 4.2.4)
    evB = np.linalg.eigvalsh(B)
    assert np.sum(np.abs(evB) <= 1e-11 * evB[-1]) == 2   # B vanishes on per-component constants


def test_scaling(orc):
    c = S.single(S.trefoil(32, 0.01, 1))
    B, B0 = orc.gram_dense(c.gamma, c.edges, SIG)
    lam = 2.3
    Bl, B0l = orc.gram_dense(lam * c.gamma, c.edges, SIG)
    f = lam ** (-(2 * SIG + 1))     # both terms scale alike, App. A.4.2
    np.testing.assert_allclose(Bl, f * B, rtol=1e-12, atol=1e-14 * np.abs(B).max())
    np.testing.assert_allclose(B0l, f * B0, rtol=1e-12, atol=1e-14 * np.abs(B0).max())


def test_straight_line(orc):
    n = 14
    line = np.stack([np.cumsum(np.linspace(1, 2, n)), np.zeros(n), np.zeros(n)], 1)
    B, B0 = orc.gram_dense(line, S.open_edges(n), SIG)
    assert np.all(B0 == 0.0)                      # k^2_4 vanishes on a line
    ev = np.linalg.eigvalsh(B)
    assert np.sum(np.abs(ev) <= 1e-11 * ev[-1]) == 2  # constants and arclength


def test_regular_polygon_is_circulant_and_matches_fourier_symbol(orc):
    """For a regular n-gon A is circulant.  Its eigenvalue on the Fourier mode u_j = exp(i k theta j),
    theta = 2 pi / n, follows from the quadratic forms by summing over the offset m = J - I:
       lambda_k = sum_m [ 2 w_m |e^{i theta k} - 1|^2 / l^2 (1 - cos(k theta m) <T_0, T_m>)
                          + w0s_m / 4 |1 + e^{i theta k}|^2 (1 - cos(k theta m)) ],
    with w0s_m = w0_{0m} + w0_{m0}; an independent route from the increment tables."""
    n = 16
    g = S.regular_polygon(n, 1.3)
    e = S.closed_edges(n)
    B, B0 = orc.gram_dense(g, e, SIG)
    A = B + B0
    for s in range(1, n):
        np.testing.assert_allclose(np.roll(A[:, 0], s), A[:, s], rtol=0, atol=1e-13 * A[0, 0])
    ev_dft = np.real(np.fft.fft(A[:, 0]))
    ell, T, x = orc.edge_quantities(g, e)
    p = 2 * SIG + 1
    lam = np.zeros(n)
    th = 2 * np.pi / n
    for k in range(n):
        for m in range(2, n - 1):
            w = 0.0
            w0 = 0.0
            for a in (0, 1):
                for b in (0, 1):
                    d = g[(0 + a) % n] - g[(m + b) % n]
                    r = np.linalg.norm(d)
                    w += r ** -p
                    w0 += (np.linalg.norm(np.cross(T[0], d)) ** 2 + np.linalg.norm(np.cross(T[m], d)) ** 2) / r ** 4 * r ** -p
            w *= 0.25 * ell[0] * ell[m]
            w0 *= 0.25 * ell[0] * ell[m]
            lam[k] += 2 * w * abs(np.exp(1j * th * k) - 1) ** 2 / ell[0] ** 2 * (1 - np.cos(th * k * m) * (T[0] @ T[m]))
            lam[k] += w0 / 4 * abs(1 + np.exp(1j * th * k)) ** 2 * (1 - np.cos(th * k * m))
    np.testing.assert_allclose(ev_dft, lam, rtol=1e-11, atol=1e-12 * A[0, 0])


def test_ngon_closed_form_symbol_matches_dense_gram(orc):
    for n in (8, 16, 33, 64):
        g = S.regular_polygon(n, 1.0)
        B, B0 = orc.gram_dense(g, S.closed_edges(n), SIG)
        ev = np.real(np.fft.fft((B + B0)[:, 0]))
        lam = orc.ngon_symbol_closed_form(n, SIG, normalized=False)
        np.testing.assert_allclose(lam, ev, rtol=1e-10, atol=1e-12 * ev.max())
        np.testing.assert_allclose(orc.ngon_symbol_closed_form(n, SIG), orc.circle_symbol(n, SIG), rtol=1e-9)


def test_constraint_jacobian_matches_differences(orc):
    c = S.single(S.trefoil(20, 0.01, 2))
    g, e = c.gamma, c.edges
    gr = orc.constraint_groups(g, e)
    assert np.abs(orc.phi(g, e, gr)).max() <= 1e-13
    C = orc.jacobian(g, e, gr)
    h = 1e-6
    J = np.zeros_like(C)
    for v in range(20):
        for k in range(3):
            gp, gm = g.copy(), g.copy()
            gp[v, k] += h
            gm[v, k] -= h
            J[:, v, k] = (orc.phi(gp, e, gr) - orc.phi(gm, e, gr)) / (2 * h)
    assert np.abs(J - C).max() <= 1e-8


def test_kkt_vs_projected_cg(orc):
    c = S.single(S.trefoil(64, 0.01, 0))
    g, e = c.gamma, c.edges
    gr = orc.constraint_groups(g, e)
    dE = orc.differential(g, e)
    prm = orc.Params(cg_tol=1e-12)
    gk, _ = orc.sobolev_gradient(g, e, gr, dE, prm, dense=True)
    gc, res = orc.sobolev_gradient(g, e, gr, dE, prm)
    assert res.converged
    assert np.abs(gk - gc).max() <= 1e-8 * np.abs(gk).max()
    C = orc.jacobian(g, e, gr).reshape(4, -1)
    assert np.abs(C @ gk.reshape(-1)).max() <= 1e-12 * np.abs(gk).max()
    # projected system has exactly k = 4 zero eigenvalues (range of C^T)
    B, B0 = orc.gram_dense(g, e, prm.sigma)
    Ab = np.kron(B + B0, np.eye(3))                 # vertex-major A-bar
    P = np.eye(192) - C.T @ np.linalg.solve(C @ C.T, C)
    ev = np.linalg.eigvalsh(P @ Ab @ P)
    assert np.sum(np.abs(ev) <= 1e-10 * ev[-1]) == 4


def test_regular_polygon_is_critical(orc):
    g = S.regular_polygon(10, 1.0)
    e = S.closed_edges(10)
    gr = orc.constraint_groups(g, e)
    dE = orc.differential(g, e)
    gt, _ = orc.sobolev_gradient(g, e, gr, dE, orc.Params(), dense=True)
    assert np.abs(gt).max() <= 1e-12 * np.abs(dE).max()


@pytest.mark.parametrize("ab", [(2.0, 4.5), (3.0, 6.0)])
def test_gradient_scaling(orc, ab):
    alpha, beta = ab
    prm = orc.Params(alpha=alpha, beta=beta)
    c = S.single(S.trefoil(40, 0.01, 4))
    g, e = c.gamma, c.edges
    lam = 1.9

    def grad(gg):
        gr = orc.constraint_groups(gg, e)
        return orc.sobolev_gradient(gg, e, gr, orc.differential(gg, e, alpha, beta), prm, dense=True)[0]

    # dE scales by lambda^(1 + alpha - beta), A by lambda^-(2 sigma + 1)
    ex = (1 + alpha - beta) + (2 * prm.sigma + 1)
    np.testing.assert_allclose(grad(lam * g), lam ** ex * grad(g), rtol=1e-9, atol=1e-12)


def test_descent_step_decreases_energy_and_keeps_constraints(orc):
    c = S.single(S.trefoil(48, 0.01, 0))
    g, e = c.gamma, c.edges
    gr = orc.constraint_groups(g, e)
    prm = orc.Params()
    g1, info = orc.descent_step(g, e, gr, prm)
    assert info.accepted
    assert info.E_after < info.E_before
    assert np.abs(orc.phi(g1, e, gr)).max() <= prm.proj_tol * max(1.0, gr[0].L0)
    g2, info2 = orc.descent_step(g1, e, gr, prm)
    assert info2.E_after < info2.E_before


def test_spectral_preconditioner_is_exact_on_regular_polygon(orc):
    """On a regular polygon A is circulant with a constant diagonal, so the preconditioner inverts
    A exactly on non-constant modes; with the 4 constraint rows PCG needs at most 6 iterations."""
    for n in (32, 64):
        g = S.regular_polygon(n, 1.0) + 0.0
        e = S.closed_edges(n)
        gr = orc.constraint_groups(g, e)
        rhs = np.random.default_rng(n).normal(size=(n, 3))
        lam = orc.circle_symbol(n, SIG)
        M = orc.spectral_preconditioner(orc.gram_diagonal(g, e, SIG), [0, n], {n: lam})
        P = orc.Projector(orc.jacobian(g, e, gr))
        res = orc.projected_cg(orc.make_apply(g, e, SIG), P, rhs, 1e-10, 200, M)
        plain = orc.projected_cg(orc.make_apply(g, e, SIG), P, rhs, 1e-10, 2000)
        assert res.converged and res.iters <= 6
        assert plain.iters > 4 * res.iters
        assert np.abs(res.x - plain.x).max() <= 1e-7 * np.abs(plain.x).max()


def test_rq_symbol_is_exact_on_regular_polygon(orc):
    """On a regular polygon A is circulant with a constant diagonal, so the Rayleigh quotients on the
    Fourier modes are its normalised eigenvalues and the correction is the identity."""
    for n in (40, 64, 100):
        g = S.regular_polygon(n, 1.7)
        B, B0 = orc.gram_dense(g, S.closed_edges(n), SIG)
        np.testing.assert_allclose(orc.spectral_rq_symbol(B + B0, n, SIG), orc.ngon_symbol_closed_form(n, SIG),
                                   rtol=1e-10)


def test_edge_length_jacobian_matches_differences(orc):
    """Edge-length rows (Sec. 8.1, Phi_I = l0_I - l_I) against central differences of phi: pins the
    sign and the endpoint of every row."""
    c = S.single(S.trefoil(16, 0.01, 5))
    g, e = c.gamma, c.edges
    gr = orc.constraint_groups(g, e, edge_lengths=True)
    assert gr[0].n_rows == 3 + 16
    assert np.abs(orc.phi(g, e, gr)).max() <= 1e-13
    C = orc.jacobian(g, e, gr)
    h = 1e-6
    J = np.zeros_like(C)
    for v in range(16):
        for k in range(3):
            gp, gm = g.copy(), g.copy()
            gp[v, k] += h
            gm[v, k] -= h
            J[:, v, k] = (orc.phi(gp, e, gr) - orc.phi(gm, e, gr)) / (2 * h)
    assert np.abs(J - C).max() <= 1e-8


def test_edge_length_rows_annihilate_rigid_motions(orc):
    """Every edge length is invariant under rigid motions, so the edge rows vanish on translations
    and on infinitesimal rotations v = w x gamma; a radial scaling is not isometric."""
    c = S.single(S.trefoil(24, 0.01, 6))
    g, e = c.gamma, c.edges
    gr = orc.constraint_groups(g, e, edge_lengths=True)
    C = orc.jacobian(g, e, gr)[3:].reshape(24, -1)
    w = np.array([0.3, -1.1, 0.7])
    for v in (np.tile([1.0, 2.0, -0.5], (24, 1)), np.cross(w, g)):
        assert np.abs(C @ v.reshape(-1)).max() <= 1e-13 * np.abs(v).max()
    ell = orc.edge_quantities(g, e)[0]
    # d/dt (l0 - l(g + t g)) = -l, row by row
    np.testing.assert_allclose(C @ g.reshape(-1), -ell, rtol=1e-12)


def test_edge_length_gradient_kkt_vs_projected_cg(orc):
    """With barycenter + edge-length rows the projected CG solution matches the dense KKT solve; the
    gradient is tangent to every constraint (C g = 0), and the projected operator has exactly one
    zero eigenvalue per constraint row."""
    n = 40
    c = S.single(S.trefoil(n, 0.01, 7))
    g, e = c.gamma, c.edges
    gr = orc.constraint_groups(g, e, edge_lengths=True)
    dE = orc.differential(g, e)
    prm = orc.Params(cg_tol=1e-12)
    gk, lam = orc.sobolev_gradient(g, e, gr, dE, prm, dense=True)
    gc, res = orc.sobolev_gradient(g, e, gr, dE, prm)
    assert res.converged
    assert np.abs(gk - gc).max() <= 1e-8 * np.abs(gk).max()
    C = orc.jacobian(g, e, gr).reshape(3 + n, -1)
    assert np.abs(C @ gk.reshape(-1)).max() <= 1e-12 * np.abs(gk).max()
    B, B0 = orc.gram_dense(g, e, prm.sigma)
    Ab = np.kron(B + B0, np.eye(3))
    P = np.eye(3 * n) - C.T @ np.linalg.solve(C @ C.T, C)
    ev = np.linalg.eigvalsh(P @ Ab @ P)
    assert np.sum(np.abs(ev) <= 1e-10 * ev[-1]) == 3 + n
    # the edge-length set is stricter than the total length: its gradient differs
    g4, _ = orc.sobolev_gradient(g, e, orc.constraint_groups(g, e), dE, prm, dense=True)
    assert np.abs(g4 - gk).max() >= 1e-3 * np.abs(gk).max()


def test_edge_length_descent_step_keeps_every_edge_length(orc):
    c = S.single(S.trefoil(36, 0.01, 8))
    g, e = c.gamma, c.edges
    gr = orc.constraint_groups(g, e, edge_lengths=True)
    prm = orc.Params()
    g1, info = orc.descent_step(g, e, gr, prm)
    assert info.accepted and info.E_after < info.E_before
    ell0 = orc.edge_quantities(g, e)[0]
    ell1 = orc.edge_quantities(g1, e)[0]
    assert np.abs(ell1 - ell0).max() <= prm.proj_tol * max(1.0, gr[0].L0)
    assert np.abs(orc.phi(g1, e, gr)).max() <= prm.proj_tol * max(1.0, gr[0].L0)


def test_dense_projection_matches_projected_route(orc):
    """Eq. 23 solved as the dense saddle-point system agrees with App. B.3.4's route (z = C^+ b, the
    projected solve, x = z - y) on a moved trefoil: the two formulations of the same projection."""
    g = S.trefoil(96, 0.01, 4)
    e = S.closed_edges(96)
    gr = orc.constraint_groups(g, e)
    prm = orc.Params(proj_cg_tol=1e-12, cg_maxit=200000)
    sig = prm.sigma
    B, B0 = orc.gram_dense(g, e, sig)
    moved = g - 0.05 * orc.differential(g, e) / np.linalg.norm(orc.differential(g, e))
    ap = orc.make_apply(g, e, sig)
    a, ia, oka = orc.constraint_projection(moved, e, gr, ap, prm)
    b, ib, okb = orc.constraint_projection(moved, e, gr, ap, prm, A_dense=B + B0)
    assert oka and okb and ia == ib
    assert np.abs(a - b).max() <= 1e-9 * np.abs(moved - g).max()
    assert np.abs(orc.phi(b, e, gr)).max() <= 1e-10 * max(1.0, gr[0].L0)
