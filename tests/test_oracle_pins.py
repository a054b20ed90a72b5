"""Pins of the oracle's point, tangent and surface constraints (Sec. 8.1: a vertex held at a target
position, an edge's tangent held at a unit vector, a vertex held on a quadric surface) combined with the
total length and no barycenter row.  CPU only.

The constrained gradient of Eq. 22 is checked against a route that shares nothing with the oracle's
Jacobian: the velocity space is reduced by deleting the pinned vertices' coordinates and then taking
the null space of complex-step derivatives of the length, of the tangents themselves and of the
surface function; on that space the gradient solves the reduced Gram system."""
import numpy as np
import pytest
import scipy.linalg as sla

import synth as S

SIG = (4.5 - 1.0) / 2.0 - 1.0


def total_length(gamma, edges):
    d = gamma[edges[:, 1]] - gamma[edges[:, 0]]
    return np.sqrt((d * d).sum(1)).sum()   # no conjugation: valid for complex-step arguments


def length_gradient_complex_step(gamma, edges):
    h = 1e-30
    out = np.zeros_like(gamma)
    for v in range(gamma.shape[0]):
        for k in range(3):
            gc = gamma.astype(np.complex128)
            gc[v, k] += 1j * h
            out[v, k] = total_length(gc, edges).imag / h
    return out


def reduced_gradient(gamma, edges, A, dE, pins):
    """argmin 1/2 g^T A-bar g - dE^T g over {g : g_v = 0 at the pins, dL . g = 0}, in component-major
    coordinates with the pinned coordinates deleted."""
    n = gamma.shape[0]
    free_v = np.setdiff1d(np.arange(n), pins)
    idx = np.concatenate([k * n + free_v for k in range(3)])   # component-major indices kept
    Ab = np.kron(np.eye(3), A)[np.ix_(idx, idx)]
    dL = length_gradient_complex_step(gamma, edges).T.reshape(-1)[idx]
    Z = sla.null_space(dL[None, :])
    b = dE.T.reshape(-1)[idx]
    gf = Z @ np.linalg.solve(Z.T @ Ab @ Z, Z.T @ b)
    g = np.zeros(3 * n)
    g[idx] = gf
    return g.reshape(3, n).T


@pytest.mark.parametrize("case", ["closed_one", "closed_many", "open_ends"])
def test_pinned_gradient_matches_reduced_space_solve(orc, case):
    if case == "open_ends":
        c = S.single(S.fourier_knot(18, 3, 11), closed=False)
        pins = np.array([0, 17])
    else:
        c = S.single(S.trefoil(22, 0.01, 12))
        pins = np.array([5]) if case == "closed_one" else np.array([0, 3, 9, 10, 16])
    g, e = c.gamma, c.edges
    gr = orc.constraint_groups(g, e, pins=pins, barycenter=False)
    assert gr[0].n_rows == 1 + 3 * len(pins)
    dE = orc.differential(g, e)
    gk, _ = orc.sobolev_gradient(g, e, gr, dE, orc.Params(), dense=True)
    B, B0 = orc.gram_dense(g, e, SIG)
    gr_ = reduced_gradient(g, e, B + B0, dE, pins)
    assert np.abs(gk[pins]).max() <= 1e-12 * np.abs(gk).max()
    np.testing.assert_allclose(gk, gr_, rtol=0, atol=1e-9 * np.abs(gr_).max())
    # the barycenter is free: this gradient moves it, unlike the one of the barycenter + length set
    ell, _, x = orc.edge_quantities(g, e)
    assert np.abs((ell[:, None] * 0.5 * (gk[e[:, 0]] + gk[e[:, 1]])).sum(0)).max() > 1e-6 * np.abs(gk).max()


def test_pin_rows_match_differences(orc):
    """Point rows (Phi_v = gamma_v - p0_v) and the length row against central differences of phi."""
    c = S.single(S.trefoil(12, 0.01, 13))
    g, e = c.gamma, c.edges
    gr = orc.constraint_groups(g, e, pins=np.array([2, 7]), barycenter=False)
    assert np.abs(orc.phi(g, e, gr)).max() <= 1e-13
    C = orc.jacobian(g, e, gr)
    h = 1e-6
    J = np.zeros_like(C)
    for v in range(12):
        for k in range(3):
            gp, gm = g.copy(), g.copy()
            gp[v, k] += h
            gm[v, k] -= h
            J[:, v, k] = (orc.phi(gp, e, gr) - orc.phi(gm, e, gr)) / (2 * h)
    assert np.abs(J - C).max() <= 1e-8


def test_regular_polygon_with_a_pin_is_critical(orc):
    """On a regular polygon dE is radial and uniform, a multiple of the length row's gradient, so the
    pinned problem is at a critical point too: g = 0 (the pin's multiplier vanishes)."""
    n = 16
    g = S.regular_polygon(n, 1.3)
    e = S.closed_edges(n)
    gr = orc.constraint_groups(g, e, pins=np.array([4]), barycenter=False)
    dE = orc.differential(g, e)
    gk, _ = orc.sobolev_gradient(g, e, gr, dE, orc.Params(), dense=True)
    assert np.abs(gk).max() <= 1e-9 * np.abs(dE).max()


def test_projection_restores_pins_and_length(orc):
    """Sec. 5.3.2 with point rows: from a curve whose pinned vertices moved and whose length changed,
    the projection returns the pins to their targets and the length to L0."""
    c = S.single(S.fourier_knot(30, 3, 14), closed=False)
    g, e = c.gamma, c.edges
    pins = np.array([0, 29, 12])
    gr = orc.constraint_groups(g, e, pins=pins, barycenter=False)
    rng = np.random.default_rng(15)
    moved = g + 2e-3 * rng.normal(size=g.shape)
    prm = orc.Params(proj_cg_tol=1e-12)
    out, it, ok = orc.constraint_projection(moved, e, gr, orc.make_apply(g, e, SIG), prm)
    assert ok and 1 <= it <= 4
    assert np.abs(out[pins] - g[pins]).max() <= 1e-10
    assert abs(total_length(out, e) - total_length(g, e)) <= 1e-10 * total_length(g, e)


def test_descent_with_pins_keeps_them_and_lowers_energy(orc):
    c = S.single(S.fourier_knot(24, 3, 16), closed=False)
    g, e = c.gamma, c.edges
    pins = np.array([0, 23])
    gr = orc.constraint_groups(g, e, pins=pins, barycenter=False)
    prm = orc.Params(cg_tol=1e-10, proj_cg_tol=1e-10)
    E = orc.energy(g, e)
    cur = g.copy()
    for _ in range(3):
        cur, info = orc.descent_step(cur, e, gr, prm)
        assert info.accepted and info.E_after < E
        E = info.E_after
        assert np.abs(cur[pins] - g[pins]).max() <= 1e-10
        assert abs(total_length(cur, e) - gr[0].L0) <= 1e-10 * gr[0].L0


# ------------------------------------------------------------------ tangent and surface rows (Sec. 8.1)

def _sphere(center, radius):
    """Quadric (Q, b, c) of |x - center|^2 - radius^2."""
    center = np.asarray(center, dtype=np.float64)
    return np.eye(3), -2.0 * center, float(center @ center - radius * radius)


def _plane_through(p, q, r):
    n = np.cross(q - p, r - p)
    n /= np.linalg.norm(n)
    return np.zeros((3, 3)), n, -float(n @ p)


def _complex_step_rows(fun, gamma):
    """Jacobian [m, nV, 3] of fun (complex-safe, R^{nV x 3} -> R^m) by complex steps."""
    h = 1e-30
    m = len(fun(gamma.astype(np.complex128)))
    J = np.zeros((m, gamma.shape[0], 3))
    for v in range(gamma.shape[0]):
        for k in range(3):
            gc = gamma.astype(np.complex128)
            gc[v, k] += 1j * h
            J[:, v, k] = fun(gc).imag / h
    return J


def _tangent(gamma, edges, I):
    d = gamma[edges[I, 1]] - gamma[edges[I, 0]]
    return d / np.sqrt((d * d).sum())


def test_tangent_and_surface_rows_match_differences(orc):
    c = S.single(S.fourier_knot(14, 3, 21), closed=False)
    g, e = c.gamma, c.edges
    X = np.array([[0.3, -0.5, 0.8], [1.0, 0.2, -0.1]])
    quad = _sphere(g.mean(0), 0.7)
    gr = orc.constraint_groups(g, e, pins=np.array([0]), barycenter=False, tangents=np.array([0, 12]), X=X,
                               surf=np.array([5, 9]), quad=quad)
    assert gr[0].n_rows == 1 + 3 + 4 + 2
    C = orc.jacobian(g, e, gr)
    h = 1e-6
    J = np.zeros_like(C)
    for v in range(14):
        for k in range(3):
            gp, gm = g.copy(), g.copy()
            gp[v, k] += h
            gm[v, k] -= h
            J[:, v, k] = (orc.phi(gp, e, gr) - orc.phi(gm, e, gr)) / (2 * h)
    assert np.abs(J - C).max() <= 1e-8 * max(1.0, np.abs(C).max())
    # the two tangent rows of an edge vanish exactly when T_I = X_I
    gr0 = orc.constraint_groups(g, e, pins=np.array([0]), barycenter=False, tangents=np.array([3]))
    assert np.abs(orc.phi(g, e, gr0)).max() <= 1e-15


@pytest.mark.parametrize("closed", [True, False])
def test_gradient_with_tangents_and_surface_matches_reduced_space_solve(orc, closed):
    """The velocity space is {g : g = 0 at the pins, dL g = 0, dT_I g = 0, df(gamma_v) g = 0}, built
    from complex-step derivatives of the length, of T_I itself (three rows of rank 2) and of f, not
    from the oracle's rows; the oracle's KKT gradient must be the reduced solve on it."""
    if closed:
        c = S.single(S.trefoil(24, 0.01, 22))
        pins, tans, surf = np.array([2]), np.array([6, 15]), np.array([10, 20])
    else:
        c = S.single(S.fourier_knot(22, 3, 23), closed=False)
        pins, tans, surf = np.array([0, 21]), np.array([0, 20]), np.array([11])
    g, e = c.gamma, c.edges
    quad = _sphere(g[surf].mean(0) + np.array([0.1, -0.2, 0.05]), 0.9)
    gr = orc.constraint_groups(g, e, pins=pins, barycenter=False, tangents=tans, surf=surf, quad=quad)
    dE = orc.differential(g, e)
    gk, _ = orc.sobolev_gradient(g, e, gr, dE, orc.Params(), dense=True)
    Q, b, c0 = quad

    def rows(x):
        out = [total_length(x, e)]
        for I in tans:
            out.extend(list(_tangent(x, e, I)))
        for v in surf:
            out.append(x[v] @ Q @ x[v] + b @ x[v] + c0)
        return np.array(out)

    J = _complex_step_rows(rows, g)
    n = g.shape[0]
    Jcm = np.stack([J[r].T.reshape(-1) for r in range(J.shape[0])])
    for v in pins:                      # pinned coordinates, component-major
        for k in range(3):
            row = np.zeros(3 * n)
            row[k * n + v] = 1.0
            Jcm = np.vstack([Jcm, row])
    Z = sla.null_space(Jcm)
    B, B0 = orc.gram_dense(g, e, SIG)
    Ab = np.kron(np.eye(3), B + B0)
    gz = Z @ np.linalg.solve(Z.T @ Ab @ Z, Z.T @ dE.T.reshape(-1))
    ref = gz.reshape(3, n).T
    np.testing.assert_allclose(gk, ref, rtol=0, atol=1e-9 * np.abs(ref).max())
    assert Z.shape[1] == 3 * n - (1 + 2 * len(tans) + len(surf) + 3 * len(pins))


def test_projection_reaches_tangent_and_surface_targets(orc):
    """From a perturbed open curve the projection restores the end pins, rotates the end edges onto
    their target tangents, and returns three vertices to the plane through them."""
    c = S.single(S.fourier_knot(30, 3, 24), closed=False)
    g, e = c.gamma, c.edges
    pins, tans, surf = np.array([0, 29]), np.array([0, 28]), np.array([10, 15, 20])
    quad = _plane_through(*g[surf])
    T = orc.edge_quantities(g, e)[1]
    X = np.array([T[0] + [0.0, 0.01, 0.0], T[28] + [0.01, 0.0, -0.01]])
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    gr = orc.constraint_groups(g, e, pins=pins, barycenter=False, tangents=tans, X=X, surf=surf, quad=quad)
    rng = np.random.default_rng(25)
    moved = g + 1e-3 * rng.normal(size=g.shape)
    out, it, ok = orc.constraint_projection(moved, e, gr, orc.make_apply(g, e, SIG), orc.Params(proj_cg_tol=1e-12))
    assert ok and 1 <= it <= 5
    assert np.abs(out[pins] - g[pins]).max() <= 1e-10
    for I, x in zip(tans, X):
        assert np.abs(_tangent(out, e, I) - x).max() <= 1e-10
    f, _ = orc.quadric(out[surf], *quad)
    assert np.abs(f).max() <= 1e-10
    assert abs(total_length(out, e) - gr[0].L0) <= 1e-10 * gr[0].L0


def test_descent_with_tangents_and_surface_keeps_them(orc):
    c = S.single(S.fourier_knot(26, 3, 26), closed=False)
    g, e = c.gamma, c.edges
    pins, tans, surf = np.array([0, 25]), np.array([0, 24]), np.array([12])
    quad = _sphere(np.zeros(3), float(np.linalg.norm(g[12])))
    gr = orc.constraint_groups(g, e, pins=pins, barycenter=False, tangents=tans, surf=surf, quad=quad)
    T0 = orc.edge_quantities(g, e)[1][tans]
    prm = orc.Params(cg_tol=1e-10, proj_cg_tol=1e-10)
    cur, E = g.copy(), orc.energy(g, e)
    for _ in range(2):
        cur, info = orc.descent_step(cur, e, gr, prm)
        assert info.accepted and info.E_after < E
        E = info.E_after
        assert np.abs(orc.edge_quantities(cur, e)[1][tans] - T0).max() <= 1e-9
        assert abs(np.linalg.norm(cur[12]) - np.linalg.norm(g[12])) <= 1e-10
