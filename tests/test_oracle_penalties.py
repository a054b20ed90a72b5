"""Pins of the oracle's penalties (Sec. 8.1): closed forms, homogeneity, invariances and central
differences of the energies."""
import numpy as np
import pytest

import synth as S


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle as O
    return O


def test_closed_forms(orc):
    sq, e4 = S.unit_square(), S.closed_edges(4)
    # field along x: the two edges along y have |T x X| = 1, the two along x 0
    assert orc.penalty_energy(sq, e4, orc.Penalties(w_field=1.0, field_b=np.array([1.0, 0, 0]))) == pytest.approx(2.0)
    # field normal to the plane: every edge counts its full length
    assert orc.penalty_energy(sq, e4, orc.Penalties(w_field=1.0, field_b=np.array([0, 0, 3.0]))) == pytest.approx(4.0)
    # total length of a regular n-gon of circumradius R
    for n in (5, 12):
        g = S.regular_polygon(n, 1.3)
        E = orc.penalty_energy(g, S.closed_edges(n), orc.Penalties(w_length=2.0))
        assert E == pytest.approx(2.0 * n * 2 * 1.3 * np.sin(np.pi / n), rel=1e-14)
    # a 2 x 1 rectangle: every vertex joins a long and a short edge, (2 - 1)^2 each
    rect = np.array([[0.0, 0, 0], [2, 0, 0], [2, 1, 0], [0, 1, 0]])
    assert orc.penalty_energy(rect, e4, orc.Penalties(w_length_diff=1.0)) == pytest.approx(4.0)
    # an open chain: its two end vertices have degree 1 and no term
    chain = np.array([[0.0, 0, 0], [2, 0, 0], [2, 1, 0], [0, 1, 0]])
    assert orc.penalty_energy(chain, S.open_edges(4), orc.Penalties(w_length_diff=1.0)) == pytest.approx(2.0)


def test_regular_polygon_is_stationary_for_the_length_difference(orc):
    g = S.regular_polygon(9, 1.0)
    e = S.closed_edges(9)
    pen = orc.Penalties(w_length_diff=1.0)
    assert orc.penalty_energy(g, e, pen) == pytest.approx(0.0, abs=1e-28)
    assert np.abs(orc.penalty_gradient(g, e, pen)).max() <= 1e-14


def test_homogeneity_and_translation(orc):
    g = S.trefoil(30, 0.02, 3)
    e = S.closed_edges(30)
    p1 = orc.Penalties(w_length=0.7, w_field=1.3, field_b=np.array([0.2, -0.5, 0.8]))
    p2 = orc.Penalties(w_length_diff=2.0)
    for pen, deg in ((p1, 1.0), (p2, 2.0)):
        E = orc.penalty_energy(g, e, pen)
        G = orc.penalty_gradient(g, e, pen)
        # Euler: both terms are homogeneous of degree deg in the positions (a constant field)
        assert float((g * G).sum()) == pytest.approx(deg * E, rel=1e-12)
        # translation invariance
        assert np.abs(G.sum(0)).max() <= 1e-12 * np.abs(G).max()


def test_gradient_matches_central_differences(orc):
    g = S.fourier_knot(24, 3, 17)
    e = S.closed_edges(24)
    M = np.array([[0.0, -1.0, 0.2], [1.0, 0.0, 0.0], [0.3, 0.0, 0.1]])  # a swirling, non-constant field
    pen = orc.Penalties(w_length=0.4, w_length_diff=1.7, w_field=2.2, field_M=M, field_b=np.array([0.1, 0.2, 0.5]))
    G = orc.penalty_gradient(g, e, pen)
    h = 1e-6
    F = np.zeros_like(g)
    for v in range(g.shape[0]):
        for k in range(3):
            gp, gm = g.copy(), g.copy()
            gp[v, k] += h
            gm[v, k] -= h
            F[v, k] = (orc.penalty_energy(gp, e, pen) - orc.penalty_energy(gm, e, pen)) / (2 * h)
    assert np.abs(F - G).max() <= 1e-7 * np.abs(G).max()
