"""Pins of the oracle's energy and differential to facts fixed by the paper and by mathematics
(Sec. 5.1, Eqs. 3, 17-18).  CPU only."""
import math
import os

import numpy as np
import pytest

import synth as S

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden_square():
    rows = []
    with open(os.path.join(HERE, "golden", "square_energy.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(tuple(float(x) for x in line.split()))
    return rows


def _rot(seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    return q


@pytest.mark.parametrize("row", _golden_square())
def test_square_closed_form(orc, row):
    alpha, beta, E, c = row
    g, e = S.unit_square(), S.closed_edges(4)
    assert abs(orc.energy(g, e, alpha, beta) - E) <= 1e-15 * E
    dE = orc.differential(g, e, alpha, beta)
    rhat = g / np.linalg.norm(g, axis=1, keepdims=True)
    np.testing.assert_allclose(dE, c * rhat, rtol=0, atol=1e-14)


def test_too_few_edges_and_straight_line_have_zero_energy(orc):
    tri = np.array([[0., 0, 0], [1, 0, 0], [0, 1, 0]])
    assert orc.energy(tri, S.closed_edges(3)) == 0.0          # every pair shares a vertex
    line = np.stack([np.linspace(0, 3, 12), np.zeros(12), np.zeros(12)], 1)
    assert orc.energy(line, S.open_edges(12)) == 0.0           # T x d = 0 for every pair
    assert np.all(orc.differential(line, S.open_edges(12)) == 0.0)


@pytest.mark.parametrize("ab", [(2.0, 4.5), (3.0, 6.0)])
def test_rigid_motion_reflection_scaling(orc, ab):
    alpha, beta = ab
    c = S.single(S.trefoil(48, 0.01, 3))
    E = orc.energy(c.gamma, c.edges, alpha, beta)
    R = _rot(1)
    g2 = c.gamma @ R.T + np.array([0.3, -2.0, 5.0])
    assert abs(orc.energy(g2, c.edges, alpha, beta) - E) <= 1e-12 * E
    refl = c.gamma * np.array([-1.0, 1.0, 1.0])
    assert abs(orc.energy(refl, c.edges, alpha, beta) - E) <= 1e-12 * E
    lam = 1.7
    # hat-E(lambda gamma) = lambda^(2 + alpha - beta) hat-E(gamma): kernel lambda^(alpha-beta), measure lambda^2
    assert abs(orc.energy(lam * c.gamma, c.edges, alpha, beta) - lam ** (2 + alpha - beta) * E) <= 1e-12 * E


def test_orientation_and_relabelling(orc):
    c = S.single(S.fourier_knot(40, 4, 7))
    E = orc.energy(c.gamma, c.edges)
    flipped = c.edges[:, ::-1].copy()          # reversing every edge flips T_I, |T x d| unchanged
    assert abs(orc.energy(c.gamma, flipped) - E) <= 1e-12 * E
    perm = np.random.default_rng(2).permutation(40)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(40)
    g2 = c.gamma[perm]                          # new vertex k is old vertex perm[k]
    e2 = inv[c.edges].astype(np.int32)
    eperm = np.random.default_rng(3).permutation(40)
    assert abs(orc.energy(g2, e2[eperm]) - E) <= 1e-12 * E


def test_rows_sum_to_total(orc):
    c = S.single(S.trefoil(64, 0.01, 0))
    E, rows = orc.energy(c.gamma, c.edges, rows=True)
    assert abs(rows.sum() - E) <= 1e-13 * E
    sub = orc.energy_rows(c.gamma, c.edges, [0, 5, 63])
    np.testing.assert_allclose(sub, rows[[0, 5, 63]], rtol=1e-15)


def test_zero_length_edge_is_an_error(orc):
    g = S.unit_square()
    g[1] = g[0]
    with pytest.raises(orc.OracleError):
        orc.energy(g, S.closed_edges(4))


@pytest.mark.parametrize("ab", [(2.0, 4.5), (3.0, 6.0)])
def test_differential_central_differences(orc, ab):
    alpha, beta = ab
    c = S.single(S.fourier_knot(24, 3, 11))
    g, e = c.gamma, c.edges
    dE = orc.differential(g, e, alpha, beta)
    h = 1e-6
    fd = np.zeros_like(g)
    for v in range(g.shape[0]):
        for k in range(3):
            gp, gm = g.copy(), g.copy()
            gp[v, k] += h
            gm[v, k] -= h
            fd[v, k] = (orc.energy(gp, e, alpha, beta) - orc.energy(gm, e, alpha, beta)) / (2 * h)
    assert np.abs(fd - dE).max() <= 1e-6 * np.abs(dE).max()


def test_differential_invariants(orc):
    alpha, beta = 2.0, 4.5
    c = S.single(S.trefoil(96, 0.01, 0))
    g, e = c.gamma, c.edges
    E = orc.energy(g, e, alpha, beta)
    dE = orc.differential(g, e, alpha, beta)
    scale = np.abs(dE).max() * np.abs(g).max() * len(g)
    assert np.abs(dE.sum(0)).max() <= 1e-12 * scale                       # translation
    assert np.abs(np.cross(g, dE).sum(0)).max() <= 1e-12 * scale           # rotation
    # Euler's identity for a function homogeneous of degree 2 + alpha - beta
    assert abs((g * dE).sum() - (2 + alpha - beta) * E) <= 1e-12 * abs(E) * 10
    sel = [0, 17, 95]
    np.testing.assert_allclose(orc.differential_at(g, e, sel, alpha, beta), dE[sel], rtol=0,
                               atol=1e-13 * np.abs(dE).max())


def test_two_curves_graph(orc):
    sc = S.scene([S.fourier_knot(20, 3, 1), S.fourier_knot(28, 3, 2)], spacing=2.0)
    E = orc.energy(sc.gamma, sc.edges)
    E1 = orc.energy(*sc.curve(0))
    E2 = orc.energy(*sc.curve(1))
    assert E > E1 + E2       # the cross pairs add positive energy
    dE = orc.differential(sc.gamma, sc.edges)
    assert np.abs(dE.sum(0)).max() <= 1e-12 * np.abs(dE).max() * len(dE)
