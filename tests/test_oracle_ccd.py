"""Pins of the oracle's collision time (Sec. 5.4, the isotopy-safe start of the line search):
closed-form crossings, coplanar motion, invariances, and brute force over sampled times."""
import numpy as np
import pytest

import synth as S


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle as O
    return O


Z = np.zeros(3)


def test_transversal_crossing_closed_form(orc):
    # I on the x axis at rest; J parallel to y at height 1 moving down with speed v: contact at 1 / v
    a, b = np.array([-1.0, 0, 0]), np.array([1.0, 0, 0])
    c, e = np.array([0.0, -1, 1]), np.array([0.0, 1, 1])
    for v in (1.0, 2.5, 0.8):
        dv = np.array([0, 0, v])  # gamma - tau d moves by -tau d
        assert orc.pair_collision_time(a, b, Z, Z, c, e, dv, dv, 1.5) == pytest.approx(1.0 / v, rel=1e-14) \
            or 1.0 / v > 1.5
    # beyond the horizon: no contact reported
    assert orc.pair_collision_time(a, b, Z, Z, c, e, np.array([0, 0, 0.5]), np.array([0, 0, 0.5]), 1.5) == np.inf
    # J passes beside I (shifted past its end): coplanar at tau = 1 but never touching
    assert orc.pair_collision_time(a, b, Z, Z, c + [3, 0, 0], e + [3, 0, 0], [0, 0, 1.0], [0, 0, 1.0], 1.5) == np.inf


def test_rotating_segment_closed_form(orc):
    # J's far end swings down through I: J from (0,-1,1) to (0,1,1), the end e moves by (0,0,-2 tau);
    # the segment touches the x axis when its line passes z = 0 at y = 0 within both segments:
    # z(y) = 1 + (y + 1) / 2 * (-2 tau) = 0 at y = 0  ->  tau = 1
    a, b = np.array([-1.0, 0, 0]), np.array([1.0, 0, 0])
    c, e = np.array([0.0, -1, 1]), np.array([0.0, 1, 1])
    t = orc.pair_collision_time(a, b, Z, Z, c, e, Z, np.array([0, 0, 2.0]), 1.5)
    assert t == pytest.approx(1.0, rel=1e-12)


def test_coplanar_motion_vertex_hits_segment(orc):
    # everything in the plane z = 0: J (parallel, above I) moves down with speed 1, its endpoints land
    # on I at tau = 1; a shorter approach speed gives 1 / v
    a, b = np.array([0.0, 0, 0]), np.array([1.0, 0, 0])
    c, e = np.array([0.25, 1, 0]), np.array([0.75, 1, 0])
    for v in (1.0, 2.0):
        dy = np.array([0, v, 0])
        assert orc.pair_collision_time(a, b, Z, Z, c, e, dy, dy, 1.5) == pytest.approx(1.0 / v, rel=1e-12)
    # sliding along x only: never touching
    dx = np.array([1.0, 0, 0])
    assert orc.pair_collision_time(a, b, Z, Z, c, e, dx, dx, 1.5) == np.inf


def test_invariances(orc):
    rng = np.random.default_rng(3)
    a, b = np.array([-1.0, 0, 0]), np.array([1.0, 0.1, 0])
    c, e = np.array([0.1, -1, 0.7]), np.array([-0.1, 1, 0.9])
    da, db = rng.normal(0, 0.1, 3), rng.normal(0, 0.1, 3)
    dc, de = np.array([0.05, 0, 1.0]), np.array([0, 0.05, 1.1])
    t0 = orc.pair_collision_time(a, b, da, db, c, e, dc, de, 1.5)
    assert 0 < t0 < 1.5
    # rigid motion (rotation of positions and directions, translation of positions)
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]]) @ \
        np.array([[1, 0, 0], [0, np.cos(1.1), -np.sin(1.1)], [0, np.sin(1.1), np.cos(1.1)]])
    sh = np.array([3.0, -2, 5])
    t1 = orc.pair_collision_time(R @ a + sh, R @ b + sh, R @ da, R @ db, R @ c + sh, R @ e + sh, R @ dc, R @ de, 1.5)
    assert t1 == pytest.approx(t0, rel=1e-9)
    # scaling positions and directions together leaves tau; scaling directions alone divides it
    t2 = orc.pair_collision_time(2 * a, 2 * b, 2 * da, 2 * db, 2 * c, 2 * e, 2 * dc, 2 * de, 1.5)
    assert t2 == pytest.approx(t0, rel=1e-9)
    t3 = orc.pair_collision_time(a, b, 2 * da, 2 * db, c, e, 2 * dc, 2 * de, 1.5)
    assert t3 == pytest.approx(t0 / 2, rel=1e-9)
    # the roles of the two segments and the orientation of each do not matter
    assert orc.pair_collision_time(c, e, dc, de, a, b, da, db, 1.5) == pytest.approx(t0, rel=1e-9)
    assert orc.pair_collision_time(b, a, db, da, e, c, de, dc, 1.5) == pytest.approx(t0, rel=1e-9)


def _brute_first_contact(g, e, d, T, samples):
    """First sampled tau where some disjoint pair's distance falls below its own running minimum
    bound: the sampled distance curve of each pair, and its first local minimum near zero."""
    ts = np.linspace(0.0, T, samples)
    h = ts[1] - ts[0]
    first = np.inf
    for I in range(len(e)):
        for J in range(I + 1, len(e)):
            a, b = e[I]
            c, f = e[J]
            if len({a, b, c, f}) < 4:
                continue
            P = g[[a, b, c, f]][None] - ts[:, None, None] * d[[a, b, c, f]][None]
            from oracle.oracle import segment_distance
            dist = np.array([segment_distance(p[0], p[1], p[2], p[3]) for p in P])
            speed = np.abs(np.diff(dist)).max() / h + 1e-300
            hit = np.nonzero(dist <= speed * h)[0]
            if hit.size:
                first = min(first, ts[hit[0]])
    return first


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_first_collision_time_against_sampled_distances(orc, seed):
    """A 10-gon knot with a random motion large enough to cross strands (seeds 0, 2, 3 collide inside
    the horizon, seed 1 does not): the cubic's first contact lies within two samples of the first
    sampled distance that reaches zero."""
    n = 10
    g = S.fourier_knot(n, 3, 40 + seed)
    e = S.closed_edges(n)
    d = np.random.default_rng(seed).normal(0, 2.0, (n, 3))
    T = 1.5
    t = orc.first_collision_time(g, e, d, T)[0]
    samples = 3001
    tb = _brute_first_contact(g, e, d, T, samples)
    h = T / (samples - 1)
    assert (tb == np.inf) == (seed == 1)
    if tb == np.inf:
        assert t == T
    else:
        assert t < T and abs(t - tb) <= 2 * h
    # no motion: no collision
    assert orc.first_collision_time(g, e, np.zeros_like(g), T)[0] == T


def test_isotopy_safe_descent_step_starts_below_the_collision(orc):
    c = S.single(S.trefoil(40, 0.01, 1))
    g, e = c.gamma, c.edges
    gr = orc.constraint_groups(g, e)
    prm = orc.Params(isotopy_safe=True)
    g1, info = orc.descent_step(g, e, gr, prm)
    assert info.accepted and info.E_after < info.E_before
    # the accepted tau is 2/3 of min(first collision, horizon) halved h times
    dE = orc.differential(g, e)
    gt, _ = orc.sobolev_gradient(g, e, gr, dE, prm)
    dd = gt / np.linalg.norm(gt)
    tmax = orc.first_collision_time(g, e, dd, prm.ccd_horizon)[0]
    assert info.tau == pytest.approx(2.0 / 3.0 * tmax * 0.5 ** info.halvings, rel=1e-9)
