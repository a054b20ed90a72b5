"""Pins of the Barnes-Hut oracle (oracle/bh.py, App. B.1) against facts from outside it: with eps = 0
no node is admissible and the traversal must reproduce the exact discrete energy (Eq. 17) and its
differential, which oracle.py computes independently in C; the node and pair gradients must match
central differences of the terms they differentiate; the hierarchy must partition the edges and
carry consistent node data; the split must be the minimiser a brute-force search finds; and the
approximation error must fall as eps does."""
import numpy as np
import pytest

import synth as S


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle as O
    O.build_library()
    return O


@pytest.fixture(scope="module")
def bh():
    from oracle import bh as B
    return B


def curves():
    return {
        "knot120": S.single(S.fourier_knot(120, 3, 2)),
        "scene": S.scene([S.fourier_knot(40, 2, 1), S.fourier_knot(57, 3, 4)]),
        "open": S.single(S.fourier_knot(50, 3, 9), closed=False),
    }


@pytest.mark.parametrize("name", ["knot120", "scene", "open"])
@pytest.mark.parametrize("ab", [(2.0, 4.5), (3.0, 6.0)])
def test_eps_zero_is_exact(orc, bh, name, ab):
    c = curves()[name]
    a, b = ab
    e0 = orc.energy(c.gamma, c.edges, a, b)
    assert abs(bh.energy(c.gamma, c.edges, 0.0, a, b) / e0 - 1.0) <= 1e-12
    d0 = orc.differential(c.gamma, c.edges, a, b)
    d = bh.differential(c.gamma, c.edges, 0.0, a, b)
    assert np.abs(d - d0).max() <= 1e-12 * np.abs(d0).max()


def _fd(F, g1, g2, h=1e-6):
    E = np.eye(3)
    d1 = np.array([(F(g1 + h * E[k], g2) - F(g1 - h * E[k], g2)) / (2 * h) for k in range(3)])
    d2 = np.array([(F(g1, g2 + h * E[k]) - F(g1, g2 - h * E[k])) / (2 * h) for k in range(3)])
    return d1, d2


@pytest.mark.parametrize("ab", [(2.0, 4.5), (3.0, 6.0), (2.0, 4.2)])
def test_gradients_match_central_differences(bh, ab):
    a, b = ab
    rng = np.random.default_rng(3)
    g1 = rng.normal(size=3)
    g2 = g1 + 0.1 * rng.normal(size=3)
    q1 = np.array([1.0, 0.3, 0.2])
    q2 = q1 + 0.1 * rng.normal(size=3)
    xbar, Tbar, L = np.array([2.0, 1.0, 0.5]), np.array([0.3, 0.5, 0.2]), 0.7

    def node(u, v):
        e = v - u
        l = np.linalg.norm(e)
        x = 0.5 * (u + v)
        return L * l * (bh.kernel(x, xbar, e / l, a, b) + bh.kernel(xbar, x, Tbar, a, b))

    def pair(u, v):
        e, f = v - u, q2 - q1
        l, lj = np.linalg.norm(e), np.linalg.norm(f)
        s = sum(0.25 * (bh.kernel(p, q, e / l, a, b) + bh.kernel(q, p, f / lj, a, b)) for p in (u, v) for q in (q1, q2))
        return l * lj * s

    for F, G in ((node, bh.node_target_grad(g1, g2, L, xbar, Tbar, a, b)),
                 (pair, bh.pair_target_grad(g1, g2, q1, q2, a, b))):
        f1, f2 = _fd(F, g1, g2)
        scale = max(np.abs(f1).max(), np.abs(f2).max())
        assert np.abs(G[0] - f1).max() <= 1e-6 * scale
        assert np.abs(G[1] - f2).max() <= 1e-6 * scale


def test_hierarchy_partitions_edges_and_node_data(bh):
    c = S.single(S.fourier_knot(300, 5, 3))
    x, T, ell, ends = bh.edge_points(c.gamma, c.edges)
    nodes, perm = bh.build_bvh(x, T, ell, ends, leaf_size=8)
    assert sorted(perm.tolist()) == list(range(300))
    seen = np.zeros(300, dtype=int)
    for nd in nodes:
        items = perm[nd["b"]:nd["e"]]
        assert abs(nd["L"] - ell[items].sum()) <= 1e-12 * nd["L"]
        xl, xh = x[items].min(0), x[items].max(0)
        assert np.all(nd["xbar"] >= xl - 1e-12) and np.all(nd["xbar"] <= xh + 1e-12)
        p1, p2 = ends[0][items], ends[1][items]
        box = np.maximum(p1, p2).max(0) - np.minimum(p1, p2).min(0)
        assert abs(nd["rx"] - 0.5 * np.sqrt(box @ box)) <= 1e-12 * max(nd["rx"], 1e-300)
        assert nd["rx"] >= 0.5 * ell[items].max() * (1 - 1e-12)  # the box holds every edge
        if nd["left"] < 0:
            assert 1 <= len(items) <= 8
            seen[items] += 1
        else:
            l, r = nodes[nd["left"]], nodes[nd["right"]]
            assert (l["b"], l["e"], r["b"], r["e"]) == (nd["b"], l["e"], l["e"], nd["e"])
            assert abs(l["L"] + r["L"] - nd["L"]) <= 1e-12 * nd["L"]
            # halves, and the coordinate whose median split minimises the children's squared 6-D diagonals
            assert l["e"] - l["b"] == len(items) // 2
            P = np.hstack([T, x])[items]
            best = np.inf
            for cc in range(6):
                o = np.lexsort((items, P[:, cc]))
                Q = P[o]
                k = len(items) // 2
                dl, dr = Q[:k].max(0) - Q[:k].min(0), Q[k:].max(0) - Q[k:].min(0)
                best = min(best, float(dl @ dl + dr @ dr))
            PL, PR = np.hstack([T, x])[perm[l["b"]:l["e"]]], np.hstack([T, x])[perm[r["b"]:r["e"]]]
            dl, dr = PL.max(0) - PL.min(0), PR.max(0) - PR.min(0)
            assert float(dl @ dl + dr @ dr) <= best * (1 + 1e-12)
    assert np.all(seen == 1)


def test_error_falls_with_eps(orc, bh):
    c = S.single(S.fourier_knot(200, 4, 5))
    e0 = orc.energy(c.gamma, c.edges)
    d0 = orc.differential(c.gamma, c.edges)
    errs, derrs, work = [], [], []
    for eps in (0.3, 0.15, 0.05):
        errs.append(abs(bh.energy(c.gamma, c.edges, eps) / e0 - 1.0))
        d = bh.differential(c.gamma, c.edges, eps)
        derrs.append(np.abs(d - d0).max() / np.abs(d0).max())
        work.append(sum(bh.admissible_count(c.gamma, c.edges, eps)))
    # measured: energy 4.1e-3, 7.4e-4, 4.0e-5; differential (largest entry) 0.14, 0.012, 1.3e-3 -- the
    # differential is the rougher one, as each edge's endpoints take their own admissibility
    # decisions and a vertex sums two edges whose rows nearly cancel
    assert errs[0] > errs[1] > errs[2] and errs[2] <= 1e-4
    assert derrs[0] > derrs[1] > derrs[2] and derrs[2] <= 3e-3
    assert work[0] < work[1] < work[2]
