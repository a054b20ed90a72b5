"""Barnes-Hut approximation of the discrete tangent-point energy and of its differential (App. B.1),
written plainly in numpy / Python loops for small curves.

TEST INFRASTRUCTURE ONLY: the tests and the benchmark's CPU-baseline leg may import this module; the
CUDA library never does, and this module never touches the CUDA library.  Its exact limit is the
discrete energy of Eq. 17 and its differential, which oracle.py computes independently.

What it computes, in the appendix's order:

  * tangent-points p_I = (T_I, x_I) in R^6 per edge (x_I the midpoint, T_I the unit tangent) and a
    bounding volume hierarchy over them: a node with more than `leaf_size` edges is split into two
    halves at the median of one of the six coordinates, the one whose split minimises the sum of the
    squared diameters of the two children's 6-D bounding boxes;
  * per node: mass L_N = sum l_I, centre x_N = sum l_I x_I / L_N, tangent T_N = sum l_I T_I / L_N,
    and the radii r_x, r_T (half the diagonals of the node's spatial box, over the edges' endpoints,
    and of its tangential box);
  * energy (Eq. BVHNodeTPE): a traversal from the root per target edge I; a node is admissible when
    r_x < eps |x_I - x_N| and r_T < eps (Eq. BarnesHutCondition) and then contributes
    l_I L_N |T_I x (x_I - x_N)|^alpha / |x_I - x_N|^beta; a leaf that is not admissible contributes
    its edges J (disjoint from I) exactly, l_I l_J khat_IJ with the discrete kernel of Eq. 18;
  * differential: the same traversal; an admissible node adds
    L_N d/d gamma_{i_a} [ l_I (k(x_I, x_N, T_I) + k(x_N, x_I, T_N)) ] to the target's endpoints
    (x_N, T_N, L_N held fixed), a leaf adds the target-side derivatives of l_I l_J (khat_IJ + khat_JI).

Readings (listed with their reasons in the design notes):
  * leaves use the trapezoid kernel khat of Eq. 18 rather than the midpoint kernel the appendix
    prints for them, so that eps -> 0 reproduces Eq. 17 exactly;
  * admissibility is strict (<), so that eps = 0 admits no node, not even a one-edge node;
  * a node that holds the target edge or an edge sharing a vertex with it is never admissible (the
    appendix takes for granted that the target lies in no admissible node; a one-edge node of the
    target itself has r_x = 0 and would otherwise pass the test at a rounding-size distance, and the
    neighbours are the pairs Eq. 17 omits);
  * the candidate planes are the six coordinates' medians (the appendix "cycles through all six
    coordinates"); the left child takes the first floor(n / 2) edges in that coordinate's order, equal
    values ordered by edge index, and ties between coordinates go to the lower one.  Minimising over
    every position instead peels a few edges off the end of a chain at each level (measured depth 489
    on 2,000 edges);
  * r_x, r_T are half-diagonals of axis-aligned boxes, the spatial one over the edges' endpoints (so a
    one-edge node has r_x = l / 2 and is admitted only at distances above l / (2 eps), where its
    midpoint term approximates the trapezoid one); the average tangent T_N is not normalised.

parity pinned by: eps = 0 equals oracle.energy / oracle.differential (tests/test_oracle_bh.py);
the node term's gradient matches central differences; the error falls with eps.
"""
from __future__ import annotations

import numpy as np


def edge_points(gamma, edges):
    """Midpoints x_I, unit tangents T_I and lengths l_I (and the endpoints, for the node boxes)."""
    g = np.asarray(gamma, dtype=np.float64)
    e = np.asarray(edges, dtype=np.int64)
    d = g[e[:, 1]] - g[e[:, 0]]
    ell = np.sqrt(d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2])
    T = d / ell[:, None]
    x = 0.5 * (g[e[:, 0]] + g[e[:, 1]])
    return x, T, ell, (g[e[:, 0]], g[e[:, 1]])


def _sq_diam(lo, hi):
    """Squared diagonals of boxes [lo, hi] (rows), summed coordinate by coordinate in order."""
    d = hi[:, 0] - lo[:, 0]
    s = d * d
    for c in range(1, lo.shape[1]):
        d = hi[:, c] - lo[:, c]
        s = s + d * d
    return s


def build_bvh(x, T, ell, ends, leaf_size=8):
    """The hierarchy as a list of nodes (dicts) with the root at index 0, and the edge order `perm`:
    node k covers perm[b:e]; internal nodes have children `left`, `right`."""
    P = np.hstack([T, x])  # tangent-point (T_I, x_I)
    n = P.shape[0]
    perm = np.arange(n)
    nodes = []
    stack = [(0, n, -1, 0)]  # (begin, end, parent, side)
    while stack:
        b, e, parent, side = stack.pop()
        k = len(nodes)
        nodes.append({"b": b, "e": e, "left": -1, "right": -1})
        if parent >= 0:
            nodes[parent]["left" if side == 0 else "right"] = k
        items = perm[b:e]
        if e - b > leaf_size:
            best = None
            for c in range(6):
                order = np.lexsort((items, P[items, c]))  # by coordinate c, then edge index
                s = items[order]
                Q = P[s]
                plo = np.minimum.accumulate(Q, axis=0)
                phi = np.maximum.accumulate(Q, axis=0)
                slo = np.minimum.accumulate(Q[::-1], axis=0)[::-1]
                shi = np.maximum.accumulate(Q[::-1], axis=0)[::-1]
                # split at the median: left = s[:h], right = s[h:]
                h = len(items) // 2
                cost = _sq_diam(plo[h - 1:h], phi[h - 1:h])[0] + _sq_diam(slo[h:h + 1], shi[h:h + 1])[0]
                if best is None or cost < best[0]:
                    best = (cost, c, h, s)
            _, c, ks, s = best
            perm[b:e] = s
            stack.append((b + ks, e, k, 1))
            stack.append((b, b + ks, k, 0))
        nd = nodes[k]
        L = float(np.sum(ell[items]))
        nd["L"] = L
        nd["xbar"] = (ell[items][:, None] * x[items]).sum(axis=0) / L
        nd["Tbar"] = (ell[items][:, None] * T[items]).sum(axis=0) / L
        p1, p2 = ends[0][items], ends[1][items]
        xl, xh = np.minimum(p1, p2).min(axis=0), np.maximum(p1, p2).max(axis=0)
        tl, th = T[items].min(axis=0), T[items].max(axis=0)
        nd["rx"] = 0.5 * float(np.sqrt(np.sum((xh - xl) ** 2)))
        nd["rT"] = 0.5 * float(np.sqrt(np.sum((th - tl) ** 2)))
    return nodes, perm


def kernel(x, y, T, alpha, beta):
    """k(x, y, T) = |T x (x - y)|^alpha / |x - y|^beta (Sec. 3.2)."""
    d = np.asarray(x) - np.asarray(y)
    c = np.cross(T, d)
    return float(np.dot(c, c)) ** (0.5 * alpha) / float(np.dot(d, d)) ** (0.5 * beta)


def _k_grads(d, T, alpha, beta):
    """f = |T x d|^alpha |d|^-beta and its gradients in d and in T (T not assumed unit)."""
    dd = float(np.dot(d, d))
    tt = float(np.dot(T, T))
    td = float(np.dot(T, d))
    c = tt * dd - td * td                 # |T x d|^2
    c = max(c, 0.0)
    f = c ** (0.5 * alpha) * dd ** (-0.5 * beta)
    a = 0.5 * alpha * f / c if c > 0.0 else 0.0   # d f / d c
    gd = a * 2.0 * (tt * d - td * T) - beta * f * d / dd
    gT = a * 2.0 * (dd * T - td * d)
    return f, gd, gT


def pair_target_grad(g1, g2, q1, q2, alpha, beta):
    """Gradients in the target edge's endpoints g1, g2 of l_I l_J (khat_IJ + khat_JI) (Eqs. 17-18),
    with the source edge (q1, q2) fixed."""
    e = g2 - g1
    l = float(np.sqrt(np.dot(e, e)))
    T = e / l
    f = q2 - q1
    lj = float(np.sqrt(np.dot(f, f)))
    TJ = f / lj
    P = (np.eye(3) - np.outer(T, T)) / l  # d T / d g2 (and minus it for g1)
    K = 0.0
    G = [np.zeros(3), np.zeros(3)]
    gT = np.zeros(3)
    for a, ga in enumerate((g1, g2)):
        for qb in (q1, q2):
            d = ga - qb
            fI, gdI, gTI = _k_grads(d, T, alpha, beta)      # k(g_ia, q_jb, T_I)
            fJ, gdJ, _ = _k_grads(-d, TJ, alpha, beta)      # k(q_jb, g_ia, T_J)
            K += 0.25 * (fI + fJ)
            G[a] += 0.25 * (gdI - gdJ)
            gT += 0.25 * gTI
    # F = l l_J K:  dF/dg_a = l_J [K dl/dg_a + l (dK/dg_a + dT/dg_a^T dK/dT)]
    out1 = lj * (-K * T + l * (G[0] - P @ gT))
    out2 = lj * (K * T + l * (G[1] + P @ gT))
    return out1, out2


def node_target_grad(g1, g2, L, xbar, Tbar, alpha, beta):
    """Gradients in g1, g2 of L l_I (k(x_I, xbar, T_I) + k(xbar, x_I, Tbar)) with the node fixed."""
    e = g2 - g1
    l = float(np.sqrt(np.dot(e, e)))
    T = e / l
    d = 0.5 * (g1 + g2) - xbar
    f1, gd1, gT1 = _k_grads(d, T, alpha, beta)
    f2, gd2, _ = _k_grads(d, Tbar, alpha, beta)  # |Tbar x (xbar - x_I)| = |Tbar x d|
    P = (np.eye(3) - np.outer(T, T)) / l
    core = 0.5 * (gd1 + gd2)
    out1 = L * (-(f1 + f2) * T + l * (core - P @ gT1))
    out2 = L * ((f1 + f2) * T + l * (core + P @ gT1))
    return out1, out2


def _khat(g1, g2, q1, q2, T, alpha, beta):
    return 0.25 * sum(kernel(ga, qb, T, alpha, beta) for ga in (g1, g2) for qb in (q1, q2))


def _near_positions(edges, perm):
    """For every edge, the hierarchy positions of itself and of the edges sharing a vertex with it."""
    E = np.asarray(edges, dtype=np.int64)
    pos = np.empty(E.shape[0], dtype=np.int64)
    pos[perm] = np.arange(E.shape[0])
    inc = {}
    for J, (a, b) in enumerate(E):
        inc.setdefault(int(a), []).append(J)
        inc.setdefault(int(b), []).append(J)
    return [sorted({int(pos[J]) for v in E[I] for J in inc[int(v)]}) for I in range(E.shape[0])]


def _visit(nodes, perm, I, xI, eps, near):
    """Admissible nodes and leaf edges of the traversal for target I (in traversal order)."""
    adm, leaf = [], []
    stack = [0]
    while stack:
        k = stack.pop()
        nd = nodes[k]
        dist = float(np.linalg.norm(xI - nd["xbar"]))
        holds = any(nd["b"] <= q < nd["e"] for q in near[I])
        if not holds and nd["rx"] < eps * dist and nd["rT"] < eps:
            adm.append(k)
        elif nd["left"] < 0:
            leaf.extend(int(J) for J in perm[nd["b"]:nd["e"]])
        else:
            stack.append(nd["right"])
            stack.append(nd["left"])
    return adm, leaf


def energy(gamma, edges, eps, alpha=2.0, beta=4.5, leaf_size=8):
    """Barnes-Hut energy (Eq. BVHNodeTPE at admissible nodes, Eq. 17's terms in the leaves)."""
    g = np.asarray(gamma, dtype=np.float64)
    E = np.asarray(edges, dtype=np.int64)
    x, T, ell, ends = edge_points(g, E)
    nodes, perm = build_bvh(x, T, ell, ends, leaf_size)
    near = _near_positions(E, perm)
    total = 0.0
    for I in range(E.shape[0]):
        adm, leaf = _visit(nodes, perm, I, x[I], eps, near)
        for k in adm:
            nd = nodes[k]
            total += ell[I] * nd["L"] * kernel(x[I], nd["xbar"], T[I], alpha, beta)
        i1, i2 = E[I]
        for J in leaf:
            j1, j2 = E[J]
            if len({i1, i2, j1, j2}) < 4:
                continue
            total += ell[I] * ell[J] * _khat(g[i1], g[i2], g[j1], g[j2], T[I], alpha, beta)
    return total


def differential(gamma, edges, eps, alpha=2.0, beta=4.5, leaf_size=8):
    """Barnes-Hut differential [nV][3] (App. B.1, "Differential")."""
    g = np.asarray(gamma, dtype=np.float64)
    E = np.asarray(edges, dtype=np.int64)
    x, T, ell, ends = edge_points(g, E)
    nodes, perm = build_bvh(x, T, ell, ends, leaf_size)
    near = _near_positions(E, perm)
    dE = np.zeros_like(g)
    for I in range(E.shape[0]):
        i1, i2 = E[I]
        adm, leaf = _visit(nodes, perm, I, x[I], eps, near)
        for k in adm:
            nd = nodes[k]
            o1, o2 = node_target_grad(g[i1], g[i2], nd["L"], nd["xbar"], nd["Tbar"], alpha, beta)
            dE[i1] += o1
            dE[i2] += o2
        for J in leaf:
            j1, j2 = E[J]
            if len({i1, i2, j1, j2}) < 4:
                continue
            o1, o2 = pair_target_grad(g[i1], g[i2], g[j1], g[j2], alpha, beta)
            dE[i1] += o1
            dE[i2] += o2
    return dE


def admissible_count(gamma, edges, eps, leaf_size=8):
    """(admissible nodes, leaf pairs) visited over all targets: the work of one traversal pass."""
    x, T, ell, ends = edge_points(gamma, edges)
    nodes, perm = build_bvh(x, T, ell, ends, leaf_size)
    near = _near_positions(edges, perm)
    na = nl = 0
    for I in range(x.shape[0]):
        adm, leaf = _visit(nodes, perm, I, x[I], eps, near)
        na += len(adm)
        nl += len(leaf)
    return na, nl
