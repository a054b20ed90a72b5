"""Seeded synthetic curve generators shared by the oracle tests and the GPU path.

This module only draws inputs: vertex positions, edge lists and curve offsets.
It holds none of the method's arithmetic (no energy, kernel, Gram or solver
code), so both the CPU oracle and the CUDA path can use it without sharing any
computation.

The shapes follow the workloads the method is evaluated on (closed knotted
polygons sampled at uniform parameter values); the paper's own knot datasets
are not used, and these random Fourier knots stand in for them.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "trefoil",
    "fourier_knot",
    "closed_edges",
    "open_edges",
    "regular_polygon",
    "unit_square",
    "scene",
    "batch_sizes",
    "batch_of_knots",
    "Curves",
]


def _params(n: int) -> np.ndarray:
    return 2.0 * math.pi * np.arange(n, dtype=np.float64) / n


def trefoil(n: int = 256, jitter: float = 0.01, seed: int = 0) -> np.ndarray:
    """Trefoil x(t) = (sin t + 2 sin 2t, cos t - 2 cos 2t, -sin 3t), t uniform on [0, 2pi),
    plus i.i.d. Gaussian jitter of standard deviation `jitter` (seeded). Returns [n, 3] float64."""
    t = _params(n)
    g = np.stack([np.sin(t) + 2 * np.sin(2 * t), np.cos(t) - 2 * np.cos(2 * t), -np.sin(3 * t)], axis=1)
    if jitter:
        g = g + np.random.default_rng(seed).normal(0.0, jitter, size=g.shape)
    return np.ascontiguousarray(g)


def fourier_knot(n: int, harmonics: int, seed: int) -> np.ndarray:
    """Closed random Fourier curve x(t) = sum_{k=1..K} a_k cos(kt) + b_k sin(kt), with every
    coordinate of a_k, b_k drawn from N(0, 1/k^2) (standard deviation 1/k), t uniform on
    [0, 2pi). Returns [n, 3] float64."""
    rng = np.random.default_rng(seed)
    t = _params(n)
    g = np.zeros((n, 3))
    for k in range(1, harmonics + 1):
        a = rng.normal(0.0, 1.0 / k, 3)
        b = rng.normal(0.0, 1.0 / k, 3)
        g += np.outer(np.cos(k * t), a) + np.outer(np.sin(k * t), b)
    return np.ascontiguousarray(g)


def regular_polygon(n: int, radius: float = 1.0) -> np.ndarray:
    t = _params(n)
    return np.ascontiguousarray(np.stack([radius * np.cos(t), radius * np.sin(t), np.zeros(n)], axis=1))


def unit_square() -> np.ndarray:
    """Unit square centred at the origin, counter-clockwise."""
    return np.array([[-.5, -.5, 0.], [.5, -.5, 0.], [.5, .5, 0.], [-.5, .5, 0.]])


def closed_edges(n: int, offset: int = 0) -> np.ndarray:
    """Edges (i, i+1 mod n) of a closed polygon on vertices offset..offset+n-1, int32 [n, 2]."""
    i = np.arange(n, dtype=np.int64)
    return np.ascontiguousarray(np.stack([i, (i + 1) % n], axis=1) + offset).astype(np.int32)


def open_edges(n: int, offset: int = 0) -> np.ndarray:
    i = np.arange(n - 1, dtype=np.int64)
    return np.ascontiguousarray(np.stack([i, i + 1], axis=1) + offset).astype(np.int32)


class Curves:
    """A graph of one or more polygons: positions [nV,3] float64, edges [nE,2] int32,
    and per-curve vertex/edge offsets (int32, length n_curves+1)."""

    def __init__(self, gamma, edges, vertex_offsets, edge_offsets):
        self.gamma = np.ascontiguousarray(gamma, dtype=np.float64)
        self.edges = np.ascontiguousarray(edges, dtype=np.int32)
        self.vertex_offsets = np.ascontiguousarray(vertex_offsets, dtype=np.int32)
        self.edge_offsets = np.ascontiguousarray(edge_offsets, dtype=np.int32)

    @property
    def n_vertices(self):
        return self.gamma.shape[0]

    @property
    def n_edges(self):
        return self.edges.shape[0]

    @property
    def n_curves(self):
        return len(self.vertex_offsets) - 1

    def curve(self, c):
        v0, v1 = self.vertex_offsets[c], self.vertex_offsets[c + 1]
        e0, e1 = self.edge_offsets[c], self.edge_offsets[c + 1]
        return self.gamma[v0:v1], self.edges[e0:e1] - v0


def single(gamma: np.ndarray, closed: bool = True) -> Curves:
    n = gamma.shape[0]
    e = closed_edges(n) if closed else open_edges(n)
    return Curves(gamma, e, [0, n], [0, e.shape[0]])


def scene(curves: list[np.ndarray], spacing: float | None = None) -> Curves:
    """Place closed curves at the points of a cubic lattice (2x2x2 for eight curves) with
    spacing 3x the largest curve radius, and join them into one graph."""
    k = max(1, math.ceil(len(curves) ** (1.0 / 3.0) - 1e-9))
    if spacing is None:
        rad = max(float(np.max(np.linalg.norm(c - c.mean(0), axis=1))) for c in curves)
        spacing = 3.0 * rad
    gs, es, vo, eo = [], [], [0], [0]
    for idx, c in enumerate(curves):
        ix, iy, iz = idx % k, (idx // k) % k, idx // (k * k)
        off = spacing * np.array([ix, iy, iz], dtype=np.float64)
        gs.append(c - c.mean(0) + off)
        es.append(closed_edges(c.shape[0], vo[-1]))
        vo.append(vo[-1] + c.shape[0])
        eo.append(eo[-1] + c.shape[0])
    return Curves(np.concatenate(gs), np.concatenate(es), vo, eo)


def batch_sizes(n_curves: int = 1024, lo: int = 64, hi: int = 4096, seed: int = 1000) -> np.ndarray:
    """Vertex counts drawn log-uniform in [lo, hi] (rounded), seeded."""
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), n_curves))).astype(np.int64)


def batch_of_knots(sizes, harmonics: int = 8, seed0: int = 1000) -> Curves:
    """Independent closed Fourier knots (curve c drawn with seed seed0 + 1 + c), concatenated
    into one vertex/edge array with offsets."""
    gs, es, vo, eo = [], [], [0], [0]
    for c, n in enumerate(sizes):
        g = fourier_knot(int(n), harmonics, seed0 + 1 + c)
        gs.append(g)
        es.append(closed_edges(int(n), vo[-1]))
        vo.append(vo[-1] + int(n))
        eo.append(eo[-1] + int(n))
    return Curves(np.concatenate(gs), np.concatenate(es), vo, eo)


# Named workloads (sizes and seeds) used by the tests and the benchmark.
def trefoil_256() -> Curves:
    return single(trefoil(256, 0.01, 0))


def eight_knots_4096(as_scene: bool = True, first_seed: int = 1) -> Curves:
    """Eight closed Fourier knots (K = 8, 4,096 vertices, seeds first_seed .. first_seed + 7)."""
    ks = [fourier_knot(4096, 8, s) for s in range(first_seed, first_seed + 8)]
    if as_scene:
        return scene(ks)
    gs, es, vo, eo = [], [], [0], [0]
    for k in ks:
        gs.append(k)
        es.append(closed_edges(4096, vo[-1]))
        vo.append(vo[-1] + 4096)
        eo.append(eo[-1] + 4096)
    return Curves(np.concatenate(gs), np.concatenate(es), vo, eo)


def knot_262144() -> Curves:
    return single(fourier_knot(262144, 16, 100))
