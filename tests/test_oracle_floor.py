"""The rounding floor of any FP64 evaluation of the Sobolev apply on smooth vectors.

The vertex rows of A-bar u (Secs. 5.2.2-5.2.3) are differences of edge rows divided by edge lengths,
twice over (the derivative operator D on both sides of the high-order form), so for a smooth u they
are ~n^2 smaller than the sums they come from.  The FP64 oracle's apply at sampled vertices is compared
here with the same sums evaluated in numpy's extended precision (80-bit on x86, 64-bit significand):
at n = 4,096 the two agree to ~1e-11, at n = 262,144 they differ by ~2e-5.  This is why solves at
262,144 vertices cannot certify a relative residual of 1e-6 with an FP64-class operator.

(Where numpy's long double is the 128-bit software format, this test is slow but still valid.)"""
import numpy as np
import pytest

import synth as S


def _apply_at_longdouble(gamma, edges, sigma, u, vidx):
    """(A-bar u) at the vertices vidx of a closed polygon (vertex v between edges v - 1 and v), with
    every sum in np.longdouble: rows h_I / l_I and l_I / 2 of the exact difference form."""
    L = np.longdouble
    n = gamma.shape[0]
    G, U = gamma.astype(L), u.astype(L)
    e1, e2 = edges[:, 0], edges[:, 1]
    P1, P2 = G[e1], G[e2]
    ev = P2 - P1
    ell = np.sqrt((ev * ev).sum(1))
    T = ev / ell[:, None]
    du = (U[e2] - U[e1]) / ell[:, None]
    ub = (U[e1] + U[e2]) / 2
    p = L(2.0 * sigma + 1.0)

    def row(I):
        J = np.arange(n)
        keep = (e1 != e1[I]) & (e1 != e2[I]) & (e2 != e1[I]) & (e2 != e2[I])
        J = J[keep]
        sw = np.zeros(len(J), dtype=L)
        sw0 = np.zeros(len(J), dtype=L)
        for a in (P1[I], P2[I]):
            for b in (P1[J], P2[J]):
                d = a[None, :] - b
                d2 = (d * d).sum(1)
                tI = (d * T[I][None, :]).sum(1)
                tJ = (d * T[J]).sum(1)
                f = d2 ** (-p / 2)
                sw += f
                sw0 += (2 * d2 - tI * tI - tJ * tJ) * f / (d2 * d2)
        omt = ((T[I][None, :] - T[J]) ** 2).sum(1) / 2
        A1 = ((ell[J] * sw)[:, None] * ((du[I][None, :] - du[J]) + omt[:, None] * du[J])).sum(0)
        A2 = ((ell[J] * sw0)[:, None] * (ub[I][None, :] - ub[J])).sum(0)
        return A1, A2

    out = np.zeros((len(vidx), 3), dtype=L)
    for k, v in enumerate(vidx):
        for I, sg in (((v - 1) % n, 1), (v, -1)):
            A1, A2 = row(I)
            out[k] += sg * L(0.5) * A1 + L(0.125) * ell[I] * A2
    return out.astype(np.float64)


@pytest.mark.parametrize("n,lo,hi", [(4096, 0.0, 1e-9), (262144, 5e-6, 1e-3)])
def test_fp64_apply_floor_on_a_smooth_vector(orc, n, lo, hi):
    c = S.knot_262144() if n == 262144 else S.single(S.fourier_knot(n, 16, 100))
    t = np.linspace(0, 2 * np.pi, n, endpoint=False)
    u = np.stack([np.cos(t), np.sin(2 * t), np.cos(3 * t)], 1)
    vidx = np.sort(np.random.default_rng(3).choice(n, 4, replace=False)).astype(np.int32)
    ref = orc.gram_apply_at(c.gamma, c.edges, 0.75, u, vidx)
    ext = _apply_at_longdouble(c.gamma, c.edges, 0.75, u, vidx)
    err = float(np.abs(ref - ext).max() / np.abs(ext).max())
    print(n, err)
    assert lo <= err <= hi, err
