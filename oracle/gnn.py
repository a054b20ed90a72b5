"""FP64 numpy oracle of the learned preconditioner term (test infrastructure only).

The learned term is this library's extension, not part of the paper.  Every step is written out
from its definition; the CUDA kernels (BF16 weights, FP32 accumulation) are checked against it.

Edge features (closed curves; I-1 and I+1 are the neighbours of edge I on its curve; d = diag(A)):
    f = [log(l_I / mean l), 1 - T_{I-1}.T_I, 1 - T_I.T_{I+1}, log(d_i1 / mean d), log(d_i2 / mean d),
         log(l_{I-1} / l_I), log(l_{I+1} / l_I), 1]
Network (3 layers of width 64 on the edge graph, then a linear read-out of 3 values per edge):
    h1 = relu(W1 f + b1)
    h2 = relu(W2s h1 + W2n (h1[I-1] + h1[I+1]) / 2 + b2)
    h3 = relu(W3s h2 + W3n (h2[I-1] + h2[I+1]) / 2 + b3)
    (a, b, c) = W4 h3 + b4
Preconditioner (SPD for every parameter value):
    M^-1 r = W S W r + Z (Z^T A Z)^-1 Z^T r + G r,
  * W = D^-1/2 diag(exp(c_v)), c_v = (c_{I-1} + c_I) / 2 the mean of the outputs of the two edges at
    vertex v, S = F^-1 diag(1 / lambda) F the circulant of each closed curve (per component): a learned
    rescaling of the Jacobi-scaled circulant (c = 0 gives the two-level preconditioner back);
  * G: for r with 3 components and r~ = r / sqrt(d),
    delta_I = r~_i2 - r~_i1, sigma_I = r~_i1 + r~_i2, ea = exp(2 a_I), eb = exp(2 b_I)
    (G r)_i2 += (ea delta_I + eb sigma_I) / sqrt(d_i2),  (G r)_i1 += (-ea delta_I + eb sigma_I) / sqrt(d_i1).
Training loss of one pair (r, e = A^+ r, so e^T r = ||e||_A^2): preconditioned CG does not change
when M^-1 is scaled, so the loss is the A-norm error of the best multiple of z = M^-1 r,
    L = min_a ||a z - e||_A^2 / ||e||_A^2 = 1 - (z^T r)^2 / ((z^T A z)(e^T r)),
the squared A-sine of the angle between z and e.  With s = z^T r, q = z^T A z:
    dL/dz = -2 s / (q e^T r) (r - (s / q) A z),
and through the rescaling, with z_S = W S W r and z2 = W S W (dL/dz) (S is symmetric):
    dL/dc_v = sum over components of ((dL/dz)_v (z_S)_v + r_v (z2)_v).
"""
from __future__ import annotations

import numpy as np

H = 64
F = 8
SHAPES = [("W1", (H, F)), ("b1", (H,)), ("W2s", (H, H)), ("W2n", (H, H)), ("b2", (H,)),
          ("W3s", (H, H)), ("W3n", (H, H)), ("b3", (H,)), ("W4", (3, H)), ("b4", (3,))]


def n_params():
    return sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    out, o = {}, 0
    for name, s in SHAPES:
        k = int(np.prod(s))
        out[name] = np.asarray(theta[o:o + k], dtype=np.float64).reshape(s)
        o += k
    return out


def init_params(seed=0, out_bias=-2.0):
    rng = np.random.default_rng(seed)
    parts = []
    for name, s in SHAPES:
        if name.startswith("W"):
            fan_in = s[1]
            w = rng.normal(0.0, 1.0 / np.sqrt(fan_in), size=s)
            if name == "W4":
                w *= 0.1
            parts.append(w.ravel())
        elif name == "b4":
            parts.append(np.array([out_bias, out_bias, 0.0]))   # c = 0: the plain Jacobi scaling
        else:
            parts.append(np.zeros(s))
    return np.concatenate(parts)


def neighbours(n):
    I = np.arange(n)
    return (I - 1) % n, (I + 1) % n


def features(gamma, diag):
    """Edge features of one closed curve (vertex i, edge i = (i, i+1 mod n))."""
    n = gamma.shape[0]
    e = np.roll(gamma, -1, axis=0) - gamma
    l = np.linalg.norm(e, axis=1)
    T = e / l[:, None]
    prv, nxt = neighbours(n)
    d1, d2 = diag, np.roll(diag, -1)
    dm = diag.mean()
    return np.stack([np.log(l / l.mean()), 1 - (T[prv] * T).sum(1), 1 - (T * T[nxt]).sum(1), np.log(d1 / dm),
                     np.log(d2 / dm), np.log(l[prv] / l), np.log(l[nxt] / l), np.ones(n)], axis=1)


def forward(theta, f):
    p = unpack(theta)
    n = f.shape[0]
    prv, nxt = neighbours(n)
    z1 = f @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0)
    m1 = 0.5 * (h1[prv] + h1[nxt])
    z2 = h1 @ p["W2s"].T + m1 @ p["W2n"].T + p["b2"]
    h2 = np.maximum(z2, 0)
    m2 = 0.5 * (h2[prv] + h2[nxt])
    z3 = h2 @ p["W3s"].T + m2 @ p["W3n"].T + p["b3"]
    h3 = np.maximum(z3, 0)
    out = h3 @ p["W4"].T + p["b4"]
    return out, dict(f=f, z1=z1, h1=h1, m1=m1, z2=z2, h2=h2, m2=m2, z3=z3, h3=h3)


def backward(theta, cache, dout):
    """Gradient of a scalar whose derivative w.r.t. the network outputs is dout [n, 2]."""
    p = unpack(theta)
    f = cache["f"]
    n = f.shape[0]
    prv, nxt = neighbours(n)
    g = {}
    g["W4"] = dout.T @ cache["h3"]
    g["b4"] = dout.sum(0)
    dh3 = dout @ p["W4"]
    dz3 = dh3 * (cache["z3"] > 0)
    g["W3s"] = dz3.T @ cache["h2"]
    g["W3n"] = dz3.T @ cache["m2"]
    g["b3"] = dz3.sum(0)
    dh2 = dz3 @ p["W3s"]
    dm2 = dz3 @ p["W3n"]
    dh2 = dh2 + 0.5 * (dm2[nxt] + dm2[prv])   # m2[I] = (h2[I-1] + h2[I+1]) / 2
    dz2 = dh2 * (cache["z2"] > 0)
    g["W2s"] = dz2.T @ cache["h1"]
    g["W2n"] = dz2.T @ cache["m1"]
    g["b2"] = dz2.sum(0)
    dh1 = dz2 @ p["W2s"]
    dm1 = dz2 @ p["W2n"]
    dh1 = dh1 + 0.5 * (dm1[nxt] + dm1[prv])
    dz1 = dh1 * (cache["z1"] > 0)
    g["W1"] = dz1.T @ f
    g["b1"] = dz1.sum(0)
    return np.concatenate([g[name].ravel() for name, _ in SHAPES])


def g_apply(out, diag, r):
    """(G r) for the per-edge outputs out = (a, b) of one closed curve; r [n, 3]."""
    n = r.shape[0]
    sd = np.sqrt(diag)
    rt = r / sd[:, None]
    r1, r2 = rt, np.roll(rt, -1, axis=0)      # values at i1 = I and i2 = I + 1
    ea, eb = np.exp(2 * out[:, 0]), np.exp(2 * out[:, 1])
    delta, sig = r2 - r1, r1 + r2
    c2 = ea[:, None] * delta + eb[:, None] * sig
    c1 = -ea[:, None] * delta + eb[:, None] * sig
    gr = c1 / sd[:, None] + np.roll(c2, 1, axis=0) / sd[:, None]   # vertex i receives c1 of edge i, c2 of edge i-1
    return gr


def g_out_grad(out, diag, r, gz):
    """d(gz . G r) / d out: per edge [dL/da, dL/db, 0] with gz = dL/d(G r)."""
    sd = np.sqrt(diag)
    rt = r / sd[:, None]
    gt = gz / sd[:, None]
    r1, r2 = rt, np.roll(rt, -1, axis=0)
    g1, g2 = gt, np.roll(gt, -1, axis=0)
    ea, eb = np.exp(2 * out[:, 0]), np.exp(2 * out[:, 1])
    delta, sig = r2 - r1, r1 + r2
    dea = ((g2 - g1) * delta).sum(1)
    deb = ((g1 + g2) * sig).sum(1)
    return np.stack([2 * ea * dea, 2 * eb * deb, np.zeros_like(dea)], axis=1)


def vertex_log_scale(out):
    """c_v = (c_{I-1} + c_I) / 2: vertex v is the second endpoint of edge v-1 and the first of edge v."""
    c = out[:, 2]
    return 0.5 * (np.roll(c, 1) + c)


def scaled_spectral(diag, vlog, lam, r):
    """W S W r with W = D^-1/2 diag(exp(vlog)), S = F^-1 diag(1 / lam) F per component (one closed curve)."""
    w = np.exp(vlog) / np.sqrt(diag)
    y = np.real(np.fft.ifft(np.fft.fft(w[:, None] * r, axis=0) / lam[:, None], axis=0))
    return w[:, None] * y


def loss_and_grad(theta, f, diag, A, r, e, base_z, lam=None):
    """Loss of one pair and its parameter gradient.  base_z: the part of M^-1 r that does not depend
    on the parameters (the coarse term; with lam = None, the whole fixed preconditioner).  lam: the
    circulant symbol of the curve, which switches the learned rescaling W S W r on."""
    out, cache = forward(theta, f)
    z = base_z + g_apply(out, diag, r)
    zs = None
    if lam is not None:
        zs = scaled_spectral(diag, vertex_log_scale(out), lam, r)
        z = z + zs
    Az = A @ z
    er = float((e * r).sum())
    s = float((z * r).sum())
    q = float((z * Az).sum())
    L = 1.0 - s * s / (q * er)
    gz = -2.0 * s / (q * er) * (r - (s / q) * Az)
    dout = g_out_grad(out, diag, r, gz)
    if lam is not None:
        z2 = scaled_spectral(diag, vertex_log_scale(out), lam, gz)
        dc_v = (gz * zs).sum(1) + (r * z2).sum(1)
        dout[:, 2] = 0.5 * (dc_v + np.roll(dc_v, -1))   # edge I feeds vertices I and I+1
    return L, backward(theta, cache, dout)


def loss_and_grad_balanced(theta, f, diag, A, Z, r, e, lam):
    """The same loss and gradient for the learned smoother inside the balancing two-level form:
        z = Q r + (I - Q A) y,   y = G r2 + W S W r2,   r2 = (I - A Q) r,   Q = Z (Z^T A Z)^-1 Z^T.
    The parameter-dependent part enters through y alone: dL/dy = (I - A Q) dL/dz (Q, A symmetric), and
    y depends on the outputs exactly as z does in the additive form, with r2 in place of r."""
    out, cache = forward(theta, f)
    E = Z.T @ A @ Z
    Q = lambda v: Z @ np.linalg.solve(E, Z.T @ v)
    r2 = r - A @ Q(r)
    zs = scaled_spectral(diag, vertex_log_scale(out), lam, r2)
    y = g_apply(out, diag, r2) + zs
    z = Q(r) + y - Q(A @ y)
    Az = A @ z
    er = float((e * r).sum())
    s = float((z * r).sum())
    q = float((z * Az).sum())
    L = 1.0 - s * s / (q * er)
    gz = -2.0 * s / (q * er) * (r - (s / q) * Az)
    gy = gz - A @ Q(gz)
    dout = g_out_grad(out, diag, r2, gy)
    z2 = scaled_spectral(diag, vertex_log_scale(out), lam, gy)
    dc_v = (gy * zs).sum(1) + (r2 * z2).sum(1)
    dout[:, 2] = 0.5 * (dc_v + np.roll(dc_v, -1))
    return L, backward(theta, cache, dout)
