"""FP64 oracle of the learned preconditioner and of flexible CG.

TEST INFRASTRUCTURE ONLY (test suite, smoke, benchmark CPU leg).  Plain
numpy, float64, channels-last arrays of shape (Z, Y, X, C); no code shared
with the CUDA path.  Neither the paper nor its comparison systems contain a
learned preconditioner: this follows the design the project states for it.

Conventions
  conv3   out[v, o] = sum_{t, i} W[o, t, i] * in[v + off(t), i], 3x3x3 taps
          t = (dz+1)*9 + (dy+1)*3 + (dx+1), zero padding, stride 1, no bias.
  pool2   2x2x2 average (even sizes).
  up2     nearest-neighbour doubling.
  U-net   (levels L0 full, L1 half, L2 quarter resolution; ReLU after every
          conv but the last):
            c1 (2->16), c2 (16->16) = e0
            pool, c3 (16->32), c4 (32->32) = e1
            pool, c5 (32->64), c6 (64->64)
            up, concat [up(64), e1] -> c7 (96->32)
            up, concat [up(32), e0] -> c8 (48->16)
            c9 (16->1) = output
          N acts on the Jacobi-scaled system D^{-1/2} A D^{-1/2} (D the
          operator's diagonal): input channels [s / rms(s), log k] with
          s = D^{-1/2} r; the output is multiplied by rms(s) D^{-1/2}.  A ReLU
          network is piecewise linear in (r, log k) and cannot form the
          product r / k that the coefficient contrast calls for; the scaling
          supplies it, and N stays positively homogeneous in r.
  loss    L(z) = 1/2 z.Az - z.r: the A-norm error 1/2 ||z - A^{-1}r||_A^2 up to
          the constant -1/2 r.A^{-1}r; dL/dz = A z - r.
  training loss (scale-free, sign-aware): with target e = A^{-1} r,
          a = z.Ae, c = z.Az, E = e.Ae, L(z) = 1/2 (1 - a |a| / (c E)).  For
          a >= 0 that is 1/2 ||s z - e||_A^2 / ||e||_A^2 with the best multiple
          s = a / c (a preconditioned step's line search picks it, so only the
          direction of z matters); for a < 0 it rises to 1, so the minimum
          (0) is reached only by positive multiples of e and the trained
          preconditioner keeps r.z > 0.
  Adam    Kingma & Ba, ICLR 2015, Algorithm 1 (bias-corrected moments).
  FCG     flexible CG (Notay, SIAM J. Sci. Comput. 22, 2000) with truncation m:
          p_k = z_k - sum_{i=k-m}^{k-1} (z_k.Ap_i / p_i.Ap_i) p_i,
          alpha_k = p_k.r_k / p_k.Ap_k; m = 1 is the beta form
          beta = z_{k+1}.(r_{k+1} - r_k) / (z_k.r_k).
"""
from __future__ import annotations

import numpy as np

import oracle

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
LAYERS = [("c1", 2, 16), ("c2", 16, 16), ("c3", 16, 32), ("c4", 32, 32), ("c5", 32, 64), ("c6", 64, 64),
          ("c7", 96, 32), ("c8", 48, 16), ("c9", 16, 1)]


def shift(x, dz, dy, dx):
    """y[z, y, x] = x[z + dz, y + dy, x + dx], zero outside."""
    Z, Y, X = x.shape[:3]
    out = np.zeros_like(x)
    zs, zd = (slice(dz, Z), slice(0, Z - dz)) if dz >= 0 else (slice(0, Z + dz), slice(-dz, Z))
    ys, yd = (slice(dy, Y), slice(0, Y - dy)) if dy >= 0 else (slice(0, Y + dy), slice(-dy, Y))
    xs, xd = (slice(dx, X), slice(0, X - dx)) if dx >= 0 else (slice(0, X + dx), slice(-dx, X))
    out[zd, yd, xd] = x[zs, ys, xs]
    return out


def conv3(x, W):
    """x: (Z, Y, X, Ci); W: (Co, 27, Ci) -> (Z, Y, X, Co)."""
    out = np.zeros(x.shape[:3] + (W.shape[0],))
    for t, (dz, dy, dx) in enumerate(TAPS):
        out += shift(x, dz, dy, dx) @ W[:, t, :].T
    return out


def conv3_adjoint(gy, W):
    """The adjoint of conv3 in its input: sum_t shift(gy, -off(t)) @ W_t."""
    out = np.zeros(gy.shape[:3] + (W.shape[2],))
    for t, (dz, dy, dx) in enumerate(TAPS):
        out += shift(gy, -dz, -dy, -dx) @ W[:, t, :]
    return out


def conv3_weight_grad(x, gy):
    """dL/dW for L depending on y = conv3(x, W) through gy = dL/dy."""
    Co, Ci = gy.shape[3], x.shape[3]
    g = np.zeros((Co, 27, Ci))
    gy2 = gy.reshape(-1, Co)
    for t, (dz, dy, dx) in enumerate(TAPS):
        g[:, t, :] = gy2.T @ shift(x, dz, dy, dx).reshape(-1, Ci)
    return g


def pool2(x):
    Z, Y, X, C = x.shape
    return x.reshape(Z // 2, 2, Y // 2, 2, X // 2, 2, C).mean(axis=(1, 3, 5))


def pool2_adjoint(g):
    return up2(g) / 8.0


def up2(x):
    return x.repeat(2, axis=0).repeat(2, axis=1).repeat(2, axis=2)


def up2_adjoint(g):
    Z, Y, X, C = g.shape
    return g.reshape(Z // 2, 2, Y // 2, 2, X // 2, 2, C).sum(axis=(1, 3, 5))


def relu(x):
    return np.maximum(x, 0.0)


def init_weights(seed: int = 0):
    """He-style initialisation from SplitMix64 normals (the shared input generator)."""
    from paper_2603_23343_gb300 import inputs
    return inputs.unet_init_weights(seed, LAYERS)


def net_forward(x, ws, round_fn=None):
    """U-net on input x (Z, Y, X, 2); returns (output (Z,Y,X,1), cache).

    round_fn (optional) is applied to every stored activation, to mirror a
    reduced-precision implementation layer by layer."""
    R = round_fn if round_fn is not None else (lambda a: a)
    c = {"x": x}
    a1 = R(relu(conv3(x, ws["c1"])))
    e0 = R(relu(conv3(a1, ws["c2"])))
    p1 = R(pool2(e0))
    a3 = R(relu(conv3(p1, ws["c3"])))
    e1 = R(relu(conv3(a3, ws["c4"])))
    p2 = R(pool2(e1))
    a5 = R(relu(conv3(p2, ws["c5"])))
    a6 = R(relu(conv3(a5, ws["c6"])))
    k7 = np.concatenate([R(up2(a6)), e1], axis=3)
    a7 = R(relu(conv3(k7, ws["c7"])))
    k8 = np.concatenate([R(up2(a7)), e0], axis=3)
    a8 = R(relu(conv3(k8, ws["c8"])))
    out = conv3(a8, ws["c9"])
    c.update(a1=a1, e0=e0, p1=p1, a3=a3, e1=e1, p2=p2, a5=a5, a6=a6, k7=k7, a7=a7, k8=k8, a8=a8)
    return out, c


def net_backward(gout, ws, c, round_fn=None, trace=None):
    """Gradients of a loss w.r.t. every weight and the input, given gout = dL/d(output).

    round_fn (optional) is applied to every propagated gradient that feeds a
    convolution (after its ReLU mask), mirroring an implementation that
    stores those in reduced precision; sums and skip gradients are not
    rounded.  trace (optional dict) receives, per layer, the (input,
    output gradient) pair its weight gradient is formed from."""
    R = round_fn if round_fn is not None else (lambda a: a)
    g = {}

    def wg(name, x, gy):
        if trace is not None:
            trace[name] = (x, gy)
        return conv3_weight_grad(x, gy)

    g["c9"] = wg("c9", c["a8"], gout)
    ga8 = R(conv3_adjoint(gout, ws["c9"]) * (c["a8"] > 0))
    g["c8"] = wg("c8", c["k8"], ga8)
    gk8 = conv3_adjoint(ga8, ws["c8"])
    ga7 = R(up2_adjoint(gk8[..., :32]) * (c["a7"] > 0))
    ge0 = gk8[..., 32:].copy()
    g["c7"] = wg("c7", c["k7"], ga7)
    gk7 = conv3_adjoint(ga7, ws["c7"])
    ga6 = R(up2_adjoint(gk7[..., :64]) * (c["a6"] > 0))
    ge1 = gk7[..., 64:].copy()
    g["c6"] = wg("c6", c["a5"], ga6)
    ga5 = R(conv3_adjoint(ga6, ws["c6"]) * (c["a5"] > 0))
    g["c5"] = wg("c5", c["p2"], ga5)
    ge1 = R((ge1 + pool2_adjoint(conv3_adjoint(ga5, ws["c5"]))) * (c["e1"] > 0))
    g["c4"] = wg("c4", c["a3"], ge1)
    ga3 = R(conv3_adjoint(ge1, ws["c4"]) * (c["a3"] > 0))
    g["c3"] = wg("c3", c["p1"], ga3)
    ge0 = R((ge0 + pool2_adjoint(conv3_adjoint(ga3, ws["c3"]))) * (c["e0"] > 0))
    g["c2"] = wg("c2", c["a1"], ge0)
    ga1 = R(conv3_adjoint(ge0, ws["c2"]) * (c["a1"] > 0))
    g["c1"] = wg("c1", c["x"], ga1)
    g["x"] = conv3_adjoint(ga1, ws["c1"])
    return g


def adam_step(w, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update at step t >= 1; returns (w, m, v) as new arrays."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    return w - lr * mhat / (np.sqrt(vhat) + eps), m, v


def logk_field(shape, k=None, kb=8):
    """log k at every grid point (0 for the constant-coefficient operator)."""
    if k is None:
        return np.zeros(shape)
    nz, ny, nx = shape
    full = np.repeat(np.repeat(np.repeat(np.asarray(k, dtype=np.float64), kb, 0), kb, 1), kb, 2)
    return np.log(full[:nz, :ny, :nx])


def jacobi_scale(shape, k=None, kb=8):
    """D^{-1/2} of the operator's diagonal D."""
    return 1.0 / np.sqrt(oracle.diag(shape, k, kb))


def net_input(r, logk, dsc):
    """Channels [s / rms(s), log k] with s = D^{-1/2} r (dsc = D^{-1/2}), and the output
    scale field rms(s) D^{-1/2}."""
    sr = r * dsc
    rms = float(np.sqrt(np.mean(sr * sr)))
    x = np.stack([sr / rms if rms > 0 else sr, logk], axis=3)
    return x, rms * dsc


def precond_apply(r, ws, k=None, kb=8):
    """z = N(r): the preconditioner the learned FCG applies."""
    x, scale = net_input(r, logk_field(r.shape, k, kb), jacobi_scale(r.shape, k, kb))
    out, _ = net_forward(x, ws)
    return out[..., 0] * scale


def loss(z, r, k=None, kb=8):
    """1/2 z.Az - z.r with A the solver's operator."""
    az = oracle.apply(z, k, kb)
    return 0.5 * float(np.sum(z * az)) - float(np.sum(z * r))


def loss_grad_z(z, r, k=None, kb=8):
    return oracle.apply(z, k, kb) - r


def loss_scaled(z, e, k=None, kb=8):
    """Sign-aware scale-free loss; for z.Ae >= 0 written out as 1/2 ||s z - e||_A^2 / ||e||_A^2."""
    az = oracle.apply(z, k, kb)
    ae = oracle.apply(e, k, kb)
    a = float(np.sum(z * ae))
    c = float(np.sum(z * az))
    E = float(np.sum(e * ae))
    if a >= 0.0:
        s = a / c
        d = s * z - e
        return 0.5 * float(np.sum(d * oracle.apply(d, k, kb))) / E
    return 0.5 * (1.0 + a * a / (c * E))


def loss_scaled_grad(z, e, k=None, kb=8):
    """dL/dz of loss_scaled: with a = z.Ae, c = z.Az, E = e.Ae, L = 1/2 (1 - a |a| / (c E)) and
    dL/dz = (|a| / (c E)) ((a / c) A z - A e)."""
    az = oracle.apply(z, k, kb)
    ae = oracle.apply(e, k, kb)
    a = float(np.sum(z * ae))
    c = float(np.sum(z * az))
    E = float(np.sum(e * ae))
    return (abs(a) / (c * E)) * ((a / c) * az - ae)


def fcg(b, precond, tol=1e-6, maxit=500, k=None, kb=8, x0=None, m=1, directions=None):
    """Flexible CG with truncation m: r = b - A x; repeat z = M(r);
    p = z - sum over the last m directions p_i of (z.Ap_i / p_i.Ap_i) p_i;
    alpha = p.r / p.Ap; x += alpha p; r -= alpha Ap; stop on ||r||/||b||.
    directions (optional list) receives every (p, Ap)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - oracle.apply(x, k, kb)
    bn = np.linalg.norm(b)
    hist = [np.linalg.norm(r) / bn]
    window = []
    it = 0
    while it < maxit and hist[-1] > tol:
        z = precond(r)
        p = z.copy()
        for pi, qi in window:
            p -= (float(np.sum(z * qi)) / float(np.sum(pi * qi))) * pi
        q = oracle.apply(p, k, kb)
        alpha = float(np.sum(p * r)) / float(np.sum(p * q))
        x += alpha * p
        r = r - alpha * q
        it += 1
        hist.append(np.linalg.norm(r) / bn)
        window.append((p, q))
        if directions is not None:
            directions.append((p, q))
        if len(window) > m:
            window.pop(0)
    return dict(x=x, iters=it, hist=np.array(hist))
