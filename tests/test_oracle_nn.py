"""Pins of the learned-preconditioner oracle (oracle/nn.py), CPU only."""
import numpy as np
import pytest

import oracle
import oracle.nn as nn
from paper_2603_23343_gb300 import inputs


def rnd(shape, seed):
    n = int(np.prod(shape))
    return inputs.uniform_pm1(seed, 0, n, np.float64).reshape(shape)


def test_weight_tap_order():
    """Weights are laid out (Co, 27, Ci) with tap t = (dz+1)*9 + (dy+1)*3 + (dx+1)."""
    for t, (dz, dy, dx) in enumerate(nn.TAPS):
        assert t == (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)
    x = rnd((4, 5, 6, 1), 21)
    W = np.zeros((1, 27, 1))
    W[0, 14, 0] = 1.0  # t = 14: (dz, dy, dx) = (0, 0, +1)
    np.testing.assert_array_equal(nn.conv3(x, W)[:, :, :-1], x[:, :, 1:])


def test_conv_tap_convention():
    """Tap (dz, dy, dx) = (0, 0, +1) reads the +x neighbour: out[..., x] = in[..., x + 1]."""
    x = rnd((4, 5, 6, 1), 1)
    W = np.zeros((1, 27, 1))
    W[0, nn.TAPS.index((0, 0, 1)), 0] = 1.0
    y = nn.conv3(x, W)
    np.testing.assert_array_equal(y[:, :, :-1], x[:, :, 1:])
    assert not np.any(y[:, :, -1])
    W2 = np.zeros((1, 27, 1))
    W2[0, nn.TAPS.index((-1, 0, 0)), 0] = 1.0  # reads the -z neighbour
    y2 = nn.conv3(x, W2)
    np.testing.assert_array_equal(y2[1:], x[:-1])
    assert not np.any(y2[0])


def test_conv_delta_kernel_is_identity_and_constant_input():
    x = rnd((5, 6, 7, 3), 2)
    W = np.zeros((3, 27, 3))
    W[:, 13, :] = np.eye(3)
    np.testing.assert_array_equal(nn.conv3(x, W), x)
    Wr = rnd((2, 27, 3), 3)
    c = np.ones((6, 6, 6, 3)) * 0.5
    y = nn.conv3(c, Wr)
    np.testing.assert_allclose(y[2, 2, 2], 0.5 * Wr.sum(axis=(1, 2)), rtol=1e-13)
    # a corner point sees only the 8 in-range taps
    in_corner = [t for t, (dz, dy, dx) in enumerate(nn.TAPS) if dz >= 0 and dy >= 0 and dx >= 0]
    np.testing.assert_allclose(y[0, 0, 0], 0.5 * Wr[:, in_corner, :].sum(axis=(1, 2)), rtol=1e-13)


def test_conv_adjoints_exact():
    x = rnd((4, 6, 5, 3), 4)
    y = rnd((4, 6, 5, 2), 5)
    W = rnd((2, 27, 3), 6)
    lhs = float(np.sum(nn.conv3(x, W) * y))
    assert abs(lhs - float(np.sum(x * nn.conv3_adjoint(y, W)))) <= 1e-12 * abs(lhs) + 1e-12
    E = rnd((2, 27, 3), 7)
    lhs_w = float(np.sum(nn.conv3(x, E) * y))  # conv is linear in W
    assert abs(lhs_w - float(np.sum(E * nn.conv3_weight_grad(x, y)))) <= 1e-12 * abs(lhs_w) + 1e-12


def test_pool_and_upsample_adjoints():
    a = rnd((4, 6, 8, 2), 8)
    b = rnd((2, 3, 4, 2), 9)
    assert abs(np.sum(nn.pool2(a) * b) - np.sum(a * nn.pool2_adjoint(b))) <= 1e-12
    assert abs(np.sum(nn.up2(b) * a) - np.sum(b * nn.up2_adjoint(a))) <= 1e-12
    np.testing.assert_allclose(nn.pool2(np.ones((4, 4, 4, 1))), np.ones((2, 2, 2, 1)))


def test_unet_backward_matches_finite_differences():
    shape = (8, 8, 8)
    r = rnd(shape, 10)
    k = inputs.lognormal_blocks(2, 2, 2, 11).astype(np.float64)
    logk = np.log(np.repeat(np.repeat(np.repeat(k, 4, 0), 4, 1), 4, 2))
    ws = nn.init_weights(3)
    x, scale = nn.net_input(r, logk, nn.jacobi_scale(shape, k, 4))

    def L(wset, xin):
        out, _ = nn.net_forward(xin, wset)
        z = out[..., 0] * scale
        return nn.loss(z, r, k, 4)

    out, cache = nn.net_forward(x, ws)
    z = out[..., 0] * scale
    gout = (nn.loss_grad_z(z, r, k, 4) * scale)[..., None]
    g = nn.net_backward(gout, ws, cache)
    h = 1e-6
    checks = [("c1", (3, 13, 0)), ("c2", (5, 0, 7)), ("c4", (1, 20, 3)), ("c5", (10, 13, 4)), ("c6", (63, 26, 63)),
              ("c7", (7, 5, 90)), ("c8", (15, 13, 40)), ("c9", (0, 13, 9))]
    for name, idx in checks:
        wp = {k2: v.copy() for k2, v in ws.items()}
        wm = {k2: v.copy() for k2, v in ws.items()}
        wp[name][idx] += h
        wm[name][idx] -= h
        fd = (L(wp, x) - L(wm, x)) / (2 * h)
        assert abs(fd - g[name][idx]) <= 1e-5 * max(1e-8, abs(fd)) + 1e-9, (name, fd, g[name][idx])
    for idx in [(1, 2, 3, 0), (7, 7, 0, 1), (4, 5, 6, 0)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (L(ws, xp) - L(ws, xm)) / (2 * h)
        assert abs(fd - g["x"][idx]) <= 1e-5 * max(1e-8, abs(fd)) + 1e-9


def test_loss_is_minimised_by_the_solution():
    shape = (5, 4, 6)
    r = rnd(shape, 12)
    zstar = oracle.pcg(r, tol=1e-14, maxit=500)["x"]
    assert np.max(np.abs(nn.loss_grad_z(zstar, r))) <= 1e-9 * np.max(np.abs(r))
    pert = rnd(shape, 13) * 1e-3
    assert nn.loss(zstar + pert, r) > nn.loss(zstar, r)
    np.testing.assert_allclose(nn.loss(zstar, r), -0.5 * float(np.sum(r * zstar)), rtol=1e-10)


@pytest.mark.parametrize("varcoeff", [False, True])
def test_fcg_reduces_to_pcg_for_linear_preconditioners(varcoeff):
    shape = (10, 12, 9)
    b = rnd(shape, 14)
    k = None
    if varcoeff:
        nbx, nby, nbz = inputs.block_counts(9, 12, 10, 4)
        k = inputs.lognormal_blocks(nbx, nby, nbz, 15).astype(np.float64)
    d = oracle.diag(shape, k, 4)
    ref = oracle.pcg(b, tol=1e-8, maxit=500, k=k, kb=4)
    f = nn.fcg(b, lambda r: r / d, tol=1e-8, maxit=500, k=k, kb=4)
    assert abs(f["iters"] - ref["iters"]) <= 1
    np.testing.assert_allclose(f["x"], ref["x"], rtol=0, atol=1e-7 * np.max(np.abs(ref["x"])))
    plain = oracle.pcg(b, tol=1e-8, maxit=500, k=k, kb=4, precond=None)
    f2 = nn.fcg(b, lambda r: r.copy(), tol=1e-8, maxit=500, k=k, kb=4)
    assert abs(f2["iters"] - plain["iters"]) <= 1
    f5 = nn.fcg(b, lambda r: r / d, tol=1e-8, maxit=500, k=k, kb=4, m=5)  # more memory changes nothing
    assert abs(f5["iters"] - ref["iters"]) <= 1
    np.testing.assert_allclose(f5["x"], ref["x"], rtol=0, atol=1e-7 * np.max(np.abs(ref["x"])))


def test_fcg_full_memory_keeps_directions_a_orthogonal():
    """With a nonlinear preconditioner and truncation m >= iterations, every search direction is
    A-orthogonal to all earlier ones (Notay's FCG with full orthogonalisation)."""
    shape = (6, 7, 5)
    b = rnd(shape, 60)

    def M(r):  # a small nonlinear, positively homogeneous map
        return np.maximum(r, 0.0) * 2.0 + np.minimum(r, 0.0) * 0.5 + 0.1 * oracle.apply(r) / 100.0

    dirs = []
    nn.fcg(b, M, tol=1e-10, maxit=12, m=50, directions=dirs)
    for i in range(len(dirs)):
        for j in range(i):
            pi, qi = dirs[i]
            pj, qj = dirs[j]
            assert abs(float(np.sum(pi * qj))) <= 1e-9 * np.sqrt(float(np.sum(pi * qi)) * float(np.sum(pj * qj)))


def test_adam_first_steps_closed_form():
    """Step 1 moves every weight by lr * g / (|g| + eps), i.e. lr * sign(g) for |g| >> eps; a
    constant gradient keeps that step size at every step (m_hat = g, v_hat = g^2 exactly)."""
    g = rnd((50,), 16)
    w0 = rnd((50,), 17)
    w, m, v = nn.adam_step(w0, g, np.zeros(50), np.zeros(50), 1, lr=0.01)
    np.testing.assert_allclose(w, w0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    for t in range(2, 6):
        w_prev = w
        w, m, v = nn.adam_step(w, g, m, v, t, lr=0.01)
        np.testing.assert_allclose(w_prev - w, 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)


def test_rounded_backward_reduces_to_exact_and_traces_layers():
    """With an identity round_fn the traced backward equals the plain one, and each traced
    pair rebuilds that layer's weight gradient."""
    shape = (8, 8, 8)
    r = rnd(shape, 50)
    ws = nn.init_weights(4)
    x, scale = nn.net_input(r, np.zeros(shape), nn.jacobi_scale(shape))
    out, cache = nn.net_forward(x, ws)
    gout = rnd(shape + (1,), 51)
    g0 = nn.net_backward(gout, ws, cache)
    tr = {}
    g1 = nn.net_backward(gout, ws, cache, round_fn=lambda a: a, trace=tr)
    for name, _, _ in nn.LAYERS:
        np.testing.assert_array_equal(g0[name], g1[name])
        np.testing.assert_array_equal(nn.conv3_weight_grad(*tr[name]), g0[name])


def test_scaled_loss_properties_and_gradient():
    """Scale-free sign-aware A-norm loss: 0 at any positive multiple of the target, 1 at any
    negative one, 1/2 for an A-orthogonal direction, invariant to positive scaling of z, and
    its closed-form gradient matches central differences on both sides of z.Ae = 0."""
    shape = (6, 5, 7)
    nbx, nby, nbz = inputs.block_counts(7, 5, 6, 4)
    k = inputs.lognormal_blocks(nbx, nby, nbz, 40).astype(np.float64)
    e = rnd(shape, 41)
    z = rnd(shape, 42)
    assert abs(nn.loss_scaled(3.0 * e, e, k, 4)) <= 1e-14
    assert abs(nn.loss_scaled(-0.5 * e, e, k, 4) - 1.0) <= 1e-14
    ae = oracle.apply(e, k, 4)
    zp = z - (float(np.sum(z * ae)) / float(np.sum(e * ae))) * e  # A-orthogonal to e
    assert abs(nn.loss_scaled(zp, e, k, 4) - 0.5) <= 1e-12
    for zz in (z + 0.3 * e, z - 0.3 * e):  # one with z.Ae > 0, one with z.Ae < 0
        a = float(np.sum(zz * ae))
        L = nn.loss_scaled(zz, e, k, 4)
        assert (0.0 < L < 0.5) if a > 0 else (0.5 < L < 1.0)
        assert abs(nn.loss_scaled(7.0 * zz, e, k, 4) - L) <= 1e-13
        g = nn.loss_scaled_grad(zz, e, k, 4)
        h = 1e-6
        for idx in [(0, 0, 0), (3, 2, 4), (5, 4, 6), (2, 1, 3)]:
            zp2, zm2 = zz.copy(), zz.copy()
            zp2[idx] += h
            zm2[idx] -= h
            fd = (nn.loss_scaled(zp2, e, k, 4) - nn.loss_scaled(zm2, e, k, 4)) / (2 * h)
            assert abs(fd - g[idx]) <= 1e-6 * abs(fd) + 1e-11
        assert abs(float(np.sum(g * zz))) <= 1e-12 * np.linalg.norm(g) * np.linalg.norm(zz)


def test_network_input_scaling():
    """The input is the Jacobi-scaled residual at unit rms plus log k; the output scale undoes
    both, so N is positively homogeneous in r, and a single block of constant k reduces the
    scaling to the Poisson one times k^{-1/2}."""
    shape = (8, 8, 8)
    r = rnd(shape, 70)
    k = np.full((1, 1, 1), 3.0)
    dsc = nn.jacobi_scale(shape, k, 8)
    np.testing.assert_allclose(dsc, nn.jacobi_scale(shape) / np.sqrt(3.0), rtol=1e-14)
    x, scale = nn.net_input(r, nn.logk_field(shape, k, 8), dsc)
    assert abs(float(np.mean(x[..., 0] ** 2)) - 1.0) <= 1e-12
    np.testing.assert_allclose(x[..., 1], np.log(3.0), rtol=1e-15)
    np.testing.assert_allclose(x[..., 0] * scale, r * dsc * dsc, rtol=1e-12)
    ws = nn.init_weights(7)
    z1 = nn.precond_apply(r, ws, k, 8)
    z2 = nn.precond_apply(2.5 * r, ws, k, 8)
    np.testing.assert_allclose(z2, 2.5 * z1, rtol=1e-12, atol=1e-300)
