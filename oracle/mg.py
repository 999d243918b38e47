"""FP64 oracle of the geometric multigrid preconditioner and of PCG with it.

TEST INFRASTRUCTURE ONLY (test suite, benchmark CPU leg).  Plain numpy,
float64, arrays (Z, Y, X); no code shared with the CUDA path.  The paper
names multigrid solvers as future work (conclusion) and gives no design;
this follows the design the project states for it:

Operators (every level): the seven-point operator in face-weight form,
  (A u)_c = sum over the six faces f of c of w_f (u_c - u_nb(f)),
with u_nb = 0 across the domain boundary.  It is stored as the weights of
the +x, +y, +z faces of every cell (wx, wy, wz; zero where the face lies on
the boundary) and the diagonal D = the sum of all six face weights of the
cell, boundary faces included.  Level 0 is the solver's operator (face
weight 1/h_d^2 times the face coefficient: 1 for Poisson; the harmonic mean
of the two cells' block coefficients, or the cell's own on the boundary).

Coarsening (aggregation): coarse cell I owns the 2 x 2 x 2 fine cells
2I + {0, 1}^3; the prolongation P copies a coarse value to its eight fine
cells; the coarse operator is the Galerkin product P^T A P, which is again
a face-weight operator: a coarse face carries the sum of the four fine face
weights across it, and the coarse diagonal is the sum of the eight fine
diagonals minus twice the weights of the twelve faces inside the aggregate.
Levels are added while every size is even and the coarse grid keeps at
least 4 cells per axis, down to at most MAX_LEVELS levels.

V-cycle (z = M r): at level l with right-hand side f:
  coarsest:  COARSE_SWEEPS damped Jacobi sweeps from u = 0
  otherwise: u = omega D^-1 f                     (pre-smoothing from zero)
             r = f - A u
             e = V-cycle(l + 1, P^T r)
             u = u + sigma P e                     (scaled coarse correction)
             u = u + omega D^-1 (f - A u)          (post-smoothing)
The pre- and post-smoothing are adjoint and the coarse correction is the
scaled Galerkin one, so M is symmetric; with omega D^-1 A's spectrum inside
(0, 2) and 0 < sigma < 2 it is positive definite (checked in the tests).
"""
from __future__ import annotations

import numpy as np

import oracle

OMEGA = 0.9
SIGMA = 1.5
COARSE_SWEEPS = 24
MAX_LEVELS = 8
MIN_COARSE = 4


def fine_weights(shape, k=None, kb=8):
    """(wx, wy, wz, D) of the solver's operator on a grid (Z, Y, X)."""
    nz, ny, nx = shape
    c = [1.0 / (1.0 / (n + 1)) ** 2 for n in (nx, ny, nz)]
    if k is None:
        kc = np.ones(shape)
    else:
        full = np.repeat(np.repeat(np.repeat(np.asarray(k, dtype=np.float64), kb, 0), kb, 1), kb, 2)
        kc = full[:nz, :ny, :nx]

    def hm(a, b):
        return 2.0 * a * b / (a + b)
    wx = np.zeros(shape)
    wy = np.zeros(shape)
    wz = np.zeros(shape)
    wx[:, :, :-1] = c[0] * hm(kc[:, :, :-1], kc[:, :, 1:])
    wy[:, :-1, :] = c[1] * hm(kc[:, :-1, :], kc[:, 1:, :])
    wz[:-1, :, :] = c[2] * hm(kc[:-1, :, :], kc[1:, :, :])
    # diagonal: interior faces on both sides, the cell's own coefficient on boundary faces
    D = np.zeros(shape)
    D += wx + wy + wz
    D[:, :, 1:] += wx[:, :, :-1]
    D[:, 1:, :] += wy[:, :-1, :]
    D[1:, :, :] += wz[:-1, :, :]
    D[:, :, 0] += c[0] * kc[:, :, 0]
    D[:, :, -1] += c[0] * kc[:, :, -1]
    D[:, 0, :] += c[1] * kc[:, 0, :]
    D[:, -1, :] += c[1] * kc[:, -1, :]
    D[0, :, :] += c[2] * kc[0, :, :]
    D[-1, :, :] += c[2] * kc[-1, :, :]
    return wx, wy, wz, D


def apply(op, u):
    """A u for a face-weight operator op = (wx, wy, wz, D)."""
    wx, wy, wz, D = op
    out = D * u
    out[:, :, :-1] -= wx[:, :, :-1] * u[:, :, 1:]
    out[:, :, 1:] -= wx[:, :, :-1] * u[:, :, :-1]
    out[:, :-1, :] -= wy[:, :-1, :] * u[:, 1:, :]
    out[:, 1:, :] -= wy[:, :-1, :] * u[:, :-1, :]
    out[:-1, :, :] -= wz[:-1, :, :] * u[1:, :, :]
    out[1:, :, :] -= wz[:-1, :, :] * u[:-1, :, :]
    return out


def restrict(r):
    """P^T r: the sum over each coarse cell's eight fine cells."""
    Z, Y, X = r.shape
    return r.reshape(Z // 2, 2, Y // 2, 2, X // 2, 2).sum(axis=(1, 3, 5))


def prolong(e):
    """P e: the coarse value copied to the eight fine cells."""
    return e.repeat(2, axis=0).repeat(2, axis=1).repeat(2, axis=2)


def coarsen(op):
    """The Galerkin operator P^T A P of a face-weight operator, in face-weight form."""
    wx, wy, wz, D = op

    def agg(a):
        Z, Y, X = a.shape
        return a.reshape(Z // 2, 2, Y // 2, 2, X // 2, 2)
    WX, WY, WZ = agg(wx), agg(wy), agg(wz)
    # faces between neighbouring aggregates: the +x faces of the aggregate's x = 1 cells, etc.
    cwx = WX[:, :, :, :, :, 1].sum(axis=(1, 3))
    cwy = WY[:, :, :, 1, :, :].sum(axis=(1, 4))
    cwz = WZ[:, 1, :, :, :, :].sum(axis=(2, 4))
    # twelve faces inside the aggregate: the +x faces of its x = 0 cells, ...
    inner = (WX[:, :, :, :, :, 0].sum(axis=(1, 3)) + WY[:, :, :, 0, :, :].sum(axis=(1, 4))
             + WZ[:, 0, :, :, :, :].sum(axis=(2, 4)))
    cD = restrict(D) - 2.0 * inner
    return cwx, cwy, cwz, cD


def hierarchy(shape, k=None, kb=8, max_levels=MAX_LEVELS):
    """[op_0, op_1, ...]: the solver's operator and its Galerkin coarsenings."""
    ops = [fine_weights(shape, k, kb)]
    s = shape
    while len(ops) < max_levels and all(n % 2 == 0 and n // 2 >= MIN_COARSE for n in s):
        ops.append(coarsen(ops[-1]))
        s = tuple(n // 2 for n in s)
    return ops


def jacobi_sweeps(op, f, sweeps, omega=OMEGA):
    """`sweeps` damped Jacobi sweeps from u = 0."""
    D = op[3]
    u = omega * f / D
    for _ in range(sweeps - 1):
        u = u + omega * (f - apply(op, u)) / D
    return u


def vcycle(ops, f, level=0, omega=OMEGA, sigma=SIGMA, coarse_sweeps=COARSE_SWEEPS):
    """z = M f, the V-cycle of the module docstring."""
    op = ops[level]
    if level == len(ops) - 1:
        return jacobi_sweeps(op, f, coarse_sweeps, omega)
    D = op[3]
    u = omega * f / D
    r = f - apply(op, u)
    e = vcycle(ops, restrict(r), level + 1, omega, sigma, coarse_sweeps)
    u = u + sigma * prolong(e)
    return u + omega * (f - apply(op, u)) / D


def pcg(b, ops, x0=None, tol=1e-6, maxit=500, k=None, kb=8, omega=OMEGA, sigma=SIGMA, coarse_sweeps=COARSE_SWEEPS):
    """PCG (Sec. VII's iteration) with z = V-cycle(r); the operator is the solver's (oracle.apply).
    Returns dict(x, iters, hist)."""
    def M(v):
        return vcycle(ops, v, 0, omega, sigma, coarse_sweeps)
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - oracle.apply(x, k, kb)
    bn = np.linalg.norm(b)
    hist = [np.linalg.norm(r) / bn]
    z = M(r)
    p = z.copy()
    rz = float(np.sum(r * z))
    it = 0
    while it < maxit and hist[-1] > tol:
        q = oracle.apply(p, k, kb)
        alpha = rz / float(np.sum(p * q))
        x += alpha * p
        r -= alpha * q
        it += 1
        hist.append(np.linalg.norm(r) / bn)
        if hist[-1] <= tol:
            break
        z = M(r)
        rz_new = float(np.sum(r * z))
        p = z + (rz_new / rz) * p
        rz = rz_new
    return dict(x=x, iters=it, hist=np.array(hist))
