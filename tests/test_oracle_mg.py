"""Pins of the multigrid oracle (oracle/mg.py) against what the mathematics
fixes, independent of the oracle's own arithmetic:

  - the face-weight form of the solver's operator equals the pinned
    matrix-free operator (oracle.apply), constant and block coefficients;
  - the coarse operator equals the Galerkin product P^T A P formed from dense
    matrices (A by applying the operator to unit vectors, P the aggregation
    written out), and for the Poisson operator equals the seven-point
    operator with four times the face weights (closed form);
  - the V-cycle is a symmetric positive definite operator (dense on a small
    grid), and on a single level it is the damped Jacobi polynomial;
  - PCG with it reaches the tolerance with the same solution as the Jacobi
    oracle and in far fewer iterations.
"""
import numpy as np
import pytest

import oracle
import oracle.mg as mg
from paper_2603_23343_gb300 import inputs


def block_k(shape, kb, seed):
    nz, ny, nx = shape
    nbx, nby, nbz = inputs.block_counts(nx, ny, nz, kb)
    return inputs.lognormal_blocks(nbx, nby, nbz, seed).astype(np.float64)


def dense(fn, shape):
    n = int(np.prod(shape))
    cols = []
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        cols.append(fn(e.reshape(shape)).ravel())
    return np.stack(cols, axis=1)


def aggregation(shape):
    """P (fine x coarse): 1 where the fine cell belongs to the coarse cell."""
    nz, ny, nx = shape
    cz, cy, cx = nz // 2, ny // 2, nx // 2
    P = np.zeros((nz * ny * nx, cz * cy * cx))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                P[(k * ny + j) * nx + i, ((k // 2) * cy + j // 2) * cx + i // 2] = 1.0
    return P


@pytest.mark.parametrize("shape", [(6, 4, 8), (5, 7, 3)])
@pytest.mark.parametrize("varcoeff", [False, True])
def test_face_weight_operator_is_the_solver_operator(shape, varcoeff):
    k = block_k(shape, 2, 9) if varcoeff else None
    u = inputs.uniform_rhs(shape, 10, dtype=np.float64)
    ref = oracle.apply(u, k, 2)
    np.testing.assert_allclose(mg.apply(mg.fine_weights(shape, k, 2), u), ref, rtol=0,
                               atol=1e-13 * np.max(np.abs(ref)))


@pytest.mark.parametrize("shape", [(4, 4, 8), (6, 4, 4)])
@pytest.mark.parametrize("varcoeff", [False, True])
def test_coarse_operator_is_the_galerkin_product(shape, varcoeff):
    k = block_k(shape, 2, 11) if varcoeff else None
    op = mg.fine_weights(shape, k, 2)
    A = dense(lambda v: mg.apply(op, v), shape)
    P = aggregation(shape)
    cshape = tuple(n // 2 for n in shape)
    cop = mg.coarsen(op)
    Ac = dense(lambda v: mg.apply(cop, v), cshape)
    np.testing.assert_allclose(Ac, P.T @ A @ P, rtol=0, atol=1e-12 * np.max(np.abs(A)))
    # and a second coarsening of the coarse operator, against the product of two aggregations
    if all(n % 4 == 0 for n in shape):
        P2 = aggregation(cshape)
        c2 = mg.coarsen(cop)
        A2 = dense(lambda v: mg.apply(c2, v), tuple(n // 4 for n in shape))
        np.testing.assert_allclose(A2, (P @ P2).T @ A @ (P @ P2), rtol=0, atol=1e-12 * np.max(np.abs(A)))


def test_poisson_coarse_operator_closed_form():
    shape = (8, 12, 16)
    nz, ny, nx = shape
    c = [(n + 1) ** 2 for n in (nx, ny, nz)]
    wx, wy, wz, D = mg.coarsen(mg.fine_weights(shape))
    np.testing.assert_allclose(wx[:, :, :-1], 4 * c[0], rtol=1e-15)
    np.testing.assert_allclose(wy[:, :-1, :], 4 * c[1], rtol=1e-15)
    np.testing.assert_allclose(wz[:-1, :, :], 4 * c[2], rtol=1e-15)
    assert not np.any(wx[:, :, -1]) and not np.any(wy[:, -1, :]) and not np.any(wz[-1, :, :])
    np.testing.assert_allclose(D, 8.0 * sum(c), rtol=1e-15)


@pytest.mark.parametrize("varcoeff", [False, True])
def test_vcycle_is_symmetric_positive_definite(varcoeff):
    shape = (8, 8, 8)
    k = block_k(shape, 2, 12) if varcoeff else None
    ops = mg.hierarchy(shape, k, 2)
    assert len(ops) == 2  # 8 -> 4, and 4 does not halve to >= 4
    M = dense(lambda v: mg.vcycle(ops, v), shape)
    np.testing.assert_allclose(M, M.T, rtol=0, atol=1e-12 * np.max(np.abs(M)))
    assert np.min(np.linalg.eigvalsh(0.5 * (M + M.T))) > 0.0


def test_single_level_vcycle_is_damped_jacobi():
    shape = (5, 6, 7)  # odd sizes: no coarse level
    ops = mg.hierarchy(shape)
    assert len(ops) == 1
    f = inputs.uniform_rhs(shape, 13, dtype=np.float64)
    d = oracle.diag(shape)
    u = mg.OMEGA * f / d
    for _ in range(mg.COARSE_SWEEPS - 1):
        u = u + mg.OMEGA * (f - oracle.apply(u)) / d
    np.testing.assert_allclose(mg.vcycle(ops, f), u, rtol=1e-13, atol=0)


@pytest.mark.parametrize("varcoeff", [False, True])
def test_mg_pcg_reaches_tolerance_in_few_iterations(varcoeff):
    shape = (32, 32, 32)
    k = block_k(shape, 8, 14) if varcoeff else None
    b = inputs.uniform_rhs(shape, 15, dtype=np.float64)
    ops = mg.hierarchy(shape, k, 8)
    res = mg.pcg(b, ops, tol=1e-8, maxit=200, k=k, kb=8)
    ref = oracle.pcg(b, tol=1e-8, maxit=5000, k=k, kb=8)
    assert res["hist"][-1] <= 1e-8
    assert oracle.true_relres(b, res["x"], k, 8) <= 1.1e-8
    assert res["iters"] <= ref["iters"] // 4, (res["iters"], ref["iters"])
    np.testing.assert_allclose(res["x"], ref["x"], rtol=0, atol=1e-5 * np.max(np.abs(ref["x"])))
