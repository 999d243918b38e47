"""Pins of the FP64 oracle against facts the mathematics fixes (CPU only).

Each test is chosen so that a plausible slip in ``oracle/oracle.c`` (a wrong
sign, a dropped neighbour, a transposed index, a wrong boundary value, a
wrong face coefficient, an off-by-one in the CG recurrences) fails it.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from paper_2603_23343_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def grid_coords(n):
    """Interior point coordinates (i+1) h, h = 1/(n+1), on the unit interval."""
    return np.arange(1, n + 1) / (n + 1.0)


def sine_mode(shape, a, b, c):
    nz, ny, nx = shape
    x, y, z = grid_coords(nx), grid_coords(ny), grid_coords(nz)
    return (np.sin(c * np.pi * z)[:, None, None] * np.sin(b * np.pi * y)[None, :, None]
            * np.sin(a * np.pi * x)[None, None, :])


def sine_eig(shape, a, b, c):
    """Closed-form eigenvalue of the 7-point Dirichlet Laplacian for mode (a,b,c)."""
    nz, ny, nx = shape
    lam = 0.0
    for n, m in ((nx, a), (ny, b), (nz, c)):
        h = 1.0 / (n + 1)
        lam += 4.0 / h**2 * np.sin(m * np.pi * h / 2) ** 2
    return lam


# ---------------------------------------------------------------- stencil --

@pytest.mark.parametrize("shape,mode", [((8, 8, 8), (1, 1, 1)), ((8, 8, 8), (3, 5, 8)),
                                        ((5, 7, 3), (2, 1, 3)), ((9, 4, 6), (6, 4, 9)),
                                        ((32, 32, 32), (7, 1, 30))])
def test_poisson_sine_eigenpairs(shape, mode):
    v = sine_mode(shape, *mode)
    lam = sine_eig(shape, *mode)
    av = oracle.apply_poisson(v)
    assert np.max(np.abs(av - lam * v)) <= 1e-11 * lam * np.max(np.abs(v))


@pytest.mark.parametrize("shape", [(6, 6, 6), (5, 9, 7), (16, 11, 13)])
def test_poisson_manufactured_quadratic(shape):
    """Central differences are exact on quadratics: A u* = -Lap u* at every point."""
    nz, ny, nx = shape
    x = grid_coords(nx)[None, None, :]
    y = grid_coords(ny)[None, :, None]
    z = grid_coords(nz)[:, None, None]
    gx, gy, gz = x * (1 - x), y * (1 - y), z * (1 - z)
    u = gx * gy * gz
    f = 2.0 * (gy * gz + gx * gz + gx * gy)
    assert np.max(np.abs(oracle.apply_poisson(u) - f)) <= 1e-9 * np.max(np.abs(f))


def dense_matrix(shape, k=None, kb=8):
    n = int(np.prod(shape))
    A = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = oracle.apply(e.reshape(shape), k, kb).ravel()
    return A


@pytest.mark.parametrize("shape", [(4, 4, 4), (5, 4, 3)])
def test_poisson_dense_symmetric_spd_spectrum(shape):
    A = dense_matrix(shape)
    assert np.array_equal(A, A.T)
    np.linalg.cholesky(A)
    nz, ny, nx = shape
    expect = sorted(sine_eig(shape, a, b, c) for a in range(1, nx + 1) for b in range(1, ny + 1)
                    for c in range(1, nz + 1))
    got = np.linalg.eigvalsh(A)
    np.testing.assert_allclose(got, expect, rtol=1e-10)
    # the diagonal of A is the Jacobi diagonal
    np.testing.assert_array_equal(np.diag(A), oracle.diag(shape).ravel())


def test_varcoeff_constant_k_is_scaled_poisson():
    shape = (12, 10, 9)
    u = inputs.uniform_rhs(shape, 5, dtype=np.float64)
    kb = inputs.block_counts(9, 10, 12, 4)
    c = 3.25
    k = np.full((kb[2], kb[1], kb[0]), c)
    np.testing.assert_allclose(oracle.apply_varcoeff(u, k, 4), c * oracle.apply_poisson(u),
                               rtol=1e-13, atol=1e-10)
    np.testing.assert_allclose(oracle.diag(shape, k, 4), c * oracle.diag(shape), rtol=1e-14)


def face_energy(u, kcell):
    """u.Au written as a sum over faces: interior faces carry the harmonic mean
    of the two cells' k times (u_a-u_b)^2; boundary faces carry the cell's own
    k times u_c^2 (the outside value is zero); each term is divided by h_d^2."""
    nz, ny, nx = u.shape
    e = 0.0
    for axis, n in ((2, nx), (1, ny), (0, nz)):
        h2 = (1.0 / (n + 1)) ** 2
        ua = np.moveaxis(u, axis, 0)
        ka = np.moveaxis(kcell, axis, 0)
        kf = 2 * ka[:-1] * ka[1:] / (ka[:-1] + ka[1:])
        e += np.sum(kf * (ua[1:] - ua[:-1]) ** 2) / h2
        e += (np.sum(ka[0] * ua[0] ** 2) + np.sum(ka[-1] * ua[-1] ** 2)) / h2
    return e


@pytest.mark.parametrize("shape,kb", [((6, 5, 7), 2), ((16, 16, 16), 8), ((9, 12, 10), 4)])
def test_varcoeff_energy_identity(shape, kb):
    nz, ny, nx = shape
    nbx, nby, nbz = inputs.block_counts(nx, ny, nz, kb)
    k = inputs.lognormal_blocks(nbx, nby, nbz, 11).astype(np.float64)
    kcell = np.repeat(np.repeat(np.repeat(k, kb, 0), kb, 1), kb, 2)[:nz, :ny, :nx]
    u = inputs.uniform_rhs(shape, 12, dtype=np.float64)
    lhs = float(np.sum(u * oracle.apply_varcoeff(u, k, kb)))
    assert abs(lhs - face_energy(u, kcell)) <= 1e-12 * abs(lhs)
    # the diagonal is the energy of a unit vector
    d = oracle.diag(shape, k, kb)
    for idx in [(0, 0, 0), (nz - 1, ny // 2, nx - 1), (nz // 2, ny - 1, 1)]:
        e = np.zeros(shape)
        e[idx] = 1.0
        assert abs(d[idx] - face_energy(e, kcell)) <= 1e-12 * d[idx]


def test_varcoeff_dense_symmetric_spd():
    shape, kb = (4, 5, 6), 2
    nbx, nby, nbz = inputs.block_counts(6, 5, 4, kb)
    k = inputs.lognormal_blocks(nbx, nby, nbz, 3).astype(np.float64)
    A = dense_matrix(shape, k, kb)
    np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-12 * np.max(np.abs(A)))
    np.linalg.cholesky(A)
    np.testing.assert_allclose(np.diag(A), oracle.diag(shape, k, kb).ravel(), rtol=1e-15)


# -------------------------------------------------------------- dot, axpy --

@pytest.mark.parametrize("n", [1, 7, 4096, 4097, 1_000_003])
def test_dot_integer_closed_forms(n):
    i = np.arange(n, dtype=np.float64)
    assert oracle.dot(i, np.ones(n)) == n * (n - 1) // 2
    s2 = (n - 1) * n * (2 * n - 1) // 6
    if s2 < 2**53:  # every partial sum is then an exactly representable integer
        assert oracle.dot(i, i) == s2


def test_dot_random_against_exact_rational_sum():
    from fractions import Fraction
    x = inputs.uniform_pm1(7, 0, 3001, np.float64)
    y = inputs.uniform_pm1(8, 0, 3001, np.float64)
    exact = sum(Fraction(a) * Fraction(b) for a, b in zip(x.tolist(), y.tolist()))
    assert abs(oracle.dot(x, y) - float(exact)) <= 1e-13 * float(np.sum(np.abs(x * y)))


def test_axpy_integer_exact():
    n = 10001
    x = np.arange(n, dtype=np.float64)
    y = 2.0 * np.arange(n, dtype=np.float64) + 1.0
    out = oracle.axpy(-3.0, x, y)
    np.testing.assert_array_equal(out, -np.arange(n) + 1.0)


# -------------------------------------------------------------------- PCG --

def test_pcg_single_mode_one_iteration():
    shape = (9, 9, 9)
    b = sine_mode(shape, 2, 3, 1)
    res = oracle.pcg(b, tol=1e-12, maxit=50, history=True)
    assert res["status"] == oracle.OK and res["iters"] == 1
    lam = sine_eig(shape, 2, 3, 1)
    np.testing.assert_allclose(res["x"], b / lam, rtol=0, atol=1e-13 * np.max(np.abs(b)) / lam)


@pytest.mark.parametrize("precond", ["jacobi", None])
def test_pcg_exact_termination_m_modes(precond):
    """CG on a right-hand side spanning m eigenvectors with distinct eigenvalues
    terminates in exactly m steps (exact arithmetic; FP64 to 1e-10)."""
    shape = (8, 7, 6)
    modes = [(1, 1, 1), (2, 3, 1), (5, 2, 4), (6, 7, 8)]
    b = sum((j + 1.0) * sine_mode(shape, *m) for j, m in enumerate(modes))
    res = oracle.pcg(b, tol=1e-10, maxit=50, precond=precond, history=True)
    assert res["iters"] == len(modes)
    assert res["hist"][len(modes) - 1] > 1e-6


def test_pcg_manufactured_solution():
    shape = (20, 18, 22)
    nz, ny, nx = shape
    x = grid_coords(nx)[None, None, :]
    y = grid_coords(ny)[None, :, None]
    z = grid_coords(nz)[:, None, None]
    gx, gy, gz = x * (1 - x), y * (1 - y), z * (1 - z)
    u = gx * gy * gz
    f = 2.0 * (gy * gz + gx * gz + gx * gy)
    res = oracle.pcg(f, tol=1e-12, maxit=2000)
    assert res["status"] == oracle.OK
    np.testing.assert_allclose(res["x"], u, rtol=0, atol=1e-9 * np.max(u))
    assert oracle.true_relres(f, res["x"]) <= 1e-11


def _scipy_cg_iterates(A, b, M, rtol, maxiter):
    sla = pytest.importorskip("scipy.sparse.linalg")
    xs = []
    x, info = sla.cg(A, b, rtol=rtol, atol=0.0, maxiter=maxiter, M=M, callback=lambda xk: xs.append(xk.copy()))
    return x, info, xs


@pytest.mark.parametrize("varcoeff", [False, True])
def test_pcg_matches_scipy_cg(varcoeff):
    sp = pytest.importorskip("scipy.sparse")
    shape = (7, 6, 8)
    nz, ny, nx = shape
    k = None
    if varcoeff:
        nbx, nby, nbz = inputs.block_counts(nx, ny, nz, 2)
        k = inputs.lognormal_blocks(nbx, nby, nbz, 21).astype(np.float64)
        A = sp.csr_matrix(dense_matrix(shape, k, 2))
    else:
        # independent assembly: Kronecker sum of 1D Dirichlet second differences
        def lap1d(n):
            h = 1.0 / (n + 1)
            return sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]) / h**2
        Ix, Iy, Iz = sp.identity(nx), sp.identity(ny), sp.identity(nz)
        A = (sp.kron(Iz, sp.kron(Iy, lap1d(nx))) + sp.kron(Iz, sp.kron(lap1d(ny), Ix))
             + sp.kron(lap1d(nz), sp.kron(Iy, Ix))).tocsr()
    b = inputs.uniform_rhs(shape, 4, dtype=np.float64)
    Minv = sp.diags(1.0 / A.diagonal())
    xs_ref, info, iterates = _scipy_cg_iterates(A, b.ravel(), Minv, 1e-9, 500)
    res = oracle.pcg(b, tol=1e-9, maxit=500, k=k, kb=2, history=True)
    assert info == 0 and res["status"] == oracle.OK
    assert abs(res["iters"] - len(iterates)) <= 1
    np.testing.assert_allclose(res["x"].ravel(), xs_ref, rtol=0, atol=1e-8 * np.max(np.abs(xs_ref)))
    # residual history of the first iterates agrees with scipy's
    bn = np.linalg.norm(b)
    for it in range(1, min(6, len(iterates)) + 1):
        ref = np.linalg.norm(b.ravel() - A @ iterates[it - 1]) / bn
        assert abs(res["hist"][it] - ref) <= 1e-9 * ref


def test_pcg_jacobi_equals_plain_cg_for_constant_coefficient():
    b = inputs.uniform_rhs((10, 11, 12), 9, dtype=np.float64)
    a = oracle.pcg(b, tol=1e-8, maxit=500, precond="jacobi")
    c = oracle.pcg(b, tol=1e-8, maxit=500, precond=None)
    assert a["iters"] == c["iters"]
    np.testing.assert_allclose(a["x"], c["x"], rtol=1e-10, atol=1e-14)


def test_pcg_zero_rhs_and_maxit():
    z = oracle.pcg(np.zeros((3, 4, 5)), x0=np.ones((3, 4, 5)), tol=1e-6, maxit=10)
    assert z["iters"] == 0 and z["status"] == oracle.OK and not np.any(z["x"])
    b = inputs.uniform_rhs((16, 16, 16), 0, dtype=np.float64)
    m = oracle.pcg(b, tol=1e-14, maxit=5)
    assert m["iters"] == 5 and m["status"] == oracle.NOT_CONVERGED


def test_pcg_nonzero_initial_guess():
    shape = (9, 10, 11)
    b = inputs.uniform_rhs(shape, 31, dtype=np.float64)
    x0 = inputs.uniform_rhs(shape, 32, dtype=np.float64) * 1e-3
    res = oracle.pcg(b, x0=x0, tol=1e-10, maxit=1000)
    assert res["status"] == oracle.OK
    assert oracle.true_relres(b, res["x"]) <= 1e-9


def test_refinement_reaches_tight_tolerance_and_direct_solve():
    shape = (6, 7, 5)
    nz, ny, nx = shape
    nbx, nby, nbz = inputs.block_counts(nx, ny, nz, 2)
    k = inputs.lognormal_blocks(nbx, nby, nbz, 1).astype(np.float64)
    b = inputs.uniform_rhs(shape, 1, dtype=np.float64)
    res = oracle.refine(b, tol=1e-12, inner_tol=1e-2, k=k, kb=2)
    assert res["relres"] <= 1e-12 and 2 <= res["steps"] <= 30
    x_direct = np.linalg.solve(dense_matrix(shape, k, 2), b.ravel())
    np.testing.assert_allclose(res["x"].ravel(), x_direct, rtol=0, atol=1e-10 * np.max(np.abs(x_direct)))


# ---------------------------------------------------------------- goldens --

def test_golden_config0_history_is_reproduced():
    """The stored 32^3 seed-0 history was written by tests/golden/make_golden.py
    (oracle only); re-running the oracle must give the same numbers."""
    with open(os.path.join(GOLDEN, "pcg_poisson32_seed0.json")) as f:
        g = json.load(f)
    b = inputs.poisson_problem(32, 0, np.float64)
    res = oracle.pcg(b, tol=g["tol"], maxit=g["maxit"], history=True)
    assert res["iters"] == g["iters"]
    np.testing.assert_allclose(res["hist"], g["hist"], rtol=1e-9)


def test_golden_paper_table3_grid():
    """Table 3 / Sec. VII-A: the comparison grid 512x112x64 has 3,670,016
    unknowns, which equals 56 cores x 64 tiles x 1024 elements."""
    with open(os.path.join(GOLDEN, "paper_table3_grid.txt")) as f:
        vals = [int(t) for t in f.read().split("#")[0].split()]
    nx, ny, nz, n, cores, tiles, tile = vals
    assert nx * ny * nz == n == cores * tiles * tile


def test_input_generator_published_vector():
    """SplitMix64 with seed 0 (Steele et al. 2014) begins e220a8397b1dcdaf, 6e789e6aa1b965f4."""
    z = inputs.splitmix64(0, 0, 4)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                   0x06C45D188009454F, 0xF88BB8A8724C81EC]
    u = inputs.uniform_pm1(0, 0, 1000, np.float64)
    assert np.array_equal(u.astype(np.float32).astype(np.float64), u)
    assert u.min() >= -1.0 and u.max() < 1.0


# ---------------------------------------------------------- general sparse (CSR) --

def kron_poisson(shape):
    """The seven-point Dirichlet Poisson matrix assembled independently as a Kronecker sum of 1D
    second differences (scipy CSR, float64)."""
    sp = pytest.importorskip("scipy.sparse")
    nz, ny, nx = shape

    def lap1d(n):
        h = 1.0 / (n + 1)
        return sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]) / h**2
    Ix, Iy, Iz = sp.identity(nx), sp.identity(ny), sp.identity(nz)
    return (sp.kron(Iz, sp.kron(Iy, lap1d(nx))) + sp.kron(Iz, sp.kron(lap1d(ny), Ix))
            + sp.kron(lap1d(nz), sp.kron(Iy, Ix))).tocsr()


def random_spd_csr(n, seed, deg=6):
    """A sparse symmetric positive definite matrix: the Laplacian of a random graph (seeded,
    positive edge weights) plus a positive diagonal shift."""
    sp = pytest.importorskip("scipy.sparse")
    m = n * deg // 2
    u = inputs.uniform_pm1(seed, 0, 3 * m, np.float64)
    a = ((u[:m] + 1) * 0.5 * n).astype(np.int64) % n
    b = ((u[m:2 * m] + 1) * 0.5 * n).astype(np.int64) % n
    w = 1.0 + 0.5 * (u[2 * m:] + 1)
    keep = a != b
    W = sp.coo_matrix((w[keep], (a[keep], b[keep])), shape=(n, n))
    W = (W + W.T).tocsr()
    L = sp.diags(np.asarray(W.sum(axis=1)).ravel()) - W
    shift = 0.05 + 0.5 * (inputs.uniform_pm1(seed + 1, 0, n, np.float64) + 1)
    return (L + sp.diags(shift)).tocsr()


@pytest.mark.parametrize("shape", [(4, 4, 4), (5, 3, 7), (9, 8, 6)])
def test_csr_apply_of_assembled_poisson_is_the_stencil(shape):
    A = kron_poisson(shape)
    u = inputs.uniform_rhs(shape, 31, dtype=np.float64)
    y = oracle.csr_apply(A.indptr, A.indices, A.data, u)
    ref = oracle.apply(u).ravel()
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-12 * np.max(np.abs(ref)))


def test_csr_apply_random_matrix_against_dense():
    A = random_spd_csr(300, 40)
    x = inputs.uniform_pm1(41, 0, 300, np.float64)
    np.testing.assert_allclose(oracle.csr_apply(A.indptr, A.indices, A.data, x), A.toarray() @ x, rtol=1e-13,
                               atol=1e-13)


def test_csr_pcg_equals_matrix_free_pcg_on_poisson():
    shape = (9, 8, 10)
    A = kron_poisson(shape)
    b = inputs.uniform_rhs(shape, 33, dtype=np.float64)
    ref = oracle.pcg(b, tol=1e-10, maxit=500, history=True)
    res = oracle.csr_pcg(A.indptr, A.indices, A.data, b, tol=1e-10, maxit=500, history=True)
    assert res["status"] == ref["status"] == oracle.OK
    assert res["iters"] == ref["iters"]
    np.testing.assert_allclose(res["hist"], ref["hist"], rtol=1e-9, atol=0)
    np.testing.assert_allclose(res["x"], ref["x"].ravel(), rtol=0, atol=1e-12 * np.max(np.abs(ref["x"])))


def test_csr_pcg_matches_scipy_cg_on_random_spd():
    sp = pytest.importorskip("scipy.sparse")
    A = random_spd_csr(2000, 50)
    b = inputs.uniform_pm1(51, 0, 2000, np.float64)
    Minv = sp.diags(1.0 / A.diagonal())
    xs_ref, info, iterates = _scipy_cg_iterates(A, b, Minv, 1e-10, 2000)
    res = oracle.csr_pcg(A.indptr, A.indices, A.data, b, tol=1e-10, maxit=2000, history=True)
    assert info == 0 and res["status"] == oracle.OK
    assert abs(res["iters"] - len(iterates)) <= 1
    np.testing.assert_allclose(res["x"], xs_ref, rtol=0, atol=1e-8 * np.max(np.abs(xs_ref)))
    bn = np.linalg.norm(b)
    for it in range(1, 6):
        r = np.linalg.norm(b - A @ iterates[it - 1]) / bn
        assert abs(res["hist"][it] - r) <= 1e-9 * r


def test_csr_pcg_exact_termination_two_eigenvalues():
    """2 x 2 blocks [[2, 1], [1, 2]] on the diagonal: D^-1 A has the two eigenvalues 1/2 and 3/2,
    so (preconditioned) CG ends in exactly two steps."""
    sp = pytest.importorskip("scipy.sparse")
    blk = np.array([[2.0, 1.0], [1.0, 2.0]])
    A = sp.block_diag([blk * (1.0 + i % 3) for i in range(50)]).tocsr()
    b = inputs.uniform_pm1(52, 0, 100, np.float64)
    res = oracle.csr_pcg(A.indptr, A.indices, A.data, b, tol=1e-14, maxit=10)
    assert res["status"] == oracle.OK and res["iters"] == 2
    np.testing.assert_allclose(A @ res["x"], b, rtol=0, atol=1e-13)


def test_config2_lattice_fixture_is_a_converged_oracle_solve():
    """The stored 512^3 lognormal solution (tests/golden/make_golden.py --config2, the oracle
    alone): a converged run to 1e-10 whose recursive and true residuals agree, sampled on the
    stated 16^3 lattice, with a nonzero solution."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "pcg_lognormal512_seed1_lattice.json")) as f:
        g = json.load(f)
    assert g["n"] == 512 and g["seed"] == 1 and g["kb"] == 8 and g["status"] == 0
    assert g["relres"] <= g["tol"] == 1e-10 and abs(g["true_relres"] - g["relres"]) <= 1e-3 * g["relres"]
    m = len(range(g["lattice_start"], g["n"], g["lattice_step"]))
    assert len(g["x_lattice"]) == m ** 3 == 16 ** 3
    xl = np.asarray(g["x_lattice"])
    assert np.all(np.isfinite(xl)) and 0 < np.linalg.norm(xl) <= g["x_norm2"]
