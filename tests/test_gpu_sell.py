"""Jacobi-PCG on a general sparse matrix in Sliced-ELL form (gbpcg_sell_*),
against the FP64 oracle's CSR product and CSR PCG (oracle.csr_apply,
oracle.csr_pcg), called through the C ABI.

  layout   the seven-point operator's slice widths are the slice's longest
           row (bit-exact integer check), the matrix built from CSR holds the
           CSR entries in order with zero padding;
  SpMV     |y_gpu - y| <= 2e-6 * (|A| |x|) elementwise (FP32 products and a
           7- to 20-term FP32 sum per row);
  solve    iterations within 2 of the oracle's CSR PCG, true residual
           ||b - A x|| / ||b|| <= tol by the oracle's FP64 CSR product.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_23343_gb300 import inputs

pytestmark = pytest.mark.gpu
sp = pytest.importorskip("scipy.sparse")


def stencil_csr(shape, k=None, kb=8):
    """The oracle's operator as a CSR matrix, column by column through the oracle's apply (an
    assembly independent of the library's)."""
    n = int(np.prod(shape))
    cols = []
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        cols.append(sp.csr_matrix(oracle.apply(e.reshape(shape), k, kb).reshape(n, 1)))
    return sp.hstack(cols).tocsr()


def random_spd(n, seed, deg=8):
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
    A = (L + sp.diags(shift)).tocsr()
    A.sort_indices()
    return A.astype(np.float32).astype(np.float64).tocsr()  # entries exact in FP32


def to_dev_csr(A):
    return (torch.from_numpy(A.indptr.astype(np.int64)).cuda(), torch.from_numpy(A.indices.astype(np.int32)).cuda(),
            torch.from_numpy(A.data.astype(np.float32)).cuda())


@pytest.mark.parametrize("shape,varcoeff", [((20, 24, 36), False), ((33, 17, 64), False), ((9, 13, 40), True),
                                            ((16, 16, 16), True)])
def test_sell_from_stencil_layout_and_spmv(gpu_lib, shape, varcoeff):
    nz, ny, nx = shape
    k, kd, k64 = None, None, None
    if varcoeff:
        nbx, nby, nbz = inputs.block_counts(nx, ny, nz, 4)
        k = inputs.lognormal_blocks(nbx, nby, nbz, 5)
        kd, k64 = torch.from_numpy(k).cuda(), k.astype(np.float64)
    m = gpu_lib.sell_from_stencil(shape, k_block=kd, kb=4)
    n = nx * ny * nz
    # widths: the longest row of each slice of 32 rows
    i = np.arange(n)
    x, y, z = i % nx, (i // nx) % ny, i // (nx * ny)
    rowlen = 1 + (x > 0) + (x < nx - 1) + (y > 0) + (y < ny - 1) + (z > 0) + (z < nz - 1)
    rl = np.zeros(((n + 31) // 32) * 32, np.int64)
    rl[:n] = rowlen
    widths = rl.reshape(-1, 32).max(axis=1)
    np.testing.assert_array_equal(m.slice_ptr.cpu().numpy(), np.concatenate([[0], np.cumsum(widths * 32)]))
    u = inputs.uniform_rhs(shape, 6, dtype=np.float64).astype(np.float32)
    yg = gpu_lib.sell_spmv(m, torch.from_numpy(u).cuda().ravel()).cpu().double().numpy()
    ref = oracle.apply(u.astype(np.float64), k64, 4).ravel()
    absop = oracle.apply(np.abs(u.astype(np.float64)), k64, 4).ravel()  # not |A||u|: bound below
    A = stencil_csr(shape, k64, 4) if n <= 5000 else None
    bound = (abs(A) @ np.abs(u.astype(np.float64)).ravel()) if A is not None else 4 * np.abs(absop) + \
        8 * np.abs(oracle.diag(shape, k64, 4).ravel() * u.ravel())
    assert np.all(np.abs(yg - ref) <= 2e-6 * bound + 1e-30)
    inv = m.inv_diag.cpu().double().numpy()
    np.testing.assert_allclose(inv, 1.0 / oracle.diag(shape, k64, 4).ravel(), rtol=2e-6)


def test_sell_from_csr_holds_the_csr_entries(gpu_lib):
    A = random_spd(3001, 60)
    rp, cc, vv = to_dev_csr(A)
    m = gpu_lib.sell_from_csr(rp, cc, vv)
    n = A.shape[0]
    lens = np.diff(A.indptr)
    ll = np.zeros(((n + 31) // 32) * 32, np.int64)
    ll[:n] = lens
    widths = ll.reshape(-1, 32).max(axis=1)
    sptr = m.slice_ptr.cpu().numpy()
    np.testing.assert_array_equal(sptr, np.concatenate([[0], np.cumsum(widths * 32)]))
    col, val = m.col.cpu().numpy(), m.val.cpu().numpy()
    for row in (0, 1, 31, 32, 1000, n - 1):
        s, l = row // 32, row % 32
        e = sptr[s] + l + 32 * np.arange(widths[s])
        k = lens[row]
        np.testing.assert_array_equal(col[e[:k]], A.indices[A.indptr[row]:A.indptr[row + 1]])
        np.testing.assert_array_equal(val[e[:k]], A.data[A.indptr[row]:A.indptr[row + 1]].astype(np.float32))
        assert np.all(val[e[k:]] == 0) and np.all(col[e[k:]] == row)
    x = inputs.uniform_pm1(61, 0, n)
    yg = gpu_lib.sell_spmv(m, torch.from_numpy(x).cuda()).cpu().double().numpy()
    ref = oracle.csr_apply(A.indptr, A.indices, A.data, x.astype(np.float64))
    bound = abs(A) @ np.abs(x.astype(np.float64))
    assert np.all(np.abs(yg - ref) <= 2e-6 * bound)


@pytest.mark.parametrize("shape", [(32, 32, 32), (24, 40, 36)])
def test_sell_pcg_on_the_stencil_matrix(gpu_lib, shape):
    """The assembled seven-point operator solved by the SELL path: the oracle's iteration count
    within 2 (the matrix-free oracle, whose CSR form has the same iterates), true residual."""
    b = inputs.uniform_rhs(shape, 62, dtype=np.float64)
    m = gpu_lib.sell_from_stencil(shape)
    x, res = gpu_lib.sell_pcg_solve(m, torch.from_numpy(b).cuda().ravel(), tol=1e-6, maxit=3000)
    ref = oracle.pcg(b, tol=1e-6, maxit=3000)
    assert res["status"] == gpu_lib.OK, res
    assert abs(res["iters"] - ref["iters"]) <= 2, (res["iters"], ref["iters"])
    tr = oracle.true_relres(b, x.cpu().numpy().reshape(shape))
    assert tr <= 1e-6 and abs(res["rel_res_true"] - tr) <= 1e-3 * tr


def test_sell_pcg_on_a_random_spd_matrix(gpu_lib):
    A = random_spd(50000, 63)
    b = inputs.uniform_pm1(64, 0, A.shape[0], np.float64)
    m = gpu_lib.sell_from_csr(*to_dev_csr(A))
    x, res = gpu_lib.sell_pcg_solve(m, torch.from_numpy(b).cuda(), tol=1e-8, maxit=5000)
    ref = oracle.csr_pcg(A.indptr, A.indices, A.data, b, tol=1e-8, maxit=5000)
    assert res["status"] == gpu_lib.OK and ref["status"] == oracle.OK, res
    assert abs(res["iters"] - ref["iters"]) <= 2, (res["iters"], ref["iters"])
    xr = x.cpu().numpy()
    tr = np.linalg.norm(b - oracle.csr_apply(A.indptr, A.indices, A.data, xr)) / np.linalg.norm(b)
    assert tr <= 1e-8 and abs(res["rel_res_true"] - tr) <= 1e-3 * tr


def test_sell_pcg_zero_rhs_cap_and_bad_arguments(gpu_lib):
    m = gpu_lib.sell_from_stencil((8, 8, 8))
    x0 = torch.full((512,), 2.0, dtype=torch.float64, device="cuda")
    x, res = gpu_lib.sell_pcg_solve(m, torch.zeros(512, dtype=torch.float64, device="cuda"), x0)
    assert res["status"] == gpu_lib.OK and res["iters"] == 0 and not torch.any(x)
    b = torch.from_numpy(inputs.uniform_rhs((8, 8, 8), 65, dtype=np.float64)).cuda().ravel()
    x, res = gpu_lib.sell_pcg_solve(m, b, tol=1e-12, maxit=3)
    assert res["status"] == gpu_lib.NOT_CONVERGED and res["iters"] == 3
    tr = oracle.true_relres(b.cpu().numpy().reshape(8, 8, 8), x.cpu().numpy().reshape(8, 8, 8))
    assert abs(res["rel_res_true"] - tr) <= 1e-3 * tr
