"""The multigrid preconditioner on the GPU (gbpcg_mg_vcycle, gbpcg_mg_pcg_solve)
against the FP64 oracle (oracle/mg.py), through the C ABI.

V-cycle: element by element, |z_gpu - z| <= 2e-5 * V_abs(|r|), where V_abs is
the same V-cycle run on |r| with every subtraction turned into an addition
(|A| for A, |f| for f): the sum of the magnitudes of all the terms each output
accumulates through the levels, which bounds the FP32 rounding of the GPU's
evaluation (a few dozen roundings per term at most).  Solve: iterations within
2 of the oracle's MG-PCG, true residual <= tol by the oracle's FP64 residual.
"""
import numpy as np
import pytest
import torch

import oracle
import oracle.mg as mg
from paper_2603_23343_gb300 import inputs

pytestmark = pytest.mark.gpu


def abs_op(op):
    return op  # weights and diagonal are non-negative already


def vcycle_abs(ops, f, level=0):
    """The V-cycle with |.| everywhere: an elementwise bound on the magnitude of the terms."""
    op = ops[level]
    D = op[3]
    absA = lambda u: 2 * D * u - mg.apply(op, u)  # noqa: E731  D u + sum w u_nb for u >= 0
    if level == len(ops) - 1:
        u = mg.OMEGA * f / D
        for _ in range(mg.COARSE_SWEEPS - 1):
            u = u + mg.OMEGA * (f + absA(u)) / D
        return u
    u = mg.OMEGA * f / D
    e = vcycle_abs(ops, mg.restrict(f + absA(u)), level + 1)
    u = u + mg.SIGMA * mg.prolong(e)
    return u + mg.OMEGA * (f + absA(u)) / D


def case(shape, varcoeff, seed):
    nz, ny, nx = shape
    k, kd = None, None
    if varcoeff:
        nbx, nby, nbz = inputs.block_counts(nx, ny, nz, 8)
        k = inputs.lognormal_blocks(nbx, nby, nbz, seed).astype(np.float64)
        kd = torch.from_numpy(k).float().cuda()
    return k, kd


@pytest.mark.parametrize("shape,varcoeff", [((32, 32, 32), False), ((16, 24, 32), True), ((64, 64, 64), True),
                                            ((8, 8, 12), False), ((20, 12, 44), False), ((6, 4, 8), True),
                                            ((4, 4, 4), False), ((128, 64, 64), False)])
def test_vcycle_elementwise(gpu_lib, shape, varcoeff):
    """One V-cycle against the oracle's, element by element: hierarchies of one level (6 x 4 x 8,
    4^3: the coarsest sweeps are the whole cycle), of levels all inside the one-CTA tail (32^3
    and smaller), and with level kernels above it (64^3, 128 x 64 x 64)."""
    k, kd = case(shape, varcoeff, 20)
    r = inputs.uniform_rhs(shape, 21)
    z, levels = gpu_lib.mg_vcycle(torch.from_numpy(r).cuda(), k_block=kd)
    ops = mg.hierarchy(shape, k, 8)
    assert levels == len(ops)
    r64 = r.astype(np.float64)
    ref = mg.vcycle(ops, r64)
    bound = vcycle_abs(ops, np.abs(r64))
    err = np.abs(z.cpu().double().numpy() - ref)
    assert np.all(err <= 2e-5 * bound), float(np.max(err / bound))


@pytest.mark.parametrize("shape,varcoeff", [((32, 32, 32), False), ((32, 32, 32), True), ((40, 48, 64), False),
                                            ((64, 64, 64), True)])
def test_mg_pcg_against_oracle(gpu_lib, shape, varcoeff):
    k, kd = case(shape, varcoeff, 22)
    b = inputs.uniform_rhs(shape, 23, dtype=np.float64)
    x, res = gpu_lib.mg_pcg_solve(torch.from_numpy(b).cuda(), tol=1e-6, maxit=500, k_block=kd)
    ref = mg.pcg(b, mg.hierarchy(shape, k, 8), tol=1e-6, maxit=500, k=k, kb=8)
    assert res["status"] == gpu_lib.OK, res
    assert abs(res["iters"] - ref["iters"]) <= 2, (res["iters"], ref["iters"])
    tr = oracle.true_relres(b, x.cpu().numpy(), k, 8)
    assert tr <= 1e-6 and abs(res["rel_res_true"] - tr) <= 1e-3 * tr


def test_mg_pcg_tight_tolerance_zero_rhs_and_cap(gpu_lib):
    shape = (32, 32, 32)
    b = inputs.uniform_rhs(shape, 24, dtype=np.float64)
    bd = torch.from_numpy(b).cuda()
    x, res = gpu_lib.mg_pcg_solve(bd, tol=1e-10, maxit=500)
    assert res["status"] == gpu_lib.OK and res["replacements"] >= 1
    assert oracle.true_relres(b, x.cpu().numpy()) <= 1e-10
    x0 = torch.full_like(bd, 3.0)
    xz, rz = gpu_lib.mg_pcg_solve(torch.zeros_like(bd), x0)
    assert rz["status"] == gpu_lib.OK and rz["iters"] == 0 and not torch.any(xz)
    xc, rc = gpu_lib.mg_pcg_solve(bd, tol=1e-12, maxit=3)
    assert rc["status"] == gpu_lib.NOT_CONVERGED and rc["iters"] == 3
    tr = oracle.true_relres(b, xc.cpu().numpy())
    assert abs(rc["rel_res_true"] - tr) <= 1e-3 * tr
