"""Batched solves: many independent grids in one graph launch.

Each problem's iterate sequence in the batch is the same arithmetic as its
standalone solve with the same tile configuration, so results must agree
bitwise; convergence is checked against the FP64 oracle.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_23343_gb300 import inputs

pytestmark = pytest.mark.gpu

SHAPES = [(48, 64, 96), (64, 48, 48), (37, 21, 100), (96, 64, 64), (13, 17, 19), (48, 48, 160)]


def test_batched_equals_standalone(gpu_lib):
    bs = [torch.from_numpy(inputs.uniform_rhs(s, 40 + i)).cuda() for i, s in enumerate(SHAPES)]
    xs, res = gpu_lib.pcg_solve_batched(bs, tol=1e-6, maxit=2000)
    for b, x, r in zip(bs, xs, res):
        x1, r1 = gpu_lib.pcg_solve(b, tol=1e-6, maxit=2000)
        assert r["status"] == r1["status"] == 0
        assert r["iters"] == r1["iters"]
        assert torch.equal(x, x1)


def test_batched_against_oracle(gpu_lib):
    shapes = SHAPES[:3]
    bnp = [inputs.uniform_rhs(s, 60 + i, dtype=np.float64) for i, s in enumerate(shapes)]
    bs = [torch.from_numpy(b).cuda() for b in bnp]
    xs, res = gpu_lib.pcg_solve_batched(bs, tol=1e-6, maxit=2000)
    for b, x, r in zip(bnp, xs, res):
        ref = oracle.pcg(b, tol=1e-6, maxit=2000)
        assert r["status"] == 0 and abs(r["iters"] - ref["iters"]) <= 2
        assert oracle.true_relres(b, x.cpu().numpy()) <= 1e-6


def test_autotune_and_batched_autotune(gpu_lib):
    b = torch.from_numpy(inputs.uniform_rhs((64, 64, 96), 70)).cuda()
    code, us = gpu_lib.autotune(b)
    ncfg = len(gpu_lib.tile_configs())
    assert 1 <= (code & 0xFF) <= ncfg and us > 0
    x, r = gpu_lib.pcg_solve(b, tol=1e-6, tile_cfg=code)
    assert r["status"] == 0
    bs = [b, torch.from_numpy(inputs.uniform_rhs((32, 48, 64), 71)).cuda()]
    xs, res = gpu_lib.pcg_solve_batched(bs, tol=1e-6, autotune=True)
    assert all(rr["status"] == 0 for rr in res)
    for bb, xx in zip(bs, xs):
        assert oracle.true_relres(bb.cpu().double().numpy(), xx.cpu().double().numpy()) <= 1.2e-6


@pytest.mark.slow
def test_config3_64_problems(gpu_lib):
    """64 problems, per-axis sizes uniform from {48, 64, 96, 128, 160} (seed 2), RHS
    U[-1,1) from seed 2 after the shape draws; FP64 x and b; tol 1e-6."""
    shapes = inputs.batch_shapes(64, 2)
    rhs = inputs.batch_rhs(shapes, 2, dtype=np.float64)
    bs = [torch.from_numpy(b).cuda() for b in rhs]
    xs, res = gpu_lib.pcg_solve_batched(bs, tol=1e-6, maxit=3000, autotune=True)
    assert len(res) == 64
    for b, x, r in zip(rhs, xs, res):
        assert r["status"] == 0, r
        assert oracle.true_relres(b, x.cpu().numpy()) <= 1e-6


def test_batched_problems_keep_their_own_scale(gpu_lib):
    """Each problem of a batch scales its own right-hand side: problems at 2^-200, 1 and 2^200
    in one launch take the iterations of the unscaled problem and return its solution scaled,
    bit for bit."""
    b = inputs.uniform_rhs((24, 20, 36), 77, dtype=np.float64)
    powers = (-200, 0, 200)
    bs = [torch.from_numpy(b * 2.0 ** p).cuda() for p in powers]
    xs, res = gpu_lib.pcg_solve_batched(bs, tol=1e-8, maxit=3000)
    x0 = xs[1].cpu().numpy()
    for p, x, r in zip(powers, xs, res):
        assert r["status"] == 0 and r["iters"] == res[1]["iters"], (p, r)
        assert np.array_equal(x.cpu().numpy() * 2.0 ** -p, x0), p
        assert oracle.true_relres(b * 2.0 ** p, x.cpu().numpy()) <= 1e-8
