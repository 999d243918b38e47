"""GPU parity of the Jacobi-PCG solve against the FP64 oracle.

Bar (FP32 vectors, FP64 scalars): iteration count within +-2 of the oracle's
on the same input; true residual ||b - A x||/||b|| (evaluated by the oracle
in FP64 on the GPU's x) <= tol; the library's own FP64 true residual agrees
with the oracle's evaluation.
"""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2603_23343_gb300 import inputs

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def solve(gpu_lib, b, io=np.float32, **kw):
    bd = torch.from_numpy(np.ascontiguousarray(b, dtype=io)).cuda()
    x, res = gpu_lib.pcg_solve(bd, **kw)
    return x.cpu().double().numpy(), res


def check_against_oracle(gpu_lib, b, tol=1e-6, maxit=2000, k=None, kb=8, io=np.float32, **kw):
    kd = None if k is None else torch.from_numpy(k).cuda()
    x, res = solve(gpu_lib, b, io=io, tol=tol, maxit=maxit, k_block=kd, kb=kb, **kw)
    k64 = None if k is None else k.astype(np.float64)
    ref = oracle.pcg(b.astype(np.float64), tol=tol, maxit=maxit, k=k64, kb=kb)
    true_rel = oracle.true_relres(b.astype(np.float64), x, k64, kb)
    assert res["status"] == oracle.OK, res
    assert res["replacements"] >= 1  # convergence is always confirmed on a replaced (true) residual
    assert abs(res["iters"] - ref["iters"]) <= 2, (res["iters"], ref["iters"])
    assert true_rel <= tol, true_rel
    assert abs(res["rel_res_true"] - true_rel) <= 1e-3 * true_rel + 1e-12
    # same problem, same iterate: the solutions agree to the solver's accuracy
    assert np.linalg.norm(x - ref["x"]) <= 50 * tol * np.linalg.norm(ref["x"]) + 1e-30
    return x, res, ref


@pytest.mark.parametrize("io", [np.float32, np.float64])
def test_config0_poisson32(gpu_lib, io):
    """32^3 Poisson, b ~ U[-1,1) seed 0, Jacobi, tol 1e-6, maxit 2000."""
    with open(os.path.join(GOLDEN, "pcg_poisson32_seed0.json")) as f:
        g = json.load(f)
    b = inputs.poisson_problem(32, 0)
    x, res, ref = check_against_oracle(gpu_lib, b, io=io)
    assert abs(res["iters"] - g["iters"]) <= 2


@pytest.mark.parametrize("shape", [(13, 17, 19), (40, 24, 100), (33, 9, 64), (8, 8, 8), (1, 1, 4), (64, 48, 96)])
def test_shapes_tma_and_plain_paths(gpu_lib, shape):
    b = inputs.uniform_rhs(shape, 21)
    check_against_oracle(gpu_lib, b)


@pytest.mark.parametrize("shape,kb", [((48, 48, 48), 8), ((24, 20, 36), 4), ((13, 11, 9), 3), ((10, 14, 22), 4)])
@pytest.mark.parametrize("io", [np.float32, np.float64])
def test_block_coefficient_lognormal(gpu_lib, shape, kb, io):
    """Block coefficients, including partial blocks at the far end of every axis (10 x 14 x 22
    with 4^3 blocks): the passes' FP32 face table and the residuals' FP64 face table."""
    nz, ny, nx = shape
    k, b = inputs.varcoeff_problem(nx, ny, nz, seed=1, kb=kb)
    check_against_oracle(gpu_lib, b, k=k, kb=kb, maxit=5000, io=io)


def test_zero_rhs_gives_zero(gpu_lib):
    b = np.zeros((16, 16, 16), np.float32)
    x0 = torch.ones(16, 16, 16, device="cuda")
    x, res = gpu_lib.pcg_solve(torch.from_numpy(b).cuda(), x=x0)
    assert res["iters"] == 0 and res["status"] == 0
    assert float(x.abs().max()) == 0.0


def test_maxit_limits(gpu_lib):
    b = inputs.poisson_problem(24, 0)
    _, r0 = solve(gpu_lib, b, maxit=0)
    assert r0["iters"] == 0 and r0["status"] == 3
    x5, r5 = solve(gpu_lib, b, maxit=5, tol=1e-12)
    ref = oracle.pcg(b.astype(np.float64), tol=1e-12, maxit=5, history=True)
    assert r5["iters"] == 5 and r5["status"] == 3
    assert abs(r5["rel_res_recursive"] - ref["hist"][5]) <= 1e-4 * ref["hist"][5]
    np.testing.assert_allclose(x5, ref["x"], rtol=0, atol=1e-5 * np.max(np.abs(ref["x"])))


def test_single_sine_mode_one_iteration(gpu_lib):
    n = 20
    s = np.sin(2 * np.pi * np.arange(1, n + 1) / (n + 1))
    b = (s[:, None, None] * s[None, :, None] * s[None, None, :]).astype(np.float32)
    _, res = solve(gpu_lib, b, tol=1e-5)
    assert res["iters"] == 1


def test_nonzero_initial_guess(gpu_lib):
    shape = (20, 22, 24)
    b = inputs.uniform_rhs(shape, 31)
    x0 = inputs.uniform_rhs(shape, 32) * 1e-3
    x, res = gpu_lib.pcg_solve(torch.from_numpy(b).cuda(), x=torch.from_numpy(x0).cuda(), tol=1e-6)
    ref = oracle.pcg(b.astype(np.float64), x0=x0.astype(np.float64), tol=1e-6)
    assert abs(res["iters"] - ref["iters"]) <= 2
    assert oracle.true_relres(b.astype(np.float64), x.cpu().double().numpy()) <= 1e-6


@pytest.mark.parametrize("io", [np.float32, np.float64])
def test_host_io_matches_device_and_is_deterministic(gpu_lib, io):
    b = inputs.poisson_problem(40, 7).astype(io)
    xd, rd = solve(gpu_lib, b, io=io)
    xd2, rd2 = solve(gpu_lib, b, io=io)
    assert np.array_equal(xd, xd2) and rd["iters"] == rd2["iters"]
    bh = torch.from_numpy(b).pin_memory()
    xh = torch.zeros_like(bh).pin_memory()
    x, rh = gpu_lib.pcg_solve(bh, x=xh, host_io=True)
    torch.cuda.synchronize()
    assert not x.is_cuda
    assert rh["iters"] == rd["iters"]
    assert np.array_equal(x.double().numpy(), xd)


@pytest.mark.slow
def test_config1_poisson256_full_size(gpu_lib):
    """256^3 Poisson, h = 1/257, b ~ U[-1,1) seed 0, FP64 x and b: the benchmark's launch configuration."""
    b = inputs.poisson_problem(256, 0)
    check_against_oracle(gpu_lib, b, io=np.float64)


@pytest.mark.slow
def test_table3_grid_fp64_solution(gpu_lib):
    """The paper's Table 3 grid (512 x 112 x 64), FP64 x: converges in its true residual."""
    b = inputs.uniform_rhs((64, 112, 512), 0)
    check_against_oracle(gpu_lib, b, io=np.float64)


def test_fp32_solution_accuracy_floor_stops_early(gpu_lib):
    """FP32 x cannot represent a solution of the 512 x 112 x 64 problem to 1e-6
    (the rounding of x alone leaves a larger residual): the solve must stop
    well before maxit with NOT_CONVERGED and report the true residual it has."""
    b = inputs.uniform_rhs((64, 112, 512), 0)
    x, res = solve(gpu_lib, b, tol=1e-6, maxit=2000)
    assert res["iters"] < 1500
    assert res["status"] in (0, 3)
    true_rel = oracle.true_relres(b.astype(np.float64), x)
    assert abs(res["rel_res_true"] - true_rel) <= 1e-3 * true_rel
    if res["status"] == 0:
        assert true_rel <= 1e-6


@pytest.mark.parametrize("cfg", range(10))
def test_every_tile_configuration(gpu_lib, cfg):
    """Each tile configuration, for pass A and for pass B, on ragged grids
    (whole-row configurations also on a row narrower than their 256 tile)."""
    ncfg = len(gpu_lib.tile_configs())
    assert ncfg == 10
    other = (cfg + 1) % ncfg
    for shape in [(37, 21, 100), (19, 13, 256)]:
        b = inputs.uniform_rhs(shape, 23)
        # FP64 x: the anisotropic 19x13x256 grid is below FP32 x's accuracy floor at 1e-6
        check_against_oracle(gpu_lib, b, io=np.float64, tile_cfg=gpu_lib.tile_cfg_code(cfg, other))


def test_pass_b_cuts_chunks_into_parts(gpu_lib):
    """Pass B marches pass A's z chunks; where its occupancy leaves room it cuts each chunk
    into parts, one CTA each.  Pass A on 6-stage 128x8 tiles (2 CTAs per SM) and pass B on
    3-stage 128x8 tiles over a ragged 61 x 250 x 252 grid: pass B gets at least twice pass A's
    CTAs (same tiles), and the last chunk's last part is shorter than the others.  The solve
    takes the default partition's iterations (within one: partial sums are added in another
    order) and meets the tolerance on the oracle's FP64 true residual."""
    shape = (61, 250, 252)
    b = inputs.uniform_rhs(shape, 31, dtype=np.float64)
    bd = torch.from_numpy(b).cuda()
    cfgs = gpu_lib.tile_configs()
    code = gpu_lib.tile_cfg_code(cfgs.index((128, 8, 6)), cfgs.index((128, 8, 3)))
    x, res = gpu_lib.pcg_solve(bd, tol=1e-6, maxit=3000, profile=True, tile_cfg=code)
    ctas_a, ctas_b = res["pass_ctas"]
    assert ctas_a > 0 and ctas_b % ctas_a == 0 and ctas_b // ctas_a >= 2, res["pass_ctas"]
    _, ref = gpu_lib.pcg_solve(bd, tol=1e-6, maxit=3000)
    assert res["status"] == gpu_lib.OK and ref["status"] == gpu_lib.OK
    assert abs(res["iters"] - ref["iters"]) <= 1, (res["iters"], ref["iters"])
    true_rel = oracle.true_relres(b, x.cpu().numpy())
    assert true_rel <= 1e-6
    assert abs(res["rel_res_true"] - true_rel) <= 1e-3 * true_rel


@pytest.mark.parametrize("io,powers,tol", [(np.float64, (-300, -100, -40, 40, 100, 300), 1e-8),
                                           (np.float32, (-60, -30, 30, 60), 1e-6)])
def test_right_hand_side_scale_invariance(gpu_lib, io, powers, tol):
    """Scaling b by 2^k scales the solution by 2^k and changes nothing else: the solver works on
    s b with s a power of two that brings max |b| near 1 (when it is far from 1), so the FP32
    iteration vectors and partial sums neither underflow nor overflow.  The iterations are the
    same and x comes back as the unscaled solution times 2^k, bit for bit."""
    b = inputs.uniform_rhs((24, 20, 36), 9, dtype=np.float64)
    x0, r0 = solve(gpu_lib, b.astype(io), io=io, tol=tol, maxit=3000)
    assert r0["status"] == gpu_lib.OK
    for k in powers:
        bk = (b * 2.0 ** k).astype(io)
        xk, rk = solve(gpu_lib, bk, io=io, tol=tol, maxit=3000)
        assert rk["status"] == gpu_lib.OK and rk["iters"] == r0["iters"], (k, rk)
        assert np.array_equal(xk.astype(np.float64) * 2.0 ** -k, x0.astype(np.float64)), k
        assert oracle.true_relres(bk.astype(np.float64), xk.astype(np.float64)) <= tol


def test_whole_row_configuration_rejects_wide_grids(gpu_lib):
    b = torch.zeros((4, 4, 260), dtype=torch.float32, device="cuda")
    with pytest.raises(gpu_lib.GbpcgError):
        gpu_lib.pcg_solve(b, tile_cfg=gpu_lib.tile_cfg_code(6, 6))
