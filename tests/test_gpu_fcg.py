"""Flexible CG with the learned preconditioner (gbpcg_fcg_solve), its descent
check with the Jacobi fallback, and what a network trained on the GPU gains
over Jacobi PCG.  Every solve is checked with the FP64 oracle's true residual
||b - A x|| / ||b||, evaluated on the returned x."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2603_23343_gb300 import inputs, learned

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def true_relres(b, x, k=None, kb=8):
    kk = None if k is None else k.cpu().numpy().astype(np.float64)
    return oracle.true_relres(b.cpu().numpy(), x.cpu().numpy(), kk, kb)


def test_identity_network_reproduces_jacobi_pcg(gpu_lib):
    """The network acts on the Jacobi-scaled system, so weights that pass their input through
    give N(r) = D^{-1} r (up to one BF16 rounding of the scaled residual): FCG becomes Jacobi
    PCG, and the oracle's iteration count for the 32^3 Poisson problem (seed 0, tol 1e-6)
    is reproduced."""
    with open(os.path.join(GOLDEN, "pcg_poisson32_seed0.json")) as f:
        gold = json.load(f)
    b = torch.from_numpy(inputs.poisson_problem(32, 0, np.float64)).cuda()
    w = learned.identity_weights().cuda()
    x, res = gpu_lib.fcg_solve(w, b, tol=1e-6, maxit=2000)
    assert res["status"] == gpu_lib.OK, res
    assert res["pass_launches"][1] == 0  # no fallback
    assert abs(res["iters"] - gold["iters"]) <= 2, (res["iters"], gold["iters"])
    assert true_relres(b, x) <= 1e-6
    assert abs(res["rel_res_true"] - true_relres(b, x)) <= 1e-3 * res["rel_res_true"]


@pytest.mark.parametrize("seed,m,shape", [(3, 0, (32, 32, 32)), (4, 0, (32, 32, 32)), (3, 1, (32, 32, 32)),
                                          (3, 32, (32, 32, 32)), (5, 0, (16, 32, 64))])
def test_identity_network_matches_jacobi_on_lognormal_coefficients(gpu_lib, seed, m, shape):
    """Same on the variable-coefficient operator: FCG with N(r) = D^{-1} r takes the iterations
    of the library's Jacobi PCG (within a few: one BF16 rounding per application), whatever the
    truncation depth m (0: the default) -- with a linear symmetric preconditioner every earlier
    direction is already A-orthogonal."""
    k, b = learned.problem(shape, seed)
    x, res = gpu_lib.fcg_solve(learned.identity_weights().cuda(), b, tol=1e-6, maxit=3000, k_block=k, m=m)
    _, ref = gpu_lib.pcg_solve(b.clone(), torch.zeros_like(b), tol=1e-6, maxit=3000, k_block=k)
    assert res["status"] == gpu_lib.OK and res["pass_launches"][1] == 0
    assert abs(res["iters"] - ref["iters"]) <= max(3, ref["iters"] // 20), (res["iters"], ref["iters"])
    assert true_relres(b, x, k) <= 1e-6


@pytest.mark.parametrize("how", ["nan", "negated"])
def test_descent_check_falls_back_to_jacobi(gpu_lib, how):
    """A preconditioner that is no descent direction (NaN output, or N(r) = -D^{-1} r with
    r.z < 0) is caught before it touches x; Jacobi PCG finishes the solve."""
    shape = (32, 32, 32)
    k, b = learned.problem(shape, 3)
    w = learned.identity_weights()
    if how == "nan":
        w[-1] = float("nan")  # a weight of the last layer, after which no ReLU acts
    else:
        n9 = 16 * 27
        w[-n9:] = -w[-n9:]
    x, res = gpu_lib.fcg_solve(w.cuda(), b, tol=1e-6, maxit=3000, k_block=k)
    assert res["status"] == gpu_lib.FALLBACK_USED, res
    assert res["pass_launches"][0] == 0 and res["pass_launches"][1] == res["iters"]
    _, ref = gpu_lib.pcg_solve(b.clone(), torch.zeros_like(b), tol=1e-6, maxit=3000, k_block=k)
    assert res["iters"] == ref["iters"]
    assert true_relres(b, x, k) <= 1e-6


def test_iteration_cap_reports_not_converged_truthfully(gpu_lib):
    k, b = learned.problem((32, 32, 32), 5)
    x, res = gpu_lib.fcg_solve(learned.identity_weights().cuda(), b, tol=1e-6, maxit=10, k_block=k)
    assert res["status"] == gpu_lib.NOT_CONVERGED and res["iters"] == 10
    t = true_relres(b, x, k)
    assert t > 1e-6 and abs(res["rel_res_true"] - t) <= 1e-3 * t


def test_zero_rhs_and_rejections(gpu_lib):
    b = torch.zeros((32, 32, 32), dtype=torch.float64, device="cuda")
    x = torch.ones_like(b)
    w = learned.identity_weights().cuda()
    x, res = gpu_lib.fcg_solve(w, b, x=x)
    assert res["status"] == gpu_lib.OK and res["iters"] == 0
    assert torch.count_nonzero(x).item() == 0
    with pytest.raises(gpu_lib.GbpcgError):
        gpu_lib.fcg_solve(w, torch.zeros((30, 30, 30), dtype=torch.float64, device="cuda"))
    with pytest.raises(gpu_lib.GbpcgError):
        gpu_lib.fcg_solve(w, torch.zeros((32, 32, 32), dtype=torch.float32, device="cuda"))


def test_trained_network_beats_jacobi(gpu_lib):
    """What the learned preconditioner gains: train on the GPU (residual snapshots of plain
    Jacobi PCG on 64^3 lognormal-coefficient problems, seeds 10-25, targets A^{-1} r from the
    plain solver), then solve held-out problems (seeds 100, 101) to the same 1e-6: FCG with
    the network needs under 0.3x the Jacobi PCG iterations, and the FP64 oracle confirms
    the true residual."""
    shape = (64, 64, 64)
    pairs = learned.make_pairs(shape, seeds=range(10, 26))
    w, losses, secs = learned.train(pairs, learned.initial_weights(0).cuda(), 2000, lr=1e-3, lr_final=1e-4)
    first, last = float(np.mean(losses[:20])), float(np.mean(losses[-200:]))
    assert np.all(np.isfinite(losses)) and last < 0.4 * first, (first, last)
    for seed in (100, 101):
        k, b = learned.problem(shape, seed)
        _, jac = gpu_lib.pcg_solve(b.clone(), torch.zeros_like(b), tol=1e-6, maxit=5000, k_block=k)
        x, res = gpu_lib.fcg_solve(w, b, tol=1e-6, maxit=5000, k_block=k)
        print(f"seed {seed}: Jacobi PCG {jac['iters']} iterations, learned FCG {res['iters']} "
              f"(loss {first:.3f} -> {last:.3f}, {secs:.1f} s of training)")
        assert res["status"] == gpu_lib.OK and res["pass_launches"][1] == 0, res
        assert res["iters"] < 0.3 * jac["iters"]
        assert true_relres(b, x, k) <= 1e-6


def test_right_hand_side_scale(gpu_lib):
    """Flexible CG keeps its FP32 vectors on s b (s a power of two bringing rms(b) near 1), so a
    right-hand side scaled by 2^-100 or 2^100 converges like the unscaled one and x comes back
    scaled; the network sees the residual divided by its rms either way."""
    k, b = learned.problem((32, 32, 32), 3)
    w = learned.identity_weights().cuda()
    x0, r0 = gpu_lib.fcg_solve(w, b, tol=1e-6, maxit=3000, k_block=k)
    assert r0["status"] == gpu_lib.OK
    for p in (-100, 100):
        bp = b * 2.0 ** p
        xp, rp = gpu_lib.fcg_solve(w, bp, tol=1e-6, maxit=3000, k_block=k)
        assert rp["status"] == gpu_lib.OK and abs(rp["iters"] - r0["iters"]) <= 1, (p, rp, r0)
        assert true_relres(bp, xp, k) <= 1e-6
