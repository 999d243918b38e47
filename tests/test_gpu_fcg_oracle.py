"""Flexible CG on the GPU (gbpcg_fcg_solve) against the oracle's flexible CG
(oracle/nn.py: fcg) with the same network weights.

The oracle's preconditioner is its FP64 U-net with the GPU's BF16 roundings
mirrored (weights, network input and every stored activation rounded to
BF16), so both solvers apply the same nonlinear M up to rounding-boundary
flips.  Checked: the iteration counts agree within 2, and the relative
residual history ||r_k|| / ||b|| for k = 1..5 agrees to 1e-4 relative for
the pass-through weights (one BF16 rounding of the scaled residual, mirrored
exactly) and to 2e-3 for trained weights (about 1e-4 of each layer's
activations round to the neighbouring BF16 value when the FP32 and FP64 sums
straddle a rounding boundary, and those flips compound through nine layers
into z; measured 3e-4).  The GPU's history is read from solves capped at k
iterations.  Cases: the
pass-through (identity) weights, for which M(r) = D^{-1/2} bf16(s / rms(s))
rms(s) with s = D^{-1/2} r, and weights trained on the GPU; truncation
m = 1 (the beta form) and m = 24.
"""
import numpy as np
import pytest
import torch

import oracle
import oracle.nn as onn
from paper_2603_23343_gb300 import inputs, learned

pytestmark = pytest.mark.gpu

SHAPE = (32, 32, 32)
TOL = 1e-6


def bf16(a):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).float()
    return t.to(torch.bfloat16).double().numpy()


def oracle_precond(ws, k64):
    """z = N(r) of the oracle network with the GPU's BF16 roundings mirrored."""
    wsb = {name: bf16(v) for name, v in ws.items()}
    logk = onn.logk_field(SHAPE, k64, 8)
    dsc = onn.jacobi_scale(SHAPE, k64, 8)

    def M(r):
        x, scale = onn.net_input(r, logk, dsc)
        out, _ = onn.net_forward(bf16(x), wsb, round_fn=bf16)
        return out[..., 0] * scale
    return M


def identity_precond(k64):
    """The pass-through network written out: D^{-1/2} bf16(s / rms(s)) rms(s), s = D^{-1/2} r."""
    dsc = onn.jacobi_scale(SHAPE, k64, 8)

    def M(r):
        s = r * dsc
        rms = float(np.sqrt(np.mean(s * s)))
        return bf16(s / rms) * (rms * dsc)
    return M


def gpu_history(gpu_lib, w, b, k, m, upto=5):
    out = []
    for it in range(1, upto + 1):
        _, res = gpu_lib.fcg_solve(w, b, tol=TOL, maxit=it, k_block=k, m=m)
        assert res["iters"] == it and res["pass_launches"][1] == 0, res
        out.append(res["rel_res_recursive"])
    return np.array(out)


def compare(gpu_lib, w, M, b, k, m, maxit, rtol):
    b64 = b.cpu().numpy()
    k64 = None if k is None else k.cpu().numpy().astype(np.float64)
    x, res = gpu_lib.fcg_solve(w, b, tol=TOL, maxit=maxit, k_block=k, m=m)
    assert res["status"] == gpu_lib.OK and res["pass_launches"][1] == 0, res
    ref = onn.fcg(b64, M, tol=TOL, maxit=maxit, k=k64, kb=8, m=m)
    print(f"m={m}: GPU {res['iters']} iterations, oracle {ref['iters']}")
    assert abs(res["iters"] - ref["iters"]) <= 2, (res["iters"], ref["iters"])
    assert ref["hist"][-1] <= TOL
    assert oracle.true_relres(b64, x.cpu().numpy(), k64, 8) <= TOL
    h = gpu_history(gpu_lib, w, b, k, m)
    np.testing.assert_allclose(h, ref["hist"][1:6], rtol=rtol, atol=0)


@pytest.mark.parametrize("m", [1, 24])
@pytest.mark.parametrize("varcoeff", [False, True])
def test_identity_network_fcg_matches_oracle_fcg(gpu_lib, m, varcoeff):
    if varcoeff:
        k, b = learned.problem(SHAPE, 3)
        k64 = k.cpu().numpy().astype(np.float64)
    else:
        k, k64 = None, None
        b = torch.from_numpy(inputs.poisson_problem(32, 0, np.float64)).cuda()
    ws_id = onn.init_weights(0)
    for name in ws_id:
        ws_id[name] = np.zeros_like(ws_id[name])
    w = learned.identity_weights()
    for name, v in gpu_lib.nn_unpack_weights(w).items():
        ws_id[name] = v.numpy().astype(np.float64)
    M = identity_precond(k64)
    # the closed form is the oracle network with these weights, exactly
    r0 = b.cpu().numpy()
    np.testing.assert_array_equal(M(r0), oracle_precond(ws_id, k64)(r0))
    compare(gpu_lib, w.cuda(), M, b, k, m, maxit=1000, rtol=1e-4)


@pytest.fixture(scope="module")
def trained_weights(gpu_lib):
    """A network trained on the GPU on 32^3 lognormal problems (seeds 10-17, the plain solver's
    residual snapshots and targets)."""
    pairs = learned.make_pairs(SHAPE, seeds=range(10, 18))
    w, losses, _ = learned.train(pairs, learned.initial_weights(0).cuda(), 600, lr=1e-3, lr_final=1e-4)
    assert np.all(np.isfinite(losses))
    return w


@pytest.mark.parametrize("m", [1, 24])
def test_trained_network_fcg_matches_oracle_fcg(gpu_lib, trained_weights, m):
    k, b = learned.problem(SHAPE, 100)
    k64 = k.cpu().numpy().astype(np.float64)
    ws = {name: v.numpy().astype(np.float64)
          for name, v in gpu_lib.nn_unpack_weights(trained_weights.cpu()).items()}
    compare(gpu_lib, trained_weights, oracle_precond(ws, k64), b, k, m, maxit=200, rtol=2e-3)
