"""Training of the learned preconditioner on the GPU, through the C ABI.

Data (the plain solver generates its own training pairs): for each problem
(lognormal block coefficient k and uniform right-hand side b, seeded like the
variable-coefficient workload), plain Jacobi PCG is run from x = 0 and its
residual r_m = b - A x_m is taken after m iterations for several m, so the
set spans rough early residuals and smooth late ones.  The target of each
residual is e = A^{-1} r, solved by the same plain PCG to a relative residual
of 1e-4.  A training step (gbpcg_nn_train_step) runs z = N(r), the loss
1/2 (1 - a|a| / (z.Az e.Ae)) with a = z.Ae -- for a >= 0 the relative A-norm
error of the best multiple of z, 1/2 ||s z - e||_A^2 / ||e||_A^2 with
s = a / z.Az -- and its gradient, the backward pass and Adam, all in the
library's kernels; this module only orders the calls.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import binding, inputs


def problem(shape, seed: int, kb: int = 8, device="cuda"):
    """(k_block on the device, b float64 on the device) of the seeded variable-coefficient problem."""
    nz, ny, nx = shape
    k, b = inputs.varcoeff_problem(nx, ny, nz, seed=seed, kb=kb, dtype=np.float64)
    return torch.from_numpy(k).float().to(device), torch.from_numpy(b).to(device)


def residual(b64: torch.Tensor, x64: torch.Tensor, k_block, kb: int) -> torch.Tensor:
    """b - A x in FP64 (stencil and axpy kernels)."""
    r = b64.clone()
    ax = binding.stencil_apply(x64, k_block=k_block, kb=kb)
    binding.axpy(-1.0, ax, r)
    return r


def make_pairs(shape, seeds, snapshots=(0, 2, 5, 10, 20, 40, 80), kb: int = 8, target_tol: float = 1e-4,
               device="cuda"):
    """[(k_block, r float32, e float32)] for every seed and snapshot iteration."""
    pairs = []
    for seed in seeds:
        k, b = problem(shape, seed, kb, device)
        for m in snapshots:
            if m == 0:
                r64 = b.clone()
            else:
                x, _ = binding.pcg_solve(b, torch.zeros_like(b), tol=1e-30, maxit=int(m), k_block=k, kb=kb)
                r64 = residual(b, x, k, kb)
            e, _ = binding.pcg_solve(r64, torch.zeros_like(r64), tol=target_tol, maxit=20000, k_block=k, kb=kb)
            pairs.append((k, r64.float().contiguous(), e.float().contiguous()))
    return pairs


def train(pairs, w0: torch.Tensor, steps: int, lr: float = 1e-3, kb: int = 8, seed: int = 0, log_every: int = 0,
          lr_final: float | None = None):
    """Adam on the pairs in a seeded random order, learning rate decaying geometrically from lr to
    lr_final; returns (weights, per-step losses, seconds)."""
    shape = tuple(pairs[0][1].shape)
    tr = binding.NnTrainer(w0, shape, k_block=pairs[0][0], kb=kb)
    order = inputs.choice(seed, 0, steps, list(range(len(pairs))))
    losses = torch.zeros(steps, dtype=torch.float64, device=tr.w.device)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(steps):
        k, r, e = pairs[int(order[i])]
        tr.set_coefficients(k, kb)
        a = lr if lr_final is None else lr * (lr_final / lr) ** (i / max(1, steps - 1))
        loss = tr.step(r, e, lr=a)
        losses[i] = loss
        if log_every and (i + 1) % log_every == 0:
            print(f"step {i + 1}: loss {losses[max(0, i + 1 - log_every):i + 1].mean().item():.4f}", flush=True)
    tr.status()
    torch.cuda.synchronize()
    return tr.w, losses.cpu().numpy(), time.perf_counter() - t0


def combination_schedule(steps: int, nprob: int, per_problem: int, seed: int = 0):
    """(a, b, c) for train_combined: step i combines pairs a[i] and b[i] (indices into the pair
    list, distinct, of the same problem) with coefficients c[i, 0], c[i, 1] ~ N(0, 1); seeded."""
    if nprob < 1 or per_problem < 2:
        raise ValueError("need at least one problem with at least two pairs")
    prob = inputs.choice(seed, 0, steps, list(range(nprob))).astype(np.int64)
    a = inputs.choice(seed + 1, 0, steps, list(range(per_problem))).astype(np.int64)
    shift = inputs.choice(seed + 2, 0, steps, list(range(1, per_problem))).astype(np.int64)
    b = (a + shift) % per_problem
    c = inputs.standard_normal(seed + 3, 0, 2 * steps).reshape(steps, 2)
    return prob * per_problem + a, prob * per_problem + b, c


def train_combined(pairs, per_problem: int, w0: torch.Tensor, steps: int, lr: float = 1e-3, kb: int = 8,
                   seed: int = 0, lr_final: float | None = None):
    """Adam as in train, but every step sees a fresh exact pair: c_a (r_a, e_a) + c_b (r_b, e_b) for
    two distinct pairs a, b of one problem (pairs[i * per_problem:(i + 1) * per_problem] share one
    coefficient field), with c = seeded standard normals divided by the pair's residual norm, so
    that a rough early residual (norm ~1) does not drown a smooth late one (norm ~1e-3).  A^{-1}
    is linear, so the combination is again a residual and its exact correction; `steps` steps
    train on `steps` distinct pairs without storing them.  The norms and combinations are formed
    by the library's dot and axpy kernels.  Returns (weights, per-step losses, seconds)."""
    nprob = len(pairs) // per_problem
    if nprob * per_problem != len(pairs):
        raise ValueError("pairs must hold per_problem pairs of each problem, problem by problem")
    ia, ib, coef = combination_schedule(steps, nprob, per_problem, seed)
    inv_norm = [1.0 / max(float(binding.dot(r, r)), 1e-300) ** 0.5 for _, r, _ in pairs]
    coef = coef * np.array([[inv_norm[a], inv_norm[b]] for a, b in zip(ia, ib)])
    shape = tuple(pairs[0][1].shape)
    tr = binding.NnTrainer(w0, shape, k_block=pairs[0][0], kb=kb)
    r = torch.empty_like(pairs[0][1])
    e = torch.empty_like(pairs[0][2])
    losses = torch.zeros(steps, dtype=torch.float64, device=tr.w.device)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(steps):
        ka, ra, ea = pairs[int(ia[i])]
        _, rb, eb = pairs[int(ib[i])]
        ca, cb = float(coef[i, 0]), float(coef[i, 1])
        r.zero_()
        e.zero_()
        binding.axpy(ca, ra, r)
        binding.axpy(cb, rb, r)
        binding.axpy(ca, ea, e)
        binding.axpy(cb, eb, e)
        tr.set_coefficients(ka, kb)
        step_lr = lr if lr_final is None else lr * (lr_final / lr) ** (i / max(1, steps - 1))
        losses[i] = tr.step(r, e, lr=step_lr)
    tr.status()
    torch.cuda.synchronize()
    return tr.w, losses.cpu().numpy(), time.perf_counter() - t0


def initial_weights(seed: int = 0) -> torch.Tensor:
    """Seeded He-style initial weights, packed (float32, CPU)."""
    return binding.nn_pack_weights(inputs.unet_init_weights(seed, binding.NN_LAYERS))


def identity_weights() -> torch.Tensor:
    """Weights that pass the scaled residual through, so that N(r) = D^{-1} r
    (the Jacobi preconditioner) up to the BF16 rounding of D^{-1/2} r / rms:
    c1 splits it into relu(s) and relu(-s), c2 and c8 carry them through the
    centre tap, the coarse path is zero and c9 recombines them."""
    ws = {name: np.zeros((co, 27, ci)) for name, ci, co in binding.NN_LAYERS}
    ws["c1"][0, 13, 0], ws["c1"][1, 13, 0] = 1.0, -1.0
    ws["c2"][0, 13, 0], ws["c2"][1, 13, 1] = 1.0, 1.0
    ws["c8"][0, 13, 32], ws["c8"][1, 13, 33] = 1.0, 1.0
    ws["c9"][0, 13, 0], ws["c9"][0, 13, 1] = 1.0, -1.0
    return binding.nn_pack_weights(ws)
