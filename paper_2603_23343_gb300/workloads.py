"""Fixed, seeded workloads for profilers (ncu and the like), one per hot path, each
run through the C ABI on cuda:0:

  python -m paper_2603_23343_gb300.workloads passes  --n N --reps R [--storage S] [--coef C]
      R profile-mode Jacobi-PCG solves of the N^3 Poisson problem (b ~ U[-1,1) seed 0): the
      pass kernels launch one by one, outside any graph, so a profiler sees every launch.
      --storage fp16 / bf16: 16-bit iteration vectors with FP64 refinement (tol 1e-8);
      --coef lognormal: the lognormal block-coefficient problem (8^3 blocks, seed 1)
  python -m paper_2603_23343_gb300.workloads batch   --n N --reps R
      R persistent batched solves of 16 Poisson problems with sizes drawn from {N/2, N}
      (seed 2): one cooperative kernel launch each
  python -m paper_2603_23343_gb300.workloads sell    --n N --reps R
      R Sliced-ELL products y = A x with the N^3 seven-point operator
  python -m paper_2603_23343_gb300.workloads vcycle  --n N --reps R
      R multigrid V-cycles (with the Galerkin set-up) on the N^3 Poisson operator
  python -m paper_2603_23343_gb300.workloads forward --n N --reps R
      R applications of the learned preconditioner (seeded initial weights) on the seeded
      lognormal problem at N^3
  python -m paper_2603_23343_gb300.workloads train   --n N --reps R
      R training steps on the exact pair e ~ U[-1,1), r = A e at N^3

Each prints one line with what it ran.
"""
from __future__ import annotations

import argparse

import numpy as np
import torch

from . import binding, inputs, learned


def passes(n, reps, storage="fp32", coef="poisson"):
    kd = None
    if coef == "lognormal":
        k, b64 = inputs.varcoeff_problem(n, n, n, seed=1, kb=8, dtype=np.float64)
        kd = torch.from_numpy(k).cuda()
    else:
        b64 = inputs.poisson_problem(n, 0, np.float64)
    b = torch.from_numpy(b64).cuda()
    st = {"fp32": None, "fp16": torch.float16, "bf16": torch.bfloat16}[storage]
    kw = dict(tol=1e-6, maxit=2000) if st is None else dict(tol=1e-8, maxit=8000, storage=st, max_outer=20)
    ws = binding.alloc_workspace(b.shape, kd, io_dtype=binding.F64, storage=binding._DTYPES.get(st, binding.F32))
    for _ in range(reps):
        x, r = binding.pcg_solve(b, torch.zeros_like(b), k_block=kd, workspace=ws, profile=True, **kw)
    print(f"passes {n}^3 {coef} {storage} x{reps}: {r['iters']} iterations, "
          f"pass A {1e3 * r['pass_ms'][0] / r['pass_launches'][0]:.1f} us, "
          f"pass B {1e3 * r['pass_ms'][1] / r['pass_launches'][1]:.1f} us")


def batch(n, reps):
    sizes = [n // 2, n]
    u = inputs.uniform_pm1(2, 0, 48, np.float64)
    shapes = [tuple(sizes[int(v > 0)] for v in u[3 * i:3 * i + 3]) for i in range(16)]
    bs = [torch.from_numpy(inputs.uniform_rhs(sh, 100 + i, dtype=np.float64)).cuda() for i, sh in enumerate(shapes)]
    for _ in range(reps):
        xs, res = binding.pcg_solve_batched(bs, tol=1e-6, maxit=3000)
    print(f"batch of 16 ({sizes}) x{reps}: {res[0]['pass_launches'][1]} phases, {res[0]['time_ms']:.2f} ms, "
          f"all converged: {all(r['status'] == 0 for r in res)}")


def sell(n, reps):
    m = binding.sell_from_stencil((n, n, n))
    x = torch.from_numpy(inputs.uniform_rhs((n, n, n), 3)).cuda().ravel()
    y = torch.empty_like(x)
    for _ in range(reps):
        binding.sell_spmv(m, x, y)
    torch.cuda.synchronize()
    print(f"sell spmv {n}^3 x{reps}: {m.nnz_stored} stored entries")


def vcycle(n, reps):
    r = torch.from_numpy(inputs.uniform_rhs((n, n, n), 3)).cuda()
    ws = binding.mg_workspace(r.shape)
    z = torch.empty_like(r)
    for _ in range(reps):
        _, levels = binding.mg_vcycle(r, z, workspace=ws)
    torch.cuda.synchronize()
    print(f"vcycle {n}^3 x{reps}: {levels} levels")


def forward(n, reps):
    shape = (n, n, n)
    k, b = learned.problem(shape, 100)
    w = learned.initial_weights(0).cuda()
    ws = binding.nn_workspace(shape)
    r = b.float()
    z = torch.empty_like(r)
    for _ in range(reps):
        binding.nn_forward(w, r, z, k_block=k, workspace=ws)
    torch.cuda.synchronize()
    print(f"forward {n}^3 x{reps}: max |z| = {float(z.abs().max()):.6g}")


def train(n, reps):
    shape = (n, n, n)
    k, _ = learned.problem(shape, 100)
    w = learned.initial_weights(0).cuda()
    e64 = torch.from_numpy(inputs.uniform_rhs(shape, 7, 0, np.float64)).cuda()
    r = binding.stencil_apply(e64, k_block=k).float()
    tr = binding.NnTrainer(w, shape, k_block=k)
    for _ in range(reps):
        loss = tr.step(r, e64.float())
    tr.status()
    print(f"train {n}^3 x{reps}: loss {loss.item():.6g}")


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_2603_23343_gb300.workloads")
    ap.add_argument("workload", choices=["passes", "batch", "sell", "vcycle", "forward", "train"])
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--storage", choices=["fp32", "fp16", "bf16"], default="fp32", help="passes only")
    ap.add_argument("--coef", choices=["poisson", "lognormal"], default="poisson", help="passes only")
    a = ap.parse_args(argv)
    if not torch.cuda.is_available():
        raise SystemExit("the workloads need a CUDA GPU")
    if a.workload == "passes":
        passes(a.n, a.reps, a.storage, a.coef)
    else:
        globals()[a.workload](a.n, a.reps)


if __name__ == "__main__":
    main()
