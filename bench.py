#!/usr/bin/env python
"""Benchmark of the GB300 Jacobi-PCG hot path (arxiv 2603.23343, Sec. VII).

Headline workload: 3D 7-point Poisson on a 256^3 interior grid (h = 1/257),
b ~ U[-1,1) seed 0, x0 = 0, Jacobi, stop at ||r||/||b|| <= 1e-6 (maxit 2000),
FP32 vectors, FP64 scalars.  One step = one full solve (reset x0, whole PCG
loop in one CUDA graph, FP64 true residual) with b already resident in HBM.
b and x are FP64 (only the init, the residual replacements and the finalize
touch them); the iteration vectors z, p0, p1, d are FP32.  The working set
(512 MiB) is larger than the 126 MB L2, so steps need no L2 flush.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  N > 1 (torchrun) runs N independent replicas
(one solve per GPU per step); the path has no data-path collective.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PCG time-to-1e-6 residual & HBM GB/s at 256^3, plain FP32 vs learned/mixed"
N_GRID = 256
TOL = 1e-6
MAXIT = 2000
# algorithmic bytes per grid point of each data pass (FP32): pass A reads z, p_{k-1} and the
# correction vector d and writes p_k, d; pass B reads p_k, z and writes z.  An iteration is 32 B/pt.
PASS_BYTES = {"pass_a": 20, "pass_b": 12}
ITER_BYTES = 32
THREE_KERNEL_BYTES = 44


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=N_GRID, help="grid points per axis (default 256)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-preconditioner leg")
    ap.add_argument("--learned-full", action="store_true",
                    help="learned leg at the full recipe: 128^3 training on seeds 10-99, evaluation on 100-109")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def tensor_peak():
    """Dense BF16 TFLOP/s: (burst, sustained, source)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["bf16_tflops"]), float(p["bf16_tflops_sustained"]), "measured"
    except Exception:
        return 1900.0, 1700.0, "fallback"


# U-net work per finest-level voxel (multiply-adds): level 0 c1 + c2 + c8 + c9, level 1 (1/8)
# c3 + c4 + c7, level 2 (1/64) c5 + c6; 2 FLOP per multiply-add
UNET_MACS_PER_VOXEL = (864 + 6912 + 20736 + 432) + (13824 + 27648 + 82944) / 8 + (55296 + 110592) / 64


def learned_leg(B, learned, stream, full: bool):
    """The learned-preconditioner workload: train on the GPU at 128^3 on lognormal problems (pairs from the plain
    solver), evaluate learned FCG against Jacobi PCG at 256^3 on held-out seeds, and time the
    heaviest convolution (c8, 48 -> 16 channels at 256^3) against the tensor peak."""
    import torch
    train_seeds = range(10, 100) if full else range(10, 42)
    eval_seeds = range(100, 110)
    snapshots = (0, 2, 5, 10, 20, 40, 80)
    steps = 4000
    t0 = time.perf_counter()
    pairs = learned.make_pairs((128, 128, 128), seeds=train_seeds, snapshots=snapshots)
    torch.cuda.synchronize()
    pair_s = time.perf_counter() - t0
    # the snapshot pairs themselves (training on 10^4 fresh combinations of them reached the
    # same loss but gave networks that lose the descent property in flexible CG at 256^3)
    w, losses, train_s = learned.train(pairs, learned.initial_weights(0).cuda(), steps, lr=1e-3, lr_final=1e-4)
    del pairs
    torch.cuda.empty_cache()
    evals = []
    for sd in eval_seeds:
        k, bb = learned.problem((256, 256, 256), sd)
        xj = torch.zeros_like(bb)
        B.pcg_solve(bb, xj, tol=TOL, maxit=20000, k_block=k)  # graph build
        xj.zero_()
        _, rj = B.pcg_solve(bb, xj, tol=TOL, maxit=20000, k_block=k)
        fws = B.fcg_workspace(bb.shape, k_block=k, tol=TOL, maxit=20000)
        _, rl = B.fcg_solve(w, bb, tol=TOL, maxit=20000, k_block=k, workspace=fws)
        mws = B.mg_workspace(bb.shape, k_block=k)
        xm = torch.zeros_like(bb)
        B.mg_pcg_solve(bb, xm, tol=TOL, maxit=2000, k_block=k, workspace=mws)
        xm.zero_()
        _, rm = B.mg_pcg_solve(bb, xm, tol=TOL, maxit=2000, k_block=k, workspace=mws)
        del mws, xm
        evals.append({"seed": sd, "jacobi": {"iters": rj["iters"], "ms": rj["time_ms"],
                                             "rel_res_true_fp64": rj["rel_res_true"]},
                      "multigrid": {"iters": rm["iters"], "ms": rm["time_ms"], "status": rm["status_name"],
                                    "rel_res_true_fp64": rm["rel_res_true"]},
                      "learned_fcg": {"iters": rl["iters"], "ms": rl["time_ms"], "network_ms": rl["pass_ms"][0],
                                      "fcg_iters": rl["pass_launches"][0], "fallback_iters": rl["pass_launches"][1],
                                      "status": rl["status_name"], "rel_res_true_fp64": rl["rel_res_true"]}})
        del fws, xj
        torch.cuda.empty_cache()
    # one network application and the c8 convolution alone, CUDA events on the launching stream
    n = 256
    k, bb = learned.problem((n, n, n), eval_seeds[0])
    r = bb.float()
    z = torch.empty_like(r)
    nws = B.nn_workspace(r.shape)
    B.nn_forward(w, r, z, k_block=k, workspace=nws, stream=stream)
    xin = torch.randn((n, n, n, 48), device="cuda").to(torch.bfloat16)
    w8 = (torch.randn((16, 27, 48), device="cuda") * 0.03).to(torch.bfloat16)
    cws = B.conv3_workspace((n, n, n), 48, 16)
    B.conv3_forward(xin, w8, workspace=cws, stream=stream)
    torch.cuda.synchronize()
    reps = 10
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record(stream)
    for _ in range(reps):
        B.nn_forward(w, r, z, k_block=k, workspace=nws, stream=stream)
    e1.record(stream)
    for _ in range(reps):
        B.conv3_forward(xin, w8, workspace=cws, stream=stream)
    e2.record(stream)
    torch.cuda.synchronize()
    net_ms = e0.elapsed_time(e1) / reps
    c8_ms = e1.elapsed_time(e2) / reps
    burst, sustained, src = tensor_peak()
    c8_flop = 2.0 * n ** 3 * 27 * 48 * 16
    net_flop = 2.0 * n ** 3 * UNET_MACS_PER_VOXEL
    c8_tf = c8_flop / (c8_ms * 1e-3) / 1e12
    iters_j = [e["jacobi"]["iters"] for e in evals]
    iters_l = [e["learned_fcg"]["iters"] for e in evals]
    return {
        "recipe": ("full" if full else "reduced") + f": train 128^3 lognormal seeds {train_seeds.start}-"
                  f"{train_seeds.stop - 1} x Jacobi-PCG snapshots {snapshots} with A^-1 r to 1e-4 "
                  f"({len(train_seeds) * len(snapshots)} pairs), {steps} Adam steps; "
                  f"evaluate 256^3 seeds {eval_seeds.start}-{eval_seeds.stop - 1}, tol {TOL}",
        "train_pairs": len(train_seeds) * len(snapshots),
        "pairs_s": pair_s, "train_s": train_s, "train_ms_per_step": 1e3 * train_s / steps,
        "loss_first_last": [float(np.mean(losses[:20])), float(np.mean(losses[-200:]))],
        "eval": evals,
        "iters_ratio_learned_over_jacobi": float(np.mean(iters_l) / np.mean(iters_j)),
        "iters_ratio_per_seed": [float(a / b) for a, b in zip(iters_l, iters_j)],
        "ms_ratio_multigrid_over_jacobi": float(np.mean([e["multigrid"]["ms"] for e in evals]) /
                                                np.mean([e["jacobi"]["ms"] for e in evals])),
        "ms_ratio_learned_over_jacobi": float(np.mean([e["learned_fcg"]["ms"] for e in evals]) /
                                              np.mean([e["jacobi"]["ms"] for e in evals])),
        "network_256": {"ms": net_ms, "tflops": net_flop / (net_ms * 1e-3) / 1e12,
                        "flop": net_flop},
        "roofline_conv_c8_256": {"bound": "tensor", "kernel": "conv3_tc_zmarch_kernel (48->16 channels)",
                                 "achieved": c8_tf, "peak": burst, "unit": "TFLOP/s", "frac": c8_tf / burst,
                                 "peak_source": src + " bf16 burst", "flop_per_launch": c8_flop,
                                 "avg_launch_us": c8_ms * 1e3, "traffic": None},
    }


def ablation_leg(B, inputs, stream, b64, n):
    """The paper's own experiments, repeated on GB300:
    Sec. VII  device-resident loop (one CUDA graph) vs the fused kernels with the stop flag read
              back to the host every iteration vs split kernels with host-side scalars (the
              paper's FP32 variant, and its H100 comparator's structure), at n^3;
    Sec. V    the dot product's reduction granularity and finish (gbpcg_dot_variant) from 2^16
              to 2^28 elements (the kernels replayed from a CUDA graph, so launch gaps of the
              host do not hide the small sizes);
    Sec. VI-C TMA out-of-bounds zero fill vs bounds-checked plain loads vs TMA plus an
              explicit zero fill, for the stencil apply from 32^3 to 256^3."""
    import torch

    def timed(fn, reps):
        """ms per call of fn(stream), the calls captured back to back in one CUDA graph so that
        the host's launch rate does not bound small sizes; best of three replays."""
        cs = torch.cuda.Stream()
        with torch.cuda.stream(cs):
            fn(cs)  # attributes, occupancy queries and tensor maps outside the capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cs):
            for _ in range(reps):
                fn(cs)
        g.replay()
        torch.cuda.synchronize()
        best = None
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.replay()
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / reps
            best = t if best is None else min(best, t)
        del g
        return best

    out = {}
    # Sec. VII: how the loop is driven
    b32 = b64.float()
    sec7 = {}
    for name, bb, mode in (("device_graph", b64, "graph"), ("host_readback_fused", b64, "host_loop"),
                           ("split_kernels_host_scalars", b32, "split")):
        xx = torch.zeros_like(bb)
        ws = B.alloc_workspace(bb.shape, io_dtype=B.F64 if bb.dtype == torch.float64 else B.F32, mode=mode)
        best = None
        for _ in range(2):
            xx.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, r = B.pcg_solve(bb, xx, tol=TOL, maxit=MAXIT, workspace=ws, mode=mode, stream=stream)
            wall = (time.perf_counter() - t0) * 1e3
            best = wall if best is None else min(best, wall)
        sec7[name] = {"ms": r["time_ms"], "wall_ms": best, "iters": r["iters"], "status": r["status_name"],
                      "us_per_iter": 1e3 * r["time_ms"] / max(1, r["iters"]),
                      "rel_res_recursive": r["rel_res_recursive"]}
        del ws, xx
    sec7["algorithmic_bytes_per_pt_iter"] = {"device_graph": ITER_BYTES, "host_readback_fused": ITER_BYTES,
                                             "split_kernels_host_scalars": 76}
    out[f"sec7_loop_driver_{n}"] = sec7
    # Sec. V: reduction granularity and finish
    names = ["cta_scalar_last_cta", "warp_partials_last_cta", "cta_scalar_second_kernel", "cta_scalar_fp64_atomics",
             "cta_scalar_two_level_tree"]
    gen = torch.Generator(device="cuda").manual_seed(5)
    xa = torch.empty(1 << 28, dtype=torch.float32, device="cuda").uniform_(-1.0, 1.0, generator=gen)
    ya = torch.empty(1 << 28, dtype=torch.float32, device="cuda").uniform_(-1.0, 1.0, generator=gen)
    res_d = torch.empty((), dtype=torch.float64, device="cuda")
    wsv = torch.empty(B.load().gbpcg_dot_variant_workspace_size(), dtype=torch.uint8, device="cuda")
    sec5 = {}
    for lg in (16, 20, 24, 28):
        m = 1 << lg
        reps = 200 if lg <= 20 else 50 if lg <= 24 else 5
        row = {}
        for v, nm in enumerate(names):
            us = 1e3 * timed(lambda st: B.dot_variant(v, xa[:m], ya[:m], res_d, wsv, stream=st), reps)
            row[nm] = {"us": us, "gbs": 8 * m / (us * 1e-6) / 1e9}
        sec5[f"2^{lg}"] = row
    out["sec5_dot_reduction_variants"] = sec5
    del xa, ya, wsv
    # Sec. VI-C: boundary handling of the stencil apply
    sec6 = {}
    for m in (32, 64, 128, 256):
        p = torch.from_numpy(inputs.uniform_rhs((m, m, m), 3)).cuda()
        q = torch.empty_like(p)
        reps = 200 if m <= 64 else 50 if m == 128 else 20
        row = {}
        for v, nm in enumerate(("tma_oob_zero_fill", "plain_loads_bounds_checked", "tma_plus_explicit_zero_fill")):
            us = 1e3 * timed(lambda st: B.stencil_apply_variant(v, p, q, stream=st), reps)
            row[nm] = {"us": us, "gbs": 8 * m ** 3 / (us * 1e-6) / 1e9}
        sec6[f"{m}^3"] = row
        del p, q
    out["sec6c_stencil_boundary_variants"] = sec6
    torch.cuda.empty_cache()
    return out


class ClockSampler:
    """nvidia-smi samples (every 100 ms) while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev: int):
        self.dev = dev
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.dev)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thr = threading.Thread(target=self._read, daemon=True)
            self.thr.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thr.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(n_gpus, backend=None):
    """(rank, world, local rank) from the torchrun environment; joins the process group for
    world > 1 (NCCL for GPU replicas unless a backend is named)."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend or ("nccl" if n_gpus > 1 else "gloo"))
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_baseline(n):
    """The FP64 oracle as it stands on the host cores: one complete solve of the
    same problem (b ~ U[-1,1) seed 0, x0 = 0, tol 1e-6), timed end to end."""
    import oracle
    from paper_2603_23343_gb300 import inputs
    oracle.build()
    b = inputs.poisson_problem(n, 0, np.float64)
    t0 = time.perf_counter()
    res = oracle.pcg(b, tol=TOL, maxit=MAXIT)
    dt = time.perf_counter() - t0
    cores = oracle.threads()
    return {"value": dt * 1e3, "unit": "ms", "cores": cores, "kind": "oracle",
            "sample": f"one complete {n}^3 FP64 oracle solve to {TOL} ({res['iters']} iterations, "
                      f"{dt:.1f} s, OpenMP {cores} threads), measured, not scaled",
            "oracle_iters": res["iters"]}


def source_hash():
    """Hash of the sources that define the pass kernels (the traffic figures' validity)."""
    h = hashlib.sha256()
    for f in ("engine.cuh", "launch.cuh", "common.cuh"):
        with open(os.path.join(ROOT, "paper_2603_23343_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if it matches this source."""
    try:
        with open(os.path.join(ROOT, "profiles", "pass_traffic.json")) as f:
            t = json.load(f)
        e = t[kernel]
        if e.get("source_sha") != source_hash():
            return None
        return e["dram_bytes_per_launch_full_size"]
    except Exception:
        return None


def run_reference(args):
    """The reference arm: the FP64 CPU oracle (there is no reference code).  Each timed
    step is one complete solve of the bench's problem; warm-up steps run a short
    sample of iterations (they only page in the oracle and its input)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_2603_23343_gb300 import inputs
    oracle.build()
    n = args.n
    b = inputs.poisson_problem(n, 0, np.float64)
    for _ in range(args.warmup):
        oracle.pcg(b, tol=TOL, maxit=10)
    times, iters = [], []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        t0 = time.perf_counter()
        res = oracle.pcg(b, tol=TOL, maxit=MAXIT)
        times.append((time.perf_counter() - t0) * 1e3)
        iters.append(res["iters"])
    timed_s = time.perf_counter() - t_all
    v = float(np.mean(times))
    cores = oracle.threads()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"poisson {n}^3 Jacobi-PCG to 1e-6 (b~U[-1,1) seed 0, x0=0)",
                       "n": n, "tol": TOL, "oracle_iters": iters[0], "timed_region_s": timed_s,
                       "ms_min_max": [min(times), max(times)]},
            "cpu_baseline": {"value": v, "unit": "ms", "cores": cores, "kind": "oracle",
                             "sample": f"each timed step is one complete {n}^3 FP64 oracle solve "
                                       f"({iters[0]} iterations, OpenMP {cores} threads); warm-up steps run "
                                       f"10 iterations"},
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    rank, world, local = dist_setup(args.gpus)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    from paper_2603_23343_gb300 import binding as B
    from paper_2603_23343_gb300 import inputs

    n = args.n
    N = n ** 3
    # b and x in FP64 (touched only by init, residual replacements and finalize);
    # the iteration vectors z, p, d are FP32
    b = torch.from_numpy(inputs.poisson_problem(n, 0, np.float64)).cuda()
    x = torch.zeros_like(b)
    ws = B.alloc_workspace(b.shape, io_dtype=B.F64)
    stream = torch.cuda.current_stream()

    def step():
        x.zero_()
        return B.pcg_solve(b, x, tol=TOL, maxit=MAXIT, workspace=ws, stream=stream)[1]

    for _ in range(max(3, args.warmup)):
        res = step()
    iters = res["iters"]

    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        results = [step() for _ in range(args.steps)]
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    ms_total = e0.elapsed_time(e1)
    ms_step = max_over_ranks(ms_total / args.steps, world)
    res = results[-1]
    iters = res["iters"]

    # per-kernel durations: the same solve with every pass launch bracketed by CUDA events
    x.zero_()
    _, prof = B.pcg_solve(b, x, tol=TOL, maxit=MAXIT, workspace=ws, profile=True, stream=stream)
    avg = {k: prof["pass_ms"][i] / max(1, prof["pass_launches"][i]) for i, k in enumerate(("pass_a", "pass_b"))}
    dom = "pass_a" if prof["pass_ms"][0] >= prof["pass_ms"][1] else "pass_b"
    peak, peak_kind = peaks()
    bytes_launch = PASS_BYTES[dom] * N
    achieved = bytes_launch / (avg[dom] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": ncu_traffic(dom), "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": bytes_launch, "avg_launch_us": avg[dom] * 1e3,
                "other_pass": {k: {"avg_launch_us": avg[k] * 1e3,
                                   "achieved_gbs": PASS_BYTES[k] * N / (avg[k] * 1e-3) / 1e9}
                               for k in avg}}

    # end to end through the C ABI with host buffers (copies inside the call)
    bh = b.cpu().pin_memory()
    xh = torch.zeros_like(bh).pin_memory()
    ws_io = B.alloc_workspace(b.shape, host_io=True, io_dtype=B.F64)
    B.pcg_solve(bh, xh, tol=TOL, maxit=MAXIT, workspace=ws_io, host_io=True, stream=stream)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(args.steps):
        xh.zero_()
        _, r_io = B.pcg_solve(bh, xh, tol=TOL, maxit=MAXIT, workspace=ws_io, host_io=True, stream=stream)
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(f0.elapsed_time(f1) / args.steps, world)

    # the same solve with FP32 x and b (x's own rounding then bounds the true residual)
    b32 = b.float()
    x32 = torch.zeros_like(b32)
    w32 = B.alloc_workspace(b.shape)
    for _ in range(2):
        x32.zero_()
        _, r32 = B.pcg_solve(b32, x32, tol=TOL, maxit=MAXIT, workspace=w32, stream=stream)

    # the paper's Table 3 grid (512 x 112 x 64), context for the H100's 0.28 ms/iteration
    bc = torch.from_numpy(inputs.uniform_rhs((64, 112, 512), 0, dtype=np.float64)).cuda()
    xc = torch.zeros_like(bc)
    wc = B.alloc_workspace(bc.shape, io_dtype=B.F64)
    for _ in range(2):
        xc.zero_()
        _, rc = B.pcg_solve(bc, xc, tol=TOL, maxit=MAXIT, workspace=wc, stream=stream)

    # mixed precision (16-bit iteration vectors, FP64 refinement) next to plain FP32
    def timed_solve(bb, reps=1, oracle_check=None, **kw):
        """Best of `reps` timed solves after one warm-up (graphs built and cached).  oracle_check(x)
        (optional) adds the FP64 oracle's verdict on the returned x."""
        xx = torch.zeros_like(bb)
        wsx = B.alloc_workspace(bb.shape, io_dtype=B.F64, storage=B._DTYPES.get(kw.get("storage"), B.F32),
                                k_block=kw.get("k_block"), kb=kw.get("kb", 8))
        B.pcg_solve(bb, xx, workspace=wsx, **kw)
        best = None
        for _ in range(reps):
            xx.zero_()
            torch.cuda.synchronize()
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            _, rr = B.pcg_solve(bb, xx, workspace=wsx, stream=stream, **kw)
            t1.record(stream)
            torch.cuda.synchronize()
            ms = t0.elapsed_time(t1)
            best = ms if best is None else min(best, ms)
        out = {"ms": best, "reps": reps, "iters": rr["iters"], "outer_steps": rr["refine_steps"],
               "status": rr["status_name"], "rel_res_true_fp64": rr["rel_res_true"]}
        if oracle_check is not None:
            out.update(oracle_check(xx.cpu().numpy()))
        del wsx, xx
        return out

    mixed = {"poisson256_tol1e-6": {"fp32_plain": {"ms": ms_step, "iters": iters}}}
    for name, dt in (("bf16", torch.bfloat16), ("fp16", torch.float16)):
        mixed["poisson256_tol1e-6"][name] = timed_solve(b, reps=3, tol=TOL, maxit=MAXIT, storage=dt, max_outer=20)
    if N <= 256 ** 3 and rank == 0:
        import oracle
        oracle.build()
        # config 2 at 512^3: each result's true residual as the FP64 oracle evaluates b - A x
        k512, b512 = inputs.varcoeff_problem(512, 512, 512, seed=1, kb=8)
        b512 = b512.astype(np.float64)
        k512_64 = k512.astype(np.float64)
        kd = torch.from_numpy(k512).cuda()
        bd = torch.from_numpy(b512).cuda()

        # the oracle's own 512^3 solution (to 1e-10) on a lattice of 16^3 points, stored by
        # tests/golden/make_golden.py --config2 (an hour and more of FP64 CPU time to recompute)
        with open(os.path.join(ROOT, "tests", "golden", "pcg_lognormal512_seed1_lattice.json")) as f:
            lat = json.load(f)
        lsl = slice(lat["lattice_start"], None, lat["lattice_step"])
        x_lat = np.asarray(lat["x_lattice"])

        def check512(xh):
            return {"oracle_true_relres": oracle.true_relres(b512, xh, k512_64, 8),
                    "err_vs_oracle_lattice": float(np.linalg.norm(xh[lsl, lsl, lsl].ravel() - x_lat)
                                                   / np.linalg.norm(x_lat))}
        c2 = {}
        c2["fp32_plain"] = timed_solve(bd, tol=1e-8, maxit=20000, k_block=kd, kb=8, oracle_check=check512)
        c2["fp16"] = timed_solve(bd, tol=1e-8, maxit=8000, k_block=kd, kb=8, storage=torch.float16, max_outer=20,
                                 oracle_check=check512)
        c2["bf16"] = timed_solve(bd, tol=1e-8, maxit=6000, k_block=kd, kb=8, storage=torch.bfloat16, max_outer=20,
                                 oracle_check=check512)
        mixed["config2_512_lognormal_tol1e-8"] = c2
        del bd, kd, b512, k512_64
        torch.cuda.empty_cache()
        # the same recipe at 128^3, where the FP64 oracle's own solution (to 1e-10) takes seconds
        # rather than the hour it takes at 512^3: the error of each result against it
        n2 = 128
        k128, b128 = inputs.varcoeff_problem(n2, n2, n2, seed=1, kb=8)
        b128 = b128.astype(np.float64)
        k128_64 = k128.astype(np.float64)
        t0 = time.perf_counter()
        oref = oracle.pcg(b128, tol=1e-10, maxit=20000, k=k128_64, kb=8)
        oracle_s = time.perf_counter() - t0
        xo = oref["x"]
        kd = torch.from_numpy(k128).cuda()
        bd = torch.from_numpy(b128).cuda()

        def check128(xh):
            return {"oracle_true_relres": oracle.true_relres(b128, xh, k128_64, 8),
                    "err_vs_oracle": float(np.linalg.norm(xh - xo) / np.linalg.norm(xo))}
        c2s = {"oracle": {"tol": 1e-10, "iters": oref["iters"], "s": oracle_s, "threads": oracle.threads()}}
        c2s["fp32_plain"] = timed_solve(bd, reps=3, tol=1e-8, maxit=20000, k_block=kd, kb=8, oracle_check=check128)
        c2s["fp16"] = timed_solve(bd, reps=3, tol=1e-8, maxit=8000, k_block=kd, kb=8, storage=torch.float16,
                                  max_outer=20, oracle_check=check128)
        c2s["bf16"] = timed_solve(bd, reps=3, tol=1e-8, maxit=6000, k_block=kd, kb=8, storage=torch.bfloat16,
                                  max_outer=20, oracle_check=check128)
        mixed["config2_recipe_128_lognormal_tol1e-8"] = c2s
        del bd, kd
        torch.cuda.empty_cache()

    # 64 independent grids (sizes from {48, 64, 96, 128, 160}) in one persistent kernel launch, tiles from
    # the autotuner; beside it the same batch as one CUDA graph with a branch per problem
    shapes = inputs.batch_shapes(64, 2)
    rhs = [torch.from_numpy(v).cuda() for v in inputs.batch_rhs(shapes, 2, dtype=np.float64)]
    xb = [torch.zeros_like(v) for v in rhs]

    def run_batch(graph, reps=3):
        B.pcg_solve_batched(rhs, xb, tol=TOL, maxit=3000, autotune=True, graph=graph)  # tunes, builds graphs
        best = None
        for _ in range(reps):
            for v in xb:
                v.zero_()
            torch.cuda.synchronize()
            _, rr = B.pcg_solve_batched(rhs, xb, tol=TOL, maxit=3000, autotune=True, graph=graph)
            if best is None or rr[0]["time_ms"] < best[0]["time_ms"]:
                best = rr
        return best
    gres = run_batch(True)
    bres = run_batch(False)
    batch_ms = bres[0]["time_ms"]
    seq_ms = 0.0
    for v in rhs:
        xv = torch.zeros_like(v)
        B.pcg_solve(v, xv, tol=TOL, maxit=3000)
        xv.zero_()
        _, rv = B.pcg_solve(v, xv, tol=TOL, maxit=3000)
        seq_ms += rv["time_ms"]
    pts_iters = sum(int(np.prod(sh)) * r["iters"] for sh, r in zip(shapes, bres))
    g_pts_iters = sum(int(np.prod(sh)) * r["iters"] for sh, r in zip(shapes, gres))
    batched = {"problems": 64, "points": int(sum(int(np.prod(sh)) for sh in shapes)), "ms": batch_ms,
               "kernel_launches": bres[0]["pass_launches"][0], "phases": bres[0]["pass_launches"][1],
               "persistent_tiles": ["64x16", "128x8", "32x32"][bres[0]["pass_ctas"][0]],
               "all_converged": all(r["status"] == 0 for r in bres),
               "iters_min_max": [min(r["iters"] for r in bres), max(r["iters"] for r in bres)],
               "max_rel_res_true_fp64": max(r["rel_res_true"] for r in bres),
               "aggregate_gbs": ITER_BYTES * pts_iters / (batch_ms * 1e-3) / 1e9,
               "aggregate_frac": ITER_BYTES * pts_iters / (batch_ms * 1e-3) / 1e9 / peak,
               "graph_of_branches": {"ms": gres[0]["time_ms"], "all_converged": all(r["status"] == 0 for r in gres),
                                     "aggregate_gbs": ITER_BYTES * g_pts_iters / (gres[0]["time_ms"] * 1e-3) / 1e9},
               "sequential_ms": seq_ms}
    del rhs, xb

    # f1: the same 256^3 operator assembled as a Sliced-ELL (SELL-32) matrix and solved by the general
    # sparse PCG (the paper's H100 comparator design), next to the matrix-free solve
    sell = None
    if rank == 0:
        sm = B.sell_from_stencil(b.shape)
        bs64 = b.ravel().contiguous()
        xs64 = torch.zeros_like(bs64)
        sws = None
        for _ in range(2):
            xs64.zero_()
            _, sres = B.sell_pcg_solve(sm, bs64, xs64, tol=TOL, maxit=MAXIT, stream=stream)
        pv = torch.from_numpy(inputs.uniform_rhs(b.shape, 3)).cuda().ravel()
        qv = torch.empty_like(pv)
        reps = 20
        B.sell_spmv(sm, pv, qv, stream=stream)
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(reps):
            B.sell_spmv(sm, pv, qv, stream=stream)
        s1.record(stream)
        torch.cuda.synchronize()
        spmv_us = s0.elapsed_time(s1) / reps * 1e3
        # SpMV algorithmic bytes: stored values and columns (8 B each), the gathered x once, y
        spmv_bytes = 8 * sm.nnz_stored + 8 * N
        sell = {"workload": f"poisson {n}^3 assembled as SELL-32 ({sm.nnz_stored} stored entries, "
                            f"{sm.nnz_stored / N:.3f} per row)",
                "solve": {"ms": sres["time_ms"], "iters": sres["iters"], "status": sres["status_name"],
                          "rel_res_true_fp64": sres["rel_res_true"], "replacements": sres["replacements"],
                          "us_per_iter": 1e3 * sres["time_ms"] / max(1, sres["iters"]),
                          "algorithmic_bytes_per_row_iter": 108,
                          "gbs_at_108B": 108 * N / (sres["time_ms"] * 1e-3 / max(1, sres["iters"])) / 1e9},
                "spmv": {"us": spmv_us, "algorithmic_bytes": spmv_bytes, "gbs": spmv_bytes / (spmv_us * 1e-6) / 1e9,
                         "frac": spmv_bytes / (spmv_us * 1e-6) / 1e9 / peak},
                "matrix_free_ms": ms_step}
        del sm, bs64, xs64, pv, qv
        torch.cuda.empty_cache()

    # f3: PCG with the geometric multigrid preconditioner on the headline problem and on the
    # lognormal-coefficient problem the learned preconditioner is evaluated on (seed 100)
    mgres = None
    if rank == 0:
        mgres = {}
        xm = torch.zeros_like(b)
        mws = B.mg_workspace(b.shape)
        for _ in range(2):
            xm.zero_()
            _, rm = B.mg_pcg_solve(b, xm, tol=TOL, maxit=MAXIT, workspace=mws, stream=stream)
        mgres["poisson256"] = {"ms": rm["time_ms"], "iters": rm["iters"], "levels": rm["pass_launches"][0],
                               "status": rm["status_name"], "rel_res_true_fp64": rm["rel_res_true"],
                               "jacobi_ms": ms_step, "jacobi_iters": iters,
                               "speedup_over_jacobi": ms_step / rm["time_ms"]}
        from paper_2603_23343_gb300 import learned as _learned
        k100, b100 = _learned.problem((n, n, n), 100)
        xm = torch.zeros_like(b100)
        mws = B.mg_workspace(b100.shape, k_block=k100)
        for _ in range(2):
            xm.zero_()
            _, rm = B.mg_pcg_solve(b100, xm, tol=TOL, maxit=MAXIT, k_block=k100, workspace=mws, stream=stream)
        xj = torch.zeros_like(b100)
        for _ in range(2):
            xj.zero_()
            _, rj = B.pcg_solve(b100, xj, tol=TOL, maxit=20000, k_block=k100, stream=stream)
        mgres["lognormal256_seed100"] = {"ms": rm["time_ms"], "iters": rm["iters"], "levels": rm["pass_launches"][0],
                                         "status": rm["status_name"], "rel_res_true_fp64": rm["rel_res_true"],
                                         "jacobi_ms": rj["time_ms"], "jacobi_iters": rj["iters"],
                                         "speedup_over_jacobi": rj["time_ms"] / rm["time_ms"]}
        del xm, mws, xj, b100, k100
        torch.cuda.empty_cache()

    # a6: the dot and axpy kernels on 2^28 FP32 elements (1 GiB per vector, far above L2), best of 5
    n28 = 1 << 28
    gen = torch.Generator(device="cuda").manual_seed(28)
    xa = torch.empty(n28, dtype=torch.float32, device="cuda").uniform_(-1.0, 1.0, generator=gen)
    ya = torch.empty(n28, dtype=torch.float32, device="cuda").uniform_(-1.0, 1.0, generator=gen)
    dout = torch.empty((), dtype=torch.float64, device="cuda")
    dws = torch.empty(B.dot_workspace_size(), dtype=torch.uint8, device="cuda")

    def best_us(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        t = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            t.append(e0.elapsed_time(e1) * 1e3)
        return min(t)

    t_dot = best_us(lambda: B.dot(xa, ya, dout, dws, stream=stream))
    t_axpy = best_us(lambda: B.axpy(1e-3, xa, ya, stream=stream))
    micro = {"n": n28, "dtype": "f32", "inputs": "U[-1,1) from a seeded device generator"}
    for name, us, nbytes in (("dot", t_dot, 8 * n28), ("axpy", t_axpy, 12 * n28)):
        micro[name] = {"us": us, "algorithmic_bytes": nbytes, "gbs": nbytes / (us * 1e-6) / 1e9,
                       "frac": nbytes / (us * 1e-6) / 1e9 / peak}
    del xa, ya, dws
    torch.cuda.empty_cache()

    ablations = ablation_leg(B, inputs, stream, b, n) if rank == 0 else None

    learned_res = None
    if not args.no_learned and n == 256:
        from paper_2603_23343_gb300 import learned
        learned_res = learned_leg(B, learned, stream, args.learned_full)

    iter_us = ms_step * 1e3 / max(1, iters)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(n)

    if rank == 0:
        line = {
            "metric": METRIC, "value": ms_step, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {
                "workload": f"poisson {n}^3 FP32 Jacobi-PCG to 1e-6 (b~U[-1,1) seed 0, x0=0, h=1/{n + 1})",
                "n": n, "tol": TOL, "iters": iters, "status": res["status_name"],
                "rel_res_true_fp64": res["rel_res_true"], "replicas": world,
                "residual_replacements": res["replacements"],
                "vectors": "iteration vectors z, p0, p1, d FP32; b, x FP64",
                "l2": "no flush: working set b,x (FP64) + z,p0,p1,d (FP32) = %d MiB > L2" % ((2 * 8 + 4 * 4) * N >> 20),
                "fp32_x": {"iters": r32["iters"], "status": r32["status_name"], "ms": r32["time_ms"],
                           "rel_res_true_fp64": r32["rel_res_true"]},
                "iteration": {"us": iter_us, "algorithmic_bytes_per_pt": ITER_BYTES,
                              "gbs": ITER_BYTES * N / (iter_us * 1e-6) / 1e9,
                              "frac": ITER_BYTES * N / (iter_us * 1e-6) / 1e9 / peak,
                              "gbs_44B_three_kernel_equiv": THREE_KERNEL_BYTES * N / (iter_us * 1e-6) / 1e9,
                              "frac_44B_three_kernel_equiv":
                                  THREE_KERNEL_BYTES * N / (iter_us * 1e-6) / 1e9 / peak},
                "table3_grid_512x112x64": {"iters": rc["iters"], "ms_per_iter": rc["time_ms"] / max(1, rc["iters"]),
                                           "h100_ms_per_iter_paper": 0.28},
            },
            "mixed_precision": mixed,
            "batched_config3": batched,
            "microkernels_2e28": micro,
            "ablations": ablations,
            "sell_spmv_pcg": sell,
            "multigrid_pcg": mgres,
            "learned_config4": learned_res,
            "roofline": roofline,
            "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": 2 * N * 8,
                    "d2h_bytes_per_step": N * 8 + 256},
            # per solve: reset, max |b|, initial residual, 2 per iteration, flush + residual per
            # replacement, finalize, true residual
            "gpu_launches": args.steps * (2 * iters + 5 + 2 * res["replacements"]),
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
