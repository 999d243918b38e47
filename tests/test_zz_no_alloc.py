"""The dot product that allocates nothing (gbpcg_dot_noalloc).

Some callers cannot hand the library a workspace or let it allocate: code
that runs while a stream is being captured into a CUDA graph (cudaMalloc is
not allowed there), code living under another framework's memory pool, and
latency-critical loops that cannot pay for an allocation.  For them the
library keeps a static scratch array on the device.  This test calls that
entry point through the C ABI and checks it against the ordinary
workspace-based gbpcg_dot, twice in a row (the second call must not be
disturbed by what the first left in the shared array).  The file sorts last
so that a run stopping at its first failure has already run everything else.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_23343_gb300 import inputs

pytestmark = pytest.mark.gpu


def _pair(seed, n, dtype=torch.float32):
    x = inputs.uniform_pm1(seed, 0, n)
    y = inputs.uniform_pm1(seed + 1, 0, n)
    scale = float(np.sum(np.abs(x.astype(np.float64) * y)))
    return torch.from_numpy(x).to(dtype).cuda(), torch.from_numpy(y).to(dtype).cuda(), scale


def test_dot_noalloc_matches_dot_on_two_calls_in_a_row(gpu_lib):
    # 2^24 + 5 runs the capped grid (8 blocks per SM, threads striding), 2^22 one pass per thread
    cases = [(50, 3_000_001), (52, 1 << 22), (60, (1 << 24) + 5)]
    for seed, n in cases:
        x, y, scale = _pair(seed, n)
        ref = float(gpu_lib.dot(x, y).item())
        got = float(gpu_lib.dot_noalloc(x, y).item())
        # the tolerance the kernel tests use for FP32 dots: 1e-5 of sum |x_i y_i|
        assert abs(got - ref) <= 1e-5 * scale, (n, got, ref)
        # and against the FP64 oracle on the same FP32 numbers
        xo = x.cpu().double().numpy()
        yo = y.cpu().double().numpy()
        assert abs(got - oracle.dot(xo, yo)) <= 1e-5 * scale, (n, got)
    # the same input twice in a row: bit-identical results (the ticket restarts
    # at zero and the sum order is fixed); gbpcg_dot uses another grid size, so
    # it agrees within the tolerance rather than bit for bit
    x, y, scale = _pair(54, 1_000_003)
    a = float(gpu_lib.dot_noalloc(x, y).item())
    b = float(gpu_lib.dot_noalloc(x, y).item())
    assert a == b
    assert abs(a - float(gpu_lib.dot(x, y).item())) <= 1e-5 * scale


def test_dot_noalloc_other_dtypes_and_empty(gpu_lib):
    x, y, scale = _pair(56, 100_003, torch.float64)
    assert abs(float(gpu_lib.dot_noalloc(x, y).item()) - float(gpu_lib.dot(x, y).item())) <= 1e-12 * scale
    x, y, scale = _pair(58, 100_003, torch.bfloat16)
    assert abs(float(gpu_lib.dot_noalloc(x, y).item()) - float(gpu_lib.dot(x, y).item())) <= 1e-5 * scale
    e = torch.empty(0, device="cuda")
    assert float(gpu_lib.dot_noalloc(e, e).item()) == 0.0
