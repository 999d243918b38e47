"""GPU parity of the three kernels (stencil, dot, axpy) against the FP64 oracle.

Tolerances (FP32 arithmetic, FP64 oracle on the same input values):
  stencil  |q_gpu - q| <= 1e-5 * (|A| |p|)_i elementwise, where |A||p| =
           2 D|p| - A|p| is the sum of the magnitudes of the terms (the
           natural rounding scale; a plain relative error is meaningless where
           the terms cancel).  16-bit storage adds one output rounding:
           + 2^-8 |q| (BF16) or 2^-11 |q| (FP16).
  dot      |d_gpu - d| <= 1e-5 * sum |x_i y_i|; integer-valued input is exact.
  axpy     bit-exact against the FP64 result rounded to FP32 when alpha is a
           float32 number (one fused rounding on each side).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_23343_gb300 import inputs

pytestmark = pytest.mark.gpu

SHAPES = [(3, 7, 5), (9, 17, 33), (37, 40, 64), (20, 33, 100), (32, 32, 32), (70, 50, 132), (1, 1, 4),
          (17, 5, 256)]


def abs_op_bound(u, k=None, kb=8):
    d = oracle.diag(u.shape, k, kb)
    au = np.abs(u)
    return 2.0 * d * au - oracle.apply(au, k, kb)


def to_dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


@pytest.mark.parametrize("shape", SHAPES)
def test_stencil_f32_poisson(gpu_lib, shape):
    p = inputs.uniform_rhs(shape, 3)
    q = gpu_lib.stencil_apply(to_dev(p)).cpu().double().numpy()
    ref = oracle.apply(p.astype(np.float64))
    bound = abs_op_bound(p.astype(np.float64))
    assert np.all(np.abs(q - ref) <= 1e-5 * bound + 1e-30)


def test_stencil_f32_sine_mode_eigen(gpu_lib):
    """Sine modes are eigenvectors; the GPU must reproduce A v = lambda v."""
    shape = (24, 20, 28)
    nz, ny, nx = shape
    a, b, c = 3, 2, 5
    gx = np.sin(a * np.pi * np.arange(1, nx + 1) / (nx + 1))
    gy = np.sin(b * np.pi * np.arange(1, ny + 1) / (ny + 1))
    gz = np.sin(c * np.pi * np.arange(1, nz + 1) / (nz + 1))
    v = (gz[:, None, None] * gy[None, :, None] * gx[None, None, :]).astype(np.float32)
    lam = sum(4 * (n + 1) ** 2 * np.sin(m * np.pi / (2 * (n + 1))) ** 2 for n, m in ((nx, a), (ny, b), (nz, c)))
    q = gpu_lib.stencil_apply(to_dev(v)).cpu().double().numpy()
    bound = abs_op_bound(v.astype(np.float64))
    assert np.all(np.abs(q - lam * v.astype(np.float64)) <= 1e-5 * bound)


@pytest.mark.parametrize("shape,kb", [((16, 16, 16), 8), ((37, 40, 64), 8), ((9, 17, 33), 3), ((20, 33, 100), 4)])
def test_stencil_f32_block_coefficient(gpu_lib, shape, kb):
    nz, ny, nx = shape
    nbx, nby, nbz = inputs.block_counts(nx, ny, nz, kb)
    k = inputs.lognormal_blocks(nbx, nby, nbz, 1)
    p = inputs.uniform_rhs(shape, 4)
    q = gpu_lib.stencil_apply(to_dev(p), k_block=to_dev(k), kb=kb).cpu().double().numpy()
    ref = oracle.apply(p.astype(np.float64), k.astype(np.float64), kb)
    bound = abs_op_bound(p.astype(np.float64), k.astype(np.float64), kb)
    assert np.all(np.abs(q - ref) <= 2e-5 * bound + 1e-30)


@pytest.mark.parametrize("tdtype,eps", [(torch.bfloat16, 2.0 ** -8), (torch.float16, 2.0 ** -11)])
@pytest.mark.parametrize("shape", [(9, 17, 33), (37, 40, 64), (32, 32, 32)])
def test_stencil_16bit_storage(gpu_lib, shape, tdtype, eps):
    # the scaled operator h^2 A keeps FP16 in range: feed values of size h^2
    p32 = inputs.uniform_rhs(shape, 5)
    pd = to_dev(p32, tdtype)
    nz, ny, nx = shape
    scale = 1.0 / (max(nx, ny, nz) + 1) ** 2
    pd = (pd.float() * scale).to(tdtype)
    p = pd.float().cpu().double().numpy()  # the exact values the GPU sees
    q = gpu_lib.stencil_apply(pd).float().cpu().double().numpy()
    ref = oracle.apply(p)
    bound = abs_op_bound(p)
    assert np.all(np.abs(q - ref) <= eps * np.abs(ref) + 1e-5 * bound + 1e-30)


@pytest.mark.parametrize("shape", [(9, 17, 33), (32, 32, 32)])
def test_stencil_f64(gpu_lib, shape):
    p = inputs.uniform_rhs(shape, 6, dtype=np.float64) * (1 + 1e-9)
    q = gpu_lib.stencil_apply(to_dev(p, torch.float64)).cpu().numpy()
    ref = oracle.apply(p)
    assert np.all(np.abs(q - ref) <= 1e-13 * abs_op_bound(p))


@pytest.mark.parametrize("shape,kb", [((10, 14, 22), 4), ((9, 17, 33), 3), ((16, 16, 16), 8)])
def test_stencil_f64_block_coefficient(gpu_lib, shape, kb):
    """FP64 operator with block coefficients (partial blocks at the far end of each axis where
    the edge is not a multiple of kb): harmonic-mean faces in FP64, against the oracle."""
    nz, ny, nx = shape
    nbx, nby, nbz = inputs.block_counts(nx, ny, nz, kb)
    k = inputs.lognormal_blocks(nbx, nby, nbz, 2)
    p = inputs.uniform_rhs(shape, 8, dtype=np.float64)
    q = gpu_lib.stencil_apply(to_dev(p, torch.float64), k_block=to_dev(k), kb=kb).cpu().numpy()
    ref = oracle.apply(p, k.astype(np.float64), kb)
    assert np.all(np.abs(q - ref) <= 1e-13 * abs_op_bound(p, k.astype(np.float64), kb))


@pytest.mark.parametrize("n", [1, 7, 4096, 4097, 1_000_003, 1 << 22])
def test_dot_f32(gpu_lib, n):
    x = inputs.uniform_pm1(10, 0, n)
    y = inputs.uniform_pm1(11, 0, n)
    d = float(gpu_lib.dot(to_dev(x), to_dev(y)).item())
    ref = oracle.dot(x.astype(np.float64), y.astype(np.float64))
    assert abs(d - ref) <= 1e-5 * float(np.sum(np.abs(x.astype(np.float64) * y))) + 1e-300


def test_dot_and_axpy_at_bench_size_capped_grid(gpu_lib):
    """2^26 + 3 elements: both kernels run their capped grid (8 blocks per SM) with every thread
    striding over many vectors, the regime the 2^28 microbenchmark times, plus a ragged tail."""
    n = (1 << 26) + 3
    x = inputs.uniform_pm1(40, 0, n)
    y = inputs.uniform_pm1(41, 0, n)
    xd, yd = to_dev(x), to_dev(y)
    d = float(gpu_lib.dot(xd, yd).item())
    x64, y64 = x.astype(np.float64), y.astype(np.float64)
    ref = oracle.dot(x64, y64)
    assert abs(d - ref) <= 1e-5 * float(np.sum(np.abs(x64 * y64)))
    alpha = 0.375
    gpu_lib.axpy(alpha, xd, yd)
    refa = oracle.axpy(alpha, x64, y64).astype(np.float32)
    assert np.array_equal(yd.cpu().numpy(), refa)


def test_dot_integer_exact_and_deterministic(gpu_lib):
    n = 3_000_001
    i = np.arange(n)
    x = ((i * 7919) % 7 - 3).astype(np.float32)
    y = ((i * 104729) % 5 - 2).astype(np.float32)
    exact = int(np.sum(x.astype(np.int64) * y.astype(np.int64)))
    xd, yd = to_dev(x), to_dev(y)
    ws = torch.empty(gpu_lib.dot_workspace_size(), dtype=torch.uint8, device="cuda")
    vals = {float(gpu_lib.dot(xd, yd, workspace=ws).item()) for _ in range(5)}
    assert vals == {float(exact)}
    # unaligned views take the scalar path and agree
    d_off = float(gpu_lib.dot(xd[1:], yd[1:]).item())
    assert d_off == float(exact - int(x[0]) * int(y[0]))


def test_dot_empty_and_other_dtypes(gpu_lib):
    e = torch.empty(0, device="cuda")
    assert float(gpu_lib.dot(e, e).item()) == 0.0
    x = inputs.uniform_pm1(12, 0, 100_003)
    y = inputs.uniform_pm1(13, 0, 100_003)
    ref = oracle.dot(x.astype(np.float64), y.astype(np.float64))
    d64 = float(gpu_lib.dot(to_dev(x, torch.float64), to_dev(y, torch.float64)).item())
    assert abs(d64 - ref) <= 1e-12 * float(np.sum(np.abs(x * y.astype(np.float64))))
    xb, yb = to_dev(x, torch.bfloat16), to_dev(y, torch.bfloat16)
    refb = oracle.dot(xb.float().cpu().double().numpy(), yb.float().cpu().double().numpy())
    db = float(gpu_lib.dot(xb, yb).item())
    assert abs(db - refb) <= 1e-5 * float(np.sum(np.abs(x * y.astype(np.float64))))


@pytest.mark.parametrize("n", [1, 5, 4096, 1_000_003])
def test_axpy_f32_bit_exact(gpu_lib, n):
    x = inputs.uniform_pm1(14, 0, n)
    y = inputs.uniform_pm1(15, 0, n)
    alpha = -0.75
    yd = to_dev(y)
    gpu_lib.axpy(alpha, to_dev(x), yd)
    ref = oracle.axpy(alpha, x.astype(np.float64), y.astype(np.float64)).astype(np.float32)
    assert np.array_equal(yd.cpu().numpy(), ref)


def test_axpy_unaligned_and_f64(gpu_lib):
    n = 10_001
    x = inputs.uniform_pm1(16, 0, n)
    y = inputs.uniform_pm1(17, 0, n)
    yd = to_dev(y)
    gpu_lib.axpy(0.3, to_dev(x)[1:], yd[1:])
    ref = oracle.axpy(np.float32(0.3), x[1:].astype(np.float64), y[1:].astype(np.float64))
    assert np.max(np.abs(yd[1:].cpu().double().numpy() - ref)) <= 1e-7 * 2
    assert yd[0].item() == y[0]
    y64 = to_dev(y, torch.float64)
    gpu_lib.axpy(0.3, to_dev(x, torch.float64), y64)
    ref64 = oracle.axpy(0.3, x.astype(np.float64), y.astype(np.float64))
    assert np.max(np.abs(y64.cpu().numpy() - ref64)) <= 1e-15
