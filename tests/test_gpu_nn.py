"""GPU parity of the learned preconditioner's kernels against the FP64 oracle
(oracle/nn.py), called through the C ABI.

Inputs are BF16 numbers (the kernels' operand type), so the oracle sees the
same values exactly in FP64.  Tolerances:
  convolutions   |y_gpu - y| <= 2e-5 * conv(|x|, |w|) elementwise: FP32
                 accumulation of 27 * ci products (tensor cores or FFMA);
                 the bound is the sum of the magnitudes of the terms.
  weight grads   |g_gpu - g| <= 2e-5 * wgrad(|x|, |gy|) elementwise (sums over
                 all voxels in FP32 per block, fixed-order slot sums).
  U-net forward  the oracle rounds every stored activation to BF16 as the GPU
                 does; remaining differences come from a BF16 rounding that
                 flips when FP32 and FP64 sums straddle a rounding boundary,
                 so the check is on norms: ||z_gpu - z|| <= 5e-3 ||z||.
  U-net backward the oracle rounds the propagated gradients to BF16 where the
                 GPU stores them.  A weight-gradient entry is a sum over voxels
                 with heavy cancellation (worst for the log k channel, constant
                 on 8^3 blocks), so its error is measured against the sum of the
                 magnitudes of its terms, B = wgrad(|x|, |gy|), from the
                 oracle's traced (x, gy): per layer ||g_gpu - g|| <= 5e-3 ||B||
                 (about one BF16 rounding of the terms: FP32-vs-FP64 sums make
                 some roundings land on the other side, and those compound
                 through the layers); cosine(g_gpu, g) >= 0.995 guards the direction.
  loss           FP32 stencils, FP64 dots: 1e-5 relative.
  Adam           FP32 arithmetic: per step half an FP32 ulp of w plus 1e-5 of
                 the step lr.
"""
import numpy as np
import pytest
import torch

import oracle.nn as onn
from paper_2603_23343_gb300 import inputs

pytestmark = pytest.mark.gpu


def bf16_np(a):
    """Round to BF16 (round to nearest even, via FP32) and return FP64."""
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).float().to(torch.bfloat16).double().numpy()


def rnd(shape, seed, scale=1.0):
    n = int(np.prod(shape))
    return inputs.uniform_pm1(seed, 0, n, np.float64).reshape(shape) * scale


def dev_bf16(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(torch.bfloat16).cuda()


# (nz, ny, nx): X % 128 == 0 with Y % 4 == 0 takes the halo-slab kernel, the rest the per-tap one
TC_SHAPES = [(5, 3, 128), (4, 8, 32), (8, 4, 8), (2, 2, 256), (3, 4, 128), (2, 8, 256)]
TC_CHANNELS = [(16, 16), (16, 32), (32, 32), (32, 64), (64, 64), (96, 32), (48, 16), (16, 48), (32, 96), (64, 32),
               (32, 16)]


def conv_case(shape, ci, co, seed):
    x = bf16_np(rnd(shape + (ci,), seed))
    w = bf16_np(rnd((co, 27, ci), seed + 1, 1.0 / np.sqrt(27 * ci)))
    return x, w


@pytest.mark.parametrize("shape", TC_SHAPES)
@pytest.mark.parametrize("ci,co", TC_CHANNELS)
def test_conv3_forward_tensor_cores(gpu_lib, shape, ci, co):
    x, w = conv_case(shape, ci, co, 100 + ci + co)
    y = gpu_lib.conv3_forward(dev_bf16(x), dev_bf16(w)).cpu().double().numpy()
    ref = onn.conv3(x, w)
    bound = onn.conv3(np.abs(x), np.abs(w))
    assert np.all(np.abs(y - ref) <= 2e-5 * bound + 1e-30), np.max(np.abs(y - ref) / (bound + 1e-30))


# 16 output channels on rows of 128 take the z-marching kernel, whose CTAs own 3-row columns over z
# segments.  (8, 59, 1024): 160 columns for 152 SMs, so each CTA marches up to three segments of
# four planes (its accumulators rotate through twelve output planes) and the last column has two
# rows inside the grid; (40, 7, 256): two-plane segments, the last column one row deep.
@pytest.mark.parametrize("shape,ci,relu", [((8, 59, 1024), 16, False), ((8, 59, 1024), 48, True),
                                           ((40, 7, 256), 48, False)])
def test_conv3_forward_zmarch_segments(gpu_lib, shape, ci, relu):
    x, w = conv_case(shape, ci, 16, 500 + ci)
    y = gpu_lib.conv3_forward(dev_bf16(x), dev_bf16(w), relu=relu).cpu().double().numpy()
    ref = onn.conv3(x, w)
    if relu:
        ref = onn.relu(ref)
    bound = onn.conv3(np.abs(x), np.abs(w))
    assert np.all(np.abs(y - ref) <= 2e-5 * bound + 1e-30), np.max(np.abs(y - ref) / (bound + 1e-30))


@pytest.mark.parametrize("ci,co", [(16, 32), (48, 16)])
def test_conv3_forward_relu(gpu_lib, ci, co):
    x, w = conv_case((4, 8, 32), ci, co, 7)
    y = gpu_lib.conv3_forward(dev_bf16(x), dev_bf16(w), relu=True).cpu().double().numpy()
    ref = onn.relu(onn.conv3(x, w))
    bound = onn.conv3(np.abs(x), np.abs(w))
    assert np.all(np.abs(y - ref) <= 2e-5 * bound + 1e-30)
    assert np.all(y >= 0)


@pytest.mark.parametrize("shape", [(5, 7, 9), (4, 8, 32), (1, 1, 3), (3, 5, 16), (2, 3, 64), (2, 3, 256)])
@pytest.mark.parametrize("ci,co", [(2, 16), (16, 1), (1, 16)])
def test_conv3_forward_cuda_cores(gpu_lib, shape, ci, co):
    x, w = conv_case(shape, ci, co, 200 + ci + co)
    y = gpu_lib.conv3_forward(dev_bf16(x), dev_bf16(w)).cpu().double().numpy()
    ref = onn.conv3(x, w)
    bound = onn.conv3(np.abs(x), np.abs(w))
    assert np.all(np.abs(y - ref) <= 2e-5 * bound + 1e-30)


@pytest.mark.parametrize("shape", [(5, 3, 128), (8, 4, 8), (3, 8, 128)])
@pytest.mark.parametrize("ci,co", [(16, 16), (48, 16), (96, 32), (64, 64), (16, 32), (16, 1)])
def test_conv3_backward_data(gpu_lib, shape, ci, co):
    gy = bf16_np(rnd(shape + (co,), 300 + ci))
    w = bf16_np(rnd((co, 27, ci), 301 + co, 1.0 / np.sqrt(27 * ci)))
    gx = gpu_lib.conv3_backward_data(dev_bf16(gy), dev_bf16(w)).cpu().double().numpy()
    ref = onn.conv3_adjoint(gy, w)
    bound = onn.conv3_adjoint(np.abs(gy), np.abs(w))
    assert np.all(np.abs(gx - ref) <= 2e-5 * bound + 1e-30)


@pytest.mark.parametrize("shape", [(5, 3, 128), (4, 8, 32), (8, 4, 8), (3, 5, 16)])
@pytest.mark.parametrize("ci,co", [(16, 16), (48, 16), (96, 32), (64, 64), (32, 64), (2, 16), (16, 1), (1, 16)])
def test_conv3_backward_weight(gpu_lib, shape, ci, co):
    x = bf16_np(rnd(shape + (ci,), 400 + ci))
    gy = bf16_np(rnd(shape + (co,), 401 + co))
    gw = gpu_lib.conv3_backward_weight(dev_bf16(x), dev_bf16(gy)).cpu().double().numpy()
    ref = onn.conv3_weight_grad(x, gy)
    bound = onn.conv3_weight_grad(np.abs(x), np.abs(gy))
    assert np.all(np.abs(gw - ref) <= 2e-5 * bound + 1e-30)
    gw2 = gpu_lib.conv3_backward_weight(dev_bf16(x), dev_bf16(gy)).cpu().double().numpy()
    np.testing.assert_array_equal(gw, gw2)  # fixed summation order


def test_conv3_rejects_unsupported(gpu_lib):
    x = dev_bf16(np.zeros((4, 4, 12, 16)))  # 12 does not divide 128
    w = dev_bf16(np.zeros((16, 27, 16)))
    with pytest.raises(gpu_lib.GbpcgError):
        gpu_lib.conv3_forward(x, w)
    w2 = dev_bf16(np.zeros((24, 27, 16)))  # 24 output channels: no tensor-core shape
    with pytest.raises(gpu_lib.GbpcgError):
        gpu_lib.conv3_forward(dev_bf16(np.zeros((4, 8, 32, 16))), w2)


# ----------------------------------------------------------- the U-net -----

def unet_case(shape=(32, 32, 32), seed=5, varcoeff=True, kb=8):
    r = inputs.uniform_rhs(shape, seed).astype(np.float64)
    if varcoeff:
        nbx, nby, nbz = inputs.block_counts(shape[2], shape[1], shape[0], kb)
        k = inputs.lognormal_blocks(nbx, nby, nbz, seed + 1)
        k64 = k.astype(np.float64)
        k_dev = torch.from_numpy(k).float().cuda()
    else:
        k64, k_dev = None, None
    ws = onn.init_weights(seed)
    return r, k64, k_dev, ws


def oracle_forward_bf16(r, k64, ws, kb=8):
    """The oracle U-net with the GPU's BF16 roundings of weights and activations."""
    wsb = {name: bf16_np(v) for name, v in ws.items()}
    x, scale = onn.net_input(r, onn.logk_field(r.shape, k64, kb), onn.jacobi_scale(r.shape, k64, kb))
    x = bf16_np(x)
    out, cache = onn.net_forward(x, wsb, round_fn=bf16_np)
    return out[..., 0] * scale, cache, wsb, scale


@pytest.mark.parametrize("varcoeff", [False, True])
@pytest.mark.parametrize("shape", [(32, 32, 32), (64, 64, 64), (16, 16, 128)])
def test_unet_forward(gpu_lib, varcoeff, shape):
    r, k64, k_dev, ws = unet_case(shape, 5 + shape[0], varcoeff)
    w = gpu_lib.nn_pack_weights(ws).cuda()
    z = gpu_lib.nn_forward(w, torch.from_numpy(r).float().cuda(), k_block=k_dev).cpu().double().numpy()
    # the oracle sees r as the FP32 numbers the GPU got
    zr, _, _, _ = oracle_forward_bf16(r.astype(np.float32).astype(np.float64), k64, ws)
    err = np.linalg.norm(z - zr) / np.linalg.norm(zr)
    assert err <= 5e-3, err
    # and the unrounded FP64 network agrees to BF16 accuracy
    z64 = onn.precond_apply(r, ws, k64, 8)
    assert np.linalg.norm(z - z64) / np.linalg.norm(z64) <= 5e-2


def test_unet_forward_is_positively_homogeneous(gpu_lib):
    r, k64, k_dev, ws = unet_case((32, 32, 32), 9, True)
    w = gpu_lib.nn_pack_weights(ws).cuda()
    rd = torch.from_numpy(r).float().cuda()
    z1 = gpu_lib.nn_forward(w, rd, k_block=k_dev)
    z2 = gpu_lib.nn_forward(w, rd * 4.0, k_block=k_dev)  # exact power-of-two scaling
    torch.testing.assert_close(z2, 4.0 * z1, rtol=1e-6, atol=0)


@pytest.mark.parametrize("shape", [(32, 32, 32), (16, 16, 128)])
def test_unet_backward(gpu_lib, shape):
    r, k64, k_dev, ws = unet_case(shape, 11, True)
    w = gpu_lib.nn_pack_weights(ws).cuda()
    rd = torch.from_numpy(r).float().cuda()
    wsp = gpu_lib.nn_workspace(r.shape, training=True)
    gpu_lib.nn_forward(w, rd, k_block=k_dev, workspace=wsp)
    gz = rnd(r.shape, 12)
    gw = gpu_lib.nn_backward(torch.from_numpy(gz).float().cuda(), wsp, k_block=k_dev).cpu().double().numpy()
    assert gpu_lib.nn_status(wsp) == gpu_lib.OK
    zr, cache, wsb, scale = oracle_forward_bf16(r.astype(np.float32).astype(np.float64), k64, ws)
    gout = bf16_np(gz * scale)[..., None]
    trace = {}
    g = onn.net_backward(gout, wsb, cache, round_fn=bf16_np, trace=trace)
    gg = gpu_lib.nn_unpack_weights(torch.from_numpy(gw))
    for name, _, _ in gpu_lib.NN_LAYERS:
        a = gg[name].numpy().ravel()
        b = g[name].ravel()
        xl, gyl = trace[name]
        bound = np.linalg.norm(onn.conv3_weight_grad(np.abs(xl), np.abs(gyl)))
        err = np.linalg.norm(a - b)
        cos = float(a @ b) / (np.linalg.norm(a) * np.linalg.norm(b))
        print(name, err / np.linalg.norm(b), err / bound, cos)
        assert err <= 5e-3 * bound and cos >= 0.995, (name, err / np.linalg.norm(b), err / bound, cos)


def test_loss_and_gradient(gpu_lib):
    """Scale-free sign-aware A-norm loss and its gradient against the oracle, for z on both
    sides of z.Ae = 0."""
    shape = (32, 32, 32)
    nb = 4
    k = inputs.lognormal_blocks(nb, nb, nb, 3)
    kd = torch.from_numpy(k).float().cuda()
    kk = k.astype(np.float64)
    e = inputs.uniform_rhs(shape, 21)
    wsp = gpu_lib.nn_workspace(shape, training=True)
    for sign in (1.0, -1.0):
        z = (inputs.uniform_rhs(shape, 20) + np.float32(sign * 0.5) * e).astype(np.float32)
        loss, gz = gpu_lib.nn_loss(torch.from_numpy(z).cuda(), torch.from_numpy(e).cuda(), wsp, k_block=kd)
        zd, ed = z.astype(np.float64), e.astype(np.float64)
        ref = onn.loss_scaled(zd, ed, kk, 8)
        assert abs(loss.item() - ref) <= 1e-5 * ref
        g = onn.loss_scaled_grad(zd, ed, kk, 8)
        assert np.max(np.abs(gz.cpu().double().numpy() - g)) <= 1e-5 * np.max(np.abs(g))


def test_adam(gpu_lib):
    n = gpu_lib.NN_NUM_WEIGHTS
    w0 = rnd((n,), 30).astype(np.float32)
    w = torch.from_numpy(w0).cuda()
    m = torch.zeros_like(w)
    v = torch.zeros_like(w)
    wr, mr, vr = w0.astype(np.float64), np.zeros(n), np.zeros(n)
    for t in range(1, 4):
        g = rnd((n,), 30 + t).astype(np.float32)
        gpu_lib.nn_adam(w, torch.from_numpy(g).cuda(), m, v, t, lr=1e-2)
        wr, mr, vr = onn.adam_step(wr, g.astype(np.float64), mr, vr, t, lr=1e-2)
    wg = w.cpu().double().numpy()
    assert np.all(np.abs(wg - wr) <= 3 * (6e-8 * np.abs(wr) + 1e-5 * 1e-2))


def test_training_checkpoint_resumes_bitwise(gpu_lib, tmp_path):
    """Five training steps equal three steps, a save and restore into a fresh trainer, and two
    more steps, bit for bit (every training kernel sums in a fixed order)."""
    from paper_2603_23343_gb300 import learned
    shape = (32, 32, 32)
    k, b = learned.problem(shape, 7)
    e = torch.from_numpy(inputs.uniform_rhs(shape, 8, 0, np.float64)).cuda()
    r = gpu_lib.stencil_apply(e, k_block=k).float()
    e = e.float()
    w0 = learned.initial_weights(1).cuda()
    full = gpu_lib.NnTrainer(w0, shape, k_block=k)
    for _ in range(5):
        full.step(r, e, lr=1e-3)
    part = gpu_lib.NnTrainer(w0, shape, k_block=k)
    for _ in range(3):
        part.step(r, e, lr=1e-3)
    torch.save(part.state_dict(), tmp_path / "ckpt.pt")
    resumed = gpu_lib.NnTrainer(learned.initial_weights(2).cuda(), shape, k_block=k)
    resumed.load_state_dict(torch.load(tmp_path / "ckpt.pt"))
    for _ in range(2):
        resumed.step(r, e, lr=1e-3)
    torch.testing.assert_close(resumed.w, full.w, rtol=0, atol=0)
    torch.testing.assert_close(resumed.m, full.m, rtol=0, atol=0)
    assert resumed.t == full.t == 5
    with pytest.raises(gpu_lib.GbpcgError):
        gpu_lib.NnTrainer(w0, (32, 32, 64), k_block=None).load_state_dict(part.state_dict())
