"""Element-by-element parity of every stage of the U-net, forward and
backward, against the FP64 oracle (oracle/nn.py), called through the C ABI.

Each stage is checked on the inputs the GPU itself stored for it (read back
from the workspace with gbpcg_nn_tensor_info), so BF16 rounding differences
of earlier stages cannot compound into later ones: every element of every
stored tensor must be what that stage computes from its own inputs.

For a BF16 tensor the GPU stores bf16(f(y)) where y is an FP32 sum and f a
monotone function (identity, ReLU, a mask).  With the oracle's FP64 value
y64 and the sum's error bound e (2e-5 of the sum of the magnitudes of its
terms for a 27 * ci-term convolution, 1e-6 relative for the short sums of
pooling, upsampling and scaling), the GPU's value must lie in
[bf16(f(y64 - e)), bf16(f(y64 + e))]: rounding is monotone, so that
interval holds every value an FP32 sum within the bound can round to.
Elements that need that allowance (the GPU's value differs from
bf16(f(y64)): the FP32 and FP64 sums straddle a rounding boundary) are
counted and must stay below 0.1 % over the stages.  FP32 tensors
must satisfy |g - y64| <= e at every element.  Weight gradients: per entry
|gw - gw64| <= 2e-5 * wgrad(|x|, |gy|).  Copies (upsampling into the
concatenated inputs) must be bit-exact.

The whole-network output is then compared with the oracle's own BF16-mirrored
forward pass element by element: there an early rounding that lands on the
other side of a boundary propagates, so the check is that 99.9 % of the
elements agree to 1e-2 relative (plus 1e-3 of the largest) and every element
to 5e-2 of the largest.
"""
import numpy as np
import pytest
import torch

import oracle.nn as onn
from paper_2603_23343_gb300 import inputs

pytestmark = pytest.mark.gpu

# (nz, ny, nx): 32^3 takes the per-tap tensor-core kernel at every level; x = 128 and x = 256 rows
# take the halo-slab kernel at the finest level(s)
SHAPES = [(32, 32, 32), (16, 16, 128), (8, 8, 256)]
FLIP_FRACTION = 1e-3


def bf16(a):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).float()
    return t.to(torch.bfloat16).double().numpy()


class Count:
    def __init__(self):
        self.flips = 0
        self.total = 0
        self.per = {}


def check_bf16(name, got, y, err, relu=False, mask=None, cnt=None):
    """got (BF16 values as FP64) against bf16(f(y)) with f = relu / mask, sum error <= err."""
    lo, hi = y - err, y + err
    if relu:
        lo, hi = np.maximum(lo, 0.0), np.maximum(hi, 0.0)
    if mask is not None:
        lo, hi = lo * mask, hi * mask
    blo, bhi = bf16(lo), bf16(hi)
    ok = (got >= blo) & (got <= bhi)
    bad = np.argwhere(~ok)
    assert bad.size == 0, (name, bad[:5].tolist(), got[~ok][:5], y[~ok][:5], err[~ok][:5])
    if cnt is not None:
        # elements that needed the allowance: the GPU's value differs from the FP64 value rounded
        ym = np.maximum(y, 0.0) if relu else y
        if mask is not None:
            ym = ym * mask
        flips = int(np.count_nonzero(got != bf16(ym)))
        cnt.flips += flips
        cnt.total += got.size
        cnt.per[name] = flips / got.size


def check_f32(name, got, y, err):
    bad = np.argwhere(~(np.abs(got - y) <= err))
    assert bad.size == 0, (name, bad[:5].tolist(), got[np.abs(got - y) > err][:5])


def conv_err(x, w):
    return 2e-5 * onn.conv3(np.abs(x), np.abs(w)) + 1e-30


def adj_err(gy, w):
    return 2e-5 * onn.conv3_adjoint(np.abs(gy), np.abs(w)) + 1e-30


def wgrad_check(name, got, x, gy):
    ref = onn.conv3_weight_grad(x, gy)
    bound = 2e-5 * onn.conv3_weight_grad(np.abs(x), np.abs(gy)) + 1e-30
    bad = np.argwhere(~(np.abs(got - ref) <= bound))
    assert bad.size == 0, (name, bad[:5].tolist())


def case(shape, seed):
    r = inputs.uniform_rhs(shape, seed).astype(np.float64)
    nbx, nby, nbz = inputs.block_counts(shape[2], shape[1], shape[0], 8)
    k = inputs.lognormal_blocks(nbx, nby, nbz, seed + 1)
    return r, k


def run_forward(gpu_lib, shape, seed, training):
    r, k = case(shape, seed)
    k64 = k.astype(np.float64)
    ws = onn.init_weights(seed)
    w = gpu_lib.nn_pack_weights(ws).cuda()
    wsb = {name: bf16(v) for name, v in ws.items()}
    rd = torch.from_numpy(r).float().cuda()
    kd = torch.from_numpy(k).float().cuda()
    wsp = gpu_lib.nn_workspace(shape, training=training)
    z = gpu_lib.nn_forward(w, rd, k_block=kd, workspace=wsp).cpu().double().numpy()
    T = {name: gpu_lib.nn_tensor(wsp, shape, name, training).cpu().double().numpy()
         for name in gpu_lib.NN_TENSORS[:14]}
    return r.astype(np.float32).astype(np.float64), k64, kd, wsb, w, wsp, z, T


@pytest.mark.parametrize("shape", SHAPES)
def test_unet_forward_stages_elementwise(gpu_lib, shape):
    r, k64, _, W, _, _, z, T = run_forward(gpu_lib, shape, 31, False)
    cnt = Count()
    # input: s = D^{-1/2} r, channels (s / rms(s), log k); FP32 products and one FP32 division
    dsc = onn.jacobi_scale(shape, k64, 8)
    check_f32("dsc", T["dsc"][..., 0], dsc, 2e-6 * dsc)
    check_f32("sr", T["sr"][..., 0], r * dsc, 3e-6 * np.abs(r * dsc))
    s = T["sr"][..., 0]
    rms = float(np.sqrt(np.mean(s * s)))
    assert abs(float(T["scale"]) - rms) <= 1e-6 * rms
    check_bf16("xin[s]", T["xin"][..., 0], s / rms, 1e-6 * np.abs(s / rms), cnt=cnt)
    lk = onn.logk_field(shape, k64, 8)
    check_bf16("xin[log k]", T["xin"][..., 1], lk, 1e-6 * np.abs(lk) + 1e-7, cnt=cnt)
    # level 0 and 1 encoders
    x = T["xin"]
    check_bf16("a1", T["a1"], onn.conv3(x, W["c1"]), conv_err(x, W["c1"]), relu=True, cnt=cnt)
    e0 = T["k8"][..., 32:48]
    check_bf16("e0", e0, onn.conv3(T["a1"], W["c2"]), conv_err(T["a1"], W["c2"]), relu=True, cnt=cnt)
    check_bf16("p1", T["p1"], onn.pool2(e0), 1e-6 * onn.pool2(np.abs(e0)), cnt=cnt)
    check_bf16("a3", T["a3"], onn.conv3(T["p1"], W["c3"]), conv_err(T["p1"], W["c3"]), relu=True, cnt=cnt)
    e1 = T["k7"][..., 64:96]
    check_bf16("e1", e1, onn.conv3(T["a3"], W["c4"]), conv_err(T["a3"], W["c4"]), relu=True, cnt=cnt)
    check_bf16("p2", T["p2"], onn.pool2(e1), 1e-6 * onn.pool2(np.abs(e1)), cnt=cnt)
    check_bf16("a5", T["a5"], onn.conv3(T["p2"], W["c5"]), conv_err(T["p2"], W["c5"]), relu=True, cnt=cnt)
    check_bf16("a6", T["a6"], onn.conv3(T["a5"], W["c6"]), conv_err(T["a5"], W["c6"]), relu=True, cnt=cnt)
    # decoders: upsampling copies are exact, the concatenated inputs are the stored tensors
    np.testing.assert_array_equal(T["k7"][..., 0:64], onn.up2(T["a6"]))
    check_bf16("a7", T["a7"], onn.conv3(T["k7"], W["c7"]), conv_err(T["k7"], W["c7"]), relu=True, cnt=cnt)
    np.testing.assert_array_equal(T["k8"][..., 0:32], onn.up2(T["a7"]))
    check_bf16("a8", T["a8"], onn.conv3(T["k8"], W["c8"]), conv_err(T["k8"], W["c8"]), relu=True, cnt=cnt)
    # output: FP32 c9 times rms(s) D^{-1/2}
    u = onn.conv3(T["a8"], W["c9"])[..., 0]
    sc = float(T["scale"]) * T["dsc"][..., 0]
    check_f32("z", z, u * sc, conv_err(T["a8"], W["c9"])[..., 0] * sc + 2e-6 * np.abs(u * sc))
    print({k: round(v, 6) for k, v in cnt.per.items()})
    assert cnt.flips <= FLIP_FRACTION * cnt.total, (cnt.flips, cnt.total, cnt.per)


@pytest.mark.parametrize("shape", SHAPES)
def test_unet_backward_stages_elementwise(gpu_lib, shape):
    r, k64, kd, W, w, wsp, z, T = run_forward(gpu_lib, shape, 37, True)
    gz = inputs.uniform_rhs(shape, 38).astype(np.float32)
    gw = gpu_lib.nn_backward(torch.from_numpy(gz).cuda(), wsp, k_block=kd).cpu().double().numpy()
    assert gpu_lib.nn_status(wsp) == gpu_lib.OK
    G = {name: gpu_lib.nn_tensor(wsp, shape, name, True).cpu().double().numpy()
         for name in gpu_lib.NN_TENSORS[14:]}
    gg = {name: v.numpy() for name, v in gpu_lib.nn_unpack_weights(torch.from_numpy(gw)).items()}
    cnt = Count()
    sc = float(T["scale"]) * T["dsc"][..., 0]
    gzs = gz.astype(np.float64) * sc
    check_bf16("gout", G["gout"][..., 0], gzs, 2e-6 * np.abs(gzs), cnt=cnt)
    m = lambda a: (a > 0).astype(np.float64)  # noqa: E731  ReLU masks from the stored activations
    # c9
    wgrad_check("gw c9", gg["c9"], T["a8"], G["gout"])
    check_bf16("ga8", G["ga8"], onn.conv3_adjoint(G["gout"], W["c9"]), adj_err(G["gout"], W["c9"]),
               mask=m(T["a8"]), cnt=cnt)
    # c8 on k8 = [up(a7), e0]
    wgrad_check("gw c8", gg["c8"], T["k8"], G["ga8"])
    check_f32("gk8", G["gk8"], onn.conv3_adjoint(G["ga8"], W["c8"]), adj_err(G["ga8"], W["c8"]))
    g7 = onn.up2_adjoint(G["gk8"][..., 0:32])
    check_bf16("ga7", G["ga7"], g7, 1e-6 * onn.up2_adjoint(np.abs(G["gk8"][..., 0:32])), mask=m(T["a7"]), cnt=cnt)
    # c7 on k7 = [up(a6), e1]
    wgrad_check("gw c7", gg["c7"], T["k7"], G["ga7"])
    check_f32("gk7", G["gk7"], onn.conv3_adjoint(G["ga7"], W["c7"]), adj_err(G["ga7"], W["c7"]))
    g6 = onn.up2_adjoint(G["gk7"][..., 0:64])
    check_bf16("ga6", G["ga6"], g6, 1e-6 * onn.up2_adjoint(np.abs(G["gk7"][..., 0:64])), mask=m(T["a6"]), cnt=cnt)
    # c6, c5
    wgrad_check("gw c6", gg["c6"], T["a5"], G["ga6"])
    check_bf16("ga5", G["ga5"], onn.conv3_adjoint(G["ga6"], W["c6"]), adj_err(G["ga6"], W["c6"]),
               mask=m(T["a5"]), cnt=cnt)
    wgrad_check("gw c5", gg["c5"], T["p2"], G["ga5"])
    check_f32("t5", G["t5"], onn.conv3_adjoint(G["ga5"], W["c5"]), adj_err(G["ga5"], W["c5"]))
    # e1: skip gradient + pooled-path gradient, masked by e1 > 0
    e1 = T["k7"][..., 64:96]
    skip1 = G["gk7"][..., 64:96]
    g_e1 = skip1 + onn.pool2_adjoint(G["t5"])
    check_bf16("ge1b", G["ge1b"], g_e1, 1e-6 * (np.abs(skip1) + onn.pool2_adjoint(np.abs(G["t5"]))), mask=m(e1),
               cnt=cnt)
    # c4, c3
    wgrad_check("gw c4", gg["c4"], T["a3"], G["ge1b"])
    check_bf16("ga3", G["ga3"], onn.conv3_adjoint(G["ge1b"], W["c4"]), adj_err(G["ge1b"], W["c4"]),
               mask=m(T["a3"]), cnt=cnt)
    wgrad_check("gw c3", gg["c3"], T["p1"], G["ga3"])
    check_f32("t3", G["t3"], onn.conv3_adjoint(G["ga3"], W["c3"]), adj_err(G["ga3"], W["c3"]))
    # e0: skip gradient + pooled-path gradient, masked by e0 > 0
    e0 = T["k8"][..., 32:48]
    skip0 = G["gk8"][..., 32:48]
    g_e0 = skip0 + onn.pool2_adjoint(G["t3"])
    check_bf16("ge0b", G["ge0b"], g_e0, 1e-6 * (np.abs(skip0) + onn.pool2_adjoint(np.abs(G["t3"]))), mask=m(e0),
               cnt=cnt)
    # c2, c1
    wgrad_check("gw c2", gg["c2"], T["a1"], G["ge0b"])
    check_bf16("ga1", G["ga1"], onn.conv3_adjoint(G["ge0b"], W["c2"]), adj_err(G["ge0b"], W["c2"]),
               mask=m(T["a1"]), cnt=cnt)
    wgrad_check("gw c1", gg["c1"], T["xin"], G["ga1"])
    print({k: round(v, 6) for k, v in cnt.per.items()})
    assert cnt.flips <= FLIP_FRACTION * cnt.total, (cnt.flips, cnt.total, cnt.per)


@pytest.mark.parametrize("shape", SHAPES)
def test_unet_output_elementwise_against_oracle_forward(gpu_lib, shape):
    """The GPU's output against the oracle's whole BF16-mirrored forward pass (not fed the GPU's
    intermediates): element by element, with the allowance for propagated rounding flips."""
    r, k64, _, W, _, _, z, _ = run_forward(gpu_lib, shape, 41, False)
    x, scale = onn.net_input(r, onn.logk_field(shape, k64, 8), onn.jacobi_scale(shape, k64, 8))
    out, _ = onn.net_forward(bf16(x), W, round_fn=bf16)
    zr = out[..., 0] * scale
    top = float(np.max(np.abs(zr)))
    close = np.abs(z - zr) <= 1e-2 * np.abs(zr) + 1e-3 * top
    assert np.count_nonzero(~close) <= FLIP_FRACTION * z.size, np.count_nonzero(~close)
    assert np.all(np.abs(z - zr) <= 5e-2 * top), float(np.max(np.abs(z - zr)) / top)
