"""The learned initialiser's tensor-core layers (include/gm_cnn.h) against the
FP64 CNN reference (oracle/cnn.py) on the same BF16-rounded inputs.

Tolerances: FP32 outputs (weight gradients, the last dense layer) carry only
FP32 accumulation error: |d| <= 1e-4 * sqrt(sum of squared terms) per
element.  BF16 outputs add one BF16 rounding of the result (relative 2^-8):
|d| <= 2^-8 |ref| + 1e-4 * sqrt(sum of squared terms)."""
import numpy as np
import pytest

from oracle import cnn as ref

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2404_07780_b300 import cnn
    from paper_2404_07780_b300.build import build_lib
    build_lib()
    cnn.lib()
    return cnn


def _bf(a, seed=None):
    """A BF16 CUDA tensor and the float64 values it holds."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a, np.float32)).to("cuda").to(torch.bfloat16).contiguous()
    return t, t.float().cpu().numpy().astype(np.float64)


def _f32(a):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a, np.float32)).to("cuda")
    return t, t.cpu().numpy().astype(np.float64)


def _close(got, want, scale, bf16_out):
    got = np.asarray(got, np.float64)
    tol = 1e-4 * scale + (2.0 ** -8 * np.abs(want) if bf16_out else 0.0) + 1e-30
    bad = np.abs(got - want) > tol
    assert not bad.any(), (int(bad.sum()), float(np.abs(got - want)[bad].max()), got[bad][:4], want[bad][:4])


def _np(t):
    return t.float().cpu().numpy().astype(np.float64)


# (n, h, w, ci, co): the four layers of the network, a ragged spatial size, and a batch
# large enough for many M tiles
CONVS = [(4, 64, 64, 1, 32), (4, 32, 32, 32, 64), (4, 16, 16, 64, 128), (4, 8, 8, 128, 128), (3, 13, 9, 8, 16),
         (64, 16, 16, 64, 128)]
# the tensor-map path's own cases: a last tile with images past the batch (37 and 5 images of
# 16 and 64 output pixels), every stage/tile shape (64-byte rows with 64 and 128 outputs, 128-byte
# rows with 64), and tiles that wrap the ring of stages many times
TMA_CONVS = [(37, 8, 8, 128, 128), (5, 16, 16, 64, 128), (3, 32, 32, 32, 64), (2, 16, 16, 32, 128),
             (2, 32, 32, 64, 64), (300, 16, 16, 64, 128)]


@pytest.mark.parametrize("shape", CONVS + TMA_CONVS)
def test_conv_forward(C, shape):
    n, h, w, ci, co = shape
    rng = np.random.default_rng(1)
    x, xr = _bf(rng.normal(size=(n, h, w, ci)))
    W, Wr = _bf(rng.normal(size=(co, 3, 3, ci)) / np.sqrt(9 * ci))
    b, br = _f32(rng.normal(size=co) * 0.1)
    for relu in (False, True):
        y = _np(C.conv_fwd(x, W, b, relu=relu))
        want = ref.conv_fwd(xr, Wr, br, relu=relu)
        scale = np.sqrt(ref.conv_fwd(xr ** 2, Wr ** 2) + br ** 2)
        _close(y, want, scale, True)
    C.check_device_error()


@pytest.mark.parametrize("shape", [s for s in CONVS if s[3] % 8 == 0])
def test_conv_backward_data(C, shape):
    n, h, w, ci, co = shape
    rng = np.random.default_rng(2)
    ho, wo = (h + 1) // 2, (w + 1) // 2
    dy, dyr = _bf(rng.normal(size=(n, ho, wo, co)))
    W, Wr = _bf(rng.normal(size=(co, 3, 3, ci)) / np.sqrt(9 * ci))
    mask, maskr = _bf(np.maximum(rng.normal(size=(n, h, w, ci)), 0.0))
    for m, mr in ((None, None), (mask, maskr)):
        dx = _np(C.conv_bwd_data(dy, W, h, w, mask=m))
        want = ref.conv_bwd_data(dyr, Wr, h, w, mask=mr)
        scale = np.sqrt(ref.conv_bwd_data(dyr ** 2, Wr ** 2, h, w))
        _close(dx, want, scale, True)
    C.check_device_error()


@pytest.mark.parametrize("shape", CONVS)
def test_conv_backward_weight(C, shape):
    n, h, w, ci, co = shape
    rng = np.random.default_rng(3)
    ho, wo = (h + 1) // 2, (w + 1) // 2
    x, xr = _bf(rng.normal(size=(n, h, w, ci)))
    dy, dyr = _bf(rng.normal(size=(n, ho, wo, co)))
    dw, db = C.conv_bwd_weight(x, dy)
    want_w, want_b = ref.conv_bwd_weight(xr, dyr)
    sw, sb = ref.conv_bwd_weight(xr ** 2, dyr ** 2)
    _close(_np(dw), want_w, np.sqrt(sw), False)
    _close(_np(db), want_b, np.sqrt(sb), False)
    C.check_device_error()


@pytest.mark.parametrize("n,fin,fout", [(64, 2048, 256), (300, 256, 16), (8, 64, 32), (1000, 128, 264)])
def test_dense_forward_and_backward(C, n, fin, fout):
    rng = np.random.default_rng(4)
    x, xr = _bf(rng.normal(size=(n, fin)))
    W, Wr = _bf(rng.normal(size=(fout, fin)) / np.sqrt(fin))
    b, br = _f32(rng.normal(size=fout) * 0.1)
    scale = np.sqrt((xr ** 2) @ (Wr ** 2).T + br ** 2)
    _close(_np(C.dense_fwd(x, W, b, relu=True)), ref.dense_fwd(xr, Wr, br, relu=True), scale, True)
    _close(_np(C.dense_fwd(x, W, b, relu=False, fp32_out=True)), ref.dense_fwd(xr, Wr, br), scale, False)
    dy, dyr = _bf(rng.normal(size=(n, fout)))
    mask, maskr = _bf(np.maximum(rng.normal(size=(n, fin)), 0.0))
    _close(_np(C.dense_bwd_data(dy, W, mask=mask)), ref.dense_bwd_data(dyr, Wr, mask=maskr),
           np.sqrt((dyr ** 2) @ (Wr ** 2)), True)
    dw, db = C.dense_bwd_weight(x, dy)
    ww, wb = ref.dense_bwd_weight(xr, dyr)
    _close(_np(dw), ww, np.sqrt((dyr ** 2).T @ (xr ** 2)), False)
    _close(_np(db), wb, np.sqrt((dyr ** 2).sum(0)), False)
    C.check_device_error()


@pytest.mark.parametrize("n,fin,fout", [(300, 2048, 256), (129, 64, 64), (1000, 200, 128), (4096, 2048, 256)])
def test_dense_forward_tma_path(C, n, fin, fout):
    # BF16 output on the tensor-map path against the oracle, and bit for bit against the
    # gathered GEMM's FP32 output rounded to BF16: both sum the same K = 16 MMA steps in the
    # same order, so only the final rounding differs, and it is the same rounding
    import torch
    assert C.fwd_path("dense", n, 0, 0, fin, fout) == C.PATH_TMA
    assert C.fwd_path("dense", n, 0, 0, fin, fout, fp32_out=True) == C.PATH_GATHER
    rng = np.random.default_rng(6)
    x, xr = _bf(rng.normal(size=(n, fin)))
    W, Wr = _bf(rng.normal(size=(fout, fin)) / np.sqrt(fin))
    b, br = _f32(rng.normal(size=fout) * 0.1)
    scale = np.sqrt((xr ** 2) @ (Wr ** 2).T + br ** 2)
    for relu in (False, True):
        y = C.dense_fwd(x, W, b, relu=relu)
        _close(_np(y), ref.dense_fwd(xr, Wr, br, relu=relu), scale, True)
        y32 = C.dense_fwd(x, W, b, relu=relu, fp32_out=True)
        assert torch.equal(y.view(torch.int16), y32.to(torch.bfloat16).view(torch.int16))
    C.check_device_error()


@pytest.mark.parametrize("n", [1, 3, 300])
def test_fused_first_two_convolutions(C, n):
    # the fused kernel equals the two layers it replaces bit for bit (the same single K = 16
    # MMA per row for the first, the same 18 K steps for the second), and the oracle within
    # the BF16 bounds; 300 images are 600 tiles, several per block on both accumulators
    import torch
    rng = np.random.default_rng(7)
    x, xr = _bf(rng.normal(size=(n, 64, 64, 1)))
    w1, w1r = _bf(rng.normal(size=(32, 3, 3, 1)) / 3.0)
    b1, b1r = _f32(rng.normal(size=32) * 0.1)
    w2, w2r = _bf(rng.normal(size=(64, 3, 3, 32)) / np.sqrt(9 * 32))
    b2, b2r = _f32(rng.normal(size=64) * 0.1)
    y = C.conv12_fwd(x, w1, b1, w2, b2)
    two = C.conv_fwd(C.conv_fwd(x, w1, b1, relu=True), w2, b2, relu=True)
    assert torch.equal(y.view(torch.int16), two.view(torch.int16))
    a1 = _np(C.conv_fwd(x, w1, b1, relu=True))  # the BF16 first layer both paths feed the second
    want = ref.conv_fwd(a1, w2r, b2r, relu=True)
    scale = np.sqrt(ref.conv_fwd(a1 ** 2, w2r ** 2) + b2r ** 2)
    _close(_np(y), want, scale, True)
    C.check_device_error()


def test_predict_equals_forward(C):
    # inference (fused first layers, batches of any size) against the training forward pass
    import torch
    net = C.Net(seed=3, device="cuda")
    rng = np.random.default_rng(8)
    x, _ = _bf(np.arcsinh(rng.normal(size=(700, 64, 64, 1)) * 3.0))
    assert torch.equal(net.predict(x, batch=256), net.forward(x)[1])
    C.check_device_error()


def test_conv_forward_paths_of_the_network(C):
    # the layers of the network on a training batch, each on the path the sizes select
    assert [C.fwd_path("conv", 512, h, h, i, o) for h, i, o in ((64, 1, 32), (32, 32, 64), (16, 64, 128),
                                                                 (8, 128, 128))] == [C.PATH_GATHER] + [C.PATH_TMA] * 3


def test_prep_vector_path_matches_the_scalar_one(C):
    # 128-pixel rows take the four-outputs-per-thread kernel; an image that starts 4 bytes past
    # a 16-byte boundary takes the one-output kernel: both give the same BF16 bits (same sums in
    # the same order), and the oracle within one BF16 rounding
    import torch
    rng = np.random.default_rng(9)
    G, H, W = 37, 128, 128
    a = rng.normal(size=(G, H, W)).astype(np.float32) * 20.0
    img = torch.from_numpy(a).cuda()
    buf = torch.empty(G * H * W + 1, dtype=torch.float32, device="cuda")
    off = buf[1:].view(G, H, W)
    off.copy_(img)
    fast, slow = C.prep(img, 0.5), C.prep(off, 0.5)
    assert torch.equal(fast.view(torch.int16), slow.view(torch.int16))
    want = ref.prep(a.astype(np.float64), 0.5)
    got = _np(fast)[..., 0]
    assert np.all(np.abs(got - want) <= 2.0 ** -8 * np.abs(want) + 1e-6)


def test_prep_loss_and_adam(C):
    import torch
    rng = np.random.default_rng(5)
    img, imgr = _f32(rng.normal(size=(5, 12, 10)) * 30.0)
    got = _np(C.prep(img, 0.5))[..., 0]
    want = ref.prep(imgr, 0.5)
    assert np.all(np.abs(got - want) <= 2.0 ** -8 * np.abs(want) + 1e-6)

    pred, predr = _f32(rng.normal(size=(37, 16)))
    tgt, tgtr = _f32(rng.normal(size=(37, 14)))
    loss, dpred = C.mse(pred, tgt, 14)
    wl, wd = ref.mse(predr, tgtr, 14)
    assert abs(loss.item() - wl) <= 1e-5 * wl
    assert np.all(np.abs(_np(dpred) - wd) <= 2.0 ** -8 * np.abs(wd) + 1e-12)

    p, pr = _f32(rng.normal(size=1000))
    g, gr = _f32(rng.normal(size=1000))
    m = torch.zeros(1000, device="cuda")
    v = torch.zeros(1000, device="cuda")
    pb = torch.empty(1000, dtype=torch.bfloat16, device="cuda")
    mr, vr = np.zeros(1000), np.zeros(1000)
    for step in (1, 2, 3):
        C.adam(p, g, m, v, pb, 1e-3, step)
        pr, mr, vr = ref.adam(pr, gr, mr, vr, 1e-3, 0.9, 0.999, 1e-8, step)
    np.testing.assert_allclose(p.cpu().numpy(), pr, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(_np(pb), pr, rtol=2.0 ** -8, atol=1e-6)
