"""Failure detection without a GPU fault: a kernel's bounded wait is made to run out.

gm_test_starve_next_pass arms a one-shot fault on the host: the first block of
the next tile-kernel launch skips the load of its first window, so its bounded
mbarrier wait finds nothing arriving and gives up after a short poll limit,
with no copy in flight.  Nothing faults, traps or hangs; the kernel sets its
error flag and returns.  The synchronising calls must then return GM_E_TIMEOUT
and the asynchronous ones must write NaN to every output, and the context must
stay usable: the same calls right after give the normal results bit for bit.
"""
import numpy as np
import pytest

from cases import from_batch, uneven_from
from paper_2404_07780_b300 import synth

pytestmark = pytest.mark.gpu

POLLS = 2000  # a few milliseconds of polling at most


@pytest.fixture(scope="module")
def gm():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2404_07780_b300 import gm as gmod
    from paper_2404_07780_b300.build import build_lib
    build_lib()
    gmod.load()
    return gmod


def _np(x):
    return None if x is None else x.detach().cpu().numpy()


def _starve(gm):
    assert gm.load().gm_test_starve_next_pass(POLLS) == 0


def _timeout(gm, fn):
    import torch
    _starve(gm)
    with pytest.raises(gm.GMError) as e:
        fn()
    torch.cuda.synchronize()
    assert "(-5)" in str(e.value) and "wait limit" in str(e.value), str(e.value)


def test_fit_batch_returns_timeout_and_the_context_survives(gm):
    c = from_batch(synth.draw_small(seed=3, G=8), at="init")
    t = c.torch()
    fit = lambda: gm.gm_fit_batch(c.spec, t["params"], t["image"], t["sigma"], t["mask"], t["psf"])
    ref = {k: _np(v) for k, v in fit().items()}
    _timeout(gm, fit)
    again = {k: _np(v) for k, v in fit().items()}
    for k in ref:
        np.testing.assert_array_equal(again[k], ref[k])


def test_adam_returns_timeout(gm):
    c = from_batch(synth.draw_small(seed=4, G=4), at="init")
    t = c.torch()
    adam = lambda: gm.gm_fit_adam(c.spec, t["params"], t["image"], t["sigma"], t["mask"], t["psf"], n_iter=5)
    ref = _np(adam()["chi2"])
    _timeout(gm, adam)
    np.testing.assert_array_equal(_np(adam()["chi2"]), ref)


def _check_nan_then_normal(gm, call):
    import torch
    ref = [_np(x) for x in call()]
    _starve(gm)
    bad = [_np(x) for x in call()]
    torch.cuda.synchronize()
    for x in bad:
        if x is not None:
            assert np.isnan(x).all()
    for x, y in zip([_np(x) for x in call()], ref):
        if y is not None:
            np.testing.assert_array_equal(x, y)
            assert np.isfinite(y).all()


def test_asynchronous_calls_write_nan_after_a_timeout(gm):
    c = from_batch(synth.draw_sdss(seed=6, G=5, H=64, W=80, K=25), at="init")
    t = c.torch()
    args = (c.spec, t["params"], t["image"], t["sigma"], t["mask"], t["psf"])
    _check_nan_then_normal(gm, lambda: gm.gm_model(c.spec, t["params"], t["psf"], c.H, c.W, components=True))
    _check_nan_then_normal(gm, lambda: gm.gm_chi2_grad(*args, want_grad=True, want_jtj=True))
    _check_nan_then_normal(gm, lambda: gm.gm_chi2_grad_noalloc(*args, want_grad=True, want_jtj=True))
    _check_nan_then_normal(gm, lambda: gm.gm_grad_adjoint(*args))


def test_uneven_batch_timeout(gm):
    rb = synth.draw_uneven_sersic(seed=8, geom=[(40, 56, 15), (64, 64, 41), (9, 7, 1)], mask_frac=0.1)
    c = uneven_from(rb, at="init")
    t = c.torch()
    _check_nan_then_normal(gm, lambda: gm.gm_chi2_grad(c.spec, t["params"], t["image"], t["sigma"], t["mask"],
                                                       t["psf"], want_grad=True, want_jtj=True, geom=rb.geom))
    fit = lambda: gm.gm_fit_batch(c.spec, t["params"], t["image"], t["sigma"], t["mask"], t["psf"], geom=rb.geom)
    _timeout(gm, fit)
    assert (_np(fit()["status"]) > 0).all()


def test_cnn_tma_gemm_wait_runs_out_and_recovers(gm):
    # the learned initialiser's TMA-fed GEMM: gm_cnn_test_starve_next has block 0 of the next
    # launch issue no copy for its first K slice; the MMA thread's bounded wait runs out, every
    # role of the block leaves (copies in flight drained, TMEM freed), the device flag reads 1
    # once (cleared when read), and the next call gives the normal result
    import ctypes
    import torch
    from oracle import cnn as ref
    from paper_2404_07780_b300 import cnn
    L = cnn.lib()
    rng = np.random.default_rng(21)
    bf = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda().to(torch.bfloat16)
    x = bf(rng.normal(size=(4, 16, 16, 64)))
    w = bf(rng.normal(size=(128, 3, 3, 64)) / 24.0)
    b = torch.from_numpy((rng.normal(size=128) * 0.1).astype(np.float32)).cuda()
    assert cnn.fwd_path("conv", 4, 16, 16, 64, 128) == cnn.PATH_TMA
    flag = ctypes.c_int(0)
    assert L.gm_cnn_check_error(ctypes.byref(flag)) == 0  # clear anything left before
    assert L.gm_cnn_test_starve_next(POLLS) == 0
    cnn.conv_fwd(x, w, b, relu=True)
    torch.cuda.synchronize()
    assert L.gm_cnn_check_error(ctypes.byref(flag)) == 0 and flag.value == 1
    assert L.gm_cnn_check_error(ctypes.byref(flag)) == 0 and flag.value == 0
    y = cnn.conv_fwd(x, w, b, relu=True).float().cpu().numpy().astype(np.float64)
    xr, wr, br = (t.float().cpu().numpy().astype(np.float64) for t in (x, w, b))
    want = ref.conv_fwd(xr, wr, br, relu=True)
    scale = np.sqrt(ref.conv_fwd(xr ** 2, wr ** 2) + br ** 2)
    assert np.all(np.abs(y - want) <= 2.0 ** -8 * np.abs(want) + 1e-4 * scale + 1e-30)
    cnn.check_device_error()


def test_cnn_fused_layers_wait_runs_out_and_recovers(gm):
    # the fused first two layers: block 0 of the next launch issues no copy of its first input
    # rows, so the compute warps' wait runs out; the flag reads 1 once and the next call equals
    # the two layers bit for bit
    import ctypes
    import torch
    from paper_2404_07780_b300 import cnn
    L = cnn.lib()
    rng = np.random.default_rng(22)
    bf = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda().to(torch.bfloat16)
    x = bf(rng.normal(size=(5, 64, 64, 1)))
    w1, w2 = bf(rng.normal(size=(32, 3, 3, 1)) / 3.0), bf(rng.normal(size=(64, 3, 3, 32)) / 17.0)
    b1 = torch.from_numpy((rng.normal(size=32) * 0.1).astype(np.float32)).cuda()
    b2 = torch.from_numpy((rng.normal(size=64) * 0.1).astype(np.float32)).cuda()
    flag = ctypes.c_int(0)
    assert L.gm_cnn_check_error(ctypes.byref(flag)) == 0
    assert L.gm_cnn_test_starve_next(POLLS) == 0
    cnn.conv12_fwd(x, w1, b1, w2, b2)
    torch.cuda.synchronize()
    assert L.gm_cnn_check_error(ctypes.byref(flag)) == 0 and flag.value == 1
    assert L.gm_cnn_check_error(ctypes.byref(flag)) == 0 and flag.value == 0
    y = cnn.conv12_fwd(x, w1, b1, w2, b2)
    two = cnn.conv_fwd(cnn.conv_fwd(x, w1, b1, relu=True), w2, b2, relu=True)
    assert torch.equal(y.view(torch.int16), two.view(torch.int16))
    cnn.check_device_error()
