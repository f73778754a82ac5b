"""gm_chi2_grad_noalloc: the chi^2 entry point for callers that cannot allocate.

Some callers of this library may not call cudaMalloc (or torch's allocator)
when they need chi^2 and its derivatives -- an optimiser plugged into a host
framework that owns all device memory, or a pipeline stage that forbids
allocation after start-up.  gm_chi2_grad_noalloc serves them from a fixed
scratch array inside the library.  These tests call it through the C ABI and
check it against gm_chi2_grad with a caller workspace, bit for bit, on calls in
a row (different batches, equal and uneven stamps, so stale scratch from an
earlier call would show), and that
a batch too large for the fixed array is refused with a clear error.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes
import numpy as np
import pytest

from cases import from_batch, uneven_from
from paper_2404_07780_b300 import gm, synth
from paper_2404_07780_b300.build import build_lib

GM_E_NOMEM = -3


def _lib():
    build_lib()
    lib = gm.load()
    P = ctypes.c_void_p
    lib.gm_chi2_grad_noalloc.restype = ctypes.c_int
    lib.gm_chi2_grad_noalloc.argtypes = [P, P, P, P, P, P, P]
    return lib


def _noalloc(lib, case, geom=None):
    """chi^2, grad and J^T W J from gm_chi2_grad_noalloc; outputs allocated by the test, not the library."""
    import torch
    t = case.torch()
    d = gm.desc_from_spec(case.spec)
    b, keep = gm.make_batch(t["image"], t["sigma"], t["mask"], t["psf"], geom)
    G, S = case.G, case.spec.n_slots
    # outputs poisoned with NaN: every element must be written by the call
    chi2 = torch.full((G,), float("nan"), dtype=torch.float64, device="cuda")
    grad = torch.full((G, S), float("nan"), dtype=torch.float64, device="cuda")
    jtj = torch.full((G, S, S), float("nan"), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.gm_chi2_grad_noalloc(ctypes.byref(d), ctypes.byref(b), ctypes.c_void_p(t["params"].data_ptr()),
                                  ctypes.c_void_p(chi2.data_ptr()), ctypes.c_void_p(grad.data_ptr()),
                                  ctypes.c_void_p(jtj.data_ptr()), stream)
    assert rc == 0, lib.gm_last_error()
    torch.cuda.synchronize()
    return chi2.cpu().numpy(), grad.cpu().numpy(), jtj.cpu().numpy()


def _reference(case, geom=None):
    t = case.torch()
    chi2, grad, jtj = gm.gm_chi2_grad(case.spec, t["params"], t["image"], t["sigma"], t["mask"], t["psf"],
                                      want_grad=True, want_jtj=True, geom=geom)
    return chi2.cpu().numpy(), grad.cpu().numpy(), jtj.cpu().numpy()


def _assert_same(got, ref):
    """Bit for bit: both calls run the same kernels on the same inputs in the same launch
    shape, and every sum over tiles is taken in a fixed order, so only the scratch address
    differs.  Stale scratch from an earlier call cannot hide under a tolerance."""
    for x, y in zip(got, ref):
        np.testing.assert_array_equal(x, y)
        assert np.isfinite(x).all()


@pytest.mark.gpu
def test_noalloc_matches_workspace_entry_point_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    lib = _lib()
    first = from_batch(synth.draw_sdss(seed=11, G=6, H=96, W=80, K=41), at="init")
    second = from_batch(synth.draw_small(seed=12, G=16), at="truth")
    # an uneven batch (mixed stamp and PSF sides, masked): its per-class tensor maps and
    # item tables go into the shared array as well, at offsets that depend on the batch
    rb = synth.draw_uneven_sersic(seed=13, geom=[(40, 56, 15), (64, 64, 41), (9, 7, 1), (96, 33, 25)],
                                  mask_frac=0.1)
    third = uneven_from(rb, at="init")
    for case, geom in ((first, None), (second, None), (third, rb.geom)):  # calls in a row on different batches
        _assert_same(_noalloc(lib, case, geom), _reference(case, geom))
    # the first batch again after the others: nothing stale survives in the shared array
    _assert_same(_noalloc(lib, first), _reference(first))
    _assert_same(_noalloc(lib, third, rb.geom), _reference(third, rb.geom))


def test_noalloc_rejects_batches_beyond_its_array():
    # 4,096 stamps of 128x128 need ~24 MB of per-tile partials: more than the fixed 16 MiB.
    # The size check comes before any device work, so the dummy pointers are never used.
    lib = _lib()
    spec = synth.single_sersic_sky(128, 128)
    d = gm.desc_from_spec(spec)
    fake = ctypes.c_void_p(16)
    b = gm.gm_batch(4096, 128, 128, 41, fake, fake, None, fake)
    assert lib.gm_chi2_grad_workspace_bytes(ctypes.byref(d), ctypes.byref(b)) > 16 * 1024 * 1024
    rc = lib.gm_chi2_grad_noalloc(ctypes.byref(d), ctypes.byref(b), fake, fake, None, None, None)
    assert rc == GM_E_NOMEM
    msg = lib.gm_last_error().decode()
    assert "built-in array" in msg and "gm_chi2_grad" in msg
