"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every symbol include/gm.h declares, sizes workspaces and rejects bad arguments
before touching the device."""
import ctypes
import os
import re

import pytest

from paper_2404_07780_b300 import gm, synth
from paper_2404_07780_b300.build import build_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build_lib()
    return gm.load()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "gm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gm_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    decl = declared_symbols()
    assert set(decl) == set(gm.EXPORTS), decl
    for name in decl:
        assert hasattr(lib, name), name
    assert lib.gm_version() == 100


def test_struct_layout_matches_header(lib):
    # sizes of the C structs as laid out by the C compiler for include/gm.h
    assert ctypes.sizeof(gm.gm_component) == 40
    assert ctypes.sizeof(gm.gm_model_desc) == 4 + 8 * 40 + 4 + 24 + 24 + 24 * 8 * 2
    assert ctypes.sizeof(gm.gm_batch) == 16 + 4 * 8
    assert ctypes.sizeof(gm.gm_fit_opts) == 9 * 8


def _desc_batch(G=4, H=64, W=64, K=15):
    spec = synth.single_sersic_sky(H, W)
    d = gm.desc_from_spec(spec)
    b = gm.gm_batch(G, H, W, K, None, None, None, None)
    return spec, d, b


def test_workspace_sizes(lib):
    _, d, b = _desc_batch()
    m = lib.gm_model_workspace_bytes(ctypes.byref(d), ctypes.byref(b))
    c = lib.gm_chi2_grad_workspace_bytes(ctypes.byref(d), ctypes.byref(b))
    f = lib.gm_fit_workspace_bytes(ctypes.byref(d), ctypes.byref(b))
    assert 0 < m < c < f
    # the chi2 workspace holds one FP64 partial per tile: 4 galaxies x 4 tiles x (1 + 8 + 36)
    assert c - m >= 4 * 4 * 45 * 8
    b.K = 14  # even PSF side is rejected: size query answers 0
    assert lib.gm_fit_workspace_bytes(ctypes.byref(d), ctypes.byref(b)) == 0


def test_bad_arguments_return_codes(lib):
    _, d, b = _desc_batch()
    fake = ctypes.c_void_p(16)  # never dereferenced: every call below fails validation first
    b.psf = fake
    # NULL descriptor
    assert lib.gm_model(None, ctypes.byref(b), fake, fake, None, fake, 1 << 20, None) == -1
    assert b"desc is NULL" in lib.gm_last_error()
    # even K
    b.K = 14
    assert lib.gm_model(ctypes.byref(d), ctypes.byref(b), fake, fake, None, fake, 1 << 20, None) == -1
    assert b"odd" in lib.gm_last_error()
    b.K = 15
    b.image = b.sigma = b.psf = fake
    # slot out of range
    d2 = gm.desc_from_spec(synth.single_sersic_sky(64, 64))
    d2.comp[0].slot[2] = 99
    assert lib.gm_chi2_grad(ctypes.byref(d2), ctypes.byref(b), fake, fake, None, None, fake, 1 << 20, None) == -1
    # log slot with a non-positive lower bound
    d3 = gm.desc_from_spec(synth.single_sersic_sky(64, 64))
    d3.lo[4] = 0.0
    assert lib.gm_chi2_grad(ctypes.byref(d3), ctypes.byref(b), fake, fake, None, None, fake, 1 << 20, None) == -1
    assert b"log slot" in lib.gm_last_error()
    # missing image for a fit
    b.image = None
    assert lib.gm_fit_batch(ctypes.byref(d), ctypes.byref(b), fake, None, fake, fake, fake, fake, None, fake,
                            1 << 20, None) == -1
    # empty batch is a no-op success
    b.n_gal = 0
    assert lib.gm_model(ctypes.byref(d), ctypes.byref(b), None, None, None, None, 0, None) == 0


def test_many_parameter_models_size_their_workspace(lib):
    # bulge+disk (12 free, 13 correlated channels) and bulge+bar+nucleus (15 free) run in
    # several channel-pair passes; the size queries accept them
    for spec in (synth.bulge_disk_sky(64, 64), synth.bulge_bar_nucleus_sky(64, 64)):
        d = gm.desc_from_spec(spec)
        b = gm.gm_batch(2, 64, 64, 25, None, None, None, None)
        assert lib.gm_chi2_grad_workspace_bytes(ctypes.byref(d), ctypes.byref(b)) > 0
        assert lib.gm_fit_workspace_bytes(ctypes.byref(d), ctypes.byref(b)) > 0


def test_fit_stats_before_any_fit(lib):
    st = gm.gm_fit_stats()
    assert lib.gm_fit_last_stats(ctypes.byref(st)) == -1
