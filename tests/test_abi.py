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


def declared_symbols(header="gm.h"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gm_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    from paper_2404_07780_b300 import cnn
    headers = sorted(f for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h"))
    assert headers == ["gm.h", "gm_cnn.h"], headers
    for header, bound in (("gm.h", gm.EXPORTS), ("gm_cnn.h", cnn.EXPORTS)):
        decl = declared_symbols(header)
        assert set(decl) == set(bound), (header, decl)
        for name in decl:
            assert hasattr(lib, name), name
    assert lib.gm_version() == 100


_LAYOUT_PROBE = r"""
#include <stddef.h>
#include <stdio.h>
#include "gm.h"
#define F(T, f) printf(#T "." #f " %zu\n", offsetof(T, f))
int main(void) {
  printf("gm_component %zu\n", sizeof(gm_component));
  printf("gm_model_desc %zu\n", sizeof(gm_model_desc));
  printf("gm_batch %zu\n", sizeof(gm_batch));
  printf("gm_fit_opts %zu\n", sizeof(gm_fit_opts));
  printf("gm_fit_stats %zu\n", sizeof(gm_fit_stats));
  F(gm_model_desc, lo); F(gm_model_desc, hi); F(gm_model_desc, amp_is_mag); F(gm_model_desc, mag_zero);
  F(gm_model_desc, has_box);
  F(gm_batch, image); F(gm_batch, psf); F(gm_batch, geom);
  F(gm_fit_opts, max_iter); F(gm_fit_opts, lambda0); F(gm_fit_stats, profile_ms);
  return 0;
}
"""


def test_struct_layout_matches_header(lib, tmp_path):
    # sizes and offsets of the C structs as the C compiler lays out include/gm.h, against the binding's ctypes
    import subprocess
    src = tmp_path / "probe.c"
    src.write_text(_LAYOUT_PROBE)
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                      text=True).stdout.splitlines())
    for name in ("gm_component", "gm_model_desc", "gm_batch", "gm_fit_opts", "gm_fit_stats"):
        assert int(out[name]) == ctypes.sizeof(getattr(gm, name)), name
    for key, v in out.items():
        if "." in key:
            struct, field = key.split(".")
            assert int(v) == getattr(getattr(gm, struct), field).offset, key


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


def test_empty_batch_is_a_no_op_for_every_entry(lib):
    # n_gal = 0: every compute entry point validates its arguments and returns success
    # without a device call (this runs where no GPU is present), and every size query
    # answers a small positive workspace
    _, d, b = _desc_batch(G=0)
    fake = ctypes.c_void_p(16)  # device pointers: never dereferenced on the host
    b.psf = b.image = b.sigma = fake
    R = ctypes.byref
    opts = gm.FitOptions().to_c()
    adam = gm.gm_adam_opts(10, 0.01, 0.9, 0.999, 1e-8)
    ws = 1 << 20
    assert lib.gm_model(R(d), R(b), fake, fake, None, None, 0, None) == 0
    assert lib.gm_chi2_grad(R(d), R(b), fake, fake, fake, None, fake, ws, None) == 0
    assert lib.gm_chi2_grad_noalloc(R(d), R(b), fake, fake, fake, None, None) == 0
    assert lib.gm_fit_batch(R(d), R(b), fake, R(opts), fake, fake, fake, fake, None, fake, ws, None) == 0
    assert lib.gm_grad_adjoint(R(d), R(b), fake, fake, fake, fake, ws, None) == 0
    assert lib.gm_fit_adam(R(d), R(b), fake, R(adam), fake, fake, ws, None) == 0
    assert lib.gm_bootstrap_counts(R(d), R(b), 1, 0, fake, fake, ws, None) == 0
    assert lib.gm_bootstrap(R(d), R(b), fake, 4, 1, fake, fake, fake, fake, ws, None) == 0
    for name in ("gm_model_workspace_bytes", "gm_chi2_grad_workspace_bytes", "gm_fit_workspace_bytes",
                 "gm_grad_adjoint_workspace_bytes", "gm_fit_adam_workspace_bytes", "gm_bootstrap_workspace_bytes"):
        assert 0 < getattr(lib, name)(R(d), R(b)) <= 1 << 16, name


def test_adjoint_adam_bootstrap_reject_bad_arguments_on_the_host(lib):
    # each refusal comes from host-side validation, with the documented code and message,
    # before any device call (this runs where no GPU is present)
    R = ctypes.byref
    fake = ctypes.c_void_p(16)
    spec, d, b = _desc_batch(K=14)
    b.psf = b.image = b.sigma = fake
    assert lib.gm_grad_adjoint(R(d), R(b), fake, fake, fake, fake, 1 << 20, None) == -1
    assert b"must be odd" in lib.gm_last_error()
    b.K = 15
    need = lib.gm_grad_adjoint_workspace_bytes(R(d), R(b))
    assert need > 0
    assert lib.gm_grad_adjoint(R(d), R(b), fake, fake, fake, fake, need - 1, None) == -3
    assert lib.gm_grad_adjoint(R(d), R(b), fake, fake, fake, None, need, None) == -3
    for bad in ((0, 0.01, 0.9, 0.999, 1e-8), (10, 0.0, 0.9, 0.999, 1e-8), (10, 0.01, 1.0, 0.999, 1e-8),
                (10, 0.01, 0.9, -0.1, 1e-8), (10, 0.01, 0.9, 0.999, 0.0)):
        assert lib.gm_fit_adam(R(d), R(b), fake, R(gm.gm_adam_opts(*bad)), fake, fake, 1 << 30, None) == -1, bad
        assert b"Adam options" in lib.gm_last_error()
    assert lib.gm_fit_adam(R(d), R(b), fake, None, fake, fake, 1 << 30, None) == -1
    adam = gm.gm_adam_opts(10, 0.01, 0.9, 0.999, 1e-8)
    na = lib.gm_fit_adam_workspace_bytes(R(d), R(b))
    assert lib.gm_fit_adam(R(d), R(b), fake, R(adam), fake, fake, na - 1, None) == -3
    nb = lib.gm_bootstrap_workspace_bytes(R(d), R(b))
    assert lib.gm_bootstrap(R(d), R(b), fake, 0, 1, fake, fake, fake, fake, nb, None) == -1
    assert lib.gm_bootstrap(R(d), R(b), fake, 4, 1, fake, fake, fake, fake, nb - 1, None) == -3
    assert lib.gm_bootstrap_counts(R(d), R(b), 1, 0, fake, fake, nb - 1, None) == -3
    assert lib.gm_bootstrap_counts(R(d), R(b), 1, -1, fake, fake, nb, None) == -1
    # equal stamps only: the size queries of the Adam fit and the bootstrap answer 0 for an uneven batch
    b.geom = fake
    assert lib.gm_fit_adam_workspace_bytes(R(d), R(b)) == 0
    assert lib.gm_bootstrap_workspace_bytes(R(d), R(b)) == 0


def test_cnn_entry_points_reject_bad_arguments_on_the_host(lib):
    # the initialiser's layers: channel and feature counts off the multiple of 8, NULL
    # pointers, short workspaces, odd input sides and bad optimiser steps are refused before
    # any device call; an empty batch is a no-op
    from paper_2404_07780_b300 import cnn
    L = cnn.lib()
    f = ctypes.c_void_p(256)  # never dereferenced
    assert L.gm_cnn_conv_fwd(f, f, None, f, 2, 32, 32, 12, 16, 1, None) == -1
    assert b"conv_fwd" in L.gm_cnn_last_error()
    assert L.gm_cnn_conv_fwd(f, f, None, f, 2, 32, 32, 8, 12, 1, None) == -1
    assert L.gm_cnn_conv_fwd(None, f, None, f, 2, 32, 32, 8, 16, 1, None) == -1
    assert L.gm_cnn_conv_fwd(f, f, None, f, 0, 32, 32, 8, 16, 1, None) == 0
    assert L.gm_cnn_conv_bwd_data(f, f, None, f, 2, 32, 32, 1, 16, None) == -1
    ws = L.gm_cnn_conv_bwd_weight_workspace(2, 32, 32, 8, 16)
    assert ws > 0
    assert L.gm_cnn_conv_bwd_weight(f, f, f, None, 2, 32, 32, 8, 16, f, ws - 1, None) == -3
    assert L.gm_cnn_dense_fwd(f, f, None, f, None, 4, 12, 16, 1, None) == -1
    assert L.gm_cnn_dense_fwd(f, f, None, None, None, 4, 16, 16, 1, None) == -1  # no output
    wd = L.gm_cnn_dense_bwd_weight_workspace(4, 16, 16)
    assert wd > 0
    assert L.gm_cnn_dense_bwd_weight(f, f, f, None, 4, 16, 16, f, wd - 1, None) == -3
    assert L.gm_cnn_prep(f, 2, 33, 32, 1.0, f, None) == -1
    assert L.gm_cnn_mse(f, f, 4, 8, 9, f, f, None) == -1
    assert L.gm_cnn_adam(f, f, f, f, None, 10, 0.01, 0.9, 0.999, 1e-8, 0, None) == -1
    assert L.gm_cnn_adam(f, f, f, f, None, -1, 0.01, 0.9, 0.999, 1e-8, 1, None) == -1


def test_cnn_operands_must_be_16_byte_aligned(lib):
    # every layer moves BF16 rows in 16-byte units: a misaligned operand is refused on the
    # host, before any device call
    from paper_2404_07780_b300 import cnn
    L = cnn.lib()
    f, m = ctypes.c_void_p(256), ctypes.c_void_p(256 + 2)  # never dereferenced
    for args in ((m, f, None, f), (f, m, None, f), (f, f, None, m)):
        assert L.gm_cnn_conv_fwd(*args, 2, 32, 32, 32, 64, 1, None) == -1
        assert b"16-byte aligned" in L.gm_cnn_last_error()
    assert L.gm_cnn_conv_bwd_data(f, f, m, f, 2, 32, 32, 32, 64, None) == -1
    assert L.gm_cnn_dense_fwd(f, f, None, m, None, 4, 64, 64, 1, None) == -1
    assert L.gm_cnn_dense_bwd_data(m, f, None, f, 4, 64, 64, None) == -1
    ws = L.gm_cnn_dense_bwd_weight_workspace(4, 64, 64)
    assert L.gm_cnn_dense_bwd_weight(f, m, f, None, 4, 64, 64, f, ws, None) == -1


def test_cnn_forward_layers_take_the_tensor_map_path(lib):
    # the network's layers: the single-channel first convolution (K = 9) and the FP32-output
    # last layer on the gathered GEMM, the other convolutions and the hidden dense layer on
    # the TMA-fed tensor-core GEMM (inference fuses the first two: gm_cnn_conv12_fwd)
    from paper_2404_07780_b300 import cnn
    T, G = cnn.PATH_TMA, cnn.PATH_GATHER
    side = cnn.INPUT_SIDE
    hw = side
    ci = 1
    got = []
    for kind, i, o in cnn.LAYERS:
        if kind == "conv":
            got.append(cnn.fwd_path("conv", 512, hw, hw, i, o))
            hw //= 2
        else:
            got.append(cnn.fwd_path("dense", 512, 0, 0, i, o, fp32_out=o == cnn.LAYERS[-1][2]))
    assert got == [G, T, T, T, T, G], got
    # tiles of 128 output pixels must be whole rows of whole images
    assert cnn.fwd_path("conv", 3, 13, 9, 8, 16) == G          # odd sides, 8 channels
    assert cnn.fwd_path("conv", 2, 24, 24, 32, 64) == G        # 12 x 12 output: 144 pixels
    assert cnn.fwd_path("conv", 2, 32, 32, 32, 96) == G        # co not a multiple of 64
    assert cnn.fwd_path("conv", 2, 32, 32, 32, 128) == T
    assert cnn.fwd_path("dense", 7, 0, 0, 2048, 256) == T
    assert cnn.fwd_path("dense", 7, 0, 0, 32, 64) == G         # fin below one 64-wide slice
    assert cnn.fwd_path("dense", 7, 0, 0, 256, 264) == G
    assert cnn.fwd_path("dense", 7, 0, 0, 256, 320) == G         # more than 256 outputs
    assert cnn.fwd_path("conv", 2, 16, 16, 64, 320) == G
    assert cnn.fwd_path("dense", 7, 0, 0, 256, 256, fp32_out=True) == G
    with pytest.raises(cnn.CNNError):
        cnn.fwd_path("conv", 2, 32, 32, 12, 16)


def test_many_parameter_models_size_their_workspace(lib):
    # bulge+disk (12 free, 13 correlated channels) and bulge+bar+nucleus (15 free) run in
    # several channel-pair passes; the size queries accept them
    for spec in (synth.bulge_disk_sky(64, 64), synth.bulge_bar_nucleus_sky(64, 64)):
        d = gm.desc_from_spec(spec)
        b = gm.gm_batch(2, 64, 64, 25, None, None, None, None)
        assert lib.gm_chi2_grad_workspace_bytes(ctypes.byref(d), ctypes.byref(b)) > 0
        assert lib.gm_fit_workspace_bytes(ctypes.byref(d), ctypes.byref(b)) > 0


def test_adjoint_stats_before_any_call(lib):
    st = gm.gm_adjoint_stats()
    assert lib.gm_grad_adjoint_last_stats(ctypes.byref(st)) == -1
    assert lib.gm_grad_adjoint_last_stats(None) == -1


def test_fit_stats_before_any_fit(lib):
    st = gm.gm_fit_stats()
    assert lib.gm_fit_last_stats(ctypes.byref(st)) == -1


def test_uneven_geometry_sizes_and_rejections(lib):
    spec = synth.single_sersic_sky(64, 64)
    d = gm.desc_from_spec(spec)

    def batch(geom):
        g = gm.geom_array(geom)
        return gm.gm_batch(len(g), 0, 0, 0, None, None, None, None, ctypes.c_void_p(g.ctypes.data)), g

    # 3 galaxies: 2 + 4 + 1 tiles; the chi^2 workspace holds one FP64 partial per tile
    b, keep = batch([(40, 64, 25), (64, 64, 41), (9, 7, 1)])
    m = lib.gm_model_workspace_bytes(ctypes.byref(d), ctypes.byref(b))
    c = lib.gm_chi2_grad_workspace_bytes(ctypes.byref(d), ctypes.byref(b))
    f = lib.gm_fit_workspace_bytes(ctypes.byref(d), ctypes.byref(b))
    assert 0 < m < c < f
    assert c - m >= 7 * 45 * 8
    for bad in ([(64, 64, 14)], [(0, 64, 15)], [(64, 5000, 15)], [(64, 64, 65)], [(64, 64, -1)]):
        b, keep = batch(bad)
        assert lib.gm_fit_workspace_bytes(ctypes.byref(d), ctypes.byref(b)) == 0
        assert "uneven batch" in lib.gm_last_error().decode()
    # the entry point without a workspace refuses a bad geometry with the planner's own reason
    b, keep = batch([(40, 64, 25), (64, 64, 14)])
    fake = ctypes.c_void_p(16)
    b.image = b.sigma = b.psf = fake
    rc = lib.gm_chi2_grad_noalloc(ctypes.byref(d), ctypes.byref(b), fake, fake, None, None, None)
    msg = lib.gm_last_error().decode()
    assert rc == -1 and "uneven batch" in msg and "must be odd" in msg, msg
    assert msg.count("gm_chi2_grad_noalloc") <= 1, msg
    # the adjoint gradient takes equal stamps only: refused before any device work
    b, keep = batch([(40, 64, 25)])
    fake = ctypes.c_void_p(16)
    b.image = b.sigma = b.psf = fake
    assert lib.gm_grad_adjoint_workspace_bytes(ctypes.byref(d), ctypes.byref(b)) == 0
    rc = lib.gm_grad_adjoint(ctypes.byref(d), ctypes.byref(b), fake, fake, None, fake, 1 << 20, None)
    assert rc == -4 and "equal stamps" in lib.gm_last_error().decode()


def test_tune_set_rejects_shapes_that_are_not_launch_shapes(lib):
    assert lib.gm_tune_set(41, 8, 4, 1, 4) == 0
    assert lib.gm_tune_set(41, 8, 0, 0, 0) == 0       # clears the entry
    assert lib.gm_tune_set(40, 8, 4, 1, 4) == -1      # even PSF side
    assert lib.gm_tune_set(41, 17, 4, 1, 4) == -1     # more free parameters than the ABI allows
    assert lib.gm_tune_set(41, 8, 5, 1, 4) == -1      # more than 4 pairs per pass
    assert lib.gm_tune_set(41, 8, 4, 1, 3) == -1      # a pair without a thread group
    assert lib.gm_tune_set(41, 8, 2, 2, 3) == -1      # 3 groups of 2-pair threads exceed 256 threads
    assert lib.gm_tune_set(41, 8, 4, 2, 4) == 0       # 4 groups of 2-pair threads: the row-split shape
    assert lib.gm_tune_set(41, 8, 2, 2, 4) == 0       # ... or with 2 pairs per pass, each split 4 ways
    assert lib.gm_tune_set(41, 8, 3, 2, 4) == -1      # ... but not with 3
    assert lib.gm_tune_set(41, 8, 0, 0, 0) == 0
    assert lib.gm_tune_set(41, 8, 2, 3, 1) == -1      # 3 pairs per thread is not built
    assert lib.gm_tune_clear() == 0


def test_tune_cache_round_trip(lib, tmp_path):
    from paper_2404_07780_b300 import tune
    path = str(tmp_path / "tuning.json")
    e = {"K": 41, "P": 8, "pairs_per_pass": 4, "pairs_per_thread": 1, "groups": 4, "ms": 1.0}
    tune.save([e], path, device="test-device")
    tune.save([dict(e, K=25, P=12, pairs_per_pass=2, pairs_per_thread=2, groups=2)], path, device="test-device")
    assert len(tune.read_cache(path)["test-device"]["entries"]) == 2
    assert tune.apply_cache(lib, path, device="test-device") == 2
    assert tune.apply_cache(lib, path, device="another-device") == 0
    assert all(lib.gm_tune_set(K, P, 0, 0, 0) == 0 for K, P in ((41, 8), (25, 12)))
    # every shape the tuner tries is one gm_tune_set accepts
    for shape in tune.SHAPES:
        assert lib.gm_tune_set(41, 8, *shape) == 0, shape
    assert lib.gm_tune_clear() == 0
