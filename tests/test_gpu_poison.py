"""Missing writes: every element of every output is written by the library.

Each entry point runs twice on the same inputs: once into output buffers filled with
NaN (integer outputs with -7) and once into buffers filled with zeros.  An element a
kernel never writes keeps its fill and the two runs differ there; NaNs the library
writes on purpose (the covariance of a galaxy whose normal matrix is singular) are
equal in both.  The forward model runs on the small odd shapes (stamps of 37x45, 7x9
with a 15x15 PSF larger than the stamp, 64x33 with a 1x1 PSF); every entry point runs
on 64x64 stamps with 15x15 PSFs and a random mask.  Only the outputs are filled; the
inputs and the workspace are the same in both runs."""
import ctypes

import numpy as np
import pytest

from cases import from_batch
from paper_2404_07780_b300 import gm, synth

pytestmark = pytest.mark.gpu

MODEL_SHAPES = [(37, 45, 9), (7, 9, 15), (64, 33, 1)]
ALL_SHAPES = [(64, 64, 15)]


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2404_07780_b300.build import build_lib
    build_lib()
    return gm.load()


def _case(H, W, K):
    c = from_batch(synth.draw_small(seed=H * 100 + W + K, G=5, H=H, W=W, K=K), at="init")
    c.mask = (np.random.default_rng(K).random((c.G, H, W)) < 0.1).astype(np.uint8)
    return c


def _filled(shape, dtype, fill):
    import torch
    return torch.full(shape, fill, dtype=dtype, device="cuda")


def _same(a, b, what):
    import torch
    torch.testing.assert_close(a, b, rtol=0, atol=0, equal_nan=True, msg=lambda m: f"{what}: {m}")


def _ws(n):
    import torch
    return torch.zeros(max(n, 1), dtype=torch.uint8, device="cuda")


def _run_all(lib, H, W, K, entries):
    import torch
    c = _case(H, W, K)
    t = c.torch()
    d = gm.desc_from_spec(c.spec)
    b, keep = gm.make_batch(t["image"], t["sigma"], t["mask"], t["psf"])
    G, S, NC = c.G, c.spec.n_slots, d.n_comp
    P = ctypes.c_void_p
    ptr = lambda x: P(x.data_ptr())
    st = P(torch.cuda.current_stream().cuda_stream)
    R = ctypes.byref
    f64, f32, i32 = torch.float64, torch.float32, torch.int32

    def model(fill):
        m, comp = _filled((G, H, W), f32, fill), _filled((G, NC, H, W), f32, fill)
        n = lib.gm_model_workspace_bytes(R(d), R(b))
        ws = _ws(n)
        assert lib.gm_model(R(d), R(b), ptr(t["params"]), ptr(m), ptr(comp), ptr(ws), n, st) == 0
        torch.cuda.synchronize()
        return m, comp

    def normal(fill):
        chi2, grad, jtj = _filled((G,), f64, fill), _filled((G, S), f64, fill), _filled((G, S, S), f64, fill)
        n = lib.gm_chi2_grad_workspace_bytes(R(d), R(b))
        ws = _ws(n)
        assert lib.gm_chi2_grad(R(d), R(b), ptr(t["params"]), ptr(chi2), ptr(grad), ptr(jtj), ptr(ws), n, st) == 0
        torch.cuda.synchronize()
        return chi2, grad, jtj

    def adjoint(fill):
        chi2, grad = _filled((G,), f64, fill), _filled((G, S), f64, fill)
        n = lib.gm_grad_adjoint_workspace_bytes(R(d), R(b))
        ws = _ws(n)
        assert lib.gm_grad_adjoint(R(d), R(b), ptr(t["params"]), ptr(chi2), ptr(grad), ptr(ws), n, st) == 0
        torch.cuda.synchronize()
        return chi2, grad

    def fit(fill, ifill):
        p = t["params"].clone()
        chi2, sig = _filled((G,), f64, fill), _filled((G, S), f64, fill)
        dof, iters, status = (_filled((G,), i32, ifill) for _ in range(3))
        o = gm.FitOptions(max_iter=30).to_c()
        n = lib.gm_fit_workspace_bytes(R(d), R(b))
        ws = _ws(n)
        assert lib.gm_fit_batch(R(d), R(b), ptr(p), R(o), ptr(chi2), ptr(dof), ptr(iters), ptr(status), ptr(sig),
                                ptr(ws), n, st) == 0
        torch.cuda.synchronize()  # ws stays referenced until the fit's work is done
        return p, chi2, dof, iters, status, sig

    runs = {"gm_model": lambda f, i: model(f), "gm_chi2_grad": lambda f, i: normal(f),
            "gm_grad_adjoint": lambda f, i: adjoint(f), "gm_fit_batch": fit}
    for name in entries:
        run = runs[name]
        poisoned = run(float("nan"), -7)
        clean = run(0.0, 0)
        torch.cuda.synchronize()
        for k, (x, y) in enumerate(zip(poisoned, clean)):
            _same(x, y, f"{name} output {k}")
        assert torch.isfinite(clean[0]).all(), name


@pytest.mark.parametrize("H,W,K", MODEL_SHAPES)
def test_every_model_element_is_written(lib, H, W, K):
    _run_all(lib, H, W, K, ("gm_model",))


@pytest.mark.parametrize("H,W,K", ALL_SHAPES)
def test_every_output_element_is_written(lib, H, W, K):
    _run_all(lib, H, W, K, ("gm_model", "gm_chi2_grad", "gm_grad_adjoint", "gm_fit_batch"))
