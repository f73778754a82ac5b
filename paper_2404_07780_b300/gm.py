"""Thin Python binding of libgm (include/gm.h): argument marshalling only.

Every step of the fitting path runs in the CUDA library; this module turns
torch CUDA tensors into the pointers and sizes of the C ABI, allocates the
caller-owned workspace with torch, and raises on any nonzero return.  There is
no CPU fallback: without the compiled library or a CUDA device every call
raises.

Function names follow the C ABI: ``gm_model``, ``gm_chi2_grad``,
``gm_fit_batch``.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgm.so")

MAX_COMP = 8
MAX_SLOTS = 24
KIND = {"sersic": 1, "expdisk": 2, "ferrer": 3, "king": 4, "gaussian": 5, "moffat": 6, "sky": 7, "tsky": 8}
STATUS = {0: "RUNNING", 1: "CONVERGED", 2: "MAX_ITER", 3: "STALLED", 4: "SINGULAR", 5: "NONFINITE",
          6: "BAD_INPUT", 7: "NO_DOF"}
ST_CONVERGED = 1

# every symbol include/gm.h declares
EXPORTS = ("gm_version", "gm_last_error", "gm_model_workspace_bytes", "gm_model",
           "gm_chi2_grad_workspace_bytes", "gm_chi2_grad", "gm_fit_workspace_bytes", "gm_fit_batch",
           "gm_fit_last_stats", "gm_chi2_grad_noalloc", "gm_grad_adjoint_workspace_bytes", "gm_grad_adjoint",
           "gm_tune_set", "gm_tune_clear", "gm_tune_last_shape", "gm_fit_adam_workspace_bytes", "gm_fit_adam",
           "gm_bootstrap_workspace_bytes", "gm_bootstrap_counts", "gm_bootstrap", "gm_test_starve_next_pass",
           "gm_grad_adjoint_last_stats")


class GMError(RuntimeError):
    pass


class gm_component(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("convolve", ctypes.c_int32), ("slot", ctypes.c_int32 * 8)]


class gm_model_desc(ctypes.Structure):
    _fields_ = [
        ("n_comp", ctypes.c_int32),
        ("comp", gm_component * MAX_COMP),
        ("n_slots", ctypes.c_int32),
        ("is_free", ctypes.c_uint8 * MAX_SLOTS),
        ("is_log", ctypes.c_uint8 * MAX_SLOTS),
        ("lo", ctypes.c_double * MAX_SLOTS),
        ("hi", ctypes.c_double * MAX_SLOTS),
        ("amp_is_mag", ctypes.c_uint8 * MAX_COMP),
        ("mag_zero", ctypes.c_double * MAX_COMP),
        ("has_box", ctypes.c_uint8 * MAX_COMP),
    ]


class gm_batch(ctypes.Structure):
    _fields_ = [
        ("n_gal", ctypes.c_int32),
        ("H", ctypes.c_int32),
        ("W", ctypes.c_int32),
        ("K", ctypes.c_int32),
        ("image", ctypes.c_void_p),
        ("sigma", ctypes.c_void_p),
        ("mask", ctypes.c_void_p),
        ("psf", ctypes.c_void_p),
        ("geom", ctypes.c_void_p),
    ]


class gm_fit_opts(ctypes.Structure):
    _fields_ = [
        ("tol", ctypes.c_double),
        ("xtol", ctypes.c_double),
        ("gtol", ctypes.c_double),
        ("max_iter", ctypes.c_int32),
        ("lambda0", ctypes.c_double),
        ("lambda_up", ctypes.c_double),
        ("lambda_down", ctypes.c_double),
        ("lambda_min", ctypes.c_double),
        ("lambda_max", ctypes.c_double),
        ("polish", ctypes.c_int32),
        ("canonical", ctypes.c_int32),
        ("lambda_inout", ctypes.c_void_p),
    ]


class gm_adjoint_stats(ctypes.Structure):
    _fields_ = [
        ("setup_ms", ctypes.c_double),
        ("resid_ms", ctypes.c_double),
        ("residual_ms", ctypes.c_double),
        ("grad_ms", ctypes.c_double),
        ("deriv_ms", ctypes.c_double),
    ]


class gm_adam_opts(ctypes.Structure):
    _fields_ = [
        ("n_iter", ctypes.c_int32),
        ("lr", ctypes.c_double),
        ("beta1", ctypes.c_double),
        ("beta2", ctypes.c_double),
        ("eps", ctypes.c_double),
    ]


class gm_fit_stats(ctypes.Structure):
    _fields_ = [
        ("passes", ctypes.c_int32),
        ("graph_reused", ctypes.c_int32),
        ("galaxy_evals", ctypes.c_int64),
        ("converged", ctypes.c_int64),
        ("iters_sum", ctypes.c_int64),
        ("profile_ms", ctypes.c_double),
        ("fused_ms", ctypes.c_double),
        ("step_ms", ctypes.c_double),
        ("wall_ms", ctypes.c_double),
    ]


@dataclass
class FitOptions:
    tol: float = 1e-6
    xtol: float = 1e-10
    gtol: float = 1e-10
    max_iter: int = 100
    lambda0: float = 1e-1
    lambda_up: float = 10.0
    lambda_down: float = 0.2
    lambda_min: float = 1e-7
    lambda_max: float = 1e10
    polish: int = 1
    canonical: int = 1
    lambda_inout: object = None  # None, or a float64 CUDA tensor [G]: damping in and out (checkpoint / resume)

    def to_c(self) -> gm_fit_opts:
        li = None if self.lambda_inout is None else ctypes.c_void_p(self.lambda_inout.data_ptr())
        if self.lambda_inout is not None:
            import torch
            t = self.lambda_inout
            if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
                raise GMError("lambda_inout must be a contiguous float64 CUDA tensor")
        return gm_fit_opts(self.tol, self.xtol, self.gtol, self.max_iter, self.lambda0, self.lambda_up, self.lambda_down,
                           self.lambda_min, self.lambda_max, self.polish, self.canonical, li)


_lib = None


def load() -> ctypes.CDLL:
    """Load the in-tree libgm.so (build it with paper_2404_07780_b300.build.build_lib)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise GMError(f"{LIB_PATH} is missing: build the CUDA library first (python -c "
                          "'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(LIB_PATH)
        P, S = ctypes.c_void_p, ctypes.c_size_t
        lib.gm_version.restype = ctypes.c_int
        lib.gm_version.argtypes = []
        lib.gm_last_error.restype = ctypes.c_char_p
        lib.gm_last_error.argtypes = []
        for name in ("gm_model_workspace_bytes", "gm_chi2_grad_workspace_bytes", "gm_fit_workspace_bytes"):
            f = getattr(lib, name)
            f.restype = S
            f.argtypes = [P, P]
        lib.gm_model.restype = ctypes.c_int
        lib.gm_model.argtypes = [P, P, P, P, P, P, S, P]
        lib.gm_chi2_grad.restype = ctypes.c_int
        lib.gm_chi2_grad.argtypes = [P, P, P, P, P, P, P, S, P]
        lib.gm_fit_batch.restype = ctypes.c_int
        lib.gm_fit_batch.argtypes = [P, P, P, P, P, P, P, P, P, P, S, P]
        lib.gm_chi2_grad_noalloc.restype = ctypes.c_int
        lib.gm_chi2_grad_noalloc.argtypes = [P, P, P, P, P, P, P]
        lib.gm_grad_adjoint_workspace_bytes.restype = S
        lib.gm_grad_adjoint_workspace_bytes.argtypes = [P, P]
        lib.gm_grad_adjoint.restype = ctypes.c_int
        lib.gm_grad_adjoint.argtypes = [P, P, P, P, P, P, S, P]
        lib.gm_grad_adjoint_last_stats.restype = ctypes.c_int
        lib.gm_grad_adjoint_last_stats.argtypes = [P]
        lib.gm_fit_last_stats.restype = ctypes.c_int
        lib.gm_fit_last_stats.argtypes = [P]
        lib.gm_bootstrap_workspace_bytes.restype = S
        lib.gm_bootstrap_workspace_bytes.argtypes = [P, P]
        lib.gm_bootstrap_counts.restype = ctypes.c_int
        lib.gm_bootstrap_counts.argtypes = [P, P, ctypes.c_uint64, ctypes.c_int32, P, P, S, P]
        lib.gm_bootstrap.restype = ctypes.c_int
        lib.gm_bootstrap.argtypes = [P, P, P, ctypes.c_int32, ctypes.c_uint64, P, P, P, P, S, P]
        lib.gm_fit_adam_workspace_bytes.restype = S
        lib.gm_fit_adam_workspace_bytes.argtypes = [P, P]
        lib.gm_fit_adam.restype = ctypes.c_int
        lib.gm_fit_adam.argtypes = [P, P, P, P, P, P, S, P]
        I32 = ctypes.c_int32
        lib.gm_test_starve_next_pass.restype = ctypes.c_int
        lib.gm_test_starve_next_pass.argtypes = [ctypes.c_uint32]
        lib.gm_tune_set.restype = ctypes.c_int
        lib.gm_tune_set.argtypes = [I32, I32, I32, I32, I32]
        lib.gm_tune_clear.restype = ctypes.c_int
        lib.gm_tune_clear.argtypes = []
        lib.gm_tune_last_shape.restype = ctypes.c_int
        lib.gm_tune_last_shape.argtypes = [P, P, P]
        _lib = lib
        from . import tune
        tune.apply_cache(lib)
    return _lib


def _check(rc: int, what: str):
    if rc != 0:
        raise GMError(f"{what} failed ({rc}): {load().gm_last_error().decode()}")


def desc_from_spec(spec) -> gm_model_desc:
    """C descriptor from a ModelSpec (see synth.ModelSpec)."""
    d = gm_model_desc()
    d.n_comp = len(spec.components)
    if d.n_comp > MAX_COMP or spec.n_slots > MAX_SLOTS:
        raise GMError("model too large for the C descriptor")
    for c, comp in enumerate(spec.components):
        d.comp[c].kind = KIND[comp.kind]
        d.comp[c].convolve = 1 if comp.convolve else 0
        for k, s in enumerate(comp.slots):
            d.comp[c].slot[k] = int(s)
        if comp.mag_zero is not None:
            d.amp_is_mag[c] = 1
            d.mag_zero[c] = float(comp.mag_zero)
        d.has_box[c] = 1 if getattr(comp, "boxy", False) else 0
    d.n_slots = spec.n_slots
    for s in range(spec.n_slots):
        d.is_free[s] = 1 if spec.free[s] else 0
        d.is_log[s] = 1 if spec.log[s] else 0
        d.lo[s] = float(spec.lo[s])
        d.hi[s] = float(spec.hi[s])
    return d


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _cuda_tensor(t, dtype, name):
    import torch
    if t is None:
        return None
    if not t.is_cuda:
        raise GMError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise GMError(f"{name} must be {dtype}, got {t.dtype}")
    return t.contiguous()


def geom_array(geom) -> np.ndarray:
    """Per-galaxy (h, w, k) of an uneven batch as a contiguous int32 [G, 3] array."""
    g = np.ascontiguousarray(np.asarray(geom, dtype=np.int32).reshape(-1, 3))
    return g


def _geom_ptr(g):
    return None if g is None else ctypes.c_void_p(g.ctypes.data)


def packed_sizes(geom: np.ndarray):
    """(pixels, PSF elements) of an uneven batch packed back to back."""
    g = geom.astype(np.int64)
    return int((g[:, 0] * g[:, 1]).sum()), int((g[:, 2] ** 2).sum())


def make_batch(image, sigma, mask, psf, geom=None):
    """gm_batch over CUDA tensors.

    Equal stamps (geom None): image/sigma [G,H,W] f32, mask [G,H,W] u8 or None, psf [G,K,K] f32.
    Uneven stamps: geom [G,3] = (h, w, k) per galaxy (host), image/sigma/mask packed back to back
    (sum h*w elements), psf packed (sum k*k elements).

    Returns (struct, keep) where keep holds the contiguous tensors (and geom) alive."""
    import torch
    psf = _cuda_tensor(psf, torch.float32, "psf")
    image = _cuda_tensor(image, torch.float32, "image")
    sigma = _cuda_tensor(sigma, torch.float32, "sigma")
    mask = _cuda_tensor(mask, torch.uint8, "mask")
    if image is None:
        raise GMError("image is required to size the batch (use gm_model for the forward model alone)")
    if geom is None:
        G, K = psf.shape[0], psf.shape[-1]
        H, W = image.shape[-2:]
        b = gm_batch(G, H, W, K, _ptr(image), _ptr(sigma), _ptr(mask), _ptr(psf), None)
        return b, (image, sigma, mask, psf)
    g = geom_array(geom)
    npix, npsf = packed_sizes(g)
    for name, t in (("image", image), ("sigma", sigma), ("mask", mask)):
        if t is not None and t.numel() != npix:
            raise GMError(f"{name} holds {t.numel()} elements; the geometry packs {npix}")
    if psf.numel() != npsf:
        raise GMError(f"psf holds {psf.numel()} elements; the geometry packs {npsf}")
    b = gm_batch(len(g), 0, 0, 0, _ptr(image), _ptr(sigma), _ptr(mask), _ptr(psf), _geom_ptr(g))
    return b, (image, sigma, mask, psf, g)


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def gm_model(spec_or_desc, params, psf, H: int = 0, W: int = 0, components: bool = False, geom=None):
    """Forward model of every galaxy.

    Equal stamps: returns model [G,H,W] (and [G,n_comp,H,W] if components).  Uneven stamps
    (geom [G,3] = (h, w, k), psf packed): returns the packed model [sum h*w] (and the packed
    components [sum n_comp*h*w], galaxy by galaxy, component by component)."""
    import torch
    lib = load()
    d = spec_or_desc if isinstance(spec_or_desc, gm_model_desc) else desc_from_spec(spec_or_desc)
    psf = _cuda_tensor(psf, torch.float32, "psf")
    params = _cuda_tensor(params, torch.float64, "params")
    dev = psf.device
    if geom is None:
        G, K = psf.shape[0], psf.shape[-1]
        b = gm_batch(G, H, W, K, None, None, None, _ptr(psf), None)
        shape, cshape = (G, H, W), (G, d.n_comp, H, W)
        g = None
    else:
        g = geom_array(geom)
        npix, npsf = packed_sizes(g)
        if psf.numel() != npsf:
            raise GMError(f"psf holds {psf.numel()} elements; the geometry packs {npsf}")
        b = gm_batch(len(g), 0, 0, 0, None, None, None, _ptr(psf), _geom_ptr(g))
        shape, cshape = (npix,), (d.n_comp * npix,)
    model = torch.empty(shape, dtype=torch.float32, device=dev)
    comp = torch.empty(cshape, dtype=torch.float32, device=dev) if components else None
    nbytes = lib.gm_model_workspace_bytes(ctypes.byref(d), ctypes.byref(b))
    if nbytes == 0 and b.n_gal > 0:
        raise GMError(f"gm_model_workspace_bytes: {lib.gm_last_error().decode()}")
    ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=dev)
    _check(lib.gm_model(ctypes.byref(d), ctypes.byref(b), _ptr(params), _ptr(model), _ptr(comp), _ptr(ws), nbytes,
                        _stream()), "gm_model")
    return (model, comp) if components else model


def gm_chi2_grad(spec_or_desc, params, image, sigma, mask, psf, want_grad: bool = True, want_jtj: bool = False,
                 geom=None):
    """chi^2 [G], d chi^2/dp [G,S] (physical units) and J^T W J [G,S,S] (or None); geom as make_batch."""
    import torch
    lib = load()
    d = spec_or_desc if isinstance(spec_or_desc, gm_model_desc) else desc_from_spec(spec_or_desc)
    b, keep = make_batch(image, sigma, mask, psf, geom)
    params = _cuda_tensor(params, torch.float64, "params")
    G, S = b.n_gal, d.n_slots
    dev = keep[0].device
    chi2 = torch.empty(G, dtype=torch.float64, device=dev)
    grad = torch.empty((G, S), dtype=torch.float64, device=dev) if want_grad else None
    jtj = torch.empty((G, S, S), dtype=torch.float64, device=dev) if want_jtj else None
    nbytes = lib.gm_chi2_grad_workspace_bytes(ctypes.byref(d), ctypes.byref(b))
    if nbytes == 0 and G > 0:
        raise GMError(f"gm_chi2_grad_workspace_bytes: {lib.gm_last_error().decode()}")
    ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=dev)
    _check(lib.gm_chi2_grad(ctypes.byref(d), ctypes.byref(b), _ptr(params), _ptr(chi2), _ptr(grad), _ptr(jtj),
                            _ptr(ws), nbytes, _stream()), "gm_chi2_grad")
    return chi2, grad, jtj


def gm_chi2_grad_noalloc(spec_or_desc, params, image, sigma, mask, psf, want_grad: bool = True,
                         want_jtj: bool = False, geom=None):
    """gm_chi2_grad without a workspace: the library's fixed scratch array serves the call.

    For callers that may not allocate device memory when they evaluate chi^2 (the outputs
    here are still allocated by torch; a caller with that constraint passes its own through
    the C ABI).  Calls that overlap on the GPU share the array and race."""
    import torch
    lib = load()
    d = spec_or_desc if isinstance(spec_or_desc, gm_model_desc) else desc_from_spec(spec_or_desc)
    b, keep = make_batch(image, sigma, mask, psf, geom)
    params = _cuda_tensor(params, torch.float64, "params")
    G, S = b.n_gal, d.n_slots
    dev = keep[0].device
    chi2 = torch.empty(G, dtype=torch.float64, device=dev)
    grad = torch.empty((G, S), dtype=torch.float64, device=dev) if want_grad else None
    jtj = torch.empty((G, S, S), dtype=torch.float64, device=dev) if want_jtj else None
    _check(lib.gm_chi2_grad_noalloc(ctypes.byref(d), ctypes.byref(b), _ptr(params), _ptr(chi2), _ptr(grad),
                                    _ptr(jtj), _stream()), "gm_chi2_grad_noalloc")
    return chi2, grad, jtj


def gm_grad_adjoint(spec_or_desc, params, image, sigma, mask, psf, want_grad: bool = True):
    """chi^2 [G] and d chi^2/dp [G,S] (physical units) by the adjoint correlation."""
    import torch
    lib = load()
    d = spec_or_desc if isinstance(spec_or_desc, gm_model_desc) else desc_from_spec(spec_or_desc)
    b, keep = make_batch(image, sigma, mask, psf)
    params = _cuda_tensor(params, torch.float64, "params")
    G, S = b.n_gal, d.n_slots
    dev = keep[0].device
    chi2 = torch.empty(G, dtype=torch.float64, device=dev)
    grad = torch.empty((G, S), dtype=torch.float64, device=dev) if want_grad else None
    nbytes = lib.gm_grad_adjoint_workspace_bytes(ctypes.byref(d), ctypes.byref(b))
    ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=dev)
    _check(lib.gm_grad_adjoint(ctypes.byref(d), ctypes.byref(b), _ptr(params), _ptr(chi2), _ptr(grad), _ptr(ws),
                               nbytes, _stream()), "gm_grad_adjoint")
    return chi2, grad


def gm_fit_adam(spec_or_desc, params0, image, sigma, mask, psf, n_iter: int = 1000, lr: float = 0.01,
                beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """Gradient-descent (Adam) fit on the adjoint gradient for n_iter steps; returns
    {"params": lowest-chi^2 point evaluated [G,S], "chi2": [G]} (CUDA tensors)."""
    import torch
    lib = load()
    d = spec_or_desc if isinstance(spec_or_desc, gm_model_desc) else desc_from_spec(spec_or_desc)
    b, keep = make_batch(image, sigma, mask, psf)
    params = _cuda_tensor(params0, torch.float64, "params").clone().contiguous()
    dev = params.device
    chi2 = torch.empty(b.n_gal, dtype=torch.float64, device=dev)
    nbytes = lib.gm_fit_adam_workspace_bytes(ctypes.byref(d), ctypes.byref(b))
    if nbytes == 0 and b.n_gal > 0:
        raise GMError(f"gm_fit_adam_workspace_bytes: {lib.gm_last_error().decode()}")
    ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=dev)
    o = gm_adam_opts(n_iter, lr, beta1, beta2, eps)
    _check(lib.gm_fit_adam(ctypes.byref(d), ctypes.byref(b), _ptr(params), ctypes.byref(o), _ptr(chi2), _ptr(ws),
                           nbytes, _stream()), "gm_fit_adam")
    return {"params": params, "chi2": chi2}


def _boot_ws(lib, d, b, dev):
    import torch
    nbytes = lib.gm_bootstrap_workspace_bytes(ctypes.byref(d), ctypes.byref(b))
    if nbytes == 0 and b.n_gal > 0:
        raise GMError(f"gm_bootstrap_workspace_bytes: {lib.gm_last_error().decode()}")
    return torch.empty(max(nbytes, 1), dtype=torch.uint8, device=dev), nbytes


def gm_bootstrap_counts(spec_or_desc, image, sigma, mask, psf, seed: int, replicate: int):
    """Pixel multiplicities [G,H,W] (int32 view of uint32) of one bootstrap replicate."""
    import torch
    lib = load()
    d = spec_or_desc if isinstance(spec_or_desc, gm_model_desc) else desc_from_spec(spec_or_desc)
    b, keep = make_batch(image, sigma, mask, psf)
    dev = keep[0].device
    counts = torch.empty((b.n_gal, b.H, b.W), dtype=torch.int32, device=dev)
    ws, nbytes = _boot_ws(lib, d, b, dev)
    _check(lib.gm_bootstrap_counts(ctypes.byref(d), ctypes.byref(b), seed, replicate, _ptr(counts), _ptr(ws), nbytes,
                                   _stream()), "gm_bootstrap_counts")
    return counts


def gm_bootstrap(spec_or_desc, params_best, image, sigma, mask, psf, n_boot: int = 100, seed: int = 0,
                 opts: FitOptions | None = None):
    """Bootstrap error bars (Sec. 5.2): (sigma_boot [G,S], converged replicates [G])."""
    import torch
    lib = load()
    d = spec_or_desc if isinstance(spec_or_desc, gm_model_desc) else desc_from_spec(spec_or_desc)
    b, keep = make_batch(image, sigma, mask, psf)
    params_best = _cuda_tensor(params_best, torch.float64, "params_best")
    dev = params_best.device
    sig = torch.empty((b.n_gal, d.n_slots), dtype=torch.float64, device=dev)
    nok = torch.empty(b.n_gal, dtype=torch.int32, device=dev)
    ws, nbytes = _boot_ws(lib, d, b, dev)
    o = (opts or FitOptions()).to_c()
    _check(lib.gm_bootstrap(ctypes.byref(d), ctypes.byref(b), _ptr(params_best), n_boot, seed, ctypes.byref(o),
                            _ptr(sig), _ptr(nok), _ptr(ws), nbytes, _stream()), "gm_bootstrap")
    return sig, nok


class Chi2(object):
    """chi^2 of every galaxy as a differentiable torch function of the parameters.

    ``Chi2(spec, image, sigma, mask, psf)(params)`` returns a [G] tensor whose
    backward pass multiplies the upstream gradient into d chi^2/dp from the
    hand-written adjoint kernel (gm_grad_adjoint); forward and gradient come from
    one call.  With it the paper's own fitting mode -- a torch optimiser such as
    Adam stepping the parameters on chi^2 (Sec. 5.1) -- runs on these kernels."""

    def __init__(self, spec_or_desc, image, sigma, mask, psf):
        self.d = spec_or_desc if isinstance(spec_or_desc, gm_model_desc) else desc_from_spec(spec_or_desc)
        self.image, self.sigma, self.mask, self.psf = image, sigma, mask, psf
        self._fn = _make_chi2_function()

    def __call__(self, params):
        return self._fn.apply(params, self)


def _make_chi2_function():
    import torch

    class _Chi2Fn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, params, owner):
            chi2, grad = gm_grad_adjoint(owner.d, params.detach().contiguous(), owner.image, owner.sigma,
                                         owner.mask, owner.psf, want_grad=params.requires_grad)
            ctx.save_for_backward(grad if grad is not None else torch.zeros_like(params))
            return chi2

        @staticmethod
        def backward(ctx, g_out):
            (grad,) = ctx.saved_tensors
            return g_out.to(grad.dtype)[:, None] * grad, None

    return _Chi2Fn


class Fitter:
    """Holds the workspace and output buffers of gm_fit_batch for one batch geometry
    (G equal H x W stamps with K x K PSFs, or an uneven batch given by geom [G,3])."""

    def __init__(self, spec_or_desc, G: int, H: int = 0, W: int = 0, K: int = 0, device="cuda", geom=None):
        import torch
        self.lib = load()
        self.d = spec_or_desc if isinstance(spec_or_desc, gm_model_desc) else desc_from_spec(spec_or_desc)
        self.geom = None if geom is None else geom_array(geom)
        if self.geom is not None:
            G = len(self.geom)
            b = gm_batch(G, 0, 0, 0, None, None, None, None, _geom_ptr(self.geom))
            self.shape = ("uneven", G)
        else:
            b = gm_batch(G, H, W, K, None, None, None, None, None)
            self.shape = (G, H, W, K)
        self.ws_bytes = self.lib.gm_fit_workspace_bytes(ctypes.byref(self.d), ctypes.byref(b))
        if self.ws_bytes == 0 and G > 0:
            raise GMError(f"gm_fit_workspace_bytes: {self.lib.gm_last_error().decode()}")
        S = self.d.n_slots
        self.ws = torch.empty(max(self.ws_bytes, 1), dtype=torch.uint8, device=device)
        self.chi2 = torch.empty(G, dtype=torch.float64, device=device)
        self.dof = torch.empty(G, dtype=torch.int32, device=device)
        self.iters = torch.empty(G, dtype=torch.int32, device=device)
        self.status = torch.empty(G, dtype=torch.int32, device=device)
        self.sigma_p = torch.empty((G, S), dtype=torch.float64, device=device)

    def fit(self, params, image, sigma, mask, psf, opts: FitOptions | None = None):
        """Fit in place: params [G,S] f64 CUDA is overwritten with the best fit."""
        import torch
        b, keep = make_batch(image, sigma, mask, psf, self.geom)
        shape = ("uneven", b.n_gal) if self.geom is not None else (b.n_gal, b.H, b.W, b.K)
        if shape != self.shape:
            raise GMError(f"batch shape {shape} != fitter shape {self.shape}")
        if not (params.is_cuda and params.dtype == torch.float64 and params.is_contiguous()):
            raise GMError("params must be a contiguous float64 CUDA tensor")
        if opts is not None and opts.lambda_inout is not None and opts.lambda_inout.numel() != b.n_gal:
            raise GMError(f"lambda_inout holds {opts.lambda_inout.numel()} values for {b.n_gal} galaxies")
        o = (opts or FitOptions()).to_c()
        _check(self.lib.gm_fit_batch(ctypes.byref(self.d), ctypes.byref(b), _ptr(params), ctypes.byref(o),
                                     _ptr(self.chi2), _ptr(self.dof), _ptr(self.iters), _ptr(self.status),
                                     _ptr(self.sigma_p), _ptr(self.ws), self.ws_bytes, _stream()), "gm_fit_batch")
        return {"params": params, "chi2": self.chi2, "dof": self.dof, "iters": self.iters, "status": self.status,
                "sigma_p": self.sigma_p}


def gm_tune_set(K: int, P: int, pairs_per_pass: int, pairs_per_thread: int, groups: int):
    """Launch shape of the fused pass for largest PSF side K and P free parameters (0 pairs_per_pass clears)."""
    _check(load().gm_tune_set(K, P, pairs_per_pass, pairs_per_thread, groups), "gm_tune_set")


def gm_tune_clear():
    _check(load().gm_tune_clear(), "gm_tune_clear")


def gm_tune_last_shape() -> tuple[int, int, int]:
    """(pairs_per_pass, pairs_per_thread, groups) of this thread's last planned pass."""
    a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().gm_tune_last_shape(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "gm_tune_last_shape")
    return a.value, b.value, c.value


def gm_grad_adjoint_last_stats() -> dict:
    """Kernel times (ms) of this thread's last gm_grad_adjoint: setup_ms, resid_ms, residual_ms, grad_ms,
    deriv_ms."""
    st = gm_adjoint_stats()
    _check(load().gm_grad_adjoint_last_stats(ctypes.byref(st)), "gm_grad_adjoint_last_stats")
    return {name: getattr(st, name) for name, _ in gm_adjoint_stats._fields_}


def gm_fit_last_stats() -> dict:
    """Counters of this thread's last gm_fit_batch: passes, graph_reused, galaxy_evals, converged, iters_sum,
    profile_ms, fused_ms, step_ms, wall_ms."""
    st = gm_fit_stats()
    _check(load().gm_fit_last_stats(ctypes.byref(st)), "gm_fit_last_stats")
    return {name: getattr(st, name) for name, _ in gm_fit_stats._fields_}


def gm_fit_batch(spec_or_desc, params0, image, sigma, mask, psf, opts: FitOptions | None = None, geom=None):
    """LM fit of every galaxy; returns a dict of CUDA tensors (params is a fitted copy of params0).
    geom as make_batch."""
    if geom is None:
        G, H, W = image.shape
        K = psf.shape[-1]
        f = Fitter(spec_or_desc, G, H, W, K, device=image.device)
    else:
        f = Fitter(spec_or_desc, len(geom_array(geom)), device=image.device, geom=geom)
    params = params0.clone().contiguous()
    out = f.fit(params, image, sigma, mask, psf, opts)
    return {k: v.clone() if k != "params" else v for k, v in out.items()}
