"""FP64 CPU oracle for batched galaxy-profile fitting (arxiv 2404.07780).

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path (the
CUDA library and its Python binding) never imports this package, and this
package imports nothing from the product.

The arithmetic lives in ``gm_oracle.c`` (plain C, double precision, one pixel
at a time, OpenMP over independent galaxies).  This module only compiles it
and marshals numpy arrays through ctypes.

What it computes, with the paper passage each step follows:

* ``component_image`` / ``model_images``: light profiles at pixel centres
  (Sec. 4.1-4.2: Eqs. r, rmaj, rmin, sersic-intensity, expdisk_I, ferrer_I,
  BE_S, gaussion_I, moffat_I, sky_I), summed, correlated with the PSF with
  zero padding (Sec. 2 workflow; App. C ``conv2d(..., padding="same")``), plus
  the unconvolved components.
* ``chi2``: Eq. chinu with the mask Omega.
* ``jacobian``: central finite differences of ``model`` (no analytic
  derivative anywhere in the oracle).
* ``fit``: Levenberg-Marquardt on the chi^2 of Eq. chinu (Sec. 5.1 names LM
  as the classical alternative to the paper's gradient descent) and the
  covariance uncertainty of Sec. 5.2.
* ``gammp`` / ``sersic_b``: the regularised incomplete gamma function and the
  Sersic constant nu_n defined in Sec. 4.1 (half of the light inside r_e).

Parity status: every function above is pinned by the ``-m "not gpu"`` tests
(closed forms, library special cases, invariants, brute force).  The exact LM
trajectory is path dependent and is not pinned; only converged minima are
compared.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_gm_oracle.so")
_lib = None

KIND_CODES = {"sersic": 1, "expdisk": 2, "ferrer": 3, "king": 4, "gaussian": 5, "moffat": 6, "sky": 7, "tsky": 8}

MAX_COMP = 8
MAX_SLOTS = 24

STATUS = {0: "RUNNING", 1: "CONVERGED", 2: "MAX_ITER", 3: "STALLED", 4: "SINGULAR",
          5: "NONFINITE", 6: "BAD_INPUT", 7: "NO_DOF"}


def build(force: bool = False) -> str:
    """Compile gm_oracle.c into a shared object next to it (plain gcc)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", _LIB_PATH, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB_PATH


class _Desc(ctypes.Structure):
    _fields_ = [
        ("n_comp", ctypes.c_int),
        ("kind", ctypes.c_int * MAX_COMP),
        ("convolve", ctypes.c_int * MAX_COMP),
        ("slot", (ctypes.c_int * 8) * MAX_COMP),
        ("n_slots", ctypes.c_int),
        ("is_free", ctypes.c_int * MAX_SLOTS),
        ("is_log", ctypes.c_int * MAX_SLOTS),
        ("lo", ctypes.c_double * MAX_SLOTS),
        ("hi", ctypes.c_double * MAX_SLOTS),
        ("amp_is_mag", ctypes.c_int * MAX_COMP),
        ("mag_zero", ctypes.c_double * MAX_COMP),
        ("has_box", ctypes.c_int * MAX_COMP),
    ]


class _Opts(ctypes.Structure):
    _fields_ = [
        ("tol", ctypes.c_double),
        ("xtol", ctypes.c_double),
        ("gtol", ctypes.c_double),
        ("max_iter", ctypes.c_int),
        ("lambda0", ctypes.c_double),
        ("lambda_up", ctypes.c_double),
        ("lambda_down", ctypes.c_double),
        ("lambda_min", ctypes.c_double),
        ("lambda_max", ctypes.c_double),
        ("polish", ctypes.c_int),
        ("canonical", ctypes.c_int),
        ("lambda_inout", ctypes.c_void_p),
    ]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        lib.or_gammp.restype = ctypes.c_double
        lib.or_gammp.argtypes = [ctypes.c_double, ctypes.c_double]
        lib.or_sersic_b.restype = ctypes.c_double
        lib.or_sersic_b.argtypes = [ctypes.c_double]
        lib.or_mag_amplitude.restype = ctypes.c_double
        lib.or_mag_amplitude.argtypes = [ctypes.c_int, P, ctypes.c_double]
        lib.or_component_value.restype = ctypes.c_double
        lib.or_component_value.argtypes = [ctypes.c_int, P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double]
        lib.or_rbox.restype = ctypes.c_double
        lib.or_rbox.argtypes = [ctypes.c_double]
        lib.or_component_image.restype = None
        lib.or_component_image.argtypes = [ctypes.c_int, P, ctypes.c_int, ctypes.c_int, P]
        lib.or_correlate.restype = None
        lib.or_correlate.argtypes = [P, ctypes.c_int, ctypes.c_int, P, ctypes.c_int, P]
        for name in ("or_model_batch", "or_component_images_batch"):
            f = getattr(lib, name)
            f.restype = ctypes.c_int
            f.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P]
        lib.or_chi2_batch.restype = ctypes.c_int
        lib.or_chi2_batch.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      P, P, P, P, P, P]
        lib.or_jacobian_batch.restype = ctypes.c_int
        lib.or_jacobian_batch.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          P, P, ctypes.c_int, P]
        lib.or_fit_batch.restype = ctypes.c_int
        lib.or_fit_batch.argtypes = [P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     P, P, P, P, P, P, P, P, P, P]
        lib.or_canonicalize.restype = ctypes.c_int
        lib.or_canonicalize.argtypes = [P, P]
        lib.or_max_threads.restype = ctypes.c_int
        lib.or_max_threads.argtypes = []
        _lib = lib
    return _lib


@dataclass
class FitOptions:
    """Levenberg-Marquardt controls (same meaning as the CUDA library's)."""
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


def _desc(spec) -> _Desc:
    """Convert a neutral model spec (see the package's synth module) to the C struct."""
    d = _Desc()
    d.n_comp = len(spec.components)
    for c, comp in enumerate(spec.components):
        d.kind[c] = KIND_CODES[comp.kind]
        d.convolve[c] = 1 if comp.convolve else 0
        for k, s in enumerate(comp.slots):
            d.slot[c][k] = int(s)
        if getattr(comp, "mag_zero", None) is not None:
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


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def gammp(a: float, x: float) -> float:
    """Regularised lower incomplete gamma P(a, x)."""
    return _load().or_gammp(float(a), float(x))


def sersic_b(n: float) -> float:
    """nu_n of Eq. sersic-intensity: P(2n, nu_n) = 1/2 (Sec. 4.1)."""
    return _load().or_sersic_b(float(n))


def mag_amplitude(kind: str, par, m0: float) -> float:
    """Amplitude (Ie or I0) that gives the profile with parameters par, whose amplitude
    slot holds a magnitude m, the total flux 10^(-0.4 (m - m0))."""
    return _load().or_mag_amplitude(KIND_CODES[kind], _ptr(_f64(par)), float(m0))


def component_value(kind: str, par, x: float, y: float, B: float = 0.0) -> float:
    """One profile's intensity at the point (x, y) (pixel units), boxiness B."""
    par = _f64(par)
    nu = sersic_b(par[6]) if kind == "sersic" else 0.0
    return _load().or_component_value(KIND_CODES[kind], _ptr(par), nu, float(B), float(x), float(y))


def rbox(B: float) -> float:
    """Eq. rbox: pi (2+B) / (2 beta(1/(2+B), 1/(2+B)))."""
    return _load().or_rbox(float(B))


def component_image(kind: str, par, H: int, W: int) -> np.ndarray:
    """One profile sampled at the H x W pixel centres, no PSF."""
    par = _f64(par)
    out = np.zeros((H, W), np.float64)
    _load().or_component_image(KIND_CODES[kind], _ptr(par), H, W, _ptr(out))
    return out


def correlate(img, psf) -> np.ndarray:
    """Zero-padded same-size cross-correlation of img with an odd K x K psf."""
    img = _f64(img)
    psf = _f64(psf)
    H, W = img.shape
    K = psf.shape[0]
    assert psf.shape == (K, K) and K % 2 == 1
    out = np.zeros((H, W), np.float64)
    _load().or_correlate(_ptr(img), H, W, _ptr(psf), K, _ptr(out))
    return out


def model_images(spec, params, psf, H: int, W: int) -> np.ndarray:
    """Model images [G, H, W] for params [G, n_slots] and psf [G, K, K]."""
    params = _f64(params)
    psf = _f64(psf)
    G = params.shape[0]
    K = psf.shape[-1]
    out = np.zeros((G, H, W), np.float64)
    d = _desc(spec)
    _load().or_model_batch(ctypes.byref(d), G, H, W, K, _ptr(params), _ptr(psf), _ptr(out))
    return out


def component_images(spec, params, psf, H: int, W: int) -> np.ndarray:
    """Each component's contribution to the model, [G, n_comp, H, W]."""
    params = _f64(params)
    psf = _f64(psf)
    G = params.shape[0]
    K = psf.shape[-1]
    out = np.zeros((G, len(spec.components), H, W), np.float64)
    d = _desc(spec)
    _load().or_component_images_batch(ctypes.byref(d), G, H, W, K, _ptr(params), _ptr(psf), _ptr(out))
    return out


def chi2(spec, params, psf, image, sigma, mask=None) -> np.ndarray:
    """Eq. chinu for every galaxy, [G]."""
    params = _f64(params)
    psf = _f64(psf)
    image = _f64(image)
    sigma = _f64(sigma)
    mask = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    G, H, W = image.shape
    K = psf.shape[-1]
    out = np.zeros(G, np.float64)
    d = _desc(spec)
    _load().or_chi2_batch(ctypes.byref(d), G, H, W, K, _ptr(params), _ptr(psf), _ptr(image),
                          _ptr(sigma), _ptr(mask), _ptr(out))
    return out


def jacobian(spec, params, psf, H: int, W: int, internal: bool = False) -> np.ndarray:
    """Central-difference dM/dp for the free slots, [G, n_free, H, W].

    internal=True differentiates with respect to ln p for log slots."""
    params = _f64(params)
    psf = _f64(psf)
    G = params.shape[0]
    K = psf.shape[-1]
    nf = int(sum(1 for f in spec.free if f))
    out = np.zeros((G, nf, H, W), np.float64)
    d = _desc(spec)
    _load().or_jacobian_batch(ctypes.byref(d), G, H, W, K, _ptr(params), _ptr(psf),
                              1 if internal else 0, _ptr(out))
    return out


def fit(spec, params0, psf, image, sigma, mask=None, opts: FitOptions | None = None, lambda_inout=None) -> dict:
    """Levenberg-Marquardt fit of every galaxy; returns a dict of numpy arrays.

    lambda_inout: None, or a float64 [G] array holding each galaxy's starting damping (used when
    > 0 and finite), overwritten with its damping at exit (checkpoint and resume, with
    opts.canonical = 0 for the checkpoint)."""
    opts = opts or FitOptions()
    params = _f64(params0).copy()
    psf = _f64(psf)
    image = _f64(image)
    sigma = _f64(sigma)
    mask = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    G, H, W = image.shape
    K = psf.shape[-1]
    chi2_out = np.zeros(G, np.float64)
    dof = np.zeros(G, np.int32)
    iters = np.zeros(G, np.int32)
    status = np.zeros(G, np.int32)
    sigma_p = np.zeros_like(params)
    d = _desc(spec)
    if lambda_inout is not None:
        assert isinstance(lambda_inout, np.ndarray) and lambda_inout.dtype == np.float64 and \
            lambda_inout.shape == (G,) and lambda_inout.flags.c_contiguous
    o = _Opts(opts.tol, opts.xtol, opts.gtol, opts.max_iter, opts.lambda0, opts.lambda_up, opts.lambda_down,
              opts.lambda_min, opts.lambda_max, opts.polish, opts.canonical,
              None if lambda_inout is None else lambda_inout.ctypes.data)
    _load().or_fit_batch(ctypes.byref(d), ctypes.byref(o), G, H, W, K, _ptr(params), _ptr(psf),
                         _ptr(image), _ptr(sigma), _ptr(mask), _ptr(chi2_out), _ptr(dof),
                         _ptr(iters), _ptr(status), _ptr(sigma_p))
    return {"params": params, "chi2": chi2_out, "dof": dof, "iters": iters, "status": status,
            "sigma_p": sigma_p}


def canonicalize(spec, params) -> np.ndarray:
    """Rewrite axis ratios above 1 as 1/q with PA + pi/2 and scale lengths times q (same image)."""
    out = _f64(params).copy()
    d = _desc(spec)
    for row in out.reshape(-1, spec.n_slots):
        r = np.ascontiguousarray(row)
        _load().or_canonicalize(ctypes.byref(d), _ptr(r))
        row[:] = r
    return out


def max_threads() -> int:
    """OpenMP threads the oracle's batch loops use."""
    return _load().or_max_threads()


def fit_adam(spec, params0, psf, image, sigma, mask=None, n_iter: int = 100, lr: float = 0.01, beta1: float = 0.9,
             beta2: float = 0.999, eps: float = 1e-8):
    """Gradient descent with Adam (Kingma & Ba 2015) on chi^2, the paper's own way of fitting
    (Sec. 5.1), with the gradient -2 J^T W r of the finite-difference Jacobian.  Steps in
    internal coordinates (ln p for log slots) scaled by 1 for log slots and max(|p0|, 1)
    otherwise, clamped to the bounds; returns (lowest-chi^2 point evaluated in canonical
    form, its chi^2) after n_iter steps and a final evaluation."""
    p = np.clip(_f64(params0).copy(), spec.lo, spec.hi)
    G, S = p.shape
    free = np.array(spec.free, bool)
    logs = np.array(spec.log, bool)
    scale = np.where(logs, 1.0, np.maximum(np.abs(p), 1.0))
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    best = p.copy()
    best_c2 = np.full(G, np.inf)
    img, sig = _f64(image), _f64(sigma)
    w = 1.0 / sig ** 2
    if mask is not None:
        w = w * (np.asarray(mask) == 0)
    H, W = img.shape[1:]
    for t in range(1, n_iter + 2):
        M = model_images(spec, p, psf, H, W)
        c2 = (w * (img - M) ** 2).sum((1, 2))
        better = np.isfinite(c2) & (c2 < best_c2)
        best[better], best_c2[better] = p[better], c2[better]
        if t == n_iter + 1:
            break
        J = jacobian(spec, p, psf, H, W)  # [G][free][H][W], physical units
        g = np.zeros_like(p)
        g[:, free] = -2.0 * np.einsum("gfhw,ghw->gf", J, w * (img - M))
        gu = np.where(logs, g * p, g)
        m = beta1 * m + (1 - beta1) * gu
        v = beta2 * v + (1 - beta2) * gu * gu
        du = lr * scale * (m / (1 - beta1 ** t)) / (np.sqrt(v / (1 - beta2 ** t)) + eps)
        u = np.where(logs, np.log(np.where(logs, p, 1.0)), p) - np.where(free, du, 0.0)
        p = np.clip(np.where(logs, np.exp(np.where(logs, u, 0.0)), u), spec.lo, spec.hi)
    return canonicalize(spec, best), best_c2


# ---------------------------------------------------------------------------
# bootstrap (Sec. 5.2)
# ---------------------------------------------------------------------------
_M64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


def splitmix64(z: int) -> int:
    """The SplitMix64 output function (Steele, Lea & Flood 2014) applied to state z."""
    z &= _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def bootstrap_counts(mask, seed: int, g: int, b: int) -> np.ndarray:
    """Pixel multiplicities of replicate b of galaxy g: N draws, N = unmasked pixels; draw k is
    the (k+1)-th SplitMix64 output from the state splitmix64(splitmix64(seed) ^ (g << 32 | b)),
    mapped to the floor(r N / 2^64)-th unmasked pixel in row-major order."""
    mask = np.asarray(mask)
    used = np.flatnonzero(mask.ravel() == 0)
    N = len(used)
    key = splitmix64(splitmix64(seed) ^ ((g << 32) | b))
    counts = np.zeros(mask.size, np.uint32)
    for k in range(N):
        r = splitmix64((key + (k + 1) * _GOLDEN) & _M64)
        counts[used[(r * N) >> 64]] += 1
    return counts.reshape(mask.shape)


def bootstrap(spec, params_best, psf, image, sigma, mask=None, n_boot: int = 100, seed: int = 0,
              opts: FitOptions | None = None):
    """Bootstrap error bars: refit every replicate (pixel c drawn c times: weight c, i.e. sigma /
    sqrt(c); undrawn pixels masked) from params_best; sigma^2 = (1/M) sum (p_i - mean)^2 over the
    M converged refits, position angles taken within pi/2 of the best fit's.  Returns
    (sigma_boot [G,S], M [G])."""
    params_best = _f64(params_best)
    G, S = params_best.shape
    image, sigma = _f64(image), _f64(sigma)
    base = np.zeros(image.shape, np.uint8) if mask is None else np.asarray(mask, np.uint8)
    pa = np.array([n.endswith(".pa") for n in spec.names])
    reps = []
    for b in range(n_boot):
        counts = np.stack([bootstrap_counts(base[g], seed, g, b) for g in range(G)])
        m_eff = ((base != 0) | (counts == 0)).astype(np.uint8)
        s_eff = np.where(counts > 0, sigma / np.sqrt(np.maximum(counts, 1)), 1.0)
        r = fit(spec, params_best, psf, image, s_eff, m_eff, opts)
        p = r["params"].copy()
        d = p[:, pa] - params_best[:, pa]
        p[:, pa] = params_best[:, pa] + d - np.pi * np.floor(d / np.pi + 0.5)
        reps.append((p, r["status"] == 1))
    sig = np.full((G, S), np.nan)
    M = np.zeros(G, np.int32)
    for g in range(G):
        ps = np.array([p[g] for p, ok in reps if ok[g]])
        M[g] = len(ps)
        if len(ps):
            sig[g] = np.sqrt(((ps - ps.mean(0)) ** 2).mean(0))
    return sig, M
