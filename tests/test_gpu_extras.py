"""Parity of the paper's extra components and fitting modes with the FP64 oracle:
the tilted sky of Eq. new_sky_I, magnitudes instead of amplitudes, boxiness,
bootstrap uncertainties and the gradient-descent (Adam) fit."""
import math

import numpy as np
import pytest

import oracle
from cases import Case, psf_image, scale_of
from paper_2404_07780_b300 import synth

pytestmark = pytest.mark.gpu


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


def _np(t):
    return None if t is None else t.detach().cpu().numpy()


def _case(spec, params, H, W, K, seed, noise=True):
    """Render spec at params with the oracle (Moffat PSF, FWHM 1.5), add the recipe's noise."""
    G = params.shape[0]
    psf = np.stack([psf_image("moffat", [K / 2, K / 2, 1, 0, 1, 1.5, 3.0], K) for _ in range(G)])
    M = oracle.model_images(spec, params, psf.astype(np.float64), H, W)
    z = np.random.default_rng(seed).standard_normal(M.shape) if noise else np.zeros(M.shape)
    D, S = synth.noisy_image(M, z)
    return Case(spec, params, psf, D, S, None, H, W, init=params, truth=params)


def _normal_oracle(c):
    psf, img, sig = c.psf.astype(np.float64), c.image.astype(np.float64), c.sigma.astype(np.float64)
    M = oracle.model_images(c.spec, c.params, psf, c.H, c.W)
    J = oracle.jacobian(c.spec, c.params, psf, c.H, c.W)
    w = 1.0 / sig ** 2
    r = img - M
    return (w * r * r).sum((1, 2)), np.einsum("gfhw,ghw->gf", J, w * r), np.einsum("gfhw,gehw,ghw->gfe", J, J, w)


def _check_normal(gm, c):
    t = c.torch()
    chi2, grad, jtj = (_np(x) for x in gm.gm_chi2_grad(c.spec, t["params"], t["image"], t["sigma"], t["mask"],
                                                       t["psf"], want_grad=True, want_jtj=True))
    rc2, rg, rA = _normal_oracle(c)
    np.testing.assert_allclose(chi2, rc2, rtol=1e-5)
    free = [i for i in range(c.spec.n_slots) if c.spec.free[i]]
    for g in range(c.G):
        d = np.sqrt(np.diag(rA[g]))
        assert (np.abs(grad[g, free] + 2.0 * rg[g]) <= 1e-4 * d * math.sqrt(rc2[g]) + 1e-300).all(), g
        assert (np.abs(jtj[g][np.ix_(free, free)] - rA[g]) <= 1e-4 * np.outer(d, d) + 1e-300).all(), g


def _tilted_spec(H, W, convolve_sky=False):
    return (synth.ModelSpec().add("sersic", "bulge", H, W)
            .add("tsky", "sky", H, W, convolve=convolve_sky))


def _tilted_params(G, H, W, seed):
    g = np.random.default_rng(seed)
    return np.stack([W / 2 + g.uniform(-2, 2, G), H / 2 + g.uniform(-2, 2, G), g.uniform(0.4, 0.9, G),
                     g.uniform(0, math.pi, G), 10 ** g.uniform(1, 2, G), g.uniform(3, 8, G), g.uniform(0.8, 3, G),
                     g.uniform(1, 4, G), g.uniform(-0.05, 0.05, G), g.uniform(-0.05, 0.05, G)], 1)


@pytest.mark.parametrize("convolve_sky", [False, True])
def test_tilted_sky_model_and_normal_equations(gm, convolve_sky):
    H, W, K = 72, 56, 25
    spec = _tilted_spec(H, W, convolve_sky)
    c = _case(spec, _tilted_params(5, H, W, 1), H, W, K, seed=2)
    t = c.torch()
    got = _np(gm.gm_model(spec, t["params"], t["psf"], H, W))
    ref = oracle.model_images(spec, c.params, c.psf.astype(np.float64), H, W)
    for g in range(c.G):
        assert np.abs(got[g] - ref[g]).max() <= 1e-5 * np.abs(ref[g]).max()
    c.params = c.params * np.array([1.01, 0.99, 1.02, 1.0, 0.95, 1.05, 1.02, 0.9, 1.1, 0.8])  # off the truth
    _check_normal(gm, c)


def test_tilted_sky_fit_recovers_the_plane(gm):
    H, W, K = 64, 64, 25
    spec = _tilted_spec(H, W)
    truth = _tilted_params(6, H, W, 3)
    c = _case(spec, truth, H, W, K, seed=4)
    start = truth.copy()
    start[:, 7:] = [2.5, 0.0, 0.0]  # flat start for the sky plane
    start[:, 4] *= 1.05
    t = c.torch()
    import torch
    opts = dict(tol=1e-12, xtol=1e-10, gtol=1e-13, max_iter=200)
    got = {k: _np(v) for k, v in gm.gm_fit_batch(spec, torch.from_numpy(start).cuda(), t["image"], t["sigma"], None,
                                                 t["psf"], gm.FitOptions(**opts)).items()}
    ref = oracle.fit(spec, start, c.psf.astype(np.float64), c.image.astype(np.float64), c.sigma.astype(np.float64),
                     None, oracle.FitOptions(**opts))
    assert (got["status"] == 1).all() and (ref["status"] == 1).all()
    np.testing.assert_allclose(got["chi2"], ref["chi2"], rtol=1e-5)
    tol = 1e-4 * np.maximum(np.abs(ref["params"]), scale_of(spec))
    d = np.abs(got["params"] - ref["params"])
    d[:, 3] = np.minimum(d[:, 3] % math.pi, math.pi - d[:, 3] % math.pi)
    assert (d <= tol).all(), (d / tol).max(0)
    # the fitted plane is the drawn one within its error bars
    assert (np.abs(got["params"][:, 8:] - truth[:, 8:]) <= 5 * got["sigma_p"][:, 8:]).all()


# ---------------------------------------------------------------------------
# magnitudes instead of amplitudes
# ---------------------------------------------------------------------------

def _mag_spec(H, W, which):
    """Profiles with a magnitude relation, in magnitudes (zero point 22.5), plus sky: a bulge,
    disk and bar (Sersic, exponential, Ferrer), or a galaxy with a nucleus next to a star
    (Sersic, Gaussian, Moffat)."""
    s = synth.ModelSpec()
    s.add("sersic", "bulge", H, W, mag_zero=22.5)
    if which == "bulge_disk_bar":
        s.add("expdisk", "disk", H, W, shared={"x0": 0, "y0": 1}, mag_zero=22.5)
        s.add("ferrer", "bar", H, W, shared={"x0": 0, "y0": 1}, fixed=("a",), mag_zero=22.5)
    else:
        s.add("gaussian", "nuc", H, W, shared={"x0": 0, "y0": 1}, fixed=("q", "pa"), mag_zero=22.5)
        s.add("moffat", "star", H, W, fixed=("q", "pa"), mag_zero=22.5)
    s.add("sky", "sky", H, W, convolve=False)
    if which == "bulge_disk_bar":
        s.free[s.slot("sky.Isky")] = False  # 16 free parameters at most
    return s


def _mag_params(spec, G, H, W, seed):
    g = np.random.default_rng(seed)
    vals = {"bulge.x0": W / 2 + g.uniform(-1, 1, G), "bulge.y0": H / 2 + g.uniform(-1, 1, G),
            "bulge.q": g.uniform(0.6, 0.9, G), "bulge.pa": g.uniform(0.2, 2.8, G), "bulge.mag": g.uniform(15, 16, G),
            "bulge.Re": g.uniform(2, 4, G), "bulge.n": g.uniform(1.5, 3, G),
            "disk.q": g.uniform(0.4, 0.7, G), "disk.pa": g.uniform(0.2, 2.8, G), "disk.mag": g.uniform(14.5, 15.5, G),
            "disk.rs": g.uniform(5, 8, G),
            "bar.q": g.uniform(0.25, 0.4, G), "bar.pa": g.uniform(0.2, 2.8, G), "bar.mag": g.uniform(16, 17, G),
            "bar.rout": g.uniform(8, 12, G), "bar.a": np.full(G, 2.0), "bar.b": g.uniform(0.2, 1.0, G),
            "nuc.q": np.ones(G), "nuc.pa": np.zeros(G), "nuc.mag": g.uniform(17, 18, G), "nuc.fwhm": g.uniform(1.5, 2.5, G),
            "star.x0": W / 2 + g.uniform(12, 16, G), "star.y0": H / 2 - g.uniform(10, 14, G), "star.q": np.ones(G),
            "star.pa": np.zeros(G), "star.mag": g.uniform(17, 18, G), "star.fwhm": g.uniform(2, 3, G),
            "star.n": g.uniform(2.5, 4, G), "sky.Isky": g.uniform(1, 3, G)}
    return np.stack([vals[n] for n in spec.names], 1)


@pytest.mark.parametrize("which", ["bulge_disk_bar", "nucleus_star"])
def test_magnitude_model_and_normal_equations(gm, which):
    H, W, K = 64, 72, 25
    spec = _mag_spec(H, W, which)
    p = _mag_params(spec, 3, H, W, 5)
    c = _case(spec, p, H, W, K, seed=6)
    t = c.torch()
    got = _np(gm.gm_model(spec, t["params"], t["psf"], H, W))
    ref = oracle.model_images(spec, c.params, c.psf.astype(np.float64), H, W)
    for g in range(c.G):
        assert np.abs(got[g] - ref[g]).max() <= 1e-5 * np.abs(ref[g]).max()
    # away from the truth: every chain-rule term of every profile contributes
    c.params = p + np.random.default_rng(7).normal(0, 0.02, p.shape) * np.maximum(np.abs(p), 0.1) * np.array(spec.free)
    _check_normal(gm, c)


def test_magnitude_fit_matches_oracle(gm):
    import torch
    H, W, K = 64, 64, 25
    spec = synth.ModelSpec().add("sersic", "bulge", H, W, mag_zero=22.5).add("sky", "sky", H, W, convolve=False)
    g = np.random.default_rng(8)
    G = 6
    truth = np.stack([W / 2 + g.uniform(-1, 1, G), H / 2 + g.uniform(-1, 1, G), g.uniform(0.4, 0.9, G),
                      g.uniform(0.2, 2.8, G), g.uniform(15, 17, G), g.uniform(3, 8, G), g.uniform(1, 3, G),
                      g.uniform(1, 3, G)], 1)
    c = _case(spec, truth, H, W, K, seed=9)
    start = truth * (1 + 0.03 * g.uniform(-1, 1, truth.shape))
    start[:, 2] = np.minimum(start[:, 2], 0.99)
    t = c.torch()
    opts = dict(tol=1e-12, xtol=1e-10, gtol=1e-13, max_iter=200)
    got = {k: _np(v) for k, v in gm.gm_fit_batch(spec, torch.from_numpy(start).cuda(), t["image"], t["sigma"], None,
                                                 t["psf"], gm.FitOptions(**opts)).items()}
    ref = oracle.fit(spec, start, c.psf.astype(np.float64), c.image.astype(np.float64), c.sigma.astype(np.float64),
                     None, oracle.FitOptions(**opts))
    assert (got["status"] == 1).all() and (ref["status"] == 1).all()
    np.testing.assert_allclose(got["chi2"], ref["chi2"], rtol=1e-5)
    tol = 1e-4 * np.maximum(np.abs(ref["params"]), scale_of(spec))
    d = np.abs(got["params"] - ref["params"])
    d[:, 3] = np.minimum(d[:, 3] % math.pi, math.pi - d[:, 3] % math.pi)
    assert (d <= tol).all(), (d / tol).max(0)
    np.testing.assert_allclose(got["sigma_p"][:, 4], ref["sigma_p"][:, 4], rtol=1e-4)  # magnitude error bars


def test_magnitude_for_king_is_unsupported(gm):
    import torch
    spec = synth.ModelSpec().add("king", "gc", 16, 16, mag_zero=22.5)
    p = torch.tensor([[8.0, 8.0, 1.0, 0.0, 18.0, 2.0, 10.0, 2.0]], dtype=torch.float64, device="cuda")
    psf = torch.ones((1, 1, 1), device="cuda")
    with pytest.raises(gm.GMError, match="no magnitude relation"):
        gm.gm_model(spec, p, psf, 16, 16)


# ---------------------------------------------------------------------------
# gradient-descent (Adam) fit
# ---------------------------------------------------------------------------

def test_adam_fit_follows_the_oracle(gm):
    import torch
    H, W, K = 48, 48, 15
    b = synth.draw_small(seed=41, G=5, H=H, W=W, K=K)
    spec = b.spec
    c = _case(spec, b.truth, H, W, K, seed=42)
    t = c.torch()
    start = torch.from_numpy(b.init).cuda()
    lr, n = 0.02, 12
    got = {k: _np(v) for k, v in gm.gm_fit_adam(spec, start, t["image"], t["sigma"], None, t["psf"], n_iter=n,
                                                lr=lr).items()}
    rp, rc2 = oracle.fit_adam(spec, b.init, c.psf.astype(np.float64), c.image.astype(np.float64),
                              c.sigma.astype(np.float64), None, n_iter=n, lr=lr)
    np.testing.assert_allclose(got["chi2"], rc2, rtol=1e-5)
    # each step moves a parameter by at most lr * scale; FP32 gradients change the step ratios by ~1e-5
    scale = np.where(np.array(spec.log), np.abs(rp), np.maximum(np.abs(b.init), 1.0))
    d = np.abs(got["params"] - rp)
    for s in [i for i, nm in enumerate(spec.names) if nm.endswith(".pa")]:
        d[:, s] = np.minimum(d[:, s] % math.pi, math.pi - d[:, s] % math.pi)
    assert (d <= 1e-3 * lr * scale * n + 1e-9).all(), (d / (lr * scale * n)).max()
    # gradient descent lowers chi^2 from the start
    c2_0 = oracle.chi2(spec, b.init, c.psf.astype(np.float64), c.image.astype(np.float64), c.sigma.astype(np.float64))
    assert (got["chi2"] < c2_0).all()


# ---------------------------------------------------------------------------
# bootstrap uncertainties
# ---------------------------------------------------------------------------

def test_bootstrap_counts_are_bit_exact(gm):
    import torch
    G, H, W = 3, 40, 50
    rng = np.random.default_rng(51)
    mask = (rng.uniform(size=(G, H, W)) < 0.2).astype(np.uint8)
    img = torch.zeros((G, H, W), device="cuda")
    sig = torch.ones((G, H, W), device="cuda")
    psf = torch.ones((G, 1, 1), device="cuda")
    spec = synth.single_sersic_sky(H, W)
    for b in (0, 7):
        got = _np(gm.gm_bootstrap_counts(spec, img, sig, torch.from_numpy(mask).cuda(), psf, seed=99, replicate=b))
        for g in range(G):
            np.testing.assert_array_equal(got[g], oracle.bootstrap_counts(mask[g], 99, g, b).astype(np.int32))


def test_bootstrap_error_bars_match_oracle(gm):
    import torch
    H, W, K = 40, 40, 9
    b = synth.draw_small(seed=52, G=3, H=H, W=W, K=K)
    b.truth[:, 4] = np.maximum(b.truth[:, 4], 20.0)  # bright enough for a well-defined minimum
    c = _case(b.spec, b.truth, H, W, K, seed=53)
    opts = dict(tol=1e-12, xtol=1e-10, gtol=1e-13, max_iter=200)
    best = oracle.fit(b.spec, b.truth, c.psf.astype(np.float64), c.image.astype(np.float64),
                      c.sigma.astype(np.float64), None, oracle.FitOptions(**opts))["params"]
    t = c.torch()
    sig, nok = gm.gm_bootstrap(b.spec, torch.from_numpy(best).cuda(), t["image"], t["sigma"], None, t["psf"], n_boot=4,
                               seed=5, opts=gm.FitOptions(**opts))
    sig, nok = _np(sig), _np(nok)
    rsig, rM = oracle.bootstrap(b.spec, best, c.psf.astype(np.float64), c.image.astype(np.float64),
                                c.sigma.astype(np.float64), None, n_boot=4, seed=5, opts=oracle.FitOptions(**opts))
    np.testing.assert_array_equal(nok, rM)
    free = np.array(b.spec.free, bool)
    # every replicate's refit matches the oracle's to the fit tolerance; the spread of 4 refits inherits it
    tol = 0.05 * rsig[:, free] + 1e-4 * np.maximum(np.abs(best[:, free]), 1.0)
    assert (np.abs(sig[:, free] - rsig[:, free]) <= tol).all(), (np.abs(sig - rsig)[:, free] / tol).max()
    assert (sig[:, ~free] == 0).all()


# ---------------------------------------------------------------------------
# boxiness
# ---------------------------------------------------------------------------

def _boxy_spec(H, W, mag):
    m0 = 22.5 if mag else None
    s = synth.ModelSpec()
    s.add("sersic", "bulge", H, W, mag_zero=m0, boxy=True)
    s.add("expdisk", "disk", H, W, shared={"x0": 0, "y0": 1}, mag_zero=m0, boxy=True)
    s.add("sky", "sky", H, W, convolve=False)
    return s


def _boxy_params(spec, G, H, W, seed, mag):
    g = np.random.default_rng(seed)
    amp_b = g.uniform(15, 16, G) if mag else 10 ** g.uniform(1.5, 2.5, G)
    amp_d = g.uniform(14.5, 15.5, G) if mag else 10 ** g.uniform(0.8, 1.5, G)
    vals = {"bulge.x0": W / 2 + g.uniform(-1, 1, G), "bulge.y0": H / 2 + g.uniform(-1, 1, G),
            "bulge.q": g.uniform(0.5, 0.8, G), "bulge.pa": g.uniform(0.2, 2.8, G),
            "bulge.mag" if mag else "bulge.Ie": amp_b, "bulge.Re": g.uniform(3, 5, G), "bulge.n": g.uniform(1.5, 3, G),
            "bulge.B": g.uniform(-0.5, 1.0, G),
            "disk.q": g.uniform(0.3, 0.6, G), "disk.pa": g.uniform(0.2, 2.8, G),
            "disk.mag" if mag else "disk.I0": amp_d, "disk.rs": g.uniform(6, 9, G), "disk.B": g.uniform(-0.5, 1.0, G),
            "sky.Isky": g.uniform(1, 3, G)}
    return np.stack([vals[n] for n in spec.names], 1)


@pytest.mark.parametrize("mag", [False, True])
def test_boxy_model_and_normal_equations(gm, mag):
    H, W, K = 64, 56, 25
    spec = _boxy_spec(H, W, mag)
    p = _boxy_params(spec, 3, H, W, 61, mag)
    c = _case(spec, p, H, W, K, seed=62)
    t = c.torch()
    got = _np(gm.gm_model(spec, t["params"], t["psf"], H, W))
    ref = oracle.model_images(spec, c.params, c.psf.astype(np.float64), H, W)
    for g in range(c.G):
        assert np.abs(got[g] - ref[g]).max() <= 1e-5 * np.abs(ref[g]).max()
    c.params = p + np.random.default_rng(63).normal(0, 0.02, p.shape) * np.maximum(np.abs(p), 0.1)
    _check_normal(gm, c)


def test_boxy_fit_matches_oracle(gm):
    import torch
    H, W, K = 64, 64, 15
    spec = synth.ModelSpec().add("sersic", "bulge", H, W, boxy=True).add("sky", "sky", H, W, convolve=False)
    g = np.random.default_rng(64)
    G = 5
    truth = np.stack([W / 2 + g.uniform(-1, 1, G), H / 2 + g.uniform(-1, 1, G), g.uniform(0.4, 0.7, G),
                      g.uniform(0.2, 2.8, G), 10 ** g.uniform(1.5, 2, G), g.uniform(5, 9, G), g.uniform(0.8, 2, G),
                      g.uniform(-0.6, 1.5, G), g.uniform(1, 3, G)], 1)
    c = _case(spec, truth, H, W, K, seed=65)
    start = truth * (1 + 0.03 * g.uniform(-1, 1, truth.shape))
    start[:, 7] = 0.0  # an ellipse to start from
    t = c.torch()
    opts = dict(tol=1e-12, xtol=1e-10, gtol=1e-13, max_iter=200)
    got = {k: _np(v) for k, v in gm.gm_fit_batch(spec, torch.from_numpy(start).cuda(), t["image"], t["sigma"], None,
                                                 t["psf"], gm.FitOptions(**opts)).items()}
    ref = oracle.fit(spec, start, c.psf.astype(np.float64), c.image.astype(np.float64), c.sigma.astype(np.float64),
                     None, oracle.FitOptions(**opts))
    assert (got["status"] == 1).all() and (ref["status"] == 1).all()
    np.testing.assert_allclose(got["chi2"], ref["chi2"], rtol=1e-5)
    tol = 1e-4 * np.maximum(np.abs(ref["params"]), scale_of(spec))
    d = np.abs(got["params"] - ref["params"])
    d[:, 3] = np.minimum(d[:, 3] % math.pi, math.pi - d[:, 3] % math.pi)
    assert (d <= tol).all(), (d / tol).max(0)
    # the fitted boxiness is the drawn one within its error bar
    assert (np.abs(got["params"][:, 7] - truth[:, 7]) <= 5 * got["sigma_p"][:, 7]).all()
