"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (the FP32 kernel against exact FP64 arithmetic on identical inputs):
  model   per pixel |dM| <= 1e-5 * (stamp peak of |M|)
  chi^2   relative 1e-5
  grad    |dg_s| <= 1e-4 * sqrt(A_ss chi^2)   (Cauchy-Schwarz bound on |g_s|)
  J^T W J |dA_st| <= 1e-4 * sqrt(A_ss A_tt)
  fit     |dp| <= 1e-4 * max(|p|, s_p), s_p = 1 px / 1 rad / 1 sky unit
"""
import math

import numpy as np
import pytest

import oracle
from cases import Case, angle_diff, from_batch, pa_slots, psf_image, q_of_pa, scale_of
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


def assert_model_close(got, ref, rel=1e-5):
    got = np.asarray(got, np.float64)
    for g in range(ref.shape[0]):
        peak = np.abs(ref[g]).max()
        err = np.abs(got[g] - ref[g]).max()
        assert err <= rel * max(peak, 1e-30), (g, err, peak)


def oracle_inputs(case: Case):
    return dict(psf=case.psf.astype(np.float64), image=case.image.astype(np.float64),
                sigma=case.sigma.astype(np.float64), mask=case.mask)


# ---------------------------------------------------------------------------
# forward model
# ---------------------------------------------------------------------------

def test_model_small_batch(gm):
    b = synth.draw_small(seed=1, G=16)
    c = from_batch(b, at="truth")
    t = c.torch()
    got = _np(gm.gm_model(c.spec, t["params"], t["psf"], c.H, c.W))
    ref = oracle.model_images(c.spec, c.params, c.psf.astype(np.float64), c.H, c.W)
    assert_model_close(got, ref)


def _kinds_specs(H, W):
    """Three models (<= 16 slots each) that together use every profile kind."""
    a = synth.ModelSpec()
    a.add("sersic", "ser", H, W)
    a.add("ferrer", "fer", H, W)
    a.add("sky", "sky", H, W, convolve=False)
    b = synth.ModelSpec()
    b.add("expdisk", "exp", H, W)
    b.add("king", "kng", H, W, shared={"x0": 0, "y0": 1})
    b.add("gaussian", "gau", H, W, convolve=False, shared={"x0": 0, "y0": 1})
    c = synth.ModelSpec()
    c.add("moffat", "mof", H, W)
    c.add("gaussian", "gau", H, W)
    c.add("sky", "sky", H, W, convolve=False)
    return [a, b, c]


def _all_kinds_params(spec, H, W, rng):
    vals = {"x0": lambda: W / 2 + rng.uniform(-3, 3), "y0": lambda: H / 2 + rng.uniform(-3, 3),
            "q": lambda: rng.uniform(0.3, 1.0), "pa": lambda: rng.uniform(0, math.pi),
            "Ie": lambda: rng.uniform(1, 20), "I0": lambda: rng.uniform(1, 20), "Re": lambda: rng.uniform(2, 8),
            "n": lambda: rng.uniform(0.6, 4), "rs": lambda: rng.uniform(2, 6), "rout": lambda: rng.uniform(6, 15),
            "a": lambda: rng.uniform(1.2, 3), "b": lambda: rng.uniform(0, 1.5), "rc": lambda: rng.uniform(1, 3),
            "rt": lambda: rng.uniform(8, 16), "alpha": lambda: rng.uniform(1.5, 2.5),
            "fwhm": lambda: rng.uniform(1.5, 4), "Isky": lambda: rng.uniform(0, 3)}
    p = np.array([vals[n.split(".")[-1]]() for n in spec.names])
    if "mof.n" in spec.names:
        p[spec.slot("mof.n")] = rng.uniform(2, 5)
    return p


@pytest.mark.parametrize("which", [0, 1, 2])
@pytest.mark.parametrize("H,W,K", [(37, 45, 9), (64, 33, 1), (7, 9, 15), (1, 1, 1), (96, 70, 41)])
def test_model_every_profile_ragged(gm, H, W, K, which):
    rng = np.random.default_rng(H * 1000 + W + K + which)
    spec = _kinds_specs(H, W)[which]
    G = 3
    params = np.stack([_all_kinds_params(spec, H, W, rng) for _ in range(G)])
    psf = np.stack([psf_image("moffat", [K / 2, K / 2, 1, 0, 1, 2.0, 3.0], K) for _ in range(G)])
    c = Case(spec, params, psf, np.zeros((G, H, W)), np.ones((G, H, W)), None, H, W)
    t = c.torch()
    got, comp = gm.gm_model(spec, t["params"], t["psf"], H, W, components=True)
    ref = oracle.model_images(spec, params, psf.astype(np.float64), H, W)
    rcomp = oracle.component_images(spec, params, psf.astype(np.float64), H, W)
    assert_model_close(_np(got), ref)
    comp = _np(comp)
    for k in range(len(spec.components)):
        assert_model_close(comp[:, k], rcomp[:, k])


def test_model_delta_psf_and_empty_batch(gm):
    import torch
    H, W = 40, 50
    spec = synth.single_sersic_sky(H, W)
    p = np.array([[20.3, 21.1, 0.7, 0.4, 5.0, 4.0, 2.5, 1.0]])
    psf = np.ones((1, 1, 1), np.float32)
    got = _np(gm.gm_model(spec, torch.from_numpy(p).cuda(), torch.from_numpy(psf).cuda(), H, W))
    ref = oracle.component_image("sersic", p[0, :7], H, W) + 1.0
    assert_model_close(got, ref[None])
    empty = gm.gm_model(spec, torch.zeros((0, 8), dtype=torch.float64, device="cuda"),
                        torch.zeros((0, 15, 15), dtype=torch.float32, device="cuda"), H, W)
    assert empty.shape == (0, H, W)


# ---------------------------------------------------------------------------
# chi^2, gradient and J^T W J
# ---------------------------------------------------------------------------

def _oracle_normal(case: Case):
    """chi^2, g = J^T W r and A = J^T W J with the oracle's FD Jacobian (physical units)."""
    oi = oracle_inputs(case)
    M = oracle.model_images(case.spec, case.params, oi["psf"], case.H, case.W)
    J = oracle.jacobian(case.spec, case.params, oi["psf"], case.H, case.W)
    w = 1.0 / oi["sigma"] ** 2
    if case.mask is not None:
        w = w * (case.mask == 0)
    r = oi["image"] - M
    chi2 = (w * r * r).sum((1, 2))
    g = np.einsum("gfhw,ghw->gf", J, w * r)
    A = np.einsum("gfhw,gehw,ghw->gfe", J, J, w)
    return chi2, g, A


@pytest.mark.parametrize("at", ["init", "truth"])
def test_chi2_grad_jtj_small(gm, at):
    b = synth.draw_small(seed=2, G=16)
    c = from_batch(b, at=at)
    t = c.torch()
    chi2, grad, jtj = gm.gm_chi2_grad(c.spec, t["params"], t["image"], t["sigma"], t["mask"], t["psf"],
                                      want_grad=True, want_jtj=True)
    chi2, grad, jtj = _np(chi2), _np(grad), _np(jtj)
    rchi2, rg, rA = _oracle_normal(c)
    np.testing.assert_allclose(chi2, rchi2, rtol=1e-5)
    free = [i for i in range(c.spec.n_slots) if c.spec.free[i]]
    for gi in range(c.G):
        d = np.sqrt(np.diag(rA[gi]))
        gbound = 1e-4 * d * math.sqrt(rchi2[gi])
        assert (np.abs(grad[gi, free] - (-2.0 * rg[gi])) <= gbound).all(), gi
        Asub = jtj[gi][np.ix_(free, free)]
        assert (np.abs(Asub - rA[gi]) <= 1e-4 * np.outer(d, d)).all(), gi


def test_chi2_with_mask_and_contaminants(gm):
    b = synth.draw_sdss(seed=5, G=6, H=96, W=80, K=41)
    c = from_batch(b, at="init")
    t = c.torch()
    chi2, grad, _ = gm.gm_chi2_grad(c.spec, t["params"], t["image"], t["sigma"], t["mask"], t["psf"])
    rchi2, rg, rA = _oracle_normal(c)
    np.testing.assert_allclose(_np(chi2), rchi2, rtol=1e-5)
    free = [i for i in range(c.spec.n_slots) if c.spec.free[i]]
    grad = _np(grad)
    for gi in range(c.G):
        bound = 1e-4 * np.sqrt(np.diag(rA[gi])) * math.sqrt(rchi2[gi])
        assert (np.abs(grad[gi, free] + 2.0 * rg[gi]) <= bound).all(), gi


@pytest.mark.parametrize("draw,K", [(synth.draw_bulge_disk, 25), (synth.draw_bulge_disk, 51),
                                    (synth.draw_bulge_bar_nucleus, 41), (synth.draw_bulge_disk, 63),
                                    (synth.draw_sdss, 63)])
def test_chi2_grad_many_parameters(gm, draw, K):
    # 12 and 15 free parameters: 13 and 16 correlated channels in several channel-pair
    # passes, two pairs per thread in the reduction-heavy variant; and the largest PSF side the
    # calls take (63, on a 64 x 72 stamp: the PSF nearly as wide as the stamp)
    b = draw(seed=7, G=4, H=64, W=72, K=K)
    c = from_batch(b, at="init")
    t = c.torch()
    chi2, grad, jtj = gm.gm_chi2_grad(c.spec, t["params"], t["image"], t["sigma"], t["mask"], t["psf"],
                                      want_grad=True, want_jtj=True)
    chi2, grad, jtj = _np(chi2), _np(grad), _np(jtj)
    rchi2, rg, rA = _oracle_normal(c)
    np.testing.assert_allclose(chi2, rchi2, rtol=1e-5)
    free = [i for i in range(c.spec.n_slots) if c.spec.free[i]]
    for gi in range(c.G):
        d = np.sqrt(np.diag(rA[gi]))
        assert (np.abs(grad[gi, free] + 2.0 * rg[gi]) <= 1e-4 * d * math.sqrt(rchi2[gi])).all(), gi
        Asub = jtj[gi][np.ix_(free, free)]
        assert (np.abs(Asub - rA[gi]) <= 1e-4 * np.outer(d, d)).all(), gi


# ---------------------------------------------------------------------------
# Levenberg-Marquardt fits
# ---------------------------------------------------------------------------

def _compare_fits(spec, got, ref, tol=1e-4):
    """Indices compared and the worst parameter difference in units of the tolerance.

    A parameter agrees when |dp| <= 1e-4 max(|p|, s_p) (s_p = 1 px, 1 rad, 1 sky unit)."""
    s = np.maximum(np.abs(ref["params"]), scale_of(spec))
    both = (got["status"] == 1) & (ref["status"] == 1)
    # the same minimum: chi^2 within the parity tolerance
    same = both & (np.abs(got["chi2"] - ref["chi2"]) <= 1e-5 * ref["chi2"])
    diff = np.abs(got["params"] - ref["params"])
    for ps in pa_slots(spec):
        diff[:, ps] = angle_diff(got["params"][:, ps], ref["params"][:, ps])
        qs = q_of_pa(spec, ps)
        round_ = ref["params"][:, qs] > 0.95  # PA undefined for round profiles
        diff[round_, ps] = 0.0
    rel = diff / s
    return same, rel


def near_truth(c: Case, seed=0, frac=0.02):
    """A start inside the truth's basin: scale parameters within +-frac, centre within
    +-0.3 px, position angle within +-0.05 rad, sky within +-0.2."""
    rng = np.random.default_rng(seed)
    p = c.truth.copy()
    for i, name in enumerate(c.spec.names):
        role = name.split(".")[-1]
        u = rng.uniform(-1, 1, c.G)
        if role in ("x0", "y0"):
            p[:, i] += 0.3 * u
        elif role == "pa":
            p[:, i] += 0.05 * u
        elif role == "Isky":
            p[:, i] += 0.2 * u
        elif role == "q":
            p[:, i] = np.minimum(p[:, i] * (1 + frac * u), 1.0)
        else:
            p[:, i] *= 1 + frac * u
    return p


FIT_TIGHT = dict(tol=1e-12, xtol=1e-10, gtol=1e-13, max_iter=200)


def test_fit_near_truth_matches_oracle(gm):
    # inside the truth's basin the LM minimum is unique: every fit must agree
    b = synth.draw_small(seed=0, G=16)
    c = from_batch(b, at="truth")
    c.params = near_truth(c)
    t = c.torch()
    got = gm.gm_fit_batch(c.spec, t["params"], t["image"], t["sigma"], t["mask"], t["psf"],
                          gm.FitOptions(**FIT_TIGHT))
    got = {k: _np(v) for k, v in got.items()}
    oi = oracle_inputs(c)
    ref = oracle.fit(c.spec, c.params, oi["psf"], oi["image"], oi["sigma"], c.mask, oracle.FitOptions(**FIT_TIGHT))
    assert (ref["status"] == 1).all(), ref["status"]
    assert (got["status"] == 1).all(), got["status"]
    np.testing.assert_allclose(got["chi2"], ref["chi2"], rtol=1e-5)
    same, rel = _compare_fits(c.spec, got, ref)
    assert same.all()
    assert rel.max() <= 1e-4, rel.max(axis=1)
    np.testing.assert_array_equal(got["dof"], ref["dof"])
    free = np.array(c.spec.free, bool)
    sig_rel = np.abs(got["sigma_p"] - ref["sigma_p"])[:, free] / ref["sigma_p"][:, free]
    assert sig_rel.max() <= 1e-4, sig_rel.max()


def test_fit_default_start_same_minimum(gm):
    # from the default start (the centre of the prior ranges) every fit must reach the
    # oracle's minimum: the same chi^2 and the same parameters
    b = synth.draw_small(seed=0, G=16)
    c = from_batch(b, at="init")
    t = c.torch()
    got = gm.gm_fit_batch(c.spec, t["params"], t["image"], t["sigma"], t["mask"], t["psf"],
                          gm.FitOptions(**FIT_TIGHT))
    got = {k: _np(v) for k, v in got.items()}
    oi = oracle_inputs(c)
    ref = oracle.fit(c.spec, c.params, oi["psf"], oi["image"], oi["sigma"], c.mask, oracle.FitOptions(**FIT_TIGHT))
    same, rel = _compare_fits(c.spec, got, ref)
    assert same.all(), (got["status"], ref["status"], got["chi2"], ref["chi2"])
    assert rel[same].max() <= 1e-4, rel[same].max(axis=1)


def test_fit_through_q_one_matches_oracle(gm):
    # starts whose position angle is 90 degrees off: the fits cross q = 1, are rewritten
    # with q <= 1 at the end, and the covariance is carried through the rewrite
    b = synth.draw_small(seed=5, G=8)
    c = from_batch(b, at="truth")
    start = c.truth * 1.02
    start[:, 3] = c.truth[:, 3] + math.pi / 2
    start[:, 2] = np.minimum(c.truth[:, 2] * 1.2, 1.0)
    c.params = start
    t = c.torch()
    got = gm.gm_fit_batch(c.spec, t["params"], t["image"], t["sigma"], t["mask"], t["psf"],
                          gm.FitOptions(**FIT_TIGHT))
    got = {k: _np(v) for k, v in got.items()}
    oi = oracle_inputs(c)
    ref = oracle.fit(c.spec, c.params, oi["psf"], oi["image"], oi["sigma"], c.mask, oracle.FitOptions(**FIT_TIGHT))
    assert (got["params"][:, 2] <= 1.0).all() and (ref["params"][:, 2] <= 1.0).all()
    same, rel = _compare_fits(c.spec, got, ref)
    assert same.all(), (got["status"], ref["status"], got["chi2"], ref["chi2"])
    assert rel[same].max() <= 1e-4, rel[same].max(axis=1)
    free = np.array(c.spec.free, bool)
    sig_rel = np.abs(got["sigma_p"] - ref["sigma_p"])[same][:, free] / ref["sigma_p"][same][:, free]
    assert sig_rel.max() <= 1e-4, sig_rel.max()


def test_fit_status_codes(gm):
    b = synth.draw_small(seed=3, G=4)
    c = from_batch(b, at="init")
    c.sigma[0, 5, 7] = 0.0                 # bad sigma on a used pixel
    c.mask = np.zeros((4, c.H, c.W), np.uint8)
    c.mask[1] = 1                          # all pixels masked
    c.image[2, 0, 0] = np.nan
    c.mask[2, 0, 0] = 1                    # a NaN under the mask is harmless
    t = c.torch()
    got = gm.gm_fit_batch(c.spec, t["params"], t["image"], t["sigma"], t["mask"], t["psf"])
    st = _np(got["status"])
    assert st[0] == 6 and st[1] == 7 and st[2] == 1 and st[3] == 1, st
    oi = oracle_inputs(c)
    ref = oracle.fit(c.spec, c.params, oi["psf"], oi["image"], oi["sigma"], c.mask)
    np.testing.assert_array_equal(st, ref["status"])


# ---------------------------------------------------------------------------
# adjoint gradient (gm_grad_adjoint) and the torch autograd function
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("draw,G,H,W,K", [(synth.draw_small, 7, 64, 64, 15),
                                          (synth.draw_bulge_bar_nucleus, 5, 96, 96, 41),
                                          (synth.draw_bulge_disk, 4, 64, 72, 25),
                                          (synth.draw_bulge_bar_nucleus, 3, 64, 72, 63)])
def test_grad_adjoint_matches_normal_equations(gm, draw, G, H, W, K):
    # the adjoint gradient (two correlations) against the 1+P-channel pass, odd G included
    b = draw(seed=9, G=G) if draw is synth.draw_small else draw(seed=9, G=G, H=H, W=W, K=K)
    c = from_batch(b, at="init")
    t = c.torch()
    chi2, grad = gm.gm_grad_adjoint(c.spec, t["params"], t["image"], t["sigma"], t["mask"], t["psf"])
    rchi2, rgrad, rjtj = gm.gm_chi2_grad(c.spec, t["params"], t["image"], t["sigma"], t["mask"], t["psf"],
                                         want_grad=True, want_jtj=True)
    chi2, grad, rchi2, rgrad, rjtj = map(_np, (chi2, grad, rchi2, rgrad, rjtj))
    np.testing.assert_allclose(chi2, rchi2, rtol=1e-5)
    for gi in range(c.G):
        bound = 1e-4 * np.sqrt(np.abs(np.diag(rjtj[gi]))) * math.sqrt(rchi2[gi])
        assert (np.abs(grad[gi] - rgrad[gi]) <= bound + 1e-300).all(), gi


def test_grad_adjoint_kernel_times(gm):
    # the library's CUDA events around the pass's kernel groups: all positive, summing to
    # about the call's own event time
    import torch
    c = from_batch(synth.draw_bulge_bar_nucleus(seed=4, G=64), at="init")
    t = c.torch()
    call = lambda: gm.gm_grad_adjoint(c.spec, t["params"], t["image"], t["sigma"], t["mask"], t["psf"])
    call()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    call()
    e1.record()
    st = gm.gm_grad_adjoint_last_stats()
    torch.cuda.synchronize()
    assert all(v > 0 for v in st.values()), st
    assert sum(st.values()) <= e0.elapsed_time(e1) * 1.05 + 0.05, (st, e0.elapsed_time(e1))


def test_grad_adjoint_vs_oracle_finite_differences(gm):
    # 64 galaxies of the bulge + bar + nucleus model (96x96, K = 41): d chi^2 / dp against
    # central FP64 finite differences of the oracle's chi^2 (relative step 1e-6)
    b = synth.draw_bulge_bar_nucleus(seed=31, G=64)
    c = from_batch(b, at="init")
    t = c.torch()
    chi2, grad = gm.gm_grad_adjoint(c.spec, t["params"], t["image"], t["sigma"], t["mask"], t["psf"])
    chi2, grad = _np(chi2), _np(grad)
    rchi2, rg, rA = _oracle_normal(c)
    np.testing.assert_allclose(chi2, rchi2, rtol=1e-5)
    free = [i for i in range(c.spec.n_slots) if c.spec.free[i]]
    for gi in range(c.G):
        bound = 1e-4 * np.sqrt(np.diag(rA[gi])) * math.sqrt(rchi2[gi])
        assert (np.abs(grad[gi, free] + 2.0 * rg[gi]) <= bound).all(), gi


@pytest.mark.parametrize("H,W,K", [(37, 45, 9), (7, 9, 15), (64, 33, 1), (96, 70, 41), (100, 45, 25)])
def test_normal_equations_and_adjoint_at_ragged_sizes(gm, H, W, K):
    # stamps that end inside a tile, a 1x1 PSF and a PSF larger than the stamp, with 10% of
    # the pixels masked: chi^2 and d chi^2/dp of both passes, and J^T W J of the normal
    # equations, against the oracle (5 galaxies: the last lane pair of the adjoint holds one).
    # The two taller stamps have a tile row away from the top and bottom whose left and
    # right tiles run by columns, skipping the taps outside the stamp (some of their warps
    # lie wholly outside it)
    c = from_batch(synth.draw_small(seed=H * 7 + W + K, G=5, H=H, W=W, K=K), at="init")
    c.mask = (np.random.default_rng(K + 1).random((c.G, H, W)) < 0.1).astype(np.uint8)
    t = c.torch()
    chi2, grad, jtj = map(_np, gm.gm_chi2_grad(c.spec, t["params"], t["image"], t["sigma"], t["mask"], t["psf"],
                                               want_grad=True, want_jtj=True))
    achi2, agrad = map(_np, gm.gm_grad_adjoint(c.spec, t["params"], t["image"], t["sigma"], t["mask"], t["psf"]))
    rchi2, rg, rA = _oracle_normal(c)
    free = [i for i in range(c.spec.n_slots) if c.spec.free[i]]
    for g in range(c.G):
        d = np.sqrt(np.diag(rA[g]))
        bound = 1e-4 * d * math.sqrt(rchi2[g])
        for name, x2, gr in (("normal", chi2, grad), ("adjoint", achi2, agrad)):
            assert abs(x2[g] - rchi2[g]) <= 1e-5 * rchi2[g], (name, g)
            assert (np.abs(gr[g, free] + 2.0 * rg[g]) <= bound).all(), (name, g)
        assert (np.abs(jtj[g][np.ix_(free, free)] - rA[g]) <= 1e-4 * np.outer(d, d)).all(), g


def test_grad_adjoint_block_ranges_across_pairs(gm):
    # 301 galaxies of 96x96 (K = 41): 151 lane pairs x 9 tiles = 1,359 tiles over a few
    # hundred blocks, so a block's contiguous range starts and ends inside pairs and
    # restages the PSF pair where it crosses into the next one; the last pair holds one
    # galaxy.  Slots repeat 7 oracle-rendered sources (an odd count: every pair mixes two
    # different galaxies); sampled slots against the oracle for their source.
    import torch
    S7, G = 7, 301
    c = from_batch(synth.draw_bulge_bar_nucleus(seed=41, G=S7), at="init")
    src = np.arange(G) % S7
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a[src])).cuda()
    chi2, grad = gm.gm_grad_adjoint(c.spec, t(c.params), t(c.image), t(c.sigma), t(c.mask), t(c.psf))
    chi2, grad = _np(chi2), _np(grad)
    rchi2, rg, rA = _oracle_normal(c)
    free = [i for i in range(c.spec.n_slots) if c.spec.free[i]]
    for g in (0, 1, 2, 17, 18, 149, 150, 151, 298, 299, 300):
        s = src[g]
        assert abs(chi2[g] - rchi2[s]) <= 1e-5 * rchi2[s], g
        d = np.sqrt(np.diag(rA[s]))
        assert (np.abs(grad[g, free] + 2.0 * rg[s]) <= 1e-4 * d * math.sqrt(rchi2[s])).all(), g


def test_chi2_autograd_function_and_adam(gm):
    import torch
    b = synth.draw_small(seed=13, G=6)
    c = from_batch(b, at="init")
    t = c.torch()
    f = gm.Chi2(c.spec, t["image"], t["sigma"], t["mask"], t["psf"])
    p = t["params"].clone().requires_grad_(True)
    loss = f(p).sum()
    loss.backward()
    _, grad = gm.gm_grad_adjoint(c.spec, t["params"], t["image"], t["sigma"], t["mask"], t["psf"])
    np.testing.assert_allclose(_np(p.grad), _np(grad), rtol=0, atol=0)
    # the paper's fitting mode: a torch optimiser stepping the parameters on chi^2
    q = t["params"].clone()
    free = torch.tensor(c.spec.free, device=q.device)
    u = q.clone().requires_grad_(True)
    opt = torch.optim.Adam([u], lr=0.02)
    first = None
    for _ in range(30):
        opt.zero_grad()
        val = f(torch.where(free, u, q)).sum()
        first = float(val.detach()) if first is None else first
        val.backward()
        opt.step()
    assert float(f(torch.where(free, u, q)).sum().detach()) < first


@pytest.mark.parametrize("n", [0.15, 0.2004, 3.00123, 10.19, 10.5, 11.5])
def test_sersic_index_on_both_sides_of_the_nu_table(gm, n):
    # the set-up interpolates nu_n and d nu/dn from FP64 nodes over n in [0.2, 10.2] and
    # solves directly outside it: model, chi^2, gradient and J^T W J match the oracle either
    # way (values between nodes and beyond both ends, bounds widened to 0.1..12)
    H = W = 48
    spec = synth.ModelSpec().add("sersic", "ser", H, W).add("sky", "sky", H, W, convolve=False)
    ns = spec.slot("ser.n")
    spec.lo[ns], spec.hi[ns] = 0.1, 12.0
    p = np.zeros((1, spec.n_slots))
    for name, v in (("ser.x0", W / 2 + 0.3), ("ser.y0", H / 2 - 0.2), ("ser.q", 0.7), ("ser.pa", 0.8),
                    ("ser.Ie", 5.0), ("ser.Re", 6.0), ("ser.n", n), ("sky.Isky", 1.0)):
        p[0, spec.slot(name)] = v
    truth = p.copy()
    truth[0, ns] = n * 1.03
    truth[0, spec.slot("ser.Re")] = 6.3
    psf = psf_image("gaussian", synth.psf_params("gaussian", np.array([2.0]), 9)[0], 9)[None]
    M = oracle.model_images(spec, truth, psf.astype(np.float64), H, W)
    rng = np.random.default_rng(4)
    image = (M + rng.normal(size=M.shape)).astype(np.float32)
    c = Case(spec, p, psf, image, np.ones_like(image), None, H, W)
    t = c.torch()
    model = _np(gm.gm_model(spec, t["params"], t["psf"], H, W))
    assert_model_close(model, oracle.model_images(spec, p, psf.astype(np.float64), H, W))
    chi2, grad, jtj = gm.gm_chi2_grad(spec, t["params"], t["image"], t["sigma"], None, t["psf"],
                                      want_grad=True, want_jtj=True)
    chi2, grad, jtj = _np(chi2), _np(grad), _np(jtj)
    rchi2, rg, rA = _oracle_normal(c)
    np.testing.assert_allclose(chi2, rchi2, rtol=1e-5)
    free = [i for i in range(spec.n_slots) if spec.free[i]]
    d = np.sqrt(np.diag(rA[0]))
    assert (np.abs(grad[0, free] + 2.0 * rg[0]) <= 1e-4 * d * math.sqrt(rchi2[0])).all()
    assert (np.abs(jtj[0][np.ix_(free, free)] - rA[0]) <= 1e-4 * np.outer(d, d)).all()
