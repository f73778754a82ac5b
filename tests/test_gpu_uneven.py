"""Uneven batches (per-galaxy stamp and PSF sizes, gm_batch.geom) through the C ABI.

Parity with the FP64 oracle galaxy by galaxy (the oracle fits and renders
one-galaxy batches of each size), at the tolerances of test_gpu_parity, and
bit-for-bit agreement with the equal-stamp path: an uneven batch that
interleaves two equal-stamp batches must give exactly the numbers each of
them gives alone, because every galaxy's tiles, tile order and reductions are
the same whichever batch it sits in.
"""
import math

import numpy as np
import pytest

import oracle
from cases import Case, UnevenCase, from_batch, uneven_from
from paper_2404_07780_b300 import synth

pytestmark = pytest.mark.gpu

# sizes that span several tiles with ragged tails, odd widths (a pad column in
# the pair planes), a PSF wider than its stamp, a one-pixel stamp with a delta
# PSF, and every PSF side class of the SDSS-like workloads
MIXED = [(48, 48, 25), (37, 45, 9), (64, 33, 1), (7, 9, 15), (1, 1, 1), (96, 70, 41), (33, 65, 51),
         (128, 40, 31), (70, 96, 41)]


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


def _peak_close(got, ref, rel=1e-5):
    peak = np.abs(ref).max()
    err = np.abs(np.asarray(got, np.float64) - ref).max()
    assert err <= rel * max(peak, 1e-30), (err, peak)


def test_uneven_model_matches_oracle(gm):
    rb = synth.draw_uneven_sersic(11, MIXED)
    c = uneven_from(rb, at="truth")
    t = c.torch()
    model, comp = gm.gm_model(c.spec, t["params"], t["psf"], components=True, geom=c.geom)
    per_gal = c.split(_np(model))
    per_comp = c.split(_np(comp), per_pixel=len(c.spec.components))
    for g, cg in enumerate(c.cases):
        ref = oracle.model_images(cg.spec, cg.params, cg.psf.astype(np.float64), cg.H, cg.W)[0]
        _peak_close(per_gal[g][0], ref)
        parts = oracle.component_images(cg.spec, cg.params, cg.psf.astype(np.float64), cg.H, cg.W)[0]
        for k in range(len(c.spec.components)):
            _peak_close(per_comp[g][k], parts[k])


def _oracle_normal_one(cg):
    psf, image, sigma = cg.psf.astype(np.float64), cg.image.astype(np.float64), cg.sigma.astype(np.float64)
    M = oracle.model_images(cg.spec, cg.params, psf, cg.H, cg.W)
    J = oracle.jacobian(cg.spec, cg.params, psf, cg.H, cg.W)
    w = 1.0 / sigma ** 2
    if cg.mask is not None:
        w = w * (cg.mask == 0)
    r = image - M
    return (w * r * r).sum(), np.einsum("fhw,hw->f", J[0], (w * r)[0]), np.einsum("fhw,ehw,hw->fe", J[0], J[0], w[0])


@pytest.mark.parametrize("which", ["sersic", "bulge_disk"])
def test_uneven_chi2_grad_jtj_matches_oracle(gm, which):
    if which == "sersic":
        rb = synth.draw_uneven_sersic(12, MIXED, mask_frac=0.05)
    else:
        # 12 free parameters: 13 correlated channels in several passes, two pairs per thread
        rb = synth.draw_uneven_bulge_disk(seed=13, G=5, sides=(40, 64, 72), ks=(25, 31, 51))
    c = uneven_from(rb, at="init")
    t = c.torch()
    chi2, grad, jtj = gm.gm_chi2_grad(c.spec, t["params"], t["image"], t["sigma"], t["mask"], t["psf"],
                                      want_grad=True, want_jtj=True, geom=c.geom)
    chi2, grad, jtj = _np(chi2), _np(grad), _np(jtj)
    free = [i for i in range(c.spec.n_slots) if c.spec.free[i]]
    for g, cg in enumerate(c.cases):
        rchi2, rg, rA = _oracle_normal_one(cg)
        assert abs(chi2[g] - rchi2) <= 1e-5 * rchi2, (g, chi2[g], rchi2)
        d = np.sqrt(np.diag(rA))
        assert (np.abs(grad[g, free] + 2.0 * rg) <= 1e-4 * d * math.sqrt(rchi2) + 1e-300).all(), g
        assert (np.abs(jtj[g][np.ix_(free, free)] - rA) <= 1e-4 * np.outer(d, d) + 1e-300).all(), g


FIT_TIGHT = dict(tol=1e-12, xtol=1e-10, gtol=1e-13, max_iter=200)


def _near_truth(truth, spec, seed=0, frac=0.02):
    rng = np.random.default_rng(seed)
    p = truth.copy()
    for i, name in enumerate(spec.names):
        role = name.split(".")[-1]
        u = rng.uniform(-1, 1, p.shape[0])
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


def test_uneven_fit_near_truth_matches_oracle(gm):
    # galaxies bright enough (Ie 20-100) for a well-determined minimum next to the truth
    geoms = [(48, 48, 25), (37, 45, 9), (96, 70, 41), (33, 65, 51), (128, 40, 31), (64, 64, 15)]
    rb = synth.draw_uneven_sersic(14, geoms, ie=(20.0, 100.0))
    c = uneven_from(rb, at="truth")
    c.params = _near_truth(c.truth, c.spec)
    t = c.torch()
    got = gm.gm_fit_batch(c.spec, t["params"], t["image"], t["sigma"], t["mask"], t["psf"],
                          gm.FitOptions(**FIT_TIGHT), geom=c.geom)
    got = {k: _np(v) for k, v in got.items()}
    assert (got["status"] == 1).all(), got["status"]
    for g, cg in enumerate(c.cases):
        ref = oracle.fit(cg.spec, c.params[g:g + 1], cg.psf.astype(np.float64), cg.image.astype(np.float64),
                         cg.sigma.astype(np.float64), cg.mask, oracle.FitOptions(**FIT_TIGHT))
        assert ref["status"][0] == 1
        assert abs(got["chi2"][g] - ref["chi2"][0]) <= 1e-5 * ref["chi2"][0], g
        assert got["dof"][g] == ref["dof"][0]
        scale = np.array([1.0 if n.split(".")[-1] in ("x0", "y0", "pa", "Isky") else 0.0 for n in c.spec.names])
        tol = 1e-4 * np.maximum(np.abs(ref["params"][0]), scale)
        diff = np.abs(got["params"][g] - ref["params"][0])
        pa = c.spec.slot("bulge.pa")
        d = diff[pa] % math.pi
        diff[pa] = min(d, math.pi - d) if ref["params"][0, c.spec.slot("bulge.q")] <= 0.95 else 0.0
        assert (diff <= tol).all(), (g, diff / tol)


def _interleave(batches):
    """Interleave equal-stamp cases galaxy by galaxy into one uneven case."""
    cases, geom = [], []
    n = max(len(b) for b in batches)
    for i in range(n):
        for b in batches:
            if i < len(b):
                cases.append(b[i])
                geom.append((b[i].H, b[i].W, b[i].psf.shape[-1]))
    return cases, np.asarray(geom, np.int32)


def _one_galaxy_cases(batch, at):
    """Split an equal-stamp synth batch into one-galaxy Cases (shared float32 inputs)."""
    whole = from_batch(batch, at=at)
    out = []
    for g in range(whole.G):
        out.append(Case(whole.spec, whole.params[g:g + 1], whole.psf[g:g + 1], whole.image[g:g + 1],
                        whole.sigma[g:g + 1],
                        None if whole.mask is None else whole.mask[g:g + 1], whole.H, whole.W,
                        init=whole.init[g:g + 1], truth=whole.truth[g:g + 1]))
    return whole, out


def test_uneven_batch_is_bitwise_the_equal_stamp_path(gm):
    import torch
    spec = synth.single_sersic_sky(128, 128)  # one set of bounds for every run
    A, a_cases = _one_galaxy_cases(synth.draw_small(seed=21, G=5), "init")
    B, b_cases = _one_galaxy_cases(synth.draw_sdss(seed=22, G=4, H=96, W=80, K=41), "init")
    for cc in a_cases + b_cases:
        cc.spec = spec
    cases, geom = _interleave([a_cases, b_cases])
    u = UnevenCase(spec, geom, cases)
    tu = u.torch()
    opts = gm.FitOptions(max_iter=60)

    def uniform(whole, mask_zeros):
        t = whole.torch()
        mask = t["mask"] if t["mask"] is not None else (
            torch.zeros(t["image"].shape, dtype=torch.uint8, device="cuda") if mask_zeros else None)
        m = _np(gm.gm_model(spec, t["params"], t["psf"], whole.H, whole.W))
        c2, g2, j2 = (_np(x) for x in gm.gm_chi2_grad(spec, t["params"], t["image"], t["sigma"], mask, t["psf"],
                                                      want_grad=True, want_jtj=True))
        f = gm.gm_fit_batch(spec, t["params"], t["image"], t["sigma"], mask, t["psf"], opts)
        return m, (c2, g2, j2), {k: _np(v) for k, v in f.items()}

    ra = uniform(A, True)
    rb = uniform(B, False)
    m = _np(gm.gm_model(spec, tu["params"], tu["psf"], geom=geom))
    c2, g2, j2 = (_np(x) for x in gm.gm_chi2_grad(spec, tu["params"], tu["image"], tu["sigma"], tu["mask"],
                                                  tu["psf"], want_grad=True, want_jtj=True, geom=geom))
    f = {k: _np(v) for k, v in gm.gm_fit_batch(spec, tu["params"], tu["image"], tu["sigma"], tu["mask"], tu["psf"],
                                                 opts, geom=geom).items()}
    per_gal = u.split(m)
    # position of each uneven galaxy in its source batch
    src = []
    for i in range(max(A.G, B.G)):
        if i < A.G:
            src.append((ra, i))
        if i < B.G:
            src.append((rb, i))
    for g, (r, i) in enumerate(src):
        np.testing.assert_array_equal(per_gal[g][0], r[0][i])
        assert c2[g] == r[1][0][i]
        np.testing.assert_array_equal(g2[g], r[1][1][i])
        np.testing.assert_array_equal(j2[g], r[1][2][i])
        for k in ("params", "chi2", "dof", "iters", "status", "sigma_p"):
            np.testing.assert_array_equal(f[k][g], r[2][k][i], err_msg=f"{k} of galaxy {g}")
