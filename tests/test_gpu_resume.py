"""Checkpoint and resume of gm_fit_batch on the GPU: a fit stopped at max_iter = k
(canonical = 0: the best point as the fit holds it, with each galaxy's damping in
lambda_inout) and resumed from that state ends bit for bit where the uninterrupted
fit ends, for every galaxy still running at k; the same split on the FP64 oracle
agrees with it at the parity tolerances."""
import numpy as np
import pytest

import oracle
from cases import from_batch, uneven_from
from paper_2404_07780_b300 import synth
from test_gpu_parity import _compare_fits, oracle_inputs

pytestmark = pytest.mark.gpu

TIGHT = dict(tol=1e-12, xtol=1e-10, gtol=1e-13)


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


def _np(d):
    return {k: v.cpu().numpy() for k, v in d.items()}


def _split_and_resume(gm, c, N, k, geom=None, select=None):
    import torch
    t = c.torch()
    full = _np(gm.gm_fit_batch(c.spec, t["params"], t["image"], t["sigma"], t["mask"], t["psf"],
                               gm.FitOptions(max_iter=N, **TIGHT), geom=geom))
    lam = torch.zeros(c.G, dtype=torch.float64, device="cuda")
    part = gm.gm_fit_batch(c.spec, t["params"], t["image"], t["sigma"], t["mask"], t["psf"],
                           gm.FitOptions(max_iter=k, canonical=0, lambda_inout=lam, **TIGHT), geom=geom)
    rest = gm.gm_fit_batch(c.spec, part["params"], t["image"], t["sigma"], t["mask"], t["psf"],
                           gm.FitOptions(max_iter=N - k + 1, lambda_inout=lam, **TIGHT), geom=geom)
    return full, _np(part), _np(rest), lam.cpu().numpy()


def test_resume_is_bit_exact_and_matches_the_oracle(gm):
    c = from_batch(synth.draw_small(seed=17, G=16), at="init")
    N, k = 100, 6
    full, part, rest, lam = _split_and_resume(gm, c, N, k)
    run = part["status"] == 2  # still running at k
    assert run.sum() >= 8, part["status"]
    assert (lam[run] > 0).all() and np.isfinite(lam).all()
    for key in ("params", "chi2", "status", "sigma_p", "dof"):
        np.testing.assert_array_equal(rest[key][run], full[key][run])
    np.testing.assert_array_equal(rest["iters"][run], full["iters"][run] - k + 1)
    # the oracle, split the same way, ends at the same fits
    oi = oracle_inputs(c)
    olam = np.zeros(c.G)
    opart = oracle.fit(c.spec, c.params, oi["psf"], oi["image"], oi["sigma"], c.mask,
                       oracle.FitOptions(max_iter=k, canonical=0, **TIGHT), olam)
    orun = opart["status"] == 2
    orest = oracle.fit(c.spec, opart["params"][orun], oi["psf"][orun], oi["image"][orun], oi["sigma"][orun], None,
                       oracle.FitOptions(max_iter=N - k + 1, **TIGHT), olam[orun].copy())
    both = run & orun
    sel = np.where(both)[0]
    pos = {g: i for i, g in enumerate(np.where(orun)[0])}
    ref = {key: np.asarray(orest[key])[[pos[g] for g in sel]] for key in ("params", "chi2", "status", "sigma_p")}
    got = {key: rest[key][sel] for key in ("params", "chi2", "status", "sigma_p")}
    same, rel = _compare_fits(c.spec, got, ref)
    np.testing.assert_array_equal(got["status"], ref["status"])
    assert (same == (ref["status"] == 1)).all()
    assert rel[same].max() <= 1e-4, rel[same].max(axis=1)


def test_resume_uneven_batch_is_bit_exact(gm):
    rb = synth.draw_uneven_sersic(seed=19, geom=[(48, 48, 25), (37, 45, 9), (96, 70, 41), (64, 64, 15)],
                                  ie=(20.0, 100.0))
    c = uneven_from(rb, at="init")
    full, part, rest, lam = _split_and_resume(gm, c, 100, 4, geom=rb.geom)
    run = part["status"] == 2
    assert run.any(), part["status"]
    for key in ("params", "chi2", "status", "sigma_p"):
        np.testing.assert_array_equal(rest[key][run], full[key][run])
