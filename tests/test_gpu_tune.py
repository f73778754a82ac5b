"""Launch shapes of the fused pass (gm_tune_set) and the autotuner.

Every shape computes the same normal equations: the pairs of a pass are
spread over the thread groups (a two-pair pass on two groups is split by PSF
rows instead, the second group adding its half), so only FP32 summation
orders change, in the correlation and in the reduction, and results agree
with the default shape to the parity tolerances of the chi^2 tests."""
import math

import numpy as np
import pytest

from cases import from_batch
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
    yield gmod
    gmod.gm_tune_clear()


def _np(x):
    return x.detach().cpu().numpy()


@pytest.mark.parametrize("draw,kw", [(synth.draw_small, dict(G=6)),
                                     (synth.draw_bulge_disk, dict(G=5, H=72, W=64, K=25)),
                                     (synth.draw_bulge_bar_nucleus, dict(G=4, H=64, W=64, K=41))])
def test_every_launch_shape_gives_the_same_normal_equations(gm, draw, kw):
    from paper_2404_07780_b300 import tune
    c = from_batch(draw(seed=31, **kw), at="init")
    t = c.torch()
    K, P = c.psf.shape[-1], c.spec.n_free

    def run():
        return [_np(x) for x in gm.gm_chi2_grad(c.spec, t["params"], t["image"], t["sigma"], t["mask"], t["psf"],
                                               want_grad=True, want_jtj=True)]

    gm.gm_tune_set(K, P, 0, 0, 0)
    ref_c2, ref_g, ref_A = run()
    ran = []
    for shape in tune.SHAPES:
        gm.gm_tune_set(K, P, *shape)
        c2, g, A = run()
        if gm.gm_tune_last_shape() != shape:
            continue  # an instance this P does not have, or too much shared memory
        ran.append(shape)
        np.testing.assert_allclose(c2, ref_c2, rtol=1e-5)
        for gi in range(c.G):
            d = np.sqrt(np.abs(np.diag(ref_A[gi])))
            assert (np.abs(g[gi] - ref_g[gi]) <= 1e-4 * d * math.sqrt(ref_c2[gi]) + 1e-300).all(), (shape, gi)
            assert (np.abs(A[gi] - ref_A[gi]) <= 1e-4 * np.outer(d, d) + 1e-300).all(), (shape, gi)
    gm.gm_tune_set(K, P, 0, 0, 0)
    assert len(ran) >= 4, ran


def test_autotune_sets_a_shape_that_runs(gm):
    from paper_2404_07780_b300 import tune
    b = synth.draw_bulge_disk(seed=32, G=8, H=64, W=64, K=31)
    c = from_batch(b, at="init")
    t = c.torch()
    e = tune.autotune(c.spec, t["params"], t["image"], t["sigma"], t["mask"], t["psf"], reps=1)
    assert (e["K"], e["P"]) == (31, 12)
    assert e["candidates"] and e["ms"] == min(e["candidates"].values())
    gm.gm_chi2_grad(c.spec, t["params"], t["image"], t["sigma"], t["mask"], t["psf"])
    assert gm.gm_tune_last_shape() == (e["pairs_per_pass"], e["pairs_per_thread"], e["groups"])
    gm.gm_tune_set(31, 12, 0, 0, 0)
