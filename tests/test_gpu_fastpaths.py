"""The tile and planes kernels' shortcuts against their general loops.

Two shortcuts serve the paper's usual model (one Sersic profile plus a flat
sky, Sec. 4 and Eq. new_sky_I with zero slopes):
  * a lone unconvolved flat sky is written over the output tile as its level
    and 1 x its slot scale, without evaluating the component;
  * one convolved component whose free parameters own channels 1 .. np in
    order keeps its channels in registers in the planes kernel instead of the
    shared-memory scatter.
Each test builds a second model that computes the same image through the
general loop -- the sky as a tilted plane with both slopes fixed at zero, or a
second convolved component far off the stamp with every parameter fixed --
and asks for bit-identical chi^2, gradient and J^T W J: the shortcuts perform
the general loops' floating-point operations, not approximations of them.
"""
import numpy as np
import pytest

from cases import Case, psf_image
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


def _sersic_sky_params(G, H, W, seed):
    g = np.random.default_rng(seed)
    return np.stack([W / 2 + g.uniform(-2, 2, G), H / 2 + g.uniform(-2, 2, G), g.uniform(0.4, 0.9, G),
                     g.uniform(0, np.pi, G), 10 ** g.uniform(1, 2, G), g.uniform(3, 8, G), g.uniform(0.8, 3, G),
                     g.uniform(1, 4, G)], 1)


def _data(H, W, K, G, seed):
    """Noisy float32 stamps (any content will do: both models see the same data)."""
    g = np.random.default_rng(seed)
    image = (20.0 + 5.0 * g.standard_normal((G, H, W))).astype(np.float32)
    sigma = (1.0 + 0.1 * g.random((G, H, W))).astype(np.float32)
    psf = np.stack([psf_image("moffat", [K / 2, K / 2, 1, 0, 1, 1.5, 3.0], K) for _ in range(G)])
    return image, sigma, psf


def _normal(gm, spec, params, image, sigma, psf, H, W):
    c = Case(spec, params, psf, image, sigma, None, H, W)
    t = c.torch()
    return [x.detach().cpu().numpy() for x in gm.gm_chi2_grad(spec, t["params"], t["image"], t["sigma"], None,
                                                               t["psf"], want_grad=True, want_jtj=True)]


# 72 x 56 stamps: ragged tiles, edge tiles by rows and by columns, K = 25 and 41
@pytest.mark.parametrize("K", [25, 41])
def test_flat_sky_shortcut_matches_the_general_loop(gm, K):
    H, W, G = 72, 56, 6
    flat = synth.ModelSpec().add("sersic", "bulge", H, W).add("sky", "sky", H, W, convolve=False)
    plane = (synth.ModelSpec().add("sersic", "bulge", H, W)
             .add("tsky", "sky", H, W, convolve=False, fixed=("kx", "ky")))
    p = _sersic_sky_params(G, H, W, 1)
    image, sigma, psf = _data(H, W, K, G, 2)
    c1, g1, A1 = _normal(gm, flat, p, image, sigma, psf, H, W)
    c2, g2, A2 = _normal(gm, plane, np.concatenate([p, np.zeros((G, 2))], 1), image, sigma, psf, H, W)
    assert np.isfinite(c1).all() and (c1 > 0).all()
    np.testing.assert_array_equal(c1, c2)
    np.testing.assert_array_equal(g1, g2[:, :8])
    np.testing.assert_array_equal(A1, A2[:, :8, :8])


@pytest.mark.parametrize("K", [25, 41])
def test_register_planes_match_the_scatter(gm, K):
    H, W, G = 72, 56, 6
    one = synth.ModelSpec().add("sersic", "bulge", H, W).add("sky", "sky", H, W, convolve=False)
    two = (synth.ModelSpec().add("sersic", "bulge", H, W)
           .add("gaussian", "nil", H, W, fixed=("x0", "y0", "q", "pa", "I0", "fwhm"))
           .add("sky", "sky", H, W, convolve=False))
    p = _sersic_sky_params(G, H, W, 3)
    # the extra component: a 1-pixel Gaussian 1000 pixels off the stamp, whose exponential
    # underflows to exactly 0 at every pixel (amplitudes stay positive: they are log-space slots)
    nil = np.tile([-1000.0, -1000.0, 1.0, 0.0, 1.0, 1.0], (G, 1))
    image, sigma, psf = _data(H, W, K, G, 4)
    c1, g1, A1 = _normal(gm, one, p, image, sigma, psf, H, W)
    c2, g2, A2 = _normal(gm, two, np.concatenate([p[:, :7], nil, p[:, 7:]], 1), image, sigma, psf, H, W)
    keep = list(range(7)) + [13]
    assert np.isfinite(c1).all() and (c1 > 0).all()
    np.testing.assert_array_equal(c1, c2)
    np.testing.assert_array_equal(g1, g2[:, keep])
    np.testing.assert_array_equal(A1, A2[:, keep][:, :, keep])
