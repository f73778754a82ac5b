"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms
printed in the paper, textbook special cases, library routines (scipy, mpmath
through a stored fixture), invariants and brute force.  A dropped term, a wrong
sign or index, or a transposed operand in oracle/gm_oracle.c fails one of them.
"""
import math
import os

import numpy as np
import pytest
import scipy.integrate as si
import scipy.optimize as so
import scipy.signal as ss
import scipy.special as sp

import oracle
from paper_2404_07780_b300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
FWHM_SIGMA = 2.0 * math.sqrt(2.0 * math.log(2.0))


# --------------------------------------------------------------------------
# Special functions: P(a, x) and nu_n (Sec. 4.1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("a", [0.4, 1.0, 1.7, 3.0, 8.0, 20.0])
@pytest.mark.parametrize("x", [1e-3, 0.3, 1.0, 2.5, 7.0, 30.0])
def test_gammp_matches_scipy(a, x):
    assert oracle.gammp(a, x) == pytest.approx(sp.gammainc(a, x), rel=1e-13, abs=1e-15)


@pytest.mark.parametrize("a", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("x", [0.1, 1.0, 4.0, 12.0])
def test_gammp_poisson_sum_for_integer_a(a, x):
    # P(a, x) = 1 - e^-x sum_{j<a} x^j / j! for integer a
    ref = 1.0 - math.exp(-x) * sum(x ** j / math.factorial(j) for j in range(a))
    assert oracle.gammp(a, x) == pytest.approx(ref, rel=1e-13, abs=1e-15)


def test_sersic_b_half_is_ln2():
    # n = 1/2: P(1, nu) = 1 - e^-nu = 1/2  =>  nu = ln 2 exactly
    assert oracle.sersic_b(0.5) == pytest.approx(math.log(2.0), rel=1e-14)


def test_sersic_b_golden_mpmath():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "sersic_b.txt")) if not l.startswith("#")]
    for n, nu in rows:
        assert oracle.sersic_b(float(n)) == pytest.approx(float(nu), rel=1e-13), n


@pytest.mark.parametrize("n", [0.2, 0.37, 0.9, 1.3, 2.2, 3.7, 5.5, 7.1, 9.9])
def test_sersic_b_matches_scipy_gammaincinv(n):
    assert oracle.sersic_b(n) == pytest.approx(sp.gammaincinv(2 * n, 0.5), rel=1e-12)


@pytest.mark.parametrize("n", [1.0, 1.5, 2.0, 3.0, 4.0])
def test_sersic_b_solves_poisson_sum(n):
    a = int(round(2 * n))
    nu = oracle.sersic_b(n)
    resid = 1.0 - math.exp(-nu) * sum(nu ** j / math.factorial(j) for j in range(a)) - 0.5
    assert abs(resid) < 1e-14


# --------------------------------------------------------------------------
# Geometry: pixel grid (App. C listing) and elliptical radius (Eqs. r-rmin)
# --------------------------------------------------------------------------

def _gauss_radius(par, x, y):
    """Invert a unit Gaussian profile to recover the elliptical radius the oracle used."""
    sig = par[5] / FWHM_SIGMA
    v = oracle.component_value("gaussian", par, x, y)
    return math.sqrt(-2.0 * sig * sig * math.log(v))


def test_radius_axes_and_rotation():
    x0, y0, q = 10.3, 7.9, 0.4
    par = [x0, y0, q, 0.0, 1.0, 30.0]
    # pa = 0: major axis along +x, minor along +y
    assert _gauss_radius(par, x0 + 3.0, y0) == pytest.approx(3.0, rel=1e-12)
    assert _gauss_radius(par, x0, y0 + 3.0) == pytest.approx(3.0 / q, rel=1e-12)
    # pa = pi/2 rotates the major axis onto +y
    par[3] = math.pi / 2
    assert _gauss_radius(par, x0, y0 + 3.0) == pytest.approx(3.0, rel=1e-12)
    assert _gauss_radius(par, x0 - 3.0, y0) == pytest.approx(3.0 / q, rel=1e-12)
    # pa = pi/4: the point along the diagonal (+x, +y) lies on the major axis
    par[3] = math.pi / 4
    assert _gauss_radius(par, x0 + 2.0, y0 + 2.0) == pytest.approx(math.sqrt(8.0), rel=1e-12)
    assert _gauss_radius(par, x0 - 2.0, y0 + 2.0) == pytest.approx(math.sqrt(8.0) / q, rel=1e-12)


def test_pixel_grid_convention():
    # pixel (i, j) has centre x = j + 0.5, y = H - 0.5 - i (row 0 at the top)
    H, W = 9, 7
    i, j = 2, 5
    img = oracle.component_image("gaussian", [j + 0.5, H - 0.5 - i, 1.0, 0.0, 3.0, 0.8], H, W)
    assert np.unravel_index(np.argmax(img), img.shape) == (i, j)
    # at the exact centre the radius is floored at 1e-4 px (the Sersic-cusp reading)
    sig = 0.8 / FWHM_SIGMA
    assert img[i, j] == pytest.approx(3.0 * math.exp(-1e-8 / (2 * sig * sig)), rel=1e-14)


# --------------------------------------------------------------------------
# Profiles: normalisations printed in Sec. 4 (r_box = 1 at B = 0)
# --------------------------------------------------------------------------

def _radial_flux(kind, par, rmax=np.inf, points=None):
    """2 pi q int_0^rmax I(r) r dr, with I sampled along the major axis (pa = 0)."""
    x0, y0, q = par[0], par[1], par[2]
    f = lambda r: oracle.component_value(kind, par, x0 + r, y0) * r
    v, _ = si.quad(f, 0.0, rmax, limit=400, epsabs=0, epsrel=1e-12, points=points)
    return 2 * math.pi * q * v


@pytest.mark.parametrize("n", [0.5, 1.0, 2.0, 4.0, 6.0])
def test_sersic_total_flux_and_half_light(n):
    Ie, Re, q = 2.5, 7.0, 0.6
    par = [0.0, 0.0, q, 0.0, Ie, Re, n]
    nu = oracle.sersic_b(n)
    # inverse of Eq. sersicLtot with r_box = 1: F = 2 pi q Re^2 n Gamma(2n) e^nu nu^-2n Ie
    F = 2 * math.pi * q * Re ** 2 * n * math.gamma(2 * n) * math.exp(nu) * nu ** (-2 * n) * Ie
    inner = _radial_flux("sersic", par, Re)
    outer = 2 * math.pi * q * si.quad(
        lambda r: oracle.component_value("sersic", par, r, 0.0) * r, Re, np.inf, limit=400,
        epsabs=0, epsrel=1e-12)[0]
    # the 1e-4 px radius floor moves at most pi q I(0) r_floor^2 of flux
    tol = 1e-9 + math.pi * q * Ie * math.exp(nu) * 1e-8 / F
    assert inner + outer == pytest.approx(F, rel=tol)
    assert inner == pytest.approx(F / 2, rel=tol)  # r_e holds half the light (Sec. 4.1)


def test_sersic_magnitude_relation_roundtrip():
    # Eq. sersicLtot: Ie from (m, m0); the flux 10^(-0.4(m - m0)) must come back
    m, m0, Re, q, n = 17.68, 22.5, 7.58, 0.64, 1.53
    nu = oracle.sersic_b(n)
    Ie = nu ** (2 * n) * 10 ** (-0.4 * (m - m0)) / (2 * math.pi * q * Re ** 2 * n * math.gamma(2 * n) * math.exp(nu))
    par = [0.0, 0.0, q, 0.0, Ie, Re, n]
    assert _radial_flux("sersic", par, np.inf) == pytest.approx(10 ** (-0.4 * (m - m0)), rel=1e-8)


def test_expdisk_normalisation():
    I0, rs, q = 3.0, 4.5, 0.7  # Eq. expdiskI0: F = 2 pi q rs^2 I0
    assert _radial_flux("expdisk", [0, 0, q, 0, I0, rs]) == pytest.approx(2 * math.pi * q * rs ** 2 * I0, rel=1e-9)


@pytest.mark.parametrize("a,b", [(2.0, 0.0), (2.0, 1.5), (0.7, 0.5), (3.0, -1.0)])
def test_ferrer_normalisation(a, b):
    I0, rout, q = 1.7, 9.0, 0.5  # Eq. ferrerI0: F = pi q rout^2 a B(a, 1 + 2/(2-b)) I0
    F = math.pi * q * rout ** 2 * a * sp.beta(a, 1 + 2 / (2 - b)) * I0
    assert _radial_flux("ferrer", [0, 0, q, 0, I0, rout, a, b], rout) == pytest.approx(F, rel=1e-8)
    assert oracle.component_value("ferrer", [0, 0, q, 0, I0, rout, a, b], rout + 0.01, 0) == 0.0


@pytest.mark.parametrize("n", [1.5, 3.0, 4.765])
def test_moffat_normalisation_and_fwhm(n):
    I0, fwhm, q = 2.0, 3.0, 0.8
    rd = fwhm / (2 * math.sqrt(2 ** (1 / n) - 1))  # Eq. moffat_rd
    F = math.pi * q * rd ** 2 * I0 / (n - 1)      # Eq. moffatI0
    par = [0, 0, q, 0, I0, fwhm, n]
    assert _radial_flux("moffat", par) == pytest.approx(F, rel=1e-8)
    assert oracle.component_value("moffat", par, fwhm / 2, 0) == pytest.approx(I0 / 2, rel=1e-13)


def test_gaussian_normalisation_and_fwhm():
    I0, fwhm, q = 5.0, 2.2, 0.9
    sig = fwhm / FWHM_SIGMA
    par = [0, 0, q, 0, I0, fwhm]
    assert _radial_flux("gaussian", par) == pytest.approx(2 * math.pi * q * sig ** 2 * I0, rel=1e-9)
    assert oracle.component_value("gaussian", par, fwhm / 2, 0) == pytest.approx(I0 / 2, rel=1e-13)


def test_king_alpha2_is_king1962():
    # alpha = 2 gives King (1962): I ~ [1/sqrt(1+(r/rc)^2) - 1/sqrt(1+(rt/rc)^2)]^2, I(0) = I0
    I0, rc, rt = 4.0, 1.5, 12.0
    par = [0, 0, 1.0, 0, I0, rc, rt, 2.0]
    king = lambda r: (1 / math.sqrt(1 + (r / rc) ** 2) - 1 / math.sqrt(1 + (rt / rc) ** 2)) ** 2
    for r in [0.0, 0.7, 2.0, 5.0, 11.9]:
        v = oracle.component_value("king", par, max(r, 0.0), 0.0)
        assert v == pytest.approx(I0 * king(max(r, 1e-4)) / king(0.0), rel=1e-9)
    assert oracle.component_value("king", par, rt + 0.1, 0.0) == 0.0


@pytest.mark.parametrize("al", [1.5, 2.5, 3.0])
def test_king_general_alpha_centre_edge_and_monotone(al):
    # Eq. BE_S with the bracket read as [A(r) - A(r_t)]: I(0) = I0, I(r_t) = 0, and I falls
    # monotonically in between, for every power alpha (not only King's alpha = 2)
    I0, rc, rt = 7.0, 1.3, 9.0
    par = [0.0, 0.0, 1.0, 0.0, I0, rc, rt, al]
    # (the radius floor of 1e-4 px moves I(0) by ~1e-8 relative)
    assert oracle.component_value("king", par, 0.0, 0.0) == pytest.approx(I0, rel=1e-7)
    assert oracle.component_value("king", par, rt, 0.0) == 0.0
    r = np.linspace(0.0, rt, 400)
    v = np.array([oracle.component_value("king", par, x, 0.0) for x in r])
    assert (np.diff(v) < 0).all()


@pytest.mark.parametrize("al", [1.5, 2.5, 3.0])
def test_king_general_alpha_untruncated_limit(al):
    # r_t -> infinity: A(r_t) -> 0 and [A(r)]^alpha = 1 / (1 + (r/r_c)^2) whatever alpha
    # (King's untruncated core profile), so a misplaced power of alpha shows here
    I0, rc, rt = 3.0, 2.0, 2.0e15
    par = [0.0, 0.0, 1.0, 0.0, I0, rc, rt, al]
    for x in (0.5, 1.0, 3.0, 10.0, 40.0):
        v = oracle.component_value("king", par, x, 0.0)
        assert v == pytest.approx(I0 / (1.0 + (x / rc) ** 2), rel=1e-8)


@pytest.mark.parametrize("al", [1.5, 2.5, 3.0])
def test_king_general_alpha_truncation_edge_power(al):
    # near r_t, A(r) - A(r_t) is linear in r_t - r, so I ~ (r_t - r)^alpha: the local
    # log-slope of I against (r_t - r) is alpha
    I0, rc, rt = 5.0, 1.0, 6.0
    par = [0.0, 0.0, 1.0, 0.0, I0, rc, rt, al]
    e1, e2 = 1e-4, 2e-4
    v1 = oracle.component_value("king", par, rt - e1, 0.0)
    v2 = oracle.component_value("king", par, rt - e2, 0.0)
    assert math.log(v2 / v1) / math.log(e2 / e1) == pytest.approx(al, rel=1e-4)


@pytest.mark.parametrize("al", [1.5, 2.5, 3.0])
def test_king_general_alpha_against_mpmath(al):
    # an independent restatement of Eq. BE_S in 50-digit arithmetic, written as the ratio
    # ((A(r) - A(r_t)) / (1 - A(r_t)))^alpha with A(x) = (1 + (x/r_c)^2)^(-1/alpha)
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    I0, rc, rt = 4.0, 1.7, 12.0
    par = [0.0, 0.0, 1.0, 0.0, I0, rc, rt, al]
    A = lambda x: (1 + (mpmath.mpf(x) / rc) ** 2) ** (-1 / mpmath.mpf(al))
    for x in (0.3, 1.0, 2.5, 6.0, 11.0):
        ref = I0 * ((A(x) - A(rt)) / (1 - A(rt))) ** al
        assert oracle.component_value("king", par, x, 0.0) == pytest.approx(float(ref), rel=1e-12)


def test_sersic_reduces_to_gaussian_and_exponential():
    # Sec. 4.1: n = 1/2 is a Gaussian (FWHM = 2 Re, I0 = 2 Ie); n = 1 an exponential
    # disk (rs = Re / nu_1, I0 = Ie e^nu_1)
    H, W = 24, 20
    g = [10.2, 11.7, 0.55, 0.8]
    Ie, Re = 1.3, 4.0
    s05 = oracle.component_image("sersic", g + [Ie, Re, 0.5], H, W)
    gau = oracle.component_image("gaussian", g + [2 * Ie, 2 * Re], H, W)
    np.testing.assert_allclose(s05, gau, rtol=1e-13, atol=0)
    nu1 = oracle.sersic_b(1.0)
    s1 = oracle.component_image("sersic", g + [Ie, Re, 1.0], H, W)
    ex = oracle.component_image("expdisk", g + [Ie * math.exp(nu1), Re / nu1], H, W)
    np.testing.assert_allclose(s1, ex, rtol=1e-13, atol=0)


def test_pixel_sum_converges_to_total_flux():
    # 2-D sampling: a smooth, well-resolved profile on a large stamp sums to its flux
    H = W = 240
    q, Re, n, Ie = 0.7, 18.0, 1.0, 1.0
    img = oracle.component_image("sersic", [W / 2 + 0.3, H / 2 - 0.2, q, 0.4, Ie, Re, n], H, W)
    nu = oracle.sersic_b(n)
    F = 2 * math.pi * q * Re ** 2 * n * math.gamma(2 * n) * math.exp(nu) * nu ** (-2 * n) * Ie
    assert img.sum() == pytest.approx(F, rel=2e-4)


# --------------------------------------------------------------------------
# PSF correlation (Sec. 2; App. C conv2d padding="same")
# --------------------------------------------------------------------------

def test_correlate_delta_identity_and_shift():
    g = np.random.default_rng(3)
    img = g.standard_normal((9, 11))
    delta = np.zeros((5, 5))
    delta[2, 2] = 1.0
    np.testing.assert_array_equal(oracle.correlate(img, delta), img)
    sh = np.zeros((5, 5))
    sh[3, 2] = 1.0  # tap (a, b) = (c + 1, c) reads I[i + 1, j]
    out = oracle.correlate(img, sh)
    np.testing.assert_array_equal(out[:-1], img[1:])
    np.testing.assert_array_equal(out[-1], 0.0)
    sh = np.zeros((5, 5))
    sh[2, 0] = 1.0  # tap (c, c - 2) reads I[i, j - 2]
    out = oracle.correlate(img, sh)
    np.testing.assert_array_equal(out[:, 2:], img[:, :-2])
    np.testing.assert_array_equal(out[:, :2], 0.0)


@pytest.mark.parametrize("shape,K", [((9, 11), 5), ((6, 4), 7), ((13, 13), 1), ((3, 5), 9)])
def test_correlate_matches_scipy(shape, K):
    g = np.random.default_rng(shape[0] * 100 + K)
    img = g.standard_normal(shape)
    psf = g.standard_normal((K, K))
    ref = ss.correlate2d(img, psf, mode="same", boundary="fill", fillvalue=0.0)
    np.testing.assert_allclose(oracle.correlate(img, psf), ref, rtol=1e-13, atol=1e-13)


def test_correlate_brute_force_tiny():
    g = np.random.default_rng(5)
    img = g.standard_normal((4, 6))
    psf = g.standard_normal((3, 3))
    c = 1
    ref = np.zeros_like(img)
    for i in range(4):
        for j in range(6):
            for a in range(3):
                for b in range(3):
                    ii, jj = i + a - c, j + b - c
                    if 0 <= ii < 4 and 0 <= jj < 6:
                        ref[i, j] += psf[a, b] * img[ii, jj]
    np.testing.assert_allclose(oracle.correlate(img, psf), ref, rtol=1e-14, atol=1e-14)


def test_unit_psf_conserves_flux():
    H = W = 64
    img = oracle.component_image("gaussian", [32.1, 31.6, 0.8, 0.3, 10.0, 4.0], H, W)
    psf = oracle.component_image("moffat", [7.5, 7.5, 1.0, 0.0, 1.0, 2.5, 3.0], 15, 15)
    psf /= psf.sum()
    assert oracle.correlate(img, psf).sum() == pytest.approx(img.sum(), rel=1e-12)


def test_model_is_correlated_sum_plus_unconvolved():
    H, W, K = 20, 24, 7
    spec = synth.single_sersic_sky(H, W)
    p = np.array([[11.2, 9.7, 0.6, 1.1, 5.0, 3.0, 2.2, 1.75]])
    psf = oracle.component_image("gaussian", [K / 2, K / 2, 1, 0, 1, 1.8], K, K)[None]
    m = oracle.model_images(spec, p, psf, H, W)[0]
    ser = oracle.component_image("sersic", p[0, :7], H, W)
    ref = ss.correlate2d(ser, psf[0], mode="same") + 1.75  # sky added after the PSF, unconvolved
    np.testing.assert_allclose(m, ref, rtol=1e-13, atol=1e-13)
    comps = oracle.component_images(spec, p, psf, H, W)[0]
    np.testing.assert_allclose(comps.sum(0), m, rtol=1e-13, atol=1e-13)


# --------------------------------------------------------------------------
# chi^2 (Eq. chinu)
# --------------------------------------------------------------------------

def test_chi2_hand_computed_with_mask():
    spec = synth.ModelSpec().add("sky", "sky", 3, 3, convolve=False)
    D = np.array([[[1.0, 2.0, 3.0], [4.0, 5.0, 6.0], [7.0, 8.0, 9.0]]])
    S = np.array([[[1.0, 2.0, 1.0], [0.5, 1.0, 2.0], [1.0, 1.0, 4.0]]])
    M = np.array([[[0, 0, 1], [0, 1, 0], [0, 0, 0]]], np.uint8)
    sky = 2.0
    # unmasked: (1-2)^2/1 + (2-2)^2/4 + (4-2)^2/.25 + (6-2)^2/4 + (7-2)^2 + (8-2)^2 + (9-2)^2/16
    ref = 1 + 0 + 16 + 4 + 25 + 36 + 49 / 16
    psf = np.ones((1, 1, 1))
    assert oracle.chi2(spec, [[sky]], psf, D, S, M)[0] == pytest.approx(ref, rel=1e-15)
    assert oracle.chi2(spec, [[sky]], psf, D, S, None)[0] == pytest.approx(ref + 1 + 9, rel=1e-15)


# --------------------------------------------------------------------------
# Jacobian by central differences
# --------------------------------------------------------------------------

def test_jacobian_against_textbook_gaussian_derivatives():
    # unconvolved circular Gaussian + sky: dI/dx0 = I (x - x0)/s^2, dI/dy0 = I (y - y0)/s^2,
    # dI/dI0 = I/I0, dI/dfwhm = I r^2 / (s^2 fwhm), dM/dsky = 1
    H, W = 12, 14
    spec = synth.ModelSpec().add("gaussian", "g", H, W, convolve=False, fixed=("q", "pa"))
    spec.add("sky", "sky", H, W, convolve=False)
    x0, y0, I0, fw = 6.3, 5.8, 4.0, 3.1
    p = np.array([[x0, y0, 1.0, 0.0, I0, fw, 0.5]])
    J = oracle.jacobian(spec, p, np.ones((1, 1, 1)), H, W)[0]
    yy, xx = np.meshgrid(H - 0.5 - np.arange(H), np.arange(W) + 0.5, indexing="ij")
    s2 = (fw / FWHM_SIGMA) ** 2
    r2 = (xx - x0) ** 2 + (yy - y0) ** 2
    I = I0 * np.exp(-r2 / (2 * s2))
    ref = [I * (xx - x0) / s2, I * (yy - y0) / s2, I / I0, I * r2 / (s2 * fw), np.ones_like(I)]
    for k in range(5):
        np.testing.assert_allclose(J[k], ref[k], rtol=1e-6, atol=1e-8 * I0)
    # internal coordinates: d/d ln I0 = I0 dI/dI0 = I
    Ji = oracle.jacobian(spec, p, np.ones((1, 1, 1)), H, W, internal=True)[0]
    np.testing.assert_allclose(Ji[2], I, rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(Ji[3], fw * ref[3], rtol=1e-6, atol=1e-8)


def test_jacobian_of_linear_model_is_exact_template():
    # the convolved model is linear in the amplitude: dM/dIe = M_sersic / Ie
    H, W, K = 16, 16, 5
    spec = synth.single_sersic_sky(H, W)
    p = np.array([[8.1, 7.7, 0.7, 0.3, 3.0, 2.5, 1.7, 0.0]])
    psf = oracle.component_image("gaussian", [K / 2, K / 2, 1, 0, 1, 1.5], K, K)[None]
    J = oracle.jacobian(spec, p, psf, H, W)[0]
    comps = oracle.component_images(spec, p, psf, H, W)[0]
    np.testing.assert_allclose(J[4], comps[0] / 3.0, rtol=1e-7, atol=1e-10)


# --------------------------------------------------------------------------
# Levenberg-Marquardt and covariance (Sec. 5.1-5.2)
# --------------------------------------------------------------------------

def _gauss_psf(K, fwhm):
    psf = oracle.component_image("gaussian", [K / 2, K / 2, 1.0, 0.0, 1.0, fwhm], K, K)
    return psf / psf.sum()


def test_lm_sky_only_closed_form():
    # a flat-sky fit has sky = sum(w D) / sum(w) and sigma_sky = (sum w)^-1/2 (Sec. 5.2)
    g = np.random.default_rng(11)
    H, W = 10, 12
    spec = synth.ModelSpec().add("sky", "sky", H, W, convolve=False)
    D = g.normal(3.0, 1.0, (1, H, W))
    S = g.uniform(0.5, 2.0, (1, H, W))
    M = (g.uniform(size=(1, H, W)) < 0.2).astype(np.uint8)
    w = (M == 0) / S ** 2
    res = oracle.fit(spec, [[0.0]], np.ones((1, 1, 1)), D, S, M,
                     oracle.FitOptions(gtol=0.0, tol=1e-14, max_iter=50))
    assert res["params"][0, 0] == pytest.approx((w * D).sum() / w.sum(), rel=1e-10)
    assert res["sigma_p"][0, 0] == pytest.approx(w.sum() ** -0.5, rel=1e-8)
    assert res["dof"][0] == int((M == 0).sum()) - 1


def test_lm_covariance_of_linear_model():
    # amplitude + sky with a fixed shape: J is known, cov = (J^T W J)^-1 exactly
    g = np.random.default_rng(12)
    H, W = 20, 20
    spec = synth.ModelSpec().add("gaussian", "g", H, W, convolve=False, fixed=("x0", "y0", "q", "pa", "fwhm"))
    spec.log[spec.slot("g.I0")] = False
    spec.add("sky", "sky", H, W, convolve=False)
    tmpl = oracle.component_image("gaussian", [10.2, 9.9, 0.8, 0.5, 1.0, 4.0], H, W)
    S = g.uniform(0.8, 1.5, (1, H, W))
    D = (7.0 * tmpl + 2.0 + S * g.standard_normal((H, W)))
    p0 = np.array([[10.2, 9.9, 0.8, 0.5, 1.0, 4.0, 0.0]])
    res = oracle.fit(spec, p0, np.ones((1, 1, 1)), D, S, None, oracle.FitOptions(gtol=0.0, tol=1e-15, max_iter=50))
    J = np.stack([tmpl.ravel(), np.ones(H * W)], 1)
    w = 1 / S.ravel() ** 2
    A = J.T @ (w[:, None] * J)
    sol = np.linalg.solve(A, J.T @ (w * D.ravel()))
    cov = np.linalg.inv(A)
    np.testing.assert_allclose(res["params"][0, [4, 6]], sol, rtol=1e-9)
    np.testing.assert_allclose(res["sigma_p"][0, [4, 6]], np.sqrt(np.diag(cov)), rtol=1e-6)
    # fitted in log space the amplitude has sigma_p = p sigma_(ln p): the same error bar
    spec.log[spec.slot("g.I0")] = True
    res = oracle.fit(spec, p0 * [1, 1, 1, 1, 5.0, 1, 1], np.ones((1, 1, 1)), D, S, None,
                     oracle.FitOptions(gtol=0.0, tol=1e-15, max_iter=80))
    np.testing.assert_allclose(res["params"][0, [4, 6]], sol, rtol=1e-9)
    np.testing.assert_allclose(res["sigma_p"][0, [4, 6]], np.sqrt(np.diag(cov)), rtol=1e-6)


def test_lm_exact_recovery_noiseless():
    b = synth.draw_small(seed=7, G=4)
    psf = np.stack([_gauss_psf(b.K, 1.5)] * b.G)
    truth = synth.galaxy_slots(b)
    D = oracle.model_images(b.spec, truth, psf, b.H, b.W)
    S = np.ones_like(D)
    # start a few percent away from the truth (the default start can fall into
    # other local minima; recovery, not the basin, is what this pins)
    start = truth * (1 + 0.04 * np.random.default_rng(1).uniform(-1, 1, truth.shape))
    res = oracle.fit(b.spec, start, psf, D, S, None, oracle.FitOptions(gtol=0.0, tol=1e-15, xtol=1e-11, max_iter=200))
    assert (res["status"] == 1).all(), res["status"]
    err = np.abs(res["params"] - truth)
    err[:, 3] = np.minimum(err[:, 3], math.pi - err[:, 3])  # PA modulo pi
    scale = np.maximum(np.abs(truth), 1.0)
    assert (err / scale).max() < 1e-8, err / scale


def test_lm_matches_minpack_on_tiny_galaxy():
    # same minimum as scipy.optimize.least_squares(method="lm") (MINPACK) on the oracle's own model
    H = W = 16
    K = 5
    spec = synth.single_sersic_sky(H, W)
    truth = np.array([[8.3, 7.6, 0.7, 0.9, 20.0, 3.0, 1.3, 1.5]])
    psf = _gauss_psf(K, 1.5)[None]
    Mt = oracle.model_images(spec, truth, psf, H, W)
    D, S = synth.noisy_image(Mt, np.random.default_rng(2).standard_normal(Mt.shape))
    init = np.array([[8.0, 8.0, 0.6, 1.0, 12.0, 4.0, 1.0, 1.0]])
    res = oracle.fit(spec, init, psf, D, S, None, oracle.FitOptions(gtol=0.0, tol=1e-14, max_iter=300))
    assert res["status"][0] == 1

    logs = np.array(spec.log)

    def resid(u):
        p = np.where(logs, np.exp(u), u)[None]
        return ((D - oracle.model_images(spec, p, psf, H, W)) / S).ravel()

    u0 = np.where(logs, np.log(init[0]), init[0])
    ref = so.least_squares(resid, u0, method="lm", xtol=1e-14, ftol=1e-14, gtol=1e-14)
    pref = np.where(logs, np.exp(ref.x), ref.x)
    pref[3] = pref[3] % math.pi
    np.testing.assert_allclose(res["params"][0], pref, rtol=2e-6, atol=2e-6)
    assert res["chi2"][0] == pytest.approx(2 * ref.cost, rel=1e-10)


def test_lm_reduced_chi2_near_one_at_truth():
    b = synth.draw_small(seed=21, G=16)
    psf = np.stack([_gauss_psf(b.K, 1.5)] * b.G)
    truth = synth.galaxy_slots(b)
    Mt = oracle.model_images(b.spec, truth, psf, b.H, b.W)
    D, S = synth.noisy_image(Mt, b.z)
    c2 = oracle.chi2(b.spec, truth, psf, D, S)
    k = b.H * b.W - b.spec.n_free
    # chi^2 at the truth is chi^2_k distributed: mean k, sd sqrt(2k)
    assert abs(c2.mean() / k - 1) < 4 * math.sqrt(2.0 / k) / math.sqrt(b.G)


def test_lm_pulls_have_unit_width():
    # Sec. 5.2: sigma_p from (J^T W J)^-1 is the standard error of the fitted parameter.  On
    # many noise draws of one bright, well-resolved galaxy (the linear regime), the pulls
    # (p_fit - p_true) / sigma_p of every free parameter have mean 0 and unit width; a wrong
    # factor in the covariance (a missing 2, sigma instead of sigma^2, a log slot not mapped
    # back) moves the width far outside the band.
    H = W = 24
    K = 7
    N = 600
    spec = synth.single_sersic_sky(H, W)
    truth = np.array([12.3, 11.8, 0.6, 0.7, 80.0, 3.5, 1.6, 2.0])
    psf = np.stack([_gauss_psf(K, 1.8)] * N)
    P = np.tile(truth, (N, 1))
    Mt = oracle.model_images(spec, P, psf, H, W)
    z = np.random.default_rng(2024).standard_normal((N, H, W))
    D, S = synth.noisy_image(Mt, z)
    res = oracle.fit(spec, P, psf, D, S, None, oracle.FitOptions(tol=1e-10, max_iter=100))
    assert (res["status"] == 1).all()
    pull = (res["params"] - truth) / res["sigma_p"]
    tol_sd = 0.1   # the sample sd of 600 unit normals is 1 +- 0.03
    for s in range(spec.n_slots):
        assert abs(pull[:, s].mean()) < 0.15, (spec.names[s], pull[:, s].mean())
        assert abs(pull[:, s].std() - 1.0) < tol_sd, (spec.names[s], pull[:, s].std())


def test_status_codes():
    H, W = 8, 8
    spec = synth.ModelSpec().add("sky", "sky", H, W, convolve=False)
    D = np.ones((3, H, W))
    S = np.ones((3, H, W))
    S[0, 2, 2] = 0.0                      # bad sigma on a used pixel
    M = np.zeros((3, H, W), np.uint8)
    M[1] = 1                              # everything masked: no degrees of freedom
    S[2, 3, 3] = 0.0
    M[2, 3, 3] = 1                        # bad sigma hidden by the mask is fine
    res = oracle.fit(spec, np.zeros((3, 1)), np.ones((3, 1, 1)), D, S, M)
    assert list(res["status"]) == [6, 7, 1]


# --------------------------------------------------------------------------
# Axis ratio above 1 (the fit may cross q = 1; results are rewritten with q <= 1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind,par", [
    ("sersic", [10.3, 11.2, 2.0, 0.3, 5.0, 3.0, 1.7]),
    ("expdisk", [10.3, 11.2, 1.6, 1.1, 5.0, 2.5]),
    ("ferrer", [10.3, 11.2, 1.8, 2.0, 5.0, 4.0, 2.0, 0.5]),
    ("king", [10.3, 11.2, 3.0, 0.7, 5.0, 1.5, 5.0, 2.0]),
    ("gaussian", [10.3, 11.2, 1.3, 0.2, 5.0, 2.5]),
    ("moffat", [10.3, 11.2, 2.5, 2.9, 5.0, 2.5, 3.0]),
])
def test_axis_ratio_above_one_is_the_turned_ellipse(kind, par):
    # q > 1 equals 1/q with PA + pi/2 and every scale length times q (same image)
    H, W = 22, 24
    spec = synth.ModelSpec().add(kind, "c", H, W)
    p = np.array([par], float)
    pc = oracle.canonicalize(spec, p)
    q = par[2]
    assert pc[0, 2] == pytest.approx(1.0 / q, rel=1e-15)
    assert pc[0, 3] == pytest.approx(par[3] + math.pi / 2, rel=1e-15)
    scale_idx = {"king": [5, 6]}.get(kind, [5])
    for k in range(len(par)):
        want = par[k] * q if k in scale_idx else par[k]
        if k not in (2, 3):
            assert pc[0, k] == pytest.approx(want, rel=1e-15), k
    a = oracle.component_image(kind, p[0], H, W)
    b = oracle.component_image(kind, pc[0], H, W)
    np.testing.assert_allclose(b, a, rtol=1e-12, atol=1e-14 * np.abs(a).max())


def test_canonical_rewrite_skips_shared_geometry():
    # a q slot whose scale slot is also used by a component with another q is left alone
    H, W = 16, 16
    spec = synth.ModelSpec().add("sersic", "a", H, W)
    spec.add("sersic", "b", H, W, shared={"Re": spec.slot("a.Re")})
    p = np.array([[8, 8, 2.0, 0.1, 1, 3, 1, 8, 8, 0.5, 0.2, 1, 1]], float)
    np.testing.assert_array_equal(oracle.canonicalize(spec, p), p)


def test_fit_through_q_one_ends_canonical():
    # a galaxy whose default PA is 90 degrees off: the fit crosses q = 1 and the
    # result is rewritten with q < 1, PA near the truth, same chi^2 as a start near the truth
    H = W = 48
    K = 9
    spec = synth.single_sersic_sky(H, W)
    truth = np.array([[24.2, 23.7, 0.45, 0.2, 20.0, 5.0, 1.5, 1.0]])
    psf = oracle.component_image("gaussian", [K / 2, K / 2, 1, 0, 1, 1.5], K, K)[None]
    psf /= psf.sum()
    Mt = oracle.model_images(spec, truth, psf, H, W)
    D, S = synth.noisy_image(Mt, np.random.default_rng(4).standard_normal(Mt.shape))
    start = np.array([[24.0, 24.0, 0.65, 0.2 + math.pi / 2, 10.0, 6.0, 1.4, 2.5]])
    r = oracle.fit(spec, start, psf, D, S, None, oracle.FitOptions(tol=1e-12, gtol=1e-13, max_iter=200))
    near = oracle.fit(spec, truth * 1.01, psf, D, S, None, oracle.FitOptions(tol=1e-12, gtol=1e-13, max_iter=200))
    assert r["status"][0] == 1 and near["status"][0] == 1
    assert r["params"][0, 2] <= 1.0
    assert r["chi2"][0] == pytest.approx(near["chi2"][0], rel=1e-9)
    np.testing.assert_allclose(r["params"][0], near["params"][0], rtol=1e-5, atol=1e-5)


# ---------------------------------------------------------------------------
# tilted sky (Eq. new_sky_I), measured from the stamp centre
# ---------------------------------------------------------------------------

def test_tilted_sky_is_a_plane_about_the_stamp_centre():
    H, W = 3, 4
    a, kx, ky = 2.0, 0.5, -0.25
    got = oracle.component_image("tsky", [a, kx, ky], H, W)
    for i in range(H):
        for j in range(W):
            x, y = j + 0.5, H - 0.5 - i  # pixel centre, row 0 at the top
            assert got[i, j] == pytest.approx(a + kx * (x - W / 2) + ky * (y - H / 2), abs=1e-15)
    # the centre of the stamp carries the sky level: mean over a symmetric stamp
    assert oracle.component_image("tsky", [a, kx, ky], 6, 8).mean() == pytest.approx(a, abs=1e-14)


def test_tilted_sky_jacobian_is_one_x_y():
    H, W, K = 9, 11, 3
    spec = synth.ModelSpec().add("sersic", "gal", H, W).add("tsky", "sky", H, W, convolve=False)
    p = np.array([[5.3, 4.1, 0.7, 0.4, 10.0, 2.0, 1.5, 1.0, 0.1, -0.2]])
    psf = np.zeros((1, K, K))
    psf[0, 1, 1] = 1.0
    J = oracle.jacobian(spec, p, psf, H, W)[0]
    x = (np.arange(W) + 0.5 - W / 2)[None, :] * np.ones((H, 1))
    y = (H - 0.5 - np.arange(H) - H / 2)[:, None] * np.ones((1, W))
    np.testing.assert_allclose(J[7], 1.0, atol=1e-8)
    np.testing.assert_allclose(J[8], x, atol=1e-7)
    np.testing.assert_allclose(J[9], y, atol=1e-7)


# ---------------------------------------------------------------------------
# magnitudes instead of amplitudes (Eqs. sersicLtot, expdiskI0, ferrerI0, moffatI0)
# ---------------------------------------------------------------------------

MAG_PROFILES = [
    ("sersic", [0, 0, 0.6, 0, 17.0, 5.0, 2.5]),
    ("sersic", [0, 0, 0.9, 0, 19.0, 3.0, 0.7]),
    ("expdisk", [0, 0, 0.5, 0, 18.0, 4.0]),
    ("ferrer", [0, 0, 0.4, 0, 18.5, 12.0, 2.0, 0.5]),
    ("ferrer", [0, 0, 0.7, 0, 18.5, 9.0, 1.3, -1.0]),
    ("gaussian", [0, 0, 0.8, 0, 16.0, 3.0]),
    ("moffat", [0, 0, 0.7, 0, 16.5, 2.5, 3.0]),
]


@pytest.mark.parametrize("kind,par", MAG_PROFILES)
def test_magnitude_sets_the_total_flux(kind, par):
    # the amplitude derived from m gives the profile the flux 10^(-0.4 (m - m0)):
    # 2 pi q int_0^inf I(r) r dr by quadrature along the major axis
    m0 = 22.5
    amp = oracle.mag_amplitude(kind, par, m0)
    p = list(par)
    p[4] = amp
    rmax = p[5] if kind == "ferrer" else np.inf
    f = lambda r: oracle.component_value(kind, p, r, 0.0) * r
    flux = 2 * math.pi * par[2] * si.quad(f, 0, rmax, limit=400, epsabs=0, epsrel=1e-11)[0]
    assert flux == pytest.approx(10 ** (-0.4 * (par[4] - m0)), rel=1e-8)


def test_magnitude_has_no_relation_for_king_and_the_skies():
    for kind, par in (("king", [0, 0, 1, 0, 18, 2, 10, 2]), ("sky", [18]), ("tsky", [18, 0, 0])):
        assert math.isnan(oracle.mag_amplitude(kind, par + [0] * (8 - len(par)), 22.5))


def test_model_in_magnitudes_equals_the_model_in_amplitudes():
    H, W, K = 24, 20, 5
    spec_m = synth.ModelSpec().add("sersic", "gal", H, W, mag_zero=22.5)
    spec_a = synth.ModelSpec().add("sersic", "gal", H, W)
    pm = np.array([[10.2, 11.7, 0.6, 0.3, 17.0, 4.0, 1.7]])
    pa = pm.copy()
    pa[0, 4] = oracle.mag_amplitude("sersic", pm[0], 22.5)
    psf = np.zeros((1, K, K))
    psf[0, 2, 2] = 1.0
    np.testing.assert_allclose(oracle.model_images(spec_m, pm, psf, H, W), oracle.model_images(spec_a, pa, psf, H, W),
                               rtol=1e-13)
    # one magnitude brighter is a factor 10^0.4 in every pixel
    pm2 = pm.copy()
    pm2[0, 4] -= 1.0
    np.testing.assert_allclose(oracle.model_images(spec_m, pm2, psf, H, W),
                               10 ** 0.4 * oracle.model_images(spec_m, pm, psf, H, W), rtol=1e-12)


# ---------------------------------------------------------------------------
# gradient-descent (Adam) fit, the paper's own optimiser
# ---------------------------------------------------------------------------

def _sky_case(seed=0, H=6, W=5):
    rng = np.random.default_rng(seed)
    spec = synth.ModelSpec().add("sky", "sky", H, W, convolve=False)
    D = 3.0 + rng.normal(0, 1.0, (1, H, W))
    S = rng.uniform(0.5, 2.0, (1, H, W))
    psf = np.ones((1, 1, 1))
    w = 1.0 / S ** 2
    return spec, D, S, psf, float((w * D).sum() / w.sum())


def test_adam_first_step_moves_by_lr_times_the_scale():
    # step 1 from zero moments moves u by lr * scale * sign(-g): here up by lr * max(|p0|, 1)
    spec, D, S, psf, pstar = _sky_case()
    p0 = np.array([[pstar - 5.0]])
    best, c2 = oracle.fit_adam(spec, p0, psf, D, S, n_iter=1, lr=0.1, eps=1e-12)
    assert best[0, 0] == pytest.approx(p0[0, 0] + 0.1 * abs(p0[0, 0]), rel=1e-12)
    w = 1.0 / S ** 2
    assert c2[0] == pytest.approx(float((w * (D - best[0, 0]) ** 2).sum()), rel=1e-12)


def test_adam_reaches_the_weighted_mean_of_a_flat_sky():
    spec, D, S, psf, pstar = _sky_case(1)
    best, _ = oracle.fit_adam(spec, np.array([[0.5]]), psf, D, S, n_iter=1500, lr=1e-2)
    # steps are at most lr * max(|p0|, 1) = 0.01: the minimum, 2.4 away, is reached after ~240
    # steps, and Adam with a constant rate then hovers within a few steps of it
    assert abs(best[0, 0] - pstar) <= 3e-2


# ---------------------------------------------------------------------------
# bootstrap: SplitMix64 and the resampling
# ---------------------------------------------------------------------------

def test_splitmix64_reference_outputs():
    # the published generator from state 0: the first outputs of its Weyl sequence
    s, out = 0, []
    for _ in range(4):
        s = (s + 0x9E3779B97F4A7C15) & ((1 << 64) - 1)
        out.append(oracle.splitmix64(s))
    assert out == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]


def test_bootstrap_counts_are_a_resampling_with_replacement():
    mask = np.zeros((40, 50), np.uint8)
    mask[5:15, 10:30] = 1
    N = int((mask == 0).sum())
    c = oracle.bootstrap_counts(mask, seed=7, g=3, b=11)
    assert c.sum() == N and (c[mask != 0] == 0).all()
    # multinomial with equal cells: P(count = 0) -> exp(-1), mean count 1, variance 1 - 1/N
    frac0 = float((c[mask == 0] == 0).mean())
    assert abs(frac0 - math.exp(-1)) < 4 * math.sqrt(math.exp(-1) * (1 - math.exp(-1)) / N)
    assert abs(c[mask == 0].var() - (1 - 1 / N)) < 0.1
    # replicates and galaxies draw differently; the same (seed, g, b) draws the same
    assert not np.array_equal(c, oracle.bootstrap_counts(mask, seed=7, g=3, b=12))
    assert not np.array_equal(c, oracle.bootstrap_counts(mask, seed=7, g=4, b=11))
    assert np.array_equal(c, oracle.bootstrap_counts(mask, seed=7, g=3, b=11))


def test_bootstrap_of_a_flat_sky_is_the_error_of_the_weighted_mean():
    # sky-only model with equal sigma: the refit is the weighted mean of the resampled pixels,
    # whose spread over replicates is close to the standard error of the mean of the data
    H, W = 12, 12
    rng = np.random.default_rng(5)
    spec = synth.ModelSpec().add("sky", "sky", H, W, convolve=False)
    D = 3.0 + rng.normal(0, 1.0, (1, H, W))
    S = np.ones((1, H, W))
    sig, M = oracle.bootstrap(spec, np.array([[D.mean()]]), np.ones((1, 1, 1)), D, S, n_boot=200, seed=1)
    assert M[0] == 200
    sem = D.std() / math.sqrt(H * W)
    assert abs(sig[0, 0] - sem) <= 0.15 * sem


# ---------------------------------------------------------------------------
# boxiness (Eqs. r-rmin with B != 0, Eq. rbox)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("B", [-1.0, -0.5, 0.0, 0.5, 2.0])
def test_rbox_is_pi_over_the_superellipse_area(B):
    p = 2.0 + B
    area = 4 * si.quad(lambda x: (1 - x ** p) ** (1 / p), 0, 1, epsabs=0, epsrel=1e-12)[0]
    assert oracle.rbox(B) == pytest.approx(math.pi / area, rel=1e-9)


def test_boxy_radius_limits():
    par = [0.0, 0.0, 0.5, 0.3, 1.0, 2.0]  # expdisk: I = exp(-r / 2)
    c, s = math.cos(0.3), math.sin(0.3)
    for X, Y in ((1.3, 0.2), (0.7, -0.9), (-2.0, 0.4)):
        x, y = c * X - s * Y, s * X + c * Y  # the point with rotated coordinates (X, Y)
        r0 = -2.0 * math.log(oracle.component_value("expdisk", par, x, y))
        assert r0 == pytest.approx(math.hypot(X, Y / 0.5), rel=1e-12)
        rb = -2.0 * math.log(oracle.component_value("expdisk", par, x, y, B=1.0))
        assert rb == pytest.approx((abs(X) ** 3 + abs(Y / 0.5) ** 3) ** (1 / 3), rel=1e-12)
        rbig = -2.0 * math.log(oracle.component_value("expdisk", par, x, y, B=60.0))
        assert rbig == pytest.approx(max(abs(X), abs(Y / 0.5)), rel=2e-2)  # towards a box


@pytest.mark.parametrize("B", [-0.6, 0.8])
def test_boxy_magnitude_flux_by_2d_quadrature(B):
    # the amplitude from m (with r_box) gives the boxy profile the flux 10^(-0.4 (m - m0)):
    # integrate the image over the plane
    m0, par = 22.5, [0.0, 0.0, 0.6, 0.4, 17.0, 2.0]  # gaussian, fwhm 2
    amp = oracle.mag_amplitude("gaussian", par, m0) * oracle.rbox(B)
    p = list(par)
    p[4] = amp
    f = lambda y, x: oracle.component_value("gaussian", p, x, y, B=B)
    flux = si.dblquad(f, -12, 12, -12, 12, epsabs=0, epsrel=1e-9)[0]
    assert flux == pytest.approx(10 ** (-0.4 * (par[4] - m0)), rel=1e-6)


def test_lm_checkpoint_and_resume_is_exact():
    # a fit stopped at max_iter = k with the raw best point (canonical = 0) and its damping,
    # then resumed from them with max_iter N - k + 1, ends exactly where the uninterrupted
    # N-iteration fit ends: the first resumed evaluation repeats the best point's A, g, chi^2
    b = synth.draw_small(seed=17, G=8, H=32, W=32, K=7)
    psf = np.stack([_gauss_psf(b.K, 1.5)] * b.G)
    truth = synth.galaxy_slots(b)
    Mt = oracle.model_images(b.spec, truth, psf, b.H, b.W)
    D, S = synth.noisy_image(Mt, b.z)
    N, k = 60, 5
    tight = dict(tol=1e-12, xtol=1e-10, gtol=1e-13)
    full = oracle.fit(b.spec, b.init, psf, D, S, None, oracle.FitOptions(max_iter=N, **tight))
    lam = np.zeros(b.G)
    part = oracle.fit(b.spec, b.init, psf, D, S, None, oracle.FitOptions(max_iter=k, canonical=0, **tight), lam)
    run = part["status"] == 2
    assert run.sum() >= 4 and (lam[run] > 0).all()
    rest = oracle.fit(b.spec, part["params"][run], psf[run], D[run], S[run], None,
                      oracle.FitOptions(max_iter=N - k + 1, **tight), lam[run].copy())
    for key in ("params", "chi2", "status", "sigma_p"):
        np.testing.assert_array_equal(rest[key], full[key][run])
    np.testing.assert_array_equal(rest["iters"], full["iters"][run] - k + 1)
