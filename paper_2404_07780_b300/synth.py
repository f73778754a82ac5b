"""Seeded synthetic inputs for batched galaxy-profile fitting.

This module holds configuration and random draws only: model descriptions
(which component uses which parameter slot), parameter draws from the stated
prior ranges, PSF and contaminant *descriptions*, mask geometry and the
Gaussian noise draws.  It evaluates no light profile, no convolution and no
chi^2; whoever consumes these inputs renders the images with its own forward
model (the CUDA library for benchmark workloads, the FP64 oracle for test
cases), so that the library and the oracle share nothing but these draws.

The SDSS g-band sample of the paper (Sec. 3: 128x128 stamps, 41x41 PSFs,
SExtractor masks) is not available; the draws below take its shapes and
stand in for it.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Parameter order of each component kind: the geometric subset p_G (centre,
# axis ratio, position angle) first, then the radial subset p_L (Sec. 2).
PARAM_NAMES = {
    "sersic": ("x0", "y0", "q", "pa", "Ie", "Re", "n"),
    "expdisk": ("x0", "y0", "q", "pa", "I0", "rs"),
    "ferrer": ("x0", "y0", "q", "pa", "I0", "rout", "a", "b"),
    "king": ("x0", "y0", "q", "pa", "I0", "rc", "rt", "alpha"),
    "gaussian": ("x0", "y0", "q", "pa", "I0", "fwhm"),
    "moffat": ("x0", "y0", "q", "pa", "I0", "fwhm", "n"),
    "sky": ("Isky",),
    "tsky": ("Isky", "kx", "ky"),
}

# Fitted in log space (positive scale and amplitude parameters) and default
# bounds, by parameter role.
_LOG_ROLES = {"Ie", "I0", "Re", "rs", "rout", "rc", "rt", "fwhm", "n", "alpha", "a", "q"}
_BIG = 1e30


def _default_bounds(kind: str, role: str, H: int, W: int) -> tuple[float, float]:
    if role == "x0":
        return 0.0, float(W)
    if role == "y0":
        return 0.0, float(H)
    if role == "q":
        # above 1 the same ellipse turned by pi/2: the fit may pass through q = 1 and the
        # result is rewritten with q <= 1 at the end
        return 0.05, 20.0
    if role == "pa":
        return -_BIG, _BIG
    if role in ("Ie", "I0"):
        return 1e-8, 1e8
    if role in ("Re", "rs", "rout", "rc", "rt", "fwhm"):
        return 1e-2, 1e3
    if role == "n":
        return (0.2, 10.0) if kind == "sersic" else (1.01, 100.0)
    if role == "alpha":
        return 0.1, 10.0
    if role == "a":
        return 0.05, 20.0
    if role == "b":
        return -5.0, 1.99
    return -_BIG, _BIG


@dataclass
class Component:
    kind: str
    convolve: bool
    slots: list[int]
    mag_zero: float | None = None   # amplitude slot holds a magnitude with this zero point
    boxy: bool = False              # a boxiness slot B follows the profile's parameters


@dataclass
class ModelSpec:
    """Which components make up the model and how they map onto parameter slots.

    A slot shared by several components (for example a common centre) is one
    fitted parameter.  free/log/lo/hi are per slot."""
    components: list[Component] = field(default_factory=list)
    names: list[str] = field(default_factory=list)
    free: list[bool] = field(default_factory=list)
    log: list[bool] = field(default_factory=list)
    lo: list[float] = field(default_factory=list)
    hi: list[float] = field(default_factory=list)

    @property
    def n_slots(self) -> int:
        return len(self.names)

    @property
    def n_free(self) -> int:
        return int(sum(self.free))

    def slot(self, name: str) -> int:
        return self.names.index(name)

    def add(self, kind: str, prefix: str, H: int, W: int, convolve: bool = True,
            shared: dict[str, int] | None = None, fixed: tuple[str, ...] = (),
            mag_zero: float | None = None, boxy: bool = False) -> "ModelSpec":
        """Append a component; roles in `shared` reuse an existing slot.  With mag_zero the
        amplitude slot (Ie / I0) is a magnitude with that zero point (named `mag`, fitted
        linearly, bounded to 0..40).  With boxy a boxiness slot `B` (bounds -1.9..10) follows
        the profile's parameters."""
        shared = shared or {}
        slots = []
        roles = list(PARAM_NAMES[kind]) + (["B"] if boxy else [])
        for k, role in enumerate(roles):
            if role in shared:
                slots.append(shared[role])
                continue
            is_mag = mag_zero is not None and k == 4
            lo, hi = (0.0, 40.0) if is_mag else ((-1.9, 10.0) if role == "B" else _default_bounds(kind, role, H, W))
            self.names.append(f"{prefix}.{'mag' if is_mag else role}")
            self.free.append(role not in fixed)
            self.log.append(role in _LOG_ROLES and not is_mag)
            self.lo.append(lo)
            self.hi.append(hi)
            slots.append(len(self.names) - 1)
        self.components.append(Component(kind, convolve, slots, mag_zero, boxy))
        return self


def single_sersic_sky(H: int, W: int) -> ModelSpec:
    """One Sersic component (convolved) plus a flat sky (not convolved): 8 free slots."""
    s = ModelSpec()
    s.add("sersic", "bulge", H, W)
    s.add("sky", "sky", H, W, convolve=False)
    return s


def bulge_disk_sky(H: int, W: int) -> ModelSpec:
    """Sersic bulge + Sersic disk with n fixed at 1 sharing the centre, plus sky.

    13 slots, 12 free (the bulge+disk recipe of App. B with a common centre)."""
    s = ModelSpec()
    s.add("sersic", "bulge", H, W)
    s.add("sersic", "disk", H, W, shared={"x0": 0, "y0": 1}, fixed=("n",))
    s.add("sky", "sky", H, W, convolve=False)
    return s


def bulge_bar_nucleus_sky(H: int, W: int) -> ModelSpec:
    """Sersic bulge + Ferrer bar (a fixed) + circular Gaussian nucleus + sky, common centre."""
    s = ModelSpec()
    s.add("sersic", "bulge", H, W)
    s.add("ferrer", "bar", H, W, shared={"x0": 0, "y0": 1}, fixed=("a",))
    s.add("gaussian", "nuc", H, W, shared={"x0": 0, "y0": 1}, fixed=("q", "pa"))
    s.add("sky", "sky", H, W, convolve=False)
    return s


def contaminant_spec(H: int, W: int) -> ModelSpec:
    """One free-standing Gaussian source (convolved): the contaminants of truth scenes."""
    return ModelSpec().add("gaussian", "cont", H, W)


# --------------------------------------------------------------------------
# Draws
# --------------------------------------------------------------------------

def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _logu(g: np.random.Generator, lo: float, hi: float, size) -> np.ndarray:
    return np.exp(g.uniform(math.log(lo), math.log(hi), size))


@dataclass
class Batch:
    """One synthetic batch of equal-size stamps (all arrays numpy, FP64 unless noted).

    The truth scene is the fitted model at `truth` plus, for every k, the
    contaminant component at `contaminants[:, k]` (zero amplitude when unused)."""
    spec: ModelSpec            # the fitted model
    H: int
    W: int
    K: int
    truth: np.ndarray          # [G, spec.n_slots]
    init: np.ndarray           # [G, spec.n_slots] default starting point
    psf_kind: str              # "gaussian" or "moffat"
    psf_par: np.ndarray        # [G, n] component parameters of the PSF profile
    mask: np.ndarray | None    # [G, H, W] uint8, nonzero = excluded
    z: np.ndarray              # [G, H, W] standard normal noise draws
    contaminants: np.ndarray | None = None   # [G, n_blobs, 6] Gaussian parameters
    sky_var: float = 4.0
    gain: float = 4.0

    def truth_parts(self):
        """(spec, params [G, n_slots]) pairs whose model images sum to the truth scene."""
        parts = [(self.spec, self.truth)]
        if self.contaminants is not None:
            cs = contaminant_spec(self.H, self.W)
            for k in range(self.contaminants.shape[1]):
                parts.append((cs, self.contaminants[:, k]))
        return parts

    @property
    def G(self) -> int:
        return self.truth.shape[0]


def psf_params(kind: str, fwhm: np.ndarray, K: int, beta: float = 3.0) -> np.ndarray:
    """Component parameters of a circular PSF profile centred on pixel (c, c) of a K x K grid."""
    c = K / 2.0  # centre of pixel (c, c) is at x = y = c + 0.5 = K / 2
    G = fwhm.shape[0]
    if kind == "gaussian":
        return np.stack([np.full(G, c), np.full(G, c), np.ones(G), np.zeros(G), np.ones(G), fwhm], 1)
    return np.stack([np.full(G, c), np.full(G, c), np.ones(G), np.zeros(G), np.ones(G), fwhm,
                     np.full(G, beta)], 1)


def draw_small(seed: int = 0, G: int = 16, H: int = 64, W: int = 64, K: int = 15) -> Batch:
    """Plain single-Sersic batch: 16 x 64x64, Gaussian PSF FWHM 1.5 px on 15x15, no mask.

    x0, y0 within +-2 px of the centre; Ie log-uniform 1-100; Re uniform 2-10;
    n log-uniform 0.5-4; q uniform 0.3-1; PA uniform 0-pi; sky uniform 0-5."""
    g = rng(seed)
    spec = single_sersic_sky(H, W)
    truth = np.stack([
        W / 2 + g.uniform(-2, 2, G), H / 2 + g.uniform(-2, 2, G), g.uniform(0.3, 1.0, G),
        g.uniform(0, math.pi, G), _logu(g, 1, 100, G), g.uniform(2, 10, G), _logu(g, 0.5, 4, G),
        g.uniform(0, 5, G)], 1)
    init = np.tile(np.array([W / 2, H / 2, 0.65, math.pi / 2, 10.0, 6.0, math.sqrt(2.0), 2.5]), (G, 1))
    z = g.standard_normal((G, H, W))
    return Batch(spec, H, W, K, truth, init, "gaussian", psf_params("gaussian", np.full(G, 1.5), K), None, z)


def draw_sdss(seed: int = 1000, G: int = 8192, H: int = 128, W: int = 128, K: int = 41,
              max_blobs: int = 5) -> Batch:
    """SDSS-shaped single-Sersic batch with contaminants hidden under a mask.

    Sersic + sky; n log-uniform 0.5-6; Re uniform 2-25 px; q uniform 0.2-1;
    log10 Ie uniform 0-3; centre within +-2 px; PA uniform 0-pi; sky uniform
    0-5.  Per-galaxy Moffat PSF, beta = 3, FWHM uniform 1.2-1.8 px, 41x41.
    0-5 elliptical mask blobs per stamp (semi-axis 2-8 px, q 0.3-1, centre at
    least 10 px from the galaxy), each hiding a Gaussian contaminant whose
    peak is 5-50 sky sigma."""
    g = rng(seed)
    spec = single_sersic_sky(H, W)
    x0 = W / 2 + g.uniform(-2, 2, G)
    y0 = H / 2 + g.uniform(-2, 2, G)
    gal = np.stack([x0, y0, g.uniform(0.2, 1.0, G), g.uniform(0, math.pi, G),
                    10 ** g.uniform(0, 3, G), g.uniform(2, 25, G), _logu(g, 0.5, 6, G),
                    g.uniform(0, 5, G)], 1)
    fwhm = g.uniform(1.2, 1.8, G)
    nblob = g.integers(0, max_blobs + 1, G)
    sig_sky = math.sqrt(4.0)
    cont = np.zeros((G, max_blobs, 6))
    mask = np.zeros((G, H, W), np.uint8)
    yy, xx = np.meshgrid(H - 0.5 - np.arange(H), np.arange(W) + 0.5, indexing="ij")
    for gi in range(G):
        for k in range(max_blobs):
            semi = g.uniform(2, 8)
            bq = g.uniform(0.3, 1.0)
            bpa = g.uniform(0, math.pi)
            rad = g.uniform(10 + semi, 0.5 * min(H, W) - 2)
            ang = g.uniform(0, 2 * math.pi)
            cx, cy = x0[gi] + rad * math.cos(ang), y0[gi] + rad * math.sin(ang)
            peak = g.uniform(5, 50) * sig_sky
            if k >= nblob[gi]:
                continue
            # contaminant: Gaussian with 3 sigma = semi-axis, same shape as the blob
            cont[gi, k] = [cx, cy, bq, bpa, peak, 2.0 * math.sqrt(2.0 * math.log(2.0)) * semi / 3.0]
            dx, dy = xx - cx, yy - cy
            X = math.cos(bpa) * dx + math.sin(bpa) * dy
            Y = -math.sin(bpa) * dx + math.cos(bpa) * dy
            mask[gi][(X / semi) ** 2 + (Y / (bq * semi)) ** 2 <= 1.0] = 1
    # unused contaminant slots: zero amplitude, harmless geometry
    unused = cont[:, :, 4] == 0
    cont[unused] = [W / 2, H / 2, 1.0, 0.0, 0.0, 1.0]
    init = np.tile(np.array([W / 2, H / 2, 0.6, math.pi / 2, math.sqrt(1000.0), 13.5, math.sqrt(3.0), 2.5]),
                   (G, 1))
    z = g.standard_normal((G, H, W), dtype=np.float32)
    return Batch(spec, H, W, K, gal, init, "moffat", psf_params("moffat", fwhm, K), mask, z, cont)


def draw_bulge_disk(seed: int = 2000, G: int = 64, H: int = 96, W: int = 96, K: int | None = None) -> Batch:
    """Bulge + disk batch (equal-size stamps): Sersic bulge (n 1-6) + Sersic disk with n = 1
    (Re_d = 1.5-4 x Re_b, own q and PA) + sky, common centre; Moffat PSF beta 3, FWHM 1.2-1.8 px,
    side K (odd, 25-51 when not given)."""
    g = rng(seed)
    spec = bulge_disk_sky(H, W)
    if K is None:
        K = int(g.choice(np.arange(25, 52, 2)))
    reb = g.uniform(1.5, 8, G)
    truth = np.stack([
        W / 2 + g.uniform(-2, 2, G), H / 2 + g.uniform(-2, 2, G),
        g.uniform(0.3, 1.0, G), g.uniform(0, math.pi, G), 10 ** g.uniform(0.5, 3, G), reb, g.uniform(1, 6, G),
        g.uniform(0.2, 1.0, G), g.uniform(0, math.pi, G), 10 ** g.uniform(0, 2, G), reb * g.uniform(1.5, 4, G),
        np.ones(G), g.uniform(0, 5, G)], 1)
    init = np.tile(np.array([W / 2, H / 2, 0.65, math.pi / 2, 10 ** 1.75, 4.0, math.sqrt(6.0),
                             0.6, math.pi / 2, 10.0, 11.0, 1.0, 2.5]), (G, 1))
    z = g.standard_normal((G, H, W))
    return Batch(spec, H, W, K, truth, init, "moffat", psf_params("moffat", g.uniform(1.2, 1.8, G), K), None, z)


def draw_bulge_bar_nucleus(seed: int = 3000, G: int = 64, H: int = 96, W: int = 96, K: int = 41) -> Batch:
    """Sersic bulge + Ferrer bar (r_out 5-20 px, a = 2 fixed, b 0-1.99) + circular Gaussian nucleus
    (sigma 0.5-1.5 px) + sky, common centre; Moffat PSF as draw_sdss."""
    g = rng(seed)
    spec = bulge_bar_nucleus_sky(H, W)
    fw = 2.0 * math.sqrt(2.0 * math.log(2.0))
    cols = {
        "bulge.x0": W / 2 + g.uniform(-2, 2, G), "bulge.y0": H / 2 + g.uniform(-2, 2, G),
        "bulge.q": g.uniform(0.5, 1.0, G), "bulge.pa": g.uniform(0, math.pi, G),
        "bulge.Ie": _logu(g, 1, 100, G), "bulge.Re": g.uniform(2, 10, G), "bulge.n": g.uniform(1, 4, G),
        "bar.q": g.uniform(0.2, 0.5, G), "bar.pa": g.uniform(0, math.pi, G), "bar.I0": _logu(g, 1, 30, G),
        "bar.rout": g.uniform(5, 20, G), "bar.a": np.full(G, 2.0), "bar.b": g.uniform(0, 1.99, G),
        "nuc.q": np.ones(G), "nuc.pa": np.zeros(G), "nuc.I0": _logu(g, 5, 100, G),
        "nuc.fwhm": fw * g.uniform(0.5, 1.5, G), "sky.Isky": g.uniform(0, 5, G)}
    truth = np.stack([cols[n] for n in spec.names], 1)
    init_vals = {"bulge.x0": W / 2, "bulge.y0": H / 2, "bulge.q": 0.75, "bulge.pa": math.pi / 2, "bulge.Ie": 10.0,
                 "bulge.Re": 6.0, "bulge.n": 2.0, "bar.q": 0.35, "bar.pa": math.pi / 4, "bar.I0": math.sqrt(30.0),
                 "bar.rout": 12.5, "bar.a": 2.0, "bar.b": 1.0, "nuc.q": 1.0, "nuc.pa": 0.0,
                 "nuc.I0": math.sqrt(500.0), "nuc.fwhm": fw, "sky.Isky": 2.5}
    init = np.tile(np.array([init_vals[n] for n in spec.names]), (G, 1))
    z = g.standard_normal((G, H, W))
    return Batch(spec, H, W, K, truth, init, "moffat", psf_params("moffat", g.uniform(1.2, 1.8, G), K), None, z)


@dataclass
class RaggedBatch:
    """A batch whose stamps and PSFs differ in size from galaxy to galaxy.

    geom[g] = (h, w, k): stamp rows and columns and PSF side of galaxy g.
    Per-pixel arrays are packed back to back in galaxy order (the layout of
    gm_batch.geom); `galaxy(g)` views one galaxy as a one-galaxy Batch."""
    spec: ModelSpec            # the fitted model (position bounds sized for the largest stamp)
    geom: np.ndarray           # [G, 3] int32
    truth: np.ndarray          # [G, spec.n_slots]
    init: np.ndarray           # [G, spec.n_slots]
    psf_kind: str
    psf_par: np.ndarray        # [G, n] PSF profile parameters (centred on each PSF's own grid)
    mask: np.ndarray | None    # packed uint8 [sum h*w]
    z: np.ndarray              # packed standard normal draws [sum h*w]
    sky_var: float = 4.0
    gain: float = 4.0

    @property
    def G(self) -> int:
        return self.truth.shape[0]

    def pix_offsets(self) -> np.ndarray:
        """[G+1] start of each stamp in the packed arrays."""
        hw = self.geom[:, 0].astype(np.int64) * self.geom[:, 1]
        return np.concatenate([[0], np.cumsum(hw)])

    def psf_offsets(self) -> np.ndarray:
        """[G+1] start of each PSF in the packed PSF array."""
        return np.concatenate([[0], np.cumsum(self.geom[:, 2].astype(np.int64) ** 2)])

    def galaxy(self, g: int) -> Batch:
        h, w, k = (int(v) for v in self.geom[g])
        o = self.pix_offsets()
        sl = slice(o[g], o[g + 1])
        mask = None if self.mask is None else self.mask[sl].reshape(1, h, w)
        return Batch(self.spec, h, w, k, self.truth[g:g + 1], self.init[g:g + 1], self.psf_kind,
                     self.psf_par[g:g + 1], mask, self.z[sl].reshape(1, h, w).astype(np.float64),
                     None, self.sky_var, self.gain)


def draw_uneven_bulge_disk(seed: int = 2000, G: int = 32768, sides=(48, 64, 96, 128, 192, 256),
                           ks=tuple(range(25, 52, 2)), noise: bool = True) -> RaggedBatch:
    """Uneven bulge + disk batch: square stamps with side uniform over `sides`, Moffat PSF
    (beta 3, FWHM 1.2-1.8 px) with odd side uniform over `ks`; Sersic bulge (n 1-6) + Sersic
    disk with n = 1 (Re_d = 1.5-4 x Re_b, own q and PA) + sky, common centre within +-2 px of
    the stamp centre.  Radii scale with the stamp side (bulge Re 1.5-8 px at side 96).  With
    noise=False no noise is drawn (z is empty; the caller supplies its own draws)."""
    g = rng(seed)
    side = g.choice(np.asarray(sides), G)
    k = g.choice(np.asarray(ks), G)
    geom = np.stack([side, side, k], 1).astype(np.int32)
    smax = int(max(sides))
    spec = bulge_disk_sky(smax, smax)
    f = side / 96.0
    reb = g.uniform(1.5, 8, G) * f
    truth = np.stack([
        side / 2 + g.uniform(-2, 2, G), side / 2 + g.uniform(-2, 2, G),
        g.uniform(0.3, 1.0, G), g.uniform(0, math.pi, G), 10 ** g.uniform(0.5, 3, G), reb, g.uniform(1, 6, G),
        g.uniform(0.2, 1.0, G), g.uniform(0, math.pi, G), 10 ** g.uniform(0, 2, G), reb * g.uniform(1.5, 4, G),
        np.ones(G), g.uniform(0, 5, G)], 1)
    init = np.stack([side / 2, side / 2, np.full(G, 0.65), np.full(G, math.pi / 2), np.full(G, 10 ** 1.75),
                     4.0 * f, np.full(G, math.sqrt(6.0)), np.full(G, 0.6), np.full(G, math.pi / 2),
                     np.full(G, 10.0), 11.0 * f, np.ones(G), np.full(G, 2.5)], 1)
    fwhm = g.uniform(1.2, 1.8, G)
    c = k / 2.0  # each PSF centred on pixel (c, c) of its own k x k grid, as psf_params
    psf_par = np.stack([c, c, np.ones(G), np.zeros(G), np.ones(G), fwhm, np.full(G, 3.0)], 1)
    npix = int((side.astype(np.int64) ** 2).sum())
    z = g.standard_normal(npix, dtype=np.float32) if noise else np.zeros(0, np.float32)
    return RaggedBatch(spec, geom, truth, init, "moffat", psf_par, None, z)


def draw_uneven_sersic(seed: int, geom, mask_frac: float = 0.0, ie=(1.0, 100.0)) -> RaggedBatch:
    """Single Sersic + sky on stamps of the given (h, w, k) each, Moffat PSF (beta 3, FWHM
    1.2-1.8 px): centre within +-1 px of the stamp centre, Ie log-uniform over `ie`, Re uniform
    1.5-0.3 min(h, w) (at least 1.5), n log-uniform 0.5-4, q uniform 0.3-1, PA uniform 0-pi,
    sky uniform 0-5; with mask_frac > 0 each pixel is masked with that probability."""
    g = rng(seed)
    geom = np.asarray(geom, np.int32).reshape(-1, 3)
    G = len(geom)
    h, w, k = (geom[:, i].astype(np.float64) for i in range(3))
    hmax, wmax = int(geom[:, 0].max()), int(geom[:, 1].max())
    spec = single_sersic_sky(hmax, wmax)
    re_hi = np.maximum(0.3 * np.minimum(h, w), 1.5)
    truth = np.stack([w / 2 + g.uniform(-1, 1, G), h / 2 + g.uniform(-1, 1, G), g.uniform(0.3, 1.0, G),
                      g.uniform(0, math.pi, G), _logu(g, ie[0], ie[1], G), 1.5 + g.uniform(0, 1, G) * (re_hi - 1.5),
                      _logu(g, 0.5, 4, G), g.uniform(0, 5, G)], 1)
    init = np.stack([w / 2, h / 2, np.full(G, 0.65), np.full(G, math.pi / 2), np.full(G, 10.0),
                     0.5 * (1.5 + re_hi), np.full(G, math.sqrt(2.0)), np.full(G, 2.5)], 1)
    psf_par = np.stack([k / 2, k / 2, np.ones(G), np.zeros(G), np.ones(G), g.uniform(1.2, 1.8, G),
                        np.full(G, 3.0)], 1)
    npix = int((geom[:, 0].astype(np.int64) * geom[:, 1]).sum())
    z = g.standard_normal(npix)
    mask = (g.uniform(0, 1, npix) < mask_frac).astype(np.uint8) if mask_frac > 0 else None
    return RaggedBatch(spec, geom, truth, init, "moffat", psf_par, mask, z)


def noisy_image(model_true: np.ndarray, z: np.ndarray, sky_var: float = 4.0, gain: float = 4.0):
    """Data and sigma map for a truth image: sigma^2 = sky_var + max(M, 0)/gain, D = M + sigma z."""
    sigma = np.sqrt(sky_var + np.maximum(model_true, 0.0) / gain)
    return model_true + sigma * z, sigma


def galaxy_slots(batch: Batch) -> np.ndarray:
    """The truth parameters of the fitted model."""
    return batch.truth
