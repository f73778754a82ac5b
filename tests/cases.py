"""Seeded test cases shared by the parity tests.

Inputs are drawn by paper_2404_07780_b300.synth (random numbers only) and
rendered by the FP64 oracle; everything the CUDA path receives is the float32
rounding of these arrays, and the oracle is re-run on exactly those rounded
values, so both sides see identical bits.
"""
from __future__ import annotations

import math

import numpy as np

import oracle
from paper_2404_07780_b300 import synth


def psf_image(kind: str, par, K: int) -> np.ndarray:
    """Unit-sum PSF rendered by the oracle, rounded to float32."""
    p = oracle.component_image(kind, par, K, K)
    return (p / p.sum()).astype(np.float32)


def psf_stack(batch: synth.Batch) -> np.ndarray:
    return np.stack([psf_image(batch.psf_kind, batch.psf_par[g], batch.K) for g in range(batch.G)])


class Case:
    """A batch ready for both paths: float32 arrays plus the float64 views the oracle uses."""

    def __init__(self, spec, params, psf, image, sigma, mask, H, W, init=None, truth=None):
        self.spec = spec
        self.params = np.ascontiguousarray(params, np.float64)
        self.init = None if init is None else np.ascontiguousarray(init, np.float64)
        self.truth = truth
        self.psf = np.ascontiguousarray(psf, np.float32)
        self.image = np.ascontiguousarray(image, np.float32)
        self.sigma = np.ascontiguousarray(sigma, np.float32)
        self.mask = None if mask is None else np.ascontiguousarray(mask, np.uint8)
        self.H, self.W = H, W

    @property
    def G(self):
        return self.params.shape[0]

    def torch(self, device="cuda"):
        import torch
        t = lambda a: None if a is None else torch.from_numpy(a).to(device)
        return dict(params=t(self.params), psf=t(self.psf), image=t(self.image), sigma=t(self.sigma),
                    mask=t(self.mask))


def from_batch(b: synth.Batch, at: str = "init") -> Case:
    """Render the truth scene of a synth batch with the oracle and add the drawn noise."""
    psf = psf_stack(b)
    Mt = sum(oracle.model_images(sp, pa, psf.astype(np.float64), b.H, b.W) for sp, pa in b.truth_parts())
    D, S = synth.noisy_image(Mt, b.z.astype(np.float64), b.sky_var, b.gain)
    truth = synth.galaxy_slots(b)
    params = b.init if at == "init" else truth
    return Case(b.spec, params, psf, D, S, b.mask, b.H, b.W, init=b.init, truth=truth)


def scale_of(spec) -> np.ndarray:
    """Per-slot absolute scale used for parameter tolerances: 1 px (centre), 1 rad (position
    angle), 1 sky unit (sky level, and per pixel for the tilted sky's slopes), 1 for the
    boxiness B (its exponent is B + 2); 0 (purely relative) for the rest."""
    s = np.zeros(spec.n_slots)
    for i, name in enumerate(spec.names):
        role = name.split(".")[-1]
        s[i] = 1.0 if role in ("x0", "y0", "pa", "Isky", "kx", "ky", "B") else 0.0
    return s


def pa_slots(spec):
    return [i for i, n in enumerate(spec.names) if n.endswith(".pa")]


def q_of_pa(spec, pa_slot):
    """The axis-ratio slot of the component whose position angle lives in pa_slot."""
    for comp in spec.components:
        if comp.kind != "sky" and comp.slots[3] == pa_slot:
            return comp.slots[2]
    return None


def angle_diff(a, b):
    d = np.abs(a - b) % math.pi
    return np.minimum(d, math.pi - d)


class UnevenCase:
    """An uneven batch (stamps and PSFs of per-galaxy size) as packed float32 arrays, plus the
    one-galaxy Cases the oracle runs on."""

    def __init__(self, spec, geom, cases):
        self.spec = spec
        self.geom = np.ascontiguousarray(geom, np.int32)
        self.cases = cases
        self.params = np.concatenate([c.params for c in cases])
        self.init = np.concatenate([c.init for c in cases])
        self.truth = np.concatenate([c.truth for c in cases])
        self.psf = np.concatenate([c.psf.ravel() for c in cases])
        self.image = np.concatenate([c.image.ravel() for c in cases])
        self.sigma = np.concatenate([c.sigma.ravel() for c in cases])
        masked = [c.mask is not None for c in cases]
        self.mask = (np.concatenate([(c.mask if c.mask is not None else np.zeros(c.image.shape, np.uint8)).ravel()
                                     for c in cases]) if any(masked) else None)

    @property
    def G(self):
        return len(self.cases)

    def offsets(self):
        hw = self.geom[:, 0].astype(np.int64) * self.geom[:, 1]
        return np.concatenate([[0], np.cumsum(hw)])

    def split(self, packed, per_pixel=1):
        """Per-galaxy [per_pixel, h, w] views of a packed per-pixel array."""
        o = self.offsets() * per_pixel
        return [np.asarray(packed[o[g]:o[g + 1]]).reshape(per_pixel, self.geom[g, 0], self.geom[g, 1])
                for g in range(self.G)]

    def torch(self, device="cuda"):
        import torch
        t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(device)
        return dict(params=t(self.params), psf=t(self.psf), image=t(self.image), sigma=t(self.sigma),
                    mask=t(self.mask))


def uneven_from(rb: synth.RaggedBatch, at: str = "init") -> UnevenCase:
    """Render every galaxy of an uneven synth batch with the oracle (one-galaxy batches)."""
    cases = [from_batch(rb.galaxy(g), at=at) for g in range(rb.G)]
    return UnevenCase(rb.spec, rb.geom, cases)
