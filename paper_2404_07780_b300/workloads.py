"""Synthetic workloads on the device, rendered by the library's own forward model.

The draws (parameters, PSF shapes, masks, noise) come from synth.py; the
images are rendered by gm_model: PSFs as unconvolved Moffat/Gaussian
components on their own grids, normalised to unit sum; the truth scene as
the model (plus contaminants); data D = M + sigma z with
sigma^2 = sky_var + max(M, 0)/gain.
"""
from __future__ import annotations

import numpy as np

from . import gm, synth


def render_equal(b: synth.Batch, device):
    """(image, sigma, mask, psf) CUDA tensors of an equal-stamp batch."""
    import torch
    G, K = b.G, b.K
    kind = "moffat" if b.psf_kind == "moffat" else "gaussian"
    psfspec = synth.ModelSpec().add(kind, "psf", K, K, convolve=False)
    one = torch.ones((G, 1, 1), dtype=torch.float32, device=device)
    psf = gm.gm_model(psfspec, torch.from_numpy(np.ascontiguousarray(b.psf_par)).to(device), one, K, K)
    psf = (psf / psf.sum((1, 2), keepdim=True)).contiguous()
    M = torch.zeros((G, b.H, b.W), dtype=torch.float32, device=device)
    for spec, par in b.truth_parts():
        M += gm.gm_model(spec, torch.from_numpy(np.ascontiguousarray(par)).to(device), psf, b.H, b.W)
    sigma = torch.sqrt(b.sky_var + M.clamp(min=0) / b.gain)
    image = M + sigma * torch.from_numpy(b.z).to(device=device, dtype=torch.float32)
    mask = torch.from_numpy(b.mask).to(device) if b.mask is not None else None
    return image.contiguous(), sigma.contiguous(), mask, psf


def render_psfs_packed(kind: str, psf_par: np.ndarray, ks: np.ndarray, device):
    """Unit-sum PSFs of per-galaxy side ks, packed back to back (FP32)."""
    import torch
    G = len(ks)
    k = np.asarray(ks, np.int64)
    psf_geom = np.stack([k, k, np.ones_like(k)], 1)
    psfspec = synth.ModelSpec().add("moffat" if kind == "moffat" else "gaussian", "psf", 64, 64, convolve=False)
    one = torch.ones(G, dtype=torch.float32, device=device)
    psf = gm.gm_model(psfspec, torch.from_numpy(np.ascontiguousarray(psf_par)).to(device), one, geom=psf_geom)
    gid = torch.repeat_interleave(torch.arange(G, device=device), torch.from_numpy(k * k).to(device))
    sums = torch.zeros(G, dtype=torch.float64, device=device).index_add_(0, gid, psf.double())
    return (psf / sums[gid].float()).contiguous()


def render_uneven(rb: synth.RaggedBatch, device, z=None):
    """(image, sigma, psf) packed CUDA tensors of an uneven batch; z (packed standard normals,
    a CUDA tensor) replaces the batch's own draws when given."""
    import torch
    psf = render_psfs_packed(rb.psf_kind, rb.psf_par, rb.geom[:, 2], device)
    M = gm.gm_model(rb.spec, torch.from_numpy(np.ascontiguousarray(rb.truth)).to(device), psf, geom=rb.geom)
    sigma = torch.sqrt(rb.sky_var + M.clamp(min=0) / rb.gain)
    if z is None:
        z = torch.from_numpy(rb.z).to(device=device, dtype=torch.float32)
    image = M + sigma * z
    del M
    return image.contiguous(), sigma.contiguous(), psf
