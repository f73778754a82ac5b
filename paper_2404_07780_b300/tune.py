"""Autotuner of the fused pass's launch shape.

The fused model+Jacobian kernel has three launch knobs (include/gm.h,
gm_tune_set): channel pairs per shared-memory pass, pairs per thread and
groups of 128 threads.  Which shape is fastest depends on the PSF side K
(window size and shared memory) and on the number of free parameters P
(channels to correlate, registers of the reduction).  `autotune` times every
shape the device can run on a sample of the caller's own batch, through
gm_chi2_grad (one full pass), and keeps the fastest; `save` writes the
choices to a JSON cache keyed by device name, and `apply_cache` pushes the
cached choices for the current device into the library (the binding does
this when it loads the library).
"""
from __future__ import annotations

import json
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(_HERE, "tuning.json")

# (pairs per pass, pairs per thread, thread groups): every pair of a pass has a group and no
# group is idle in a full pass; (4, 2, 4) and (2, 2, 4) are the 512-thread shapes whose
# groups split two pairs by PSF rows, two or four groups per two pairs
SHAPES = [(pp, cpt, groups) for cpt in (1, 2) for groups in range(1, (4 if cpt == 1 else 2) + 1)
          for pp in range(1, 5) if groups <= pp <= cpt * groups] + [(4, 2, 4), (2, 2, 4)]


def device_name() -> str:
    import torch
    return torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"


def read_cache(path: str = CACHE) -> dict:
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)


def apply_cache(lib, path: str = CACHE, device: str | None = None) -> int:
    """Set every cached shape of this device in the library; returns how many."""
    data = read_cache(path)
    if not data:
        return 0
    try:
        dev = device or device_name()
    except Exception:  # no usable torch / device: nothing to apply
        return 0
    n = 0
    for e in data.get(dev, {}).get("entries", []):
        if lib.gm_tune_set(e["K"], e["P"], e["pairs_per_pass"], e["pairs_per_thread"], e["groups"]) == 0:
            n += 1
    return n


def save(entries: list[dict], path: str = CACHE, device: str | None = None):
    """Merge entries (dicts with K, P, pairs_per_pass, pairs_per_thread, groups, ms) into the cache."""
    data = read_cache(path)
    dev = device or device_name()
    old = {(e["K"], e["P"]): e for e in data.get(dev, {}).get("entries", [])}
    for e in entries:
        old[(e["K"], e["P"])] = e
    data[dev] = {"entries": sorted(old.values(), key=lambda e: (e["K"], e["P"]))}
    with open(path, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
        f.write("\n")


def autotune(spec, params, image, sigma, mask, psf, geom=None, reps: int = 3, warmup: int = 1,
             verbose: bool = False) -> dict:
    """Time every launch shape on this batch (gm_chi2_grad, CUDA events) and set the fastest.

    Returns the entry {K, P, pairs_per_pass, pairs_per_thread, groups, ms, candidates}."""
    import numpy as np
    import torch
    from . import gm
    lib = gm.load()
    d = spec if isinstance(spec, gm.gm_model_desc) else gm.desc_from_spec(spec)
    P = sum(1 for s in range(d.n_slots) if d.is_free[s])
    K = int(psf.shape[-1]) if geom is None else int(np.asarray(geom).reshape(-1, 3)[:, 2].max())
    stream = torch.cuda.current_stream()

    def run():
        gm.gm_chi2_grad(d, params, image, sigma, mask, psf, want_grad=True, want_jtj=False, geom=geom)

    prev = None
    timings = {}
    try:
        for shape in SHAPES:
            gm.gm_tune_set(K, P, *shape)
            run()
            if gm.gm_tune_last_shape() != shape:  # not a shape this batch can run
                continue
            for _ in range(warmup):
                run()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                run()
            e1.record(stream)
            torch.cuda.synchronize()
            timings[shape] = e0.elapsed_time(e1) / reps
            if verbose:
                print(f"K={K} P={P} shape {shape}: {timings[shape]:.3f} ms")
    finally:
        gm.gm_tune_set(K, P, 0, 0, 0)
    if not timings:
        raise gm.GMError("no launch shape ran")
    best = min(timings, key=timings.get)
    gm.gm_tune_set(K, P, *best)
    return {"K": K, "P": P, "pairs_per_pass": best[0], "pairs_per_thread": best[1], "groups": best[2],
            "ms": timings[best], "candidates": {f"{a},{b},{c}": t for (a, b, c), t in sorted(timings.items())}}


def tune_workloads(path: str = CACHE, G: int = 512, verbose: bool = True) -> list[dict]:
    """Tune the shapes of the library's standard workloads (a sample of G galaxies of each
    recipe, rendered by the library) and merge them into the cache."""
    import numpy as np
    import torch
    from . import gm, synth, workloads
    dev = torch.device("cuda")
    entries = []

    def render(b):
        image, sigma, mask, psf = workloads.render_equal(b, dev)
        return torch.from_numpy(b.init).to(dev), image, sigma, mask, psf

    batches = [synth.draw_small(seed=1, G=G), synth.draw_sdss(seed=1000, G=G)]
    batches += [synth.draw_bulge_disk(seed=2000, G=G, H=128, W=128, K=k) for k in range(25, 52, 2)]
    batches += [synth.draw_bulge_bar_nucleus(seed=3000, G=G, H=96, W=96, K=41)]
    for b in batches:
        p0, image, sigma, mask, psf = render(b)
        e = autotune(b.spec, p0, image, sigma, mask, psf, verbose=verbose)
        entries.append(e)
        if verbose:
            print(f"K={e['K']} P={e['P']}: best {e['pairs_per_pass']},{e['pairs_per_thread']},{e['groups']} "
                  f"{e['ms']:.3f} ms", flush=True)
    save(entries, path)
    return entries


if __name__ == "__main__":
    import sys
    sys.exit(0 if tune_workloads() else 1)
