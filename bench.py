"""Benchmark: converged galaxy fits/s on the SDSS-shaped single-Sersic workload.

Workload (synthetic, stands in for the paper's 8,289 SDSS g-band stamps):
8,192 galaxies, 128x128 float32 stamps, Sersic + sky (8 free parameters),
per-galaxy Moffat PSF (beta 3, FWHM 1.2-1.8 px, 41x41), sigma^2 = 4 + M/4,
uint8 masks hiding 0-5 Gaussian contaminants, default-start Levenberg-Marquardt
to a relative chi^2 decrease < 1e-6 (max 200 evaluations).

A step is one gm_fit_batch call over the whole batch (validation, set-up,
every LM iteration of fused model+Jacobian+chi^2 pass and FP64 step, final
covariance).  `value` counts galaxies that ended CONVERGED.  Inputs are 1.2 GB
per batch, larger than the 126 MB L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--no-extra]

On one GPU the default line also carries `other_workloads`: the small, gradient, inference,
uneven and learned-start workloads, each run once at its full size in a child process after the fit's own
measurement (a few minutes in all; --no-extra leaves them out, and so does a run on N > 1 GPUs).
Their figures are context: `value`, `e2e` and `roofline` are the SDSS-shaped fit's.

The reference arm (--impl reference) is the FP64 CPU oracle timed on this
host's cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

_ROOT = os.path.dirname(os.path.abspath(__file__))
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)

from paper_2404_07780_b300 import synth  # noqa: E402

METRIC = "converged galaxy fits/sec on 1 B300 at matched χ² tol; model+Jacobian Gpix/s"
UNIT = "fits/s"
TOL = 1e-6
MAX_ITER = 200
PEAKS_PATH = os.path.join(_ROOT, "MEASURED_PEAKS.json")
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12  # SMs x FP32 lanes x 2 FLOP x max SM clock
# DRAM bytes (read + write) of the SDSS-shaped fit's fused pass (k_fused<NORMAL, 8, 2, WIDE>, the
# tuned shape) per galaxy evaluated, from one ncu capture of a 1,024-galaxy pass of this workload
# (705.6 MB); traffic grows in proportion to the galaxies a pass evaluates, so a launch's traffic is
# this times its galaxies
FUSED_DRAM_BYTES_PER_GALAXY = 705.609e6 / 1024


def fused_name(P, shape):
    """The fused-pass instance a launch shape (pairs per pass, per thread, groups) runs."""
    pp, cpt, groups = shape
    wide = ",WIDE" if cpt == 2 and groups > 2 else ""
    return f"k_fused<NORMAL,{P},{cpt}{wide}> ({pp} pairs per pass, {cpt} per thread, {groups} x 128 threads)"


# the same for the uneven workload's fused pass (k_fused<NORMAL, 12, 2, WIDE>, the tuned shape), per
# stamp pixel evaluated (2,617.4 MB for a 2,048-galaxy pass of 45.59 M pixels)
UNEVEN_DRAM_BYTES_PER_PIXEL = 2617.424e6 / 45591296


def workload_config(G, H, K):
    return {"workload": f"SDSS-shaped single-Sersic+sky fit, {G} x {H}x{H} float32 stamps, per-galaxy Moffat PSF "
                        f"{K}x{K}, masked contaminants, default-start LM to dchi2/chi2<{TOL:g}",
            "galaxies": G, "stamp": [H, H], "psf": [K, K], "free_params": 8, "tol": TOL, "max_iter": MAX_ITER,
            "l2": "inputs 1.2 GB per batch > 126 MB L2 (no flush)"}


# ---------------------------------------------------------------------------
# multi-process plumbing (one process per GPU; galaxies are independent, so
# every rank fits its own batch: weak scaling, no data-path collective)
# ---------------------------------------------------------------------------

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def reduce_max(x: float, world: int, device=None) -> float:
    """Max of a host scalar over ranks (the timing reduction; no data path)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def rank_seed(rank: int) -> int:
    """Each rank draws its own batch of the same recipe."""
    return 1000 + rank


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int = 0):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def stop(self) -> dict:
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[3 + k] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ---------------------------------------------------------------------------
# workload on the device (rendered by the library's own forward model)
# ---------------------------------------------------------------------------

def render_workload(b: synth.Batch, device):
    """PSFs, truth images, noisy data and sigma maps on the device, rendered by gm_model."""
    from paper_2404_07780_b300 import workloads
    return workloads.render_equal(b, device)


def inbounds_taps(H, W, K):
    """Sum over output pixels of the PSF taps that fall inside the stamp."""
    c = (K - 1) // 2
    rows = sum(min(K, H - i + c) - max(0, c - i) for i in range(H))
    cols = sum(min(K, W - j + c) - max(0, c - j) for j in range(W))
    return rows * cols


# ---------------------------------------------------------------------------
# CPU oracle timing (the cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

def oracle_sample_fit(b: synth.Batch, idx, keep=None, max_iter=None):
    """Render galaxies idx of the workload with the oracle and fit them with its LM; returns (converged, seconds).
    With keep (a dict), also stores the float32 inputs, the start and the oracle's result there."""
    import oracle
    sub = synth.Batch(b.spec, b.H, b.W, b.K, b.truth[idx], b.init[idx], b.psf_kind, b.psf_par[idx],
                      None if b.mask is None else b.mask[idx], b.z[idx],
                      None if b.contaminants is None else b.contaminants[idx])
    psf = np.stack([oracle.component_image(sub.psf_kind, sub.psf_par[g], sub.K, sub.K) for g in range(len(idx))])
    psf = (psf / psf.sum((1, 2), keepdims=True)).astype(np.float32).astype(np.float64)
    Mt = sum(oracle.model_images(sp, pa, psf, sub.H, sub.W) for sp, pa in sub.truth_parts())
    D, S = synth.noisy_image(Mt, sub.z.astype(np.float64), sub.sky_var, sub.gain)
    D = D.astype(np.float32).astype(np.float64)
    S = S.astype(np.float32).astype(np.float64)
    t0 = time.perf_counter()
    r = oracle.fit(sub.spec, sub.init, psf, D, S, sub.mask, oracle.FitOptions(tol=TOL, max_iter=max_iter or MAX_ITER))
    dt = time.perf_counter() - t0
    if keep is not None:
        keep.update(spec=sub.spec, init=sub.init, psf=psf.astype(np.float32), image=D.astype(np.float32),
                    sigma=S.astype(np.float32), mask=sub.mask, ref=r)
    return int((r["status"] == 1).sum()), dt


TIGHT = dict(tol=1e-12, xtol=1e-10, gtol=1e-13)  # the parity tests' stopping rule


def oracle_match(keep, device, max_iter=None, tight=False) -> dict:
    """The GPU fit of the galaxies the oracle fitted (same float32 inputs, start and options) against the
    oracle's: the fraction that ends with the oracle's status and, when converged, at its minimum (chi^2
    within 1e-5 relative and every parameter within 1e-4 max(|p|, s_p), s_p = 1 px / 1 rad / 1 sky
    unit); and the fractions whose chi^2 is above / below the oracle's by more than sqrt(2 dof)."""
    import torch
    from paper_2404_07780_b300 import gm
    import oracle
    spec, ref = keep["spec"], keep["ref"]
    kw = dict(TIGHT) if tight else dict(tol=TOL)
    kw["max_iter"] = max_iter or MAX_ITER
    if tight:  # the oracle refits the sample with the tight rule (not timed)
        f64 = lambda a: None if a is None else a.astype(np.float64)
        ref = oracle.fit(spec, keep["init"], f64(keep["psf"]), f64(keep["image"]), f64(keep["sigma"]), keep["mask"],
                         oracle.FitOptions(**kw))
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(device)
    got = gm.gm_fit_batch(spec, t(keep["init"]), t(keep["image"]), t(keep["sigma"]), t(keep["mask"]),
                          t(keep["psf"]), gm.FitOptions(**kw))
    got = {k: v.cpu().numpy() for k, v in got.items()}
    scale = np.array([1.0 if n.split(".")[-1] in ("x0", "y0", "pa", "Isky") else 0.0 for n in spec.names])
    bar = 1e-4 * np.maximum(np.abs(ref["params"]), scale)
    diff = np.abs(got["params"] - ref["params"])
    for s_, n in enumerate(spec.names):
        if n.endswith(".pa"):
            d = diff[:, s_] % np.pi
            diff[:, s_] = np.minimum(d, np.pi - d)
            diff[ref["params"][:, s_ - 1] > 0.95, s_] = 0.0  # q precedes PA; PA undefined for round profiles
    conv = ref["status"] == 1
    same_status = got["status"] == ref["status"]
    chi2_ok = np.abs(got["chi2"] - ref["chi2"]) <= 1e-5 * ref["chi2"]
    params_ok = (diff <= bar).all(axis=1)
    match = same_status & (~conv | (chi2_ok & params_ok))
    sd = np.sqrt(2.0 * np.maximum(ref["dof"], 1))
    n = len(ref["status"])
    return {"oracle_match_frac": float(match.mean()), "galaxies": n, "same_status_frac": float(same_status.mean()),
            "chi2_within_1e-5_frac": float((chi2_ok | (got["chi2"] < ref["chi2"])).mean()),
            "gpu_chi2_higher_by_sigma_frac": float((got["chi2"] - ref["chi2"] > sd).mean()),
            "gpu_chi2_lower_by_sigma_frac": float((ref["chi2"] - got["chi2"] > sd).mean()),
            "worst_param_over_bar": float(np.max(diff[conv] / bar[conv])) if conv.any() else None,
            "options": f"tol {kw['tol']:g}, max_iter {kw['max_iter']}, same start (the default start) and float32 "
                       "inputs"}


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args, world, rank):
    """The FP64 oracle as it stands, on this host's cores, on bounded samples of the workload."""
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    threads = oracle.max_threads()
    per_step = max(1, min(64, threads))
    b = synth.draw_sdss(seed=rank_seed(0), G=per_step * (args.warmup + args.steps))
    conv = 0
    secs = 0.0
    for s in range(args.warmup + args.steps):
        idx = np.arange(s * per_step, (s + 1) * per_step)
        c, dt = oracle_sample_fit(b, idx)
        if s >= args.warmup:
            conv += c
            secs += dt
    value = conv / secs if secs > 0 else 0.0
    G, H, K = args.galaxies, 128, 41
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(G, H, K),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{per_step} galaxies of the workload per step, {args.steps} timed steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------

def run_gpu(args, world, rank, local):
    import torch
    from paper_2404_07780_b300 import gm
    from paper_2404_07780_b300.build import build_lib

    build_lib()
    gm.load()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = dist_init(world, "nccl")
    G, H, K = args.galaxies, 128, 41
    b = synth.draw_sdss(seed=rank_seed(rank), G=G, H=H, W=H, K=K)
    image, sigma, mask, psf = render_workload(b, dev)
    p0 = torch.from_numpy(b.init).to(dev)
    fitter = gm.Fitter(b.spec, G, H, H, K, device=dev)
    opts = gm.FitOptions(tol=TOL, max_iter=MAX_ITER)
    params = torch.empty_like(p0)

    def step():
        params.copy_(p0)
        return fitter.fit(params, image, sigma, mask, psf, opts)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    converged = 0
    fused_ms = 0.0
    evals = 0
    launches = 0
    iters = []
    torch.cuda.synchronize()
    e0.record(stream)
    stats = []
    for _ in range(args.steps):
        # library calls only: torch ops here would be slowed by the nvidia-smi sampler
        step()
        stats.append(gm.gm_fit_last_stats())
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    for st in stats:
        fused_ms += st["fused_ms"]
        evals += st["galaxy_evals"]
        launches += 4 + 3 * st["passes"]  # geometry, validation, init, finish; k_planes, k_fused, k_lm_step per pass
        converged += st["converged"]
        iters.append(st["iters_sum"] / G)
        print(f"step: library wall {st['wall_ms']:.1f} ms, profile {st['profile_ms']:.1f} ms, "
              f"fused {st['fused_ms']:.1f} ms, lm steps {st['step_ms']:.1f} ms, passes {st['passes']}",
              file=sys.stderr)
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms_max = reduce_max(ms, world, dev)
    conv_all = reduce_sum(converged, world, dev)
    value = conv_all / (ms_max / 1e3)

    # end to end through the public API from pinned host buffers
    h_img = image.cpu().pin_memory()
    h_sig = sigma.cpu().pin_memory()
    h_msk = mask.cpu().pin_memory()
    h_psf = psf.cpu().pin_memory()
    h_p0 = p0.cpu().pin_memory()
    h_out_p = torch.empty_like(h_p0).pin_memory()
    h_out_st = torch.empty(G, dtype=torch.int32).pin_memory()
    h_out_c2 = torch.empty(G, dtype=torch.float64).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in (h_img, h_sig, h_msk, h_psf, h_p0))
    d2h = sum(t.numel() * t.element_size() for t in (h_out_p, h_out_st, h_out_c2))
    e_steps = max(1, args.steps)
    # two device input sets: step k+1's inputs are copied on a second stream while step k
    # fits (every step still copies its own inputs from pinned host memory and reads its
    # results back); the sets are allocated before the timed region
    hosts = (h_img, h_sig, h_msk, h_psf, h_p0)
    dbuf = [tuple(torch.empty_like(h, device=dev) for h in hosts) for _ in range(2)]
    copy_stream = torch.cuda.Stream(device=dev)
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    used = [torch.cuda.Event(), torch.cuda.Event()]

    def issue_copy(k):
        with torch.cuda.stream(copy_stream):
            if k >= 2:
                copy_stream.wait_event(used[k % 2])  # the fit of step k-2 is done with this set
            for d, h in zip(dbuf[k % 2], hosts):
                d.copy_(h, non_blocking=True)
            copied[k % 2].record(copy_stream)

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e_conv = 0
    issue_copy(0)
    for k in range(e_steps):
        if k + 1 < e_steps:
            issue_copy(k + 1)
        stream.wait_event(copied[k % 2])
        d_img, d_sig, d_msk, d_psf, d_p = dbuf[k % 2]
        out = fitter.fit(d_p, d_img, d_sig, d_msk, d_psf, opts)
        used[k % 2].record(stream)
        h_out_p.copy_(out["params"], non_blocking=True)
        h_out_st.copy_(out["status"], non_blocking=True)
        h_out_c2.copy_(out["chi2"], non_blocking=True)
        stream.synchronize()
        e_conv += int((h_out_st == gm.ST_CONVERGED).sum().item())
    torch.cuda.synchronize()
    e_secs = reduce_max(time.perf_counter() - t0, world, dev)
    e_value = reduce_sum(e_conv, world, dev) / e_secs

    # roofline of the dominant kernel: the fused pass, FP32 ALU bound
    taps = inbounds_taps(H, H, K)
    nch = 1 + 7  # model + one channel per free parameter of the convolved Sersic
    flops = 2.0 * nch * taps * evals
    achieved = flops / (fused_ms / 1e3) / 1e12
    gpix = evals * H * H / (fused_ms / 1e3) / 1e9
    launches_fused = sum(st["passes"] for st in stats)
    roof = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP32_PEAK_TFLOPS,
            "traffic": FUSED_DRAM_BYTES_PER_GALAXY * evals / max(launches_fused, 1),
            "traffic_unit": "bytes per launch (average launch)",
            "algorithmic_bytes": (9 + 32) * H * H * evals / max(launches_fused, 1),
            "kernel": fused_name(8, gm.gm_tune_last_shape()),
            "peak_source": "derived: 148 SMs x 128 FP32 FMA/clk x 2 FLOP x 2032 MHz (no FP32 figure is measured)"}

    cpu = None
    match = match_tight = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        threads = oracle.max_threads()
        n = max(1, min(64, threads))
        cb = synth.draw_sdss(seed=rank_seed(0), G=n, H=H, W=H, K=K)
        keep = {}
        c, dt = oracle_sample_fit(cb, np.arange(n), keep)
        cpu = {"value": c / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"first {n} galaxies of the workload recipe (seed {rank_seed(0)}), rendered and fitted by "
                         f"the FP64 oracle, default start, tol {TOL:g}"}
        match = oracle_match(keep, dev)
        match_tight = oracle_match(keep, dev, tight=True)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": workload_config(G, H, K), "gpix_per_s": gpix,
                "converged_frac": converged / (G * args.steps), "mean_iters": float(np.mean(iters)),
                "roofline": roof, "cpu_baseline": cpu, "oracle_match": match, "oracle_match_tight": match_tight,
                "e2e": {"value": e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "gpu_launches": launches, "clocks": clocks}
        if world == 1 and not args.no_extra:
            line["other_workloads"] = run_other_workloads()
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# the other workloads, summarised in the default line
# ---------------------------------------------------------------------------

# (workload, extra arguments, child time limit in s): each runs at its full size in a process of its
# own after the SDSS-shaped fit's line is complete, so that nothing there can change that line
OTHER_WORKLOADS = (("small", (), 180), ("gradient", ("--no-cpu-baseline",), 240), ("inference", (), 180),
                   ("uneven", ("--no-cpu-baseline", "--steps", "1", "--warmup", "1"), 360),
                   ("learned", ("--steps", "1", "--warmup", "1"), 420))


def summarize_workload(name: str, l: dict) -> dict:
    """The figures of a workload's own JSON line that the default line carries."""
    keys = ("value", "unit", "ms_per_step", "steps", "warmup", "converged_frac", "mean_iters", "gpu_launches")
    s = {k: l[k] for k in keys if k in l}
    s["workload"] = l["config"]["workload"]
    r = l.get("roofline") or {}
    s["roofline"] = {k: r[k] for k in ("bound", "achieved", "peak", "unit", "frac", "pass_frac", "kernel") if k in r}
    if l.get("e2e"):
        s["e2e"] = l["e2e"]["value"]
    c = l.get("clocks") or {}
    s["clocks"] = {"sm_mhz": c.get("sm_mhz"), "sm_max_mhz": c.get("sm_max_mhz"), "reasons": c.get("reasons")}
    if name == "small":
        s["us_per_iteration"] = l["us_per_iteration"]
        s["us_per_iteration_kernels"] = l["us_per_iteration_kernels"]
        if l.get("cpu_baseline"):
            s["oracle_fits_per_s"] = l["cpu_baseline"]["value"]
            s["oracle_us_per_iteration"] = l["cpu_baseline"]["us_per_iteration"]
        if l.get("oracle_match"):
            s["oracle_match_frac"] = l["oracle_match"]["oracle_match_frac"]
    elif name == "gradient":
        s["normal_equations_ms_per_step"] = l["normal_equations_ms_per_step"]
        s["speedup_vs_normal_equations"] = l["speedup_vs_normal_equations"]
        s["adam_vs_lm"] = l["adam_vs_lm"]
    elif name == "inference":
        s["tensor"] = l["tensor"]
        s["layers_ms"] = {k: v["ms"] for k, v in l["layers"].items()}
    elif name == "learned":
        s["speedup_vs_default_start"] = l["speedup_vs_default_start"]
        s["default_start"] = l["default_start"]
        s["learned_start"] = l["learned_start"]
        s["inference"] = {k: l["inference"][k] for k in ("ms", "tflops", "frac")}
        s["train_s"] = l["training"]["train_s"]
    return s


def run_other_workloads() -> dict:
    """Run every other workload of this file once, in a child process each, and summarise its line;
    a child that fails or runs out of time is recorded as such."""
    out = {}
    for name, extra, limit in OTHER_WORKLOADS:
        cmd = [sys.executable, os.path.abspath(__file__), "--workload", name, "--no-extra", *extra]
        t0 = time.perf_counter()
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=limit, cwd=_ROOT)
        except subprocess.TimeoutExpired:
            out[name] = {"error": f"no line within {limit} s", "args": list(extra)}
            continue
        lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
        if r.returncode != 0 or not lines:
            tail = (r.stderr.strip().splitlines() or ["(no output)"])[-1]
            out[name] = {"error": f"exit {r.returncode}: {tail[:200]}", "args": list(extra)}
            continue
        try:
            s = summarize_workload(name, json.loads(lines[-1]))
        except (KeyError, TypeError, ValueError) as e:
            s = {"error": f"unreadable line: {e!r}"}
        s["args"] = list(extra)
        s["wall_s"] = time.perf_counter() - t0
        out[name] = s
    return out


# ---------------------------------------------------------------------------
# uneven workload: stamps and PSFs of per-galaxy size in one batch
# ---------------------------------------------------------------------------

UNEVEN_SIDES = (48, 64, 96, 128, 192, 256)
UNEVEN_KS = tuple(range(25, 52, 2))


def render_uneven(rb: synth.RaggedBatch, device):
    """Packed PSFs (unit sum), data and sigma of an uneven batch, rendered by gm_model."""
    from paper_2404_07780_b300 import workloads
    return workloads.render_uneven(rb, device)


def uneven_config(G):
    return {"workload": f"uneven bulge+disk+sky fit, {G} stamps of side uniform over {list(UNEVEN_SIDES)} "
                        f"(float32), per-galaxy Moffat PSF of odd side 25-51, 12 free parameters, default-start LM "
                        f"to dchi2/chi2<{TOL:g}",
            "galaxies": G, "sides": list(UNEVEN_SIDES), "psf_sides": [UNEVEN_KS[0], UNEVEN_KS[-1]],
            "free_params": 12, "tol": TOL, "max_iter": MAX_ITER,
            "l2": "inputs ~5.8 GB per batch > 126 MB L2 (no flush)"}


def run_uneven(args, world, rank, local):
    """Uneven workload: G bulge+disk+sky galaxies on square stamps of mixed side with mixed PSF
    sides, one gm_fit_batch call per step (one persistent pass per LM iteration, CUDA graph)."""
    import torch
    from paper_2404_07780_b300 import gm
    from paper_2404_07780_b300.build import build_lib

    build_lib()
    gm.load()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = dist_init(world, "nccl")
    G = args.galaxies
    rb = synth.draw_uneven_bulge_disk(seed=2000 + rank, G=G, sides=UNEVEN_SIDES, ks=UNEVEN_KS)
    image, sigma, psf = render_uneven(rb, dev)
    p0 = torch.from_numpy(rb.init).to(dev)
    fitter = gm.Fitter(rb.spec, G, device=dev, geom=rb.geom)
    opts = gm.FitOptions(tol=TOL, max_iter=MAX_ITER)
    params = torch.empty_like(p0)

    def step():
        params.copy_(p0)
        return fitter.fit(params, image, sigma, None, psf, opts)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    stats = []
    for _ in range(args.steps):
        step()
        stats.append(gm.gm_fit_last_stats())
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    for st in stats:
        print(f"step: library wall {st['wall_ms']:.1f} ms, profile {st['profile_ms']:.1f} ms, "
              f"fused {st['fused_ms']:.1f} ms, lm steps {st['step_ms']:.1f} ms, passes {st['passes']}",
              file=sys.stderr)
    converged = sum(st["converged"] for st in stats)
    fused_ms = sum(st["fused_ms"] for st in stats)
    launches = sum(4 + 3 * st["passes"] for st in stats)
    ms_max = reduce_max(ms, world, dev)
    value = reduce_sum(converged, world, dev) / (ms_max / 1e3)

    # per-galaxy work: every step repeats the same deterministic fits
    iters = fitter.iters.cpu().numpy().astype(np.float64)
    taps = np.zeros(G)
    for side in UNEVEN_SIDES:
        for k in UNEVEN_KS:
            sel = (rb.geom[:, 0] == side) & (rb.geom[:, 2] == k)
            if sel.any():
                taps[sel] = inbounds_taps(side, side, k)
    nch = 1 + 11  # model + one channel per free parameter of the convolved bulge and disk
    flops = args.steps * float((2.0 * nch * taps * iters).sum())
    pix = args.steps * float((rb.geom[:, 0].astype(np.float64) * rb.geom[:, 1] * iters).sum())
    achieved = flops / (fused_ms / 1e3) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP32_PEAK_TFLOPS,
            "traffic": UNEVEN_DRAM_BYTES_PER_PIXEL * pix / max(sum(st["passes"] for st in stats), 1),
            "traffic_unit": "bytes per launch (average launch)",
            "algorithmic_bytes": 56.0 * pix / max(sum(st["passes"] for st in stats), 1),
            "kernel": fused_name(12, gm.gm_tune_last_shape()) + ", uneven items, per-class TMA maps",
            "peak_source": "derived: 148 SMs x 128 FP32 FMA/clk x 2 FLOP x 2032 MHz (no FP32 figure is measured)"}

    # end to end through the public API from pinned host buffers
    h_img = image.cpu().pin_memory()
    h_sig = sigma.cpu().pin_memory()
    h_psf = psf.cpu().pin_memory()
    h_p0 = p0.cpu().pin_memory()
    h_out_p = torch.empty_like(h_p0).pin_memory()
    h_out_st = torch.empty(G, dtype=torch.int32).pin_memory()
    h_out_c2 = torch.empty(G, dtype=torch.float64).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in (h_img, h_sig, h_psf, h_p0))
    d2h = sum(t.numel() * t.element_size() for t in (h_out_p, h_out_st, h_out_c2))
    e_steps = max(1, min(args.steps, 2))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e_conv = 0
    for _ in range(e_steps):
        d_img = h_img.to(dev, non_blocking=True)
        d_sig = h_sig.to(dev, non_blocking=True)
        d_psf = h_psf.to(dev, non_blocking=True)
        d_p = h_p0.to(dev, non_blocking=True)
        out = fitter.fit(d_p, d_img, d_sig, None, d_psf, opts)
        h_out_p.copy_(out["params"], non_blocking=True)
        h_out_st.copy_(out["status"], non_blocking=True)
        h_out_c2.copy_(out["chi2"], non_blocking=True)
        torch.cuda.synchronize()
        e_conv += int((h_out_st == gm.ST_CONVERGED).sum().item())
    e_secs = reduce_max(time.perf_counter() - t0, world, dev)
    e_value = reduce_sum(e_conv, world, dev) / e_secs

    cpu = None
    match = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        threads = oracle.max_threads()
        n = max(1, min(32, threads))
        # one class of the recipe (96x96 stamps, 41x41 PSF): the oracle fits a batch of equal stamps
        cb = synth.draw_uneven_bulge_disk(seed=2000, G=n, sides=(96,), ks=(41,))
        sub = synth.Batch(cb.spec, 96, 96, 41, cb.truth, cb.init, cb.psf_kind, cb.psf_par, None,
                          cb.z.reshape(n, 96, 96).astype(np.float64))
        c, dt = oracle_sample_fit(sub, np.arange(n))
        cpu = {"value": c / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{n} galaxies of the recipe's 96x96 / K=41 class (seed 2000), rendered and fitted by the "
                         f"FP64 oracle, default start, tol {TOL:g}"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": uneven_config(G), "gpix_per_s": pix / (fused_ms / 1e3) / 1e9,
                "converged_frac": converged / (G * args.steps), "mean_iters": float(iters.mean()),
                "roofline": roof, "cpu_baseline": cpu,
                "e2e": {"value": e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "gpu_launches": launches, "clocks": clocks}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# small workload: the plain single-Sersic batch, launch-latency bound
# ---------------------------------------------------------------------------

SMALL_MAX_ITER = 100


def run_small(args, world, rank, local):
    """16 x 64x64 single-Sersic+sky fits with a 15x15 Gaussian PSF (FWHM 1.5 px), no mask, LM from the
    default start, max_iter 100: one gm_fit_batch call per step.  At this size a pass is a few tiles,
    so the time per LM iteration (the three kernels of a pass and the host poll) is what is reported."""
    import torch
    from paper_2404_07780_b300 import gm
    from paper_2404_07780_b300.build import build_lib

    build_lib()
    gm.load()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = dist_init(world, "nccl")
    G = args.galaxies
    b = synth.draw_small(seed=rank_seed(rank), G=G)
    image, sigma, mask, psf = render_workload(b, dev)
    p0 = torch.from_numpy(b.init).to(dev)
    fitter = gm.Fitter(b.spec, G, b.H, b.W, b.K, device=dev)
    opts = gm.FitOptions(tol=TOL, max_iter=SMALL_MAX_ITER)
    params = torch.empty_like(p0)

    def step():
        params.copy_(p0)
        return fitter.fit(params, image, sigma, mask, psf, opts)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    stats = []
    for _ in range(args.steps):
        step()
        stats.append(gm.gm_fit_last_stats())
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    passes = sum(st["passes"] for st in stats)
    converged = sum(st["converged"] for st in stats)
    fused_ms = sum(st["fused_ms"] for st in stats)
    profile_ms = sum(st["profile_ms"] for st in stats)
    step_ms = sum(st["step_ms"] for st in stats)
    evals = sum(st["galaxy_evals"] for st in stats)
    ms_max = reduce_max(ms, world, dev)
    value = reduce_sum(converged, world, dev) / (ms_max / 1e3)
    iters = fitter.iters.cpu().numpy().astype(np.float64)
    taps = inbounds_taps(b.H, b.W, b.K)
    achieved = 2.0 * 8 * taps * evals / (fused_ms / 1e3) / 1e12

    # end to end through the public API from pinned host buffers
    hosts = [t.cpu().pin_memory() for t in (image, sigma, psf, p0)]
    h_out = [torch.empty_like(fitter.status, device="cpu").pin_memory(),
             torch.empty_like(fitter.chi2, device="cpu").pin_memory(), torch.empty_like(p0, device="cpu").pin_memory()]
    h2d = sum(t.numel() * t.element_size() for t in hosts)
    d2h = sum(t.numel() * t.element_size() for t in h_out)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e_conv = 0
    for _ in range(args.steps):
        d_img, d_sig, d_psf, d_p = (h.to(dev, non_blocking=True) for h in hosts)
        out = fitter.fit(d_p, d_img, d_sig, None, d_psf, opts)
        h_out[0].copy_(out["status"], non_blocking=True)
        h_out[1].copy_(out["chi2"], non_blocking=True)
        h_out[2].copy_(out["params"], non_blocking=True)
        stream.synchronize()
        e_conv += int((h_out[0] == gm.ST_CONVERGED).sum().item())
    e_secs = reduce_max(time.perf_counter() - t0, world, dev)
    e_value = reduce_sum(e_conv, world, dev) / e_secs

    cpu = None
    match = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        threads = oracle.max_threads()
        keep = {}
        c, dt = oracle_sample_fit(b, np.arange(G), keep, max_iter=SMALL_MAX_ITER)
        cpu = {"value": c / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"the whole workload ({G} galaxies, seed {rank_seed(0)}), rendered and fitted by the FP64 "
                         f"oracle, default start, tol {TOL:g}, max_iter {SMALL_MAX_ITER}",
               "us_per_iteration": 1e6 * dt / max(int(keep["ref"]["iters"].max()), 1)}
        match = oracle_match(keep, dev, max_iter=SMALL_MAX_ITER)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"plain single-Sersic+sky fit, {G} x {b.H}x{b.W} float32 stamps, Gaussian PSF "
                                       f"FWHM 1.5 px on {b.K}x{b.K}, no mask, default-start LM to dchi2/chi2<{TOL:g}",
                           "galaxies": G, "stamp": [b.H, b.W], "psf": [b.K, b.K], "free_params": 8, "tol": TOL,
                           "max_iter": SMALL_MAX_ITER, "l2": "inputs 0.5 MB, resident in L2 (a latency-bound case)"},
                "us_per_iteration": 1e3 * ms_max / max(passes, 1),
                "us_per_iteration_kernels": {"k_planes": 1e3 * profile_ms / max(passes, 1),
                                             "k_fused": 1e3 * fused_ms / max(passes, 1),
                                             "k_lm_step": 1e3 * step_ms / max(passes, 1)},
                "passes_per_fit": passes / args.steps,
                "converged_frac": converged / (G * args.steps), "mean_iters": float(iters.mean()),
                "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                             "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None,
                             "kernel": fused_name(8, gm.gm_tune_last_shape()) + " (a few tiles per launch: latency)",
                             "peak_source": "derived: 148 SMs x 128 FP32 FMA/clk x 2 FLOP x 2032 MHz"},
                "cpu_baseline": cpu, "oracle_match": match,
                "e2e": {"value": e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "gpu_launches": sum(4 + 3 * st["passes"] for st in stats), "clocks": clocks}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# learned-initialiser workload
# ---------------------------------------------------------------------------

def run_learned(args, world, rank, local):
    """Learned initialiser: train the CNN on the GPU on `--train-samples` stamps rendered by
    gm_model, then time the learned pipeline (network input preparation, inference, LM fit from
    the predicted start, default-start refits of the galaxies that do not converge) on 65,536
    bulge+disk galaxies of 128x128 with per-galaxy Moffat PSFs of side 25-51.  The default-start
    fit of the same batch is timed beside it."""
    import torch
    from paper_2404_07780_b300 import cnn, gm, workloads
    from paper_2404_07780_b300.build import build_lib

    build_lib()
    gm.load()
    cnn.lib()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = dist_init(world, "nccl")
    G = args.galaxies
    side = 128

    # training (a one-off cost, timed on its own)
    t0 = time.perf_counter()
    X, T, codec = cnn.make_training_set(args.train_samples, seed=4000 + rank, side=side, device=dev)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    net = cnn.Net(seed=rank, device=dev)
    t0 = time.perf_counter()
    losses = cnn.train(net, X, T, codec.dv, epochs=args.epochs, batch=512, lr=2e-3,
                       log=lambda m: print(m, file=sys.stderr))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del X, T

    rb = synth.draw_uneven_bulge_disk(seed=4100 + rank, G=G, sides=(side,), ks=UNEVEN_KS)
    image, sigma, psf = workloads.render_uneven(rb, dev)
    p_def = torch.from_numpy(rb.init).to(dev)
    fitter = gm.Fitter(rb.spec, G, device=dev, geom=rb.geom)
    opts = gm.FitOptions(tol=TOL, max_iter=MAX_ITER)
    stream = torch.cuda.current_stream()
    img3 = image.view(G, side, side)

    def learned_step():
        p0 = cnn.learned_start(net, img3, codec, rb.spec)
        return cnn.fit_with_fallback(fitter, rb.spec, p0, p_def, image, sigma, None, psf, opts, geom=rb.geom)

    # the default-start fit of the same batch (one warm-up, one timed)
    params = torch.empty_like(p_def)
    params.copy_(p_def)
    fitter.fit(params, image, sigma, None, psf, opts)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    params.copy_(p_def)
    torch.cuda.synchronize()
    e0.record(stream)
    d = {k: v.clone() for k, v in fitter.fit(params, image, sigma, None, psf, opts).items()}
    e1.record(stream)
    torch.cuda.synchronize()
    ms_default = e0.elapsed_time(e1)

    for _ in range(args.warmup):
        learned_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    torch.cuda.synchronize()
    e0.record(stream)
    conv = 0
    evals = 0
    refits = 0
    fused_ms = 0.0
    for _ in range(args.steps):
        r, info = learned_step()
        conv += int((r["status"] == gm.ST_CONVERGED).sum().item())
        evals += info["evals"]
        refits += info["refits"]
        fused_ms += info["fused_ms"]
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms_max = reduce_max(ms, world, dev)
    value = reduce_sum(conv, world, dev) / (ms_max / 1e3)

    # inference alone (network input preparation + forward), for the tensor-core roofline
    inf_ms = []
    for _ in range(3):
        torch.cuda.synchronize()
        e0.record(stream)
        net.predict(cnn.prep(img3, 1.0 / cnn.SKY_SIGMA))
        e1.record(stream)
        torch.cuda.synchronize()
        inf_ms.append(e0.elapsed_time(e1))
    macs = 0
    hw = 64
    for kind, i, o in cnn.LAYERS:
        if kind == "conv":
            hw //= 2
            macs += hw * hw * o * 9 * i
        else:
            macs += i * o
    inf_tflops = 2.0 * macs * G / (min(inf_ms) / 1e3) / 1e12
    peak_bf16 = None
    try:
        with open(PEAKS_PATH) as f:
            peak_bf16 = json.load(f).get("bf16_tflops")
    except (OSError, ValueError):
        pass

    # roofline of the dominant kernel (the fused pass): algorithmic FLOPs of the evaluations
    # spent, at the mean in-bounds taps of the batch's PSF sides
    taps = np.array([inbounds_taps(side, side, int(k)) for k in rb.geom[:, 2]], np.float64)
    flops = 2.0 * (1 + 11) * taps.mean() * evals
    achieved = flops / (fused_ms / 1e3) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None,
            "kernel": fused_name(12, gm.gm_tune_last_shape()) + ", evaluations x mean taps of the batch",
            "peak_source": "derived: 148 SMs x 128 FP32 FMA/clk x 2 FLOP x 2032 MHz (no FP32 figure is measured)"}
    c2_d, c2_l = d["chi2"].cpu().numpy(), r["chi2"].cpu().numpy()
    dof = d["dof"].cpu().numpy().astype(np.float64)
    dchi = (c2_l - c2_d) / np.sqrt(2 * dof)
    it_d = float(d["iters"].float().mean().item())
    it_l = evals / (G * args.steps)
    conv_d = int((d["status"] == gm.ST_CONVERGED).sum().item())

    # end to end through the public API from pinned host buffers
    h_img, h_sig, h_psf = image.cpu().pin_memory(), sigma.cpu().pin_memory(), psf.cpu().pin_memory()
    h_out = torch.empty((G, rb.spec.n_slots), dtype=torch.float64).pin_memory()
    h_st = torch.empty(G, dtype=torch.int32).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in (h_img, h_sig, h_psf))
    d2h = h_out.numel() * 8 + h_st.numel() * 4
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e_conv = 0
    for _ in range(max(1, min(args.steps, 2))):
        di, ds, dp = h_img.to(dev, non_blocking=True), h_sig.to(dev, non_blocking=True), h_psf.to(dev, non_blocking=True)
        p0 = cnn.learned_start(net, di.view(G, side, side), codec, rb.spec)
        out, _ = cnn.fit_with_fallback(fitter, rb.spec, p0, p_def, di, ds, None, dp, opts, geom=rb.geom)
        h_out.copy_(out["params"], non_blocking=True)
        h_st.copy_(out["status"], non_blocking=True)
        torch.cuda.synchronize()
        e_conv += int((h_st == gm.ST_CONVERGED).sum().item())
    e_secs = reduce_max(time.perf_counter() - t0, world, dev)
    e_value = reduce_sum(e_conv, world, dev) / e_secs

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32 fit, bf16 network", "data": "synthetic",
                "config": {"workload": f"learned initialiser + LM refinement, {G} bulge+disk+sky galaxies, "
                                       f"{side}x{side} float32 stamps, per-galaxy Moffat PSF of odd side 25-51, "
                                       f"12 free parameters, tol {TOL:g}; network trained on "
                                       f"{args.train_samples} rendered stamps, {args.epochs} epoch(s)",
                           "galaxies": G, "train_samples": args.train_samples, "epochs": args.epochs,
                           "l2": "inputs ~1.1 GB per batch > 126 MB L2 (no flush)"},
                "default_start": {"fits_per_s": conv_d / (ms_default / 1e3), "ms": ms_default,
                                  "converged_frac": conv_d / G, "mean_iters": it_d},
                "learned_start": {"converged_frac": conv / (G * args.steps), "mean_iters": it_l,
                                  "fallback_refits_per_step": refits / args.steps,
                                  "chi2_better_by_1sigma_frac": float(np.mean(dchi < -1)),
                                  "chi2_worse_by_1sigma_frac": float(np.mean(dchi > 1))},
                "speedup_vs_default_start": value / (conv_d / (ms_default / 1e3)),
                "training": {"samples": args.train_samples, "epochs": args.epochs, "data_s": t_data,
                             "train_s": t_train, "samples_per_s": args.train_samples * args.epochs / t_train,
                             "loss_per_epoch": losses},
                "inference": {"ms": min(inf_ms), "stamps_per_s": G / (min(inf_ms) / 1e3),
                              "tflops": inf_tflops, "bf16_peak_tflops": peak_bf16,
                              "frac": (inf_tflops / peak_bf16) if peak_bf16 else None},
                "roofline": roof,
                "cpu_baseline": None,
                "e2e": {"value": e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "clocks": clocks}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


# algorithmic DRAM bytes of one stamp through the network input preparation and the forward
# layers: each layer reads its input activation and writes its output once (BF16 NHWC; weights
# are shared by the batch and negligible per stamp)
def inference_bytes_per_stamp() -> dict:
    """Per kernel of Net.predict: the input preparation, the fused first two convolutions (the
    input read, the second layer's output written), then one kernel per layer."""
    from paper_2404_07780_b300 import cnn
    side = 2 * cnn.INPUT_SIDE
    b = {"prep": side * side * 4 + cnn.INPUT_SIDE * cnn.INPUT_SIDE * 2}
    hw, feats = cnn.INPUT_SIDE, cnn.INPUT_SIDE * cnn.INPUT_SIDE
    for li, (kind, i, o) in enumerate(cnn.LAYERS):
        last = li == len(cnn.LAYERS) - 1
        if kind == "conv":
            hw //= 2
            out = hw * hw * o
        else:
            out = o
        if li == 0:
            first = feats * 2
        elif li == 1:
            b["conv12"] = first + out * 2
        else:
            b[f"{kind}{li + 1}"] = feats * 2 + out * (4 if last else 2)
        feats = out
    return b


def inference_flops_per_stamp() -> float:
    from paper_2404_07780_b300 import cnn
    macs, hw = 0, cnn.INPUT_SIDE
    for kind, i, o in cnn.LAYERS:
        if kind == "conv":
            hw //= 2
            macs += hw * hw * o * 9 * i
        else:
            macs += i * o
    return 2.0 * macs


def run_inference(args, world, rank, local):
    """The learned initialiser's inference alone: network input preparation (2x2 block mean,
    asinh) of G float32 128x128 stamps and the forward pass in batches, with the network's seeded
    initial weights (the timing does not depend on the weights' values).  One step = one predict()
    of the whole set; each layer is also timed on its own in one extra pass."""
    import torch
    from paper_2404_07780_b300 import cnn, gm
    from paper_2404_07780_b300.build import build_lib

    build_lib()
    gm.load()
    cnn.lib()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    G = args.galaxies
    side = 2 * cnn.INPUT_SIDE
    gen = torch.Generator(device=dev)
    gen.manual_seed(5000 + rank)
    image = 2.0 * torch.randn((G, side, side), generator=gen, device=dev)  # sky noise, sigma 2
    net = cnn.Net(seed=rank, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        return net.predict(cnn.prep(image, 1.0 / cnn.SKY_SIGMA), batch=args.infer_batch)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps

    # each kernel on its own (events between the calls, one pass over the whole set)
    names = ["prep", "conv12"] + [f"{k}{li + 1}" for li, (k, _, _) in enumerate(cnn.LAYERS) if li >= 2]
    layer_ms = dict.fromkeys(names, 0.0)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)]
    x = cnn.prep(image, 1.0 / cnn.SKY_SIGMA)
    torch.cuda.synchronize()
    ev[0].record(stream)
    x = cnn.prep(image, 1.0 / cnn.SKY_SIGMA)
    ev[1].record(stream)
    torch.cuda.synchronize()
    layer_ms["prep"] = ev[0].elapsed_time(ev[1])
    for s0 in range(0, G, args.infer_batch):
        a = x[s0:s0 + args.infer_batch].contiguous()
        ev[1].record(stream)
        a = cnn.conv12_fwd(a, net.w(0), net.b(0), net.w(1), net.b(1))
        ev[2].record(stream)
        for li in range(2, len(cnn.LAYERS)):
            kind, i, o = cnn.LAYERS[li]
            last = li == len(cnn.LAYERS) - 1
            if kind == "conv":
                a = cnn.conv_fwd(a, net.w(li), net.b(li), relu=True)
            else:
                a = cnn.dense_fwd(a.reshape(a.shape[0], -1), net.w(li), net.b(li), relu=not last, fp32_out=last)
            ev[li + 1].record(stream)
        torch.cuda.synchronize()
        for k in range(1, len(names)):
            layer_ms[names[k]] += ev[k].elapsed_time(ev[k + 1])
    bpp = inference_bytes_per_stamp()
    peaks = {}
    try:
        with open(PEAKS_PATH) as f:
            peaks = json.load(f)
    except (OSError, ValueError):
        pass
    hbm, bf16 = peaks.get("hbm_gbs"), peaks.get("bf16_tflops")
    flops = inference_flops_per_stamp() * G
    tflops = flops / (ms / 1e3) / 1e12
    gbs = sum(bpp.values()) * G / (ms / 1e3) / 1e9
    layers = {}
    hw = cnn.INPUT_SIDE // 4
    for k, name in enumerate(names):
        t = layer_ms[name]
        d = {"ms": t, "gbs": bpp[name] * G / (t / 1e3) / 1e9}
        if k == 1:
            d["path"] = "fused conv1 + conv2 (tensor cores, conv1 kept in shared memory)"
        elif k > 1:
            kind, i, o = cnn.LAYERS[k]
            last = k == len(cnn.LAYERS) - 1
            if kind == "conv":
                d["path"] = ["gather", "tma"][cnn.fwd_path("conv", args.infer_batch, hw, hw, i, o)]
                hw //= 2
            else:
                d["path"] = ["gather", "tma"][cnn.fwd_path("dense", args.infer_batch, 0, 0, i, o, fp32_out=last)]
        if hbm:
            d["hbm_frac"] = d["gbs"] / hbm
        layers[name] = d
    line = {"metric": "CNN initialiser inference (input preparation + forward)", "value": G / (ms / 1e3),
            "unit": "stamps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16 (FP32 accumulate)",
            "data": "synthetic",
            "config": {"workload": f"{G} float32 128x128 stamps (sky noise) -> 64x64 BF16 input -> 4 conv + 2 dense "
                                   f"layers (the first two fused), batches of {args.infer_batch}", "stamps": G, "batch": args.infer_batch,
                       "l2": f"inputs {G * side * side * 4 / 1e9:.1f} GB > 126 MB L2 (no flush)"},
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                         "frac": gbs / hbm if hbm else None, "traffic": None,
                         "algorithmic_bytes_per_stamp": sum(bpp.values()),
                         "kernel": "whole inference (prep, fused conv1+conv2, 4 more layers): each kernel's input read once, "
                                   "output written once",
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs"},
            "tensor": {"tflops": tflops, "bf16_peak_tflops": bf16, "frac": tflops / bf16 if bf16 else None,
                       "flops_per_stamp": inference_flops_per_stamp()},
            "layers": layers, "gpu_launches": None, "clocks": clocks}
    print(json.dumps(line))
    return 0


def run_gradient(args, world, rank, local):
    """Gradient workload: d chi^2/dp of the bulge + bar + nucleus + sky model (15 free
    parameters) for 4,096 galaxies of 96x96 with a 41x41 Moffat PSF, by the adjoint
    correlation (gm_grad_adjoint); the 1+P-channel normal-equation pass (gm_chi2_grad) is
    timed beside it.  One step = one gradient of the whole batch."""
    import torch
    from paper_2404_07780_b300 import gm
    from paper_2404_07780_b300.build import build_lib

    build_lib()
    gm.load()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    G, H, K = 4096, 96, 41
    b = synth.draw_bulge_bar_nucleus(seed=3000 + rank, G=G, H=H, W=H, K=K)
    image, sigma, mask, psf = render_workload(b, dev)
    p0 = torch.from_numpy(b.init).to(dev)
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    kstats = []

    def adjoint_call():
        gm.gm_grad_adjoint(b.spec, p0, image, sigma, mask, psf)
        kstats.append(gm.gm_grad_adjoint_last_stats())  # the library's CUDA events around its kernels

    sampler = ClockSampler(local)
    sampler.start()
    ms_adj = timed(adjoint_call)
    clocks = sampler.stop()
    kst = {k: float(np.mean([s[k] for s in kstats[-args.steps:]])) for k in kstats[-1]}
    ms_ne = timed(lambda: gm.gm_chi2_grad(b.spec, p0, image, sigma, mask, psf, want_grad=True, want_jtj=False))
    taps = inbounds_taps(H, H, K)
    flops_corr = 2.0 * taps * G  # one single-channel correlation of every galaxy
    achieved = 2 * flops_corr / ((kst["resid_ms"] + kst["grad_ms"]) / 1e3) / 1e12
    pass_tflops = 2 * flops_corr / (ms_adj / 1e3) / 1e12
    gpix = G * H * H / (ms_adj / 1e3) / 1e9

    # the paper's optimiser (Adam, 1,000 steps, as its examples) against LM on the same batch
    adam_iters = args.adam_iters
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    ad = gm.gm_fit_adam(b.spec, p0, image, sigma, mask, psf, n_iter=adam_iters, lr=0.01)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_adam = e0.elapsed_time(e1)
    lm = gm.gm_fit_batch(b.spec, p0, image, sigma, mask, psf, gm.FitOptions(tol=TOL, max_iter=MAX_ITER))
    torch.cuda.synchronize()
    e0.record(stream)
    lm = gm.gm_fit_batch(b.spec, p0, image, sigma, mask, psf, gm.FitOptions(tol=TOL, max_iter=MAX_ITER))
    e1.record(stream)
    torch.cuda.synchronize()
    ms_lm = e0.elapsed_time(e1)
    c2_ad, c2_lm = ad["chi2"].cpu().numpy(), lm["chi2"].cpu().numpy()
    dof = lm["dof"].cpu().numpy().astype(np.float64)
    dchi = (c2_ad - c2_lm) / np.sqrt(2 * dof)
    if rank == 0:
        print(json.dumps({
            "metric": "chi^2 gradient throughput (adjoint correlation)", "value": gpix, "unit": "Gpix/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_adj,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"bulge+bar+nucleus+sky gradient, {G} x {H}x{H}, Moffat PSF {K}x{K}, 15 free "
                                   "parameters, default start", "galaxies": G},
            "normal_equations_ms_per_step": ms_ne, "speedup_vs_normal_equations": ms_ne / ms_adj,
            "adam_vs_lm": {"adam_iters": adam_iters, "adam_lr": 0.01, "adam_ms": ms_adam, "lm_ms": ms_lm,
                           "lm_converged_frac": float((lm["status"] == gm.ST_CONVERGED).float().mean().item()),
                           "lm_mean_iters": float(lm["iters"].float().mean().item()),
                           "adam_chi2_above_lm_by_1sigma_frac": float(np.mean(dchi > 1)),
                           "adam_chi2_below_lm_by_1sigma_frac": float(np.mean(dchi < -1)),
                           "median_chi2_excess_sigma": float(np.median(dchi))},
            "kernel_ms_per_step": kst,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None,
                         "kernel": "k_adjoint<RESID> and k_adjoint<GRAD> (the two correlations, 2 x in-bounds taps "
                                   "x 2 FLOP per pixel; their own CUDA-event times)",
                         "pass_achieved": pass_tflops, "pass_frac": pass_tflops / FP32_PEAK_TFLOPS,
                         "peak_source": "derived: 148 SMs x 128 FP32 FMA/clk x 2 FLOP x 2032 MHz"},
            "clocks": clocks}))
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--galaxies", type=int, default=None,
                    help="batch size per GPU (default 8192 for fit, 32768 for uneven; profiling runs use less)")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing (profiling runs)")
    ap.add_argument("--no-extra", action="store_true",
                    help="fit workload: leave out the summaries of the other workloads (each run in a child process)")
    ap.add_argument("--train-samples", type=int, default=1 << 20, help="learned workload: training stamps")
    ap.add_argument("--adam-iters", type=int, default=1000, help="gradient workload: Adam steps (the paper's 1,000)")
    ap.add_argument("--epochs", type=int, default=1, help="learned workload: training epochs")
    ap.add_argument("--infer-batch", type=int, default=16384, help="inference workload: stamps per forward batch")
    ap.add_argument("--workload", default="fit",
                    choices=["fit", "uneven", "gradient", "learned", "small", "inference"],
                    help="fit: the LM fit of the SDSS-shaped batch (default); uneven: bulge+disk fits on stamps and "
                         "PSFs of mixed size; gradient: adjoint chi^2 gradient; learned: the CNN start; small: 16 "
                         "stamps of 64x64 (time per LM iteration); inference: the CNN initialiser's forward pass")
    args = ap.parse_args()
    if args.galaxies is None:
        args.galaxies = {"uneven": 32768, "learned": 65536, "small": 16, "inference": 65536}.get(args.workload, 8192)
    world, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.workload == "gradient":
        return run_gradient(args, world, rank, local)
    if args.workload == "uneven":
        return run_uneven(args, world, rank, local)
    if args.workload == "learned":
        return run_learned(args, world, rank, local)
    if args.workload == "small":
        return run_small(args, world, rank, local)
    if args.workload == "inference":
        return run_inference(args, world, rank, local)
    return run_gpu(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
