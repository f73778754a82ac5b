"""Host logic of bench.py's default line, on CPU: the summaries of the other workloads it carries.

Every other workload runs in a child process of its own and its JSON line is cut down to the
figures the default line keeps; a child that fails or gives no line is recorded as an error and
never stops the fit's own line from printing."""
import bench


def _line(**extra):
    base = {"value": 10.0, "unit": "fits/s", "ms_per_step": 5.0, "steps": 1, "warmup": 1, "converged_frac": 1.0,
            "mean_iters": 12.0, "gpu_launches": 40, "config": {"workload": "w"},
            "roofline": {"bound": "alu", "achieved": 1.0, "peak": 2.0, "unit": "TFLOP/s", "frac": 0.5, "traffic": 3},
            "e2e": {"value": 9.0}, "clocks": {"sm_mhz": 1900.0, "sm_max_mhz": 2032.0, "reasons": []}}
    base.update(extra)
    return base


def test_summary_keeps_the_common_figures():
    s = bench.summarize_workload("uneven", _line())
    assert s["value"] == 10.0 and s["e2e"] == 9.0 and s["workload"] == "w"
    assert s["roofline"] == {"bound": "alu", "achieved": 1.0, "peak": 2.0, "unit": "TFLOP/s", "frac": 0.5}
    assert s["clocks"]["reasons"] == []


def test_summary_of_each_workload():
    small = bench.summarize_workload("small", _line(
        us_per_iteration=100.0, us_per_iteration_kernels={"k_fused": 50.0},
        cpu_baseline={"value": 40.0, "us_per_iteration": 9e4}, oracle_match={"oracle_match_frac": 1.0}))
    assert small["us_per_iteration"] == 100.0 and small["oracle_fits_per_s"] == 40.0
    assert small["oracle_match_frac"] == 1.0
    grad = bench.summarize_workload("gradient", _line(
        normal_equations_ms_per_step=30.0, speedup_vs_normal_equations=5.0, adam_vs_lm={"adam_ms": 7000.0}))
    assert grad["speedup_vs_normal_equations"] == 5.0 and grad["adam_vs_lm"]["adam_ms"] == 7000.0
    learned = bench.summarize_workload("learned", _line(
        speedup_vs_default_start=1.8, default_start={"fits_per_s": 3000.0}, learned_start={"mean_iters": 8.0},
        inference={"ms": 20.0, "tflops": 80.0, "frac": 0.05, "stamps_per_s": 3e6}, training={"train_s": 6.0}))
    assert learned["speedup_vs_default_start"] == 1.8
    assert learned["inference"] == {"ms": 20.0, "tflops": 80.0, "frac": 0.05}
    inf = bench.summarize_workload("inference", _line(
        tensor={"tflops": 360.0, "frac": 0.2}, layers={"prep": {"ms": 0.8, "gbs": 6000.0}}))
    assert inf["tensor"]["frac"] == 0.2 and inf["layers_ms"] == {"prep": 0.8}


def test_failing_child_is_recorded(monkeypatch):
    # on a host without a GPU the child exits non-zero: the error is recorded, nothing raises
    monkeypatch.setattr(bench, "OTHER_WORKLOADS", (("small", ("--galaxies", "2"), 120),))
    out = bench.run_other_workloads()
    assert set(out) == {"small"}
    assert out["small"]["error"].startswith("exit ")
    assert out["small"]["args"] == ["--galaxies", "2"]
