"""bench.py's one-line JSON contract: the reference arm (the CPU oracle) runs here; our arm runs
on a GPU at a tiny size.  Both lines must carry the keys the benchmark contract asks for."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BASE_KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
             "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"}


def _run(args, timeout):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                       capture_output=True, text=True, timeout=timeout)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.strip().splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def test_reference_arm_line():
    d = _run(["--impl", "reference", "--steps", "1", "--warmup", "1", "--cpu-seconds", "1"], 600)
    assert BASE_KEYS <= set(d)
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert cb["single_thread"]["cores"] == 1 and cb["single_thread"]["value"] > 0
    assert cb["cpu"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"]


@pytest.mark.gpu
def test_our_arm_line_small():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = _run(["--per-density", "4", "--sweeps", "20", "--steps", "2", "--warmup", "3",
              "--no-gap", "--no-ragged", "--cpu-seconds", "1", "--ksweep-sweeps", "4"], 900)
    assert BASE_KEYS <= set(d) and d["value"] > 0
    r = d["roofline"]
    assert {"bound", "achieved", "peak", "unit", "frac", "traffic"} <= set(r)
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-9
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] > 0
    assert d["cpu_baseline"]["single_thread"]["value"] > 0
    assert {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"} <= set(d["e2e"])
    assert d["gpu_launches"] > 0
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= set(d["clocks"])
    ks = d["blocked_k"]
    for k in ("16", "32", "64"):
        assert ks[k]["value"] > 0 and ks[k]["cycles_per_spin_step"] > 0 and ks[k]["kernel"]
    assert ks["plain"]["value"] > 0
    for case in ("n250_m5", "n500_m30"):
        assert d["plain_mkp"][case]["value"] > 0 and d["plain_mkp"][case]["kernel"] == "plain"
    lat = d["roofline"]["latency"]
    assert lat["cycles_per_spin_step"] > 0 and 0 < lat["smsp_issue_active"] <= 1


@pytest.mark.gpu
def test_our_arm_optional_sections_small():
    """The best-in-run / tightening section and the paper-scale section at tiny sizes: their
    keys and the accounting of samples (no quality claim at these sizes)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = _run(["--per-density", "2", "--sweeps", "20", "--steps", "1", "--warmup", "3",
              "--no-gap", "--no-ragged", "--no-e2e", "--no-plain", "--no-cpu", "--run-best",
              "--rb-instances", "2", "--rb-iters", "3", "--paper-scale", "--ps-per-class", "1",
              "--ps-iters", "256"], 900)
    rb = d["run_best_mkp"]
    for name in ("last_sample", "run_best", "run_best_tight_0.95", "run_best_tight_0.9"):
        assert {"within_1pct", "any_feasible", "median_gap", "feasible_sample_fraction",
                "device_ms"} <= set(rb[name])
        assert 0.0 <= rb[name]["feasible_sample_fraction"] <= 1.0
    ps = d["paper_scale_qkp"]
    assert ps["instances"] == 12
    assert ps["paper_single_chain"]["samples_per_instance"] == 256
    assert ps["batched_equal_samples"]["samples_per_instance"] == 256
    assert ps["batched_equal_iterations"]["samples_per_instance"] == 256 * 128
    for run in ("paper_single_chain", "batched_equal_samples", "batched_equal_iterations"):
        for n in ("100", "200", "300"):
            acc = ps[run]["accuracy_by_size"][n]
            assert 0.0 <= acc["min_accuracy_pct"] <= acc["median_accuracy_pct"] <= 100.0


@pytest.mark.gpu
def test_target_run_small(tmp_path):
    """The target section end to end at a tiny size: a best-known table written by
    --make-best-known (every state checked by the oracle), then the warm-started blocked,
    cold plain and cold blocked runs against it.  Cold plain and cold blocked draw identical
    samples, so they reach the gap at the same iterations."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    bk = str(tmp_path / "bk.json")
    common = ["--target-per-density", "1", "--target-iters", "3", "--sweeps", "30",
              "--best-known", bk]
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--make-best-known",
                        *common], cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    table = json.load(open(bk))
    assert len(table["instances"]) == 4
    assert all(row["cost"] is None or row["cost"] <= 0 for row in table["instances"])
    d = _run(["--per-density", "2", "--steps", "1", "--warmup", "3", "--no-ragged", "--no-e2e",
              "--no-plain", "--no-cpu", "--no-ksweep", "--target-train", "40", *common], 900)
    g = d["gap_1pct"]
    assert g["instances"] == 4
    known = 4 - g["instances_without_best_known"]
    for arm in ("warm_blocked", "cold_plain", "cold_blocked"):
        assert g[arm]["all"]["of"] == known and 0 <= g[arm]["all"]["reached"] <= known
        assert g[arm]["iterations_run"] <= 3
        assert g[arm]["better_than_best_known"] >= 0
    assert g["cold_plain"]["all"]["reached"] == g["cold_blocked"]["all"]["reached"]
    assert g["cold_plain"]["median_iterations_reached"] == \
        g["cold_blocked"]["median_iterations_reached"]
