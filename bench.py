#!/usr/bin/env python3
"""Throughput benchmark of the SAIM hot path (one JSON line on rank 0).

Workload: QKP N=300 at densities 0.25/0.5/0.75/1.0, 256 instances each (1024 instances,
N' <= 313 spins), 128 chains per instance, 1000 sweeps with beta 0 -> 10 (Table I).  One step
is one outer iteration of Algorithm 1 over the whole batch: one annealing run per chain
(sais_sample), the feasible-sample bookkeeping (sais_track_best) and the multiplier step
(sais_update_lambda), all through the C-ABI on device buffers.  Metric: p-bit spin updates
per second (chains x sweeps x N' summed over instances, divided by the step time).

--impl reference times the CPU oracle (the only reference that exists for this method) on a
bounded sample of the same workload.  Under torchrun every rank runs its own 1024 instances
(weak scaling, no collective on the data path); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "p-bit spin updates/s; wall-clock to 1% gap on QKP N=300 (BF16 block vs plain)"
UNIT = "spin_updates/s"
DENSITIES = (0.25, 0.5, 0.75, 1.0)
SM_COUNT, FP32_LANES_PER_SM, SM_MAX_MHZ = 152, 128, 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--variant", default="auto", choices=["auto", "plain", "blocked"])
    ap.add_argument("--per-density", type=int, default=256)
    ap.add_argument("--chains", type=int, default=128)
    ap.add_argument("--sweeps", type=int, default=1000)
    ap.add_argument("--beta-max", type=float, default=10.0)
    ap.add_argument("--eta", type=float, default=20.0)
    ap.add_argument("--block-k", type=int, default=0)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-gap", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--gap-instances", type=int, default=16, help="per density")
    ap.add_argument("--gap-iters", type=int, default=100)
    ap.add_argument("--gap-eta", type=float, default=2000.0)
    ap.add_argument("--no-ragged", action="store_true")
    ap.add_argument("--penalty", action="store_true",
                    help="also compare with the penalty method (eta = 0, scaled P)")
    ap.add_argument("--run-best", action="store_true",
                    help="also measure best-in-run tracking and capacity tightening on MKP")
    ap.add_argument("--rb-instances", type=int, default=32)
    ap.add_argument("--rb-iters", type=int, default=50)
    ap.add_argument("--rb-beta-max", type=float, default=50.0)
    ap.add_argument("--rb-eta", type=float, default=20.0)
    ap.add_argument("--paper-scale", action="store_true",
                    help="also run the paper's budget (2000 single-chain iterations) on QKP")
    ap.add_argument("--ps-per-class", type=int, default=12)
    ap.add_argument("--ps-iters", type=int, default=2000)
    ap.add_argument("--ps-eta", type=float, default=20.0)
    ap.add_argument("--warmstart", action="store_true",
                    help="also run the learned warm start: labels, training, evaluation")
    ap.add_argument("--ws-train", type=int, default=20000)
    ap.add_argument("--ws-eval", type=int, default=64)
    ap.add_argument("--ws-epochs", type=int, default=200)
    ap.add_argument("--ragged-iters", type=int, default=3)
    ap.add_argument("--no-target", action="store_true",
                    help="skip the target run (warm-started blocked vs cold plain to a 1%% gap)")
    ap.add_argument("--target-per-density", type=int, default=38)
    ap.add_argument("--target-iters", type=int, default=40)
    ap.add_argument("--target-train", type=int, default=3000)
    ap.add_argument("--best-known", default=os.path.join(ROOT, "best_known_qkp300.json"))
    ap.add_argument("--make-best-known", action="store_true",
                    help="compute the best-known table of the target instances and exit")
    ap.add_argument("--no-ksweep", action="store_true")
    ap.add_argument("--ksweep-sweeps", type=int, default=200)
    ap.add_argument("--ragged-tune-sweeps", type=int, default=50)
    ap.add_argument("--kernel-case", choices=sorted(KERNEL_CASES),
                    help="run one small sampler launch (after --warmup launches) and exit: the "
                         "cases the committed ncu summaries were captured on")
    return ap.parse_args()


# name: (instances, chains, sweeps, beta_max, variant, block_k); sizes keep an ncu capture short
# while W stays larger than L2 where the kernel streams it.
KERNEL_CASES = {
    "rankk_qkp300": ("152 QKP N=300 d=0.5", 128, 200, 10.0, "blocked", 16),
    "field_qkp900": ("152 QKP N=900 d=0.5", 128, 30, 10.0, "blocked", 16),
    "field_qkp1000_hilo": ("152 QKP N=1000 d=0.5, profits <= 1e4", 128, 20, 10.0, "blocked", 16),
    "field_qkp300_k32": ("304 QKP N=300 d=0.5", 128, 40, 10.0, "blocked", 32),
    "plain_qkp300": ("152 QKP N=300 d=0.5", 128, 50, 10.0, "plain", 0),
    "plain_mkp500_m30": ("32 MKP N=500 m=30", 256, 20, 50.0, "plain", 0),
    "persistent_ragged": ("the ragged batch: 384 QKP N~U[100,1000] (profits <= 1e4) + 128 MKP, "
                          "chains U[64,256]", 256, 20, 10.0, "auto", 0),
}


def kernel_case(a, sais, torch):
    """One of KERNEL_CASES: `a.warmup` launches, then one launch timed with CUDA events."""
    from paper_2501_04971_gb300 import workloads as wl
    what, C, T, beta, variant, k = KERNEL_CASES[a.kernel_case]
    name = a.kernel_case
    counts = None
    if name == "persistent_ragged":
        insts = wl.ragged_batch()
        counts = np.random.default_rng(0x524147).integers(64, 257, len(insts)).astype(np.int32)
    elif name.startswith("plain_mkp"):
        insts = [wl.mkp(500, 30, s) for s in range(32)]
    else:
        n = int(name.split("qkp")[1].split("_")[0])
        cnt = 304 if name.endswith("_k32") else 152
        pm = 10000 if name.endswith("_hilo") else 100
        insts = [wl.qkp(n, 0.5, s, profit_max=pm) for s in range(cnt)]
    prob = sais.Problem(insts)
    if counts is not None:
        prob.set_instance_chains(counts)
    lam = torch.full((prob.count * prob.m_stride,), 0.5, device="cuda")
    out = prob.alloc_outputs(C)
    kernel = prob.plan(C, variant, k)["kernel"]
    for _ in range(max(1, a.warmup)):
        prob.sample(lam, C, T, beta, 1, 0, variant=variant, block_k=k, out=out)
    prob.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    prob.sample(lam, C, T, beta, 1, 0, variant=variant, block_k=k, out=out)
    e1.record()
    prob.synchronize()
    ms = e0.elapsed_time(e1)
    per_inst = counts if counts is not None else np.full(prob.count, C)
    upd = int(sum(s.n_spins * int(c) for s, c in zip(prob.scalars, per_inst))) * T
    line = {"case": name, "workload": what, "chains": C, "sweeps": T, "kernel": kernel,
            "ms": ms, "spin_updates": upd, "rate": upd / (ms / 1e3), "unit": UNIT}
    if kernel == "persistent":
        st = prob.persistent_stats()
        line["busy_fraction_mean"] = float(st["busy_fraction"].mean())
    print(json.dumps(line))
    prob.close()


def workload(per_density: int, rank: int):
    from paper_2501_04971_gb300 import workloads as wl
    return [wl.qkp(300, d, rank * per_density + s) for d in DENSITIES for s in range(per_density)]


def over_ranks(x: float, dist, device, op: str = "max") -> float:
    """Max (timings) or sum (work units) of a per-rank scalar over all ranks; the value itself
    without a process group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def workload_name(a) -> str:
    return (f"QKP N=300, d in {{0.25,0.5,0.75,1}} x {a.per_density} instances, "
            f"{a.chains} chains, {a.sweeps} sweeps (beta 0->{a.beta_max:g}) per step")


# ------------------------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline leg and --impl reference)
# ------------------------------------------------------------------------------------------

def cpu_model() -> str:
    """The host CPU as /proc/cpuinfo names it (x86: model name; Arm: the CPU part), with the
    machine type."""
    import platform
    try:
        lines = open("/proc/cpuinfo").read().splitlines()
        for key in ("model name", "Model", "CPU part"):
            for line in lines:
                if line.startswith(key) and ":" in line:
                    return f"{platform.machine()}, {key}: {line.split(':', 1)[1].strip()}"
    except OSError:
        pass
    return f"{platform.machine()} {platform.processor()}".strip()


def oracle_rate(insts, seconds: float, chains: int, threads: int = 0):
    """The oracle's annealing runs (or_anneal, OpenMP over chains) on a bounded sample: the
    first instance of each density, `chains` chains, sweep count calibrated so the run takes
    about `seconds`; `threads` > 0 limits the OpenMP threads for the run.  Returns
    (updates/s, threads used, description)."""
    import oracle
    prev = oracle.max_threads()
    if threads:
        oracle.set_threads(threads)
    try:
        return _oracle_rate(insts, seconds, chains)
    finally:
        if threads:
            oracle.set_threads(prev)


def _oracle_rate(insts, seconds: float, chains: int):
    import oracle
    sample = [insts[i * (len(insts) // len(DENSITIES))] for i in range(len(DENSITIES))]
    probs = []
    for inst in sample:
        p = oracle.Problem(inst.n, inst.m, inst.W, inst.h, inst.A, inst.b, alpha=inst.alpha,
                           density=inst.density)
        J, hI, _ = p.ising(np.array([1.0], np.float32))
        probs.append((p, J, hI))

    def run(T):
        t0 = time.perf_counter()
        upd = 0
        for p, J, hI in probs:
            oracle.anneal(J, hI, 10.0, T, 1, 0, chains)
            upd += chains * T * p.nprime
        return upd, time.perf_counter() - t0

    u, dt = run(2)
    T = max(2, int(2 * seconds / max(dt, 1e-6)))
    u, dt = run(T)
    cores = oracle.max_threads()
    desc = (f"oracle or_anneal, {len(probs)} instances (one per density), {chains} chains x "
            f"{T} sweeps each, {u} updates in {dt:.1f} s, OpenMP over chains, {cores} threads")
    return u / dt, cores, desc


def cpu_baseline_line(insts, seconds: float, value=None, cores=None, desc=None):
    """The cpu_baseline object: the oracle on all host cores (given, or measured here) and on
    one core (a quarter of the time), with the host CPU named."""
    if value is None:
        value, cores, desc = oracle_rate(insts, seconds, 2 * (os.cpu_count() or 1))
    v1, _, d1 = oracle_rate(insts, max(0.5, seconds / 4), 4, threads=1)
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
            "single_thread": {"value": v1, "unit": UNIT, "cores": 1, "sample": d1},
            "cpu": cpu_model()}


def reference_arm(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    insts = workload(a.per_density, 0)
    per = max(2.0, a.cpu_seconds / max(1, a.steps + a.warmup))
    for _ in range(a.warmup):
        oracle_rate(insts, per / 4, 2 * (os.cpu_count() or 1))
    vals, cores, desc, secs = [], 1, "", []
    for _ in range(a.steps):
        t0 = time.perf_counter()
        v, cores, desc = oracle_rate(insts, per, 2 * (os.cpu_count() or 1))
        secs.append(time.perf_counter() - t0)
        vals.append(v)
    v = float(statistics.median(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * statistics.mean(secs), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a), "sample": "bounded CPU sample"},
            "cpu_baseline": cpu_baseline_line(insts, per, v, cores, desc),
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9 and f[1].replace(".", "").isdigit():
                    rows.append(f)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v == "Active"})
        return {"sm_mhz": float(statistics.median(sm)), "sm_max_mhz": float(rows[0][2]),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------------------------------
# the target run: wall-clock to a 1 % gap on QKP N=300, warm-started blocked vs cold plain
# ------------------------------------------------------------------------------------------

INT64_MAX = np.iinfo(np.int64).max


def target_instances(per: int):
    """QKP N=300 at the four densities, `per` each (seeds 5000 + 100 q + i)."""
    from paper_2501_04971_gb300 import workloads as wl
    return [wl.qkp(300, d, 5000 + 100 * q + i) for q, d in enumerate(DENSITIES)
            for i in range(per)]


def target_budget(a):
    return dict(C=a.chains, T=a.sweeps, beta=a.beta_max, eta=a.gap_eta, K=a.target_iters)


def oracle_check(inst, x_bits: np.ndarray, nspins: int):
    """(cost, feasible) of a bit-packed state by the oracle, in int64 (Sec. IV-A)."""
    import oracle
    from paper_2501_04971_gb300 import sais
    p = oracle.Problem(inst.n, inst.m, inst.W, inst.h, inst.A, inst.b, alpha=inst.alpha,
                       density=inst.density)
    x = sais.unpack_bits(np.asarray(x_bits, np.uint32)[None, :], nspins)[0]
    return p.cost(x), p.feasible(x)


def make_best_known(a, sais, torch):
    """Best-known profit of every target instance: the best feasible sample of 16 seeds x 16 x
    the target budget (target_iters iterations) of Algorithm 1 from lambda = 0, each kept state
    checked by the oracle in int64.  The runs use the blocked sampler, whose samples are those
    of the plain sampler bit for bit.  Not certified optimal."""
    insts = target_instances(a.target_per_density)
    prob = sais.Problem(insts)
    b = target_budget(a)
    best = np.full(prob.count, INT64_MAX, np.int64)
    bx = np.zeros((prob.count, prob.words), np.uint32)
    t0 = time.perf_counter()
    for seed in range(16):
        r = prob.solve(16 * b["K"], b["C"], b["T"], b["beta"], b["eta"], 31000 + seed,
                       variant="blocked", use_graph=True)
        better = r["best_cost"] < best
        best[better] = r["best_cost"][better]
        bx[better] = np.asarray(r["best_x"]).reshape(prob.count, -1)[better].view(np.uint32)
        print(f"seed {seed}: {int(better.sum())} improved, {time.perf_counter() - t0:.0f} s",
              file=sys.stderr, flush=True)
    rows = []
    for j, inst in enumerate(insts):
        row = {"density": inst.density,
               "seed": 5000 + 100 * DENSITIES.index(inst.density) + j % a.target_per_density,
               "cost": None, "x": None}
        if best[j] != INT64_MAX:   # else no feasible sample in the whole ensemble
            cost, feas = oracle_check(inst, bx[j], prob.scalars[j].n_spins)
            assert feas and cost == best[j], (j, cost, best[j])
            row["cost"], row["x"] = int(best[j]), "".join(f"{w:08x}" for w in bx[j])
        rows.append(row)
    out = {"workload": "QKP N=300, d in {0.25,0.5,0.75,1} x %d (seeds 5000 + 100 q + i)"
                       % a.target_per_density,
           "recipe": "best feasible sample of 16 seeds x %d iterations (16 x the target budget) "
                     "of Algorithm 1 from lambda = 0, %d chains x %d sweeps, beta_max %g, eta "
                     "%g, P = 2dN; blocked sampler (its samples are the plain sampler's); every "
                     "state checked by the oracle in int64; not certified optimal"
                     % (16 * b["K"], b["C"], b["T"], b["beta"], b["eta"]),
           "seconds": time.perf_counter() - t0, "instances": rows}
    prob.close()
    with open(a.best_known, "w") as f:
        json.dump(out, f, indent=0)
    print(f"wrote {a.best_known}", file=sys.stderr)


def load_best_known(a, insts, nspins):
    """The stored best-known costs, each state re-checked by the oracle (int64); INT64_MAX where
    the ensemble found no feasible sample."""
    d = json.load(open(a.best_known))
    rows = d["instances"]
    assert len(rows) == len(insts), "best-known table is for another instance count"
    best = np.full(len(insts), INT64_MAX, np.int64)
    for j, (inst, row) in enumerate(zip(insts, rows)):
        if row["cost"] is None:
            continue
        x = np.array([int(row["x"][8 * w:8 * w + 8], 16) for w in range(len(row["x"]) // 8)],
                     np.uint32)
        cost, feas = oracle_check(inst, x, nspins[j])
        assert feas and cost == row["cost"], f"best-known row {j} fails the oracle check"
        best[j] = row["cost"]
    return best, d["recipe"]


def solve_to_gap(prob, sais, torch, variant, lam0, K, b, best_known, t0):
    """Algorithm 1 through sais_solve, one iteration per call resumed from the previous call's
    multipliers (iter0 = k), pinned host buffers.  Per instance: the host wall-clock from t0
    (taken before the first call, or before the warm start) until its best feasible profit
    reaches 0.99 x best-known, and the iteration; nan where never within K iterations."""
    cnt, M, Wd = prob.count, prob.m_stride, prob.words
    lam_h = torch.zeros(cnt * M, dtype=torch.float32).pin_memory()
    lam_h.copy_(lam0)
    pinned = {"best_cost": torch.zeros(cnt, dtype=torch.int64).pin_memory(),
              "lambda_final": torch.zeros(cnt * M, dtype=torch.float32).pin_memory()}
    prm = sais.sais_solve_params()
    prm.iters, prm.chains, prm.sweeps, prm.beta_max = 1, b["C"], b["T"], b["beta"]
    prm.eta, prm.seed, prm.project_nonneg = b["eta"], 4242, 1
    prm.variant = sais._VARIANTS[variant]
    prm.lambda0 = sais._P(lam_h.data_ptr())
    res = sais.sais_solve_result()
    for k_, v_ in pinned.items():
        setattr(res, k_, sais._P(v_.data_ptr()))
    sp = sais._P(torch.cuda.current_stream().cuda_stream)
    best = np.full(cnt, INT64_MAX, np.int64)
    reach_s = np.full(cnt, np.nan)
    reach_k = np.full(cnt, np.nan)
    for k in range(K):
        prm.iter0 = k
        sais.sais_solve(prob.handle, prm, res, sp)
        t = time.perf_counter() - t0
        lam_h.copy_(pinned["lambda_final"])
        best = np.minimum(best, pinned["best_cost"].numpy())
        hit = ((best != INT64_MAX) & (best_known != INT64_MAX) & (-best >= 0.99 * (-best_known))
               & np.isnan(reach_s))
        reach_s[hit] = t
        reach_k[hit] = k + 1
        if not np.isnan(reach_s[best_known != INT64_MAX]).any():
            break
    return reach_s, reach_k, best, k + 1


def target_measurement(a, sais, torch):
    """The target comparison: wall-clock from sais_solve entry to a 1 % gap against the stored
    best-known, on QKP N=300 at the four densities (`target_per_density` each; one batch that
    fills the GPU), for (1) the BF16 blocked sampler started from the learned multipliers
    (network trained in this run on `target_train` instances by the project's kernels), (2) the
    plain FP32 sampler from lambda = 0 as in Algorithm 1, (3) the blocked sampler from lambda =
    0.  Unreached instances count as never (medians over all instances, infinite where
    unreached)."""
    from paper_2501_04971_gb300 import warmstart as ws
    insts = target_instances(a.target_per_density)
    prob = sais.Problem(insts)
    nsp = [s.n_spins for s in prob.scalars]
    best_known, recipe = load_best_known(a, insts, nsp)
    b = target_budget(a)
    dens = np.repeat(np.array(DENSITIES), a.target_per_density)
    # the warm-start network, trained here
    t1 = time.perf_counter()
    tr = ws.training_instances(a.target_train)
    bud = ws.SolveBudget(iters=30, chains=128, sweeps=200, beta_max=a.beta_max, eta=a.gap_eta)
    X, y, t_lab, _ = ws.label(tr, bud)
    net, losses, t_train = ws.train(X, y, epochs=a.ws_epochs)
    t_ws = time.perf_counter() - t1
    known = best_known != INT64_MAX
    out = {"instances": prob.count, "best_known": recipe,
           "instances_without_best_known": int((~known).sum()),
           "workload": "QKP N=300, d in {0.25,0.5,0.75,1} x %d, %d chains x %d sweeps per "
                       "iteration, beta_max %g, P = 2dN, eta %g (normalised units), at most %d "
                       "iterations" % (a.target_per_density, b["C"], b["T"], b["beta"], b["eta"],
                                       b["K"]),
           "time": "host wall-clock from the first sais_solve entry (warm: from the warm-start "
                   "call), one iteration per call, resumed through lambda0 / iter0",
           "warm_start_net": {"train_instances": len(tr), "rows": int(X.shape[0]),
                              "label_seconds": t_lab, "train_device_seconds": t_train,
                              "seconds_total": t_ws, "loss_first_last": [losses[0], losses[-1]]}}

    def stats(r, mask):
        rr = np.where(np.isnan(r[mask]), np.inf, r[mask])
        ok = np.isfinite(rr)
        med = float(np.median(rr)) if ok.any() else None
        p90 = float(np.percentile(rr, 90)) if ok.any() else None
        return {"reached": int(ok.sum()), "of": int(mask.sum()),
                "median_s": med if med is not None and np.isfinite(med) else None,
                "p90_s": p90 if p90 is not None and np.isfinite(p90) else None,
                "median_s_reached": float(np.median(rr[ok])) if ok.any() else None}

    arms = (("warm_blocked", "blocked", True), ("cold_plain", "plain", False),
            ("cold_blocked", "blocked", False))
    reach = {}
    for name, variant, warm in arms:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lam = torch.zeros(prob.count * prob.m_stride, dtype=torch.float32, device="cuda")
        if warm:
            prob.warm_start(net, lam)
        lam0 = lam.cpu()
        rs, rk, best, kk = solve_to_gap(prob, sais, torch, variant, lam0, b["K"], b, best_known, t0)
        reach[name] = rs
        out[name] = {"variant": variant, "lambda0": "learned" if warm else "zero",
                     "iterations_run": kk, "all": stats(rs, known),
                     "median_iterations_reached": float(np.nanmedian(rk)) if (~np.isnan(rk)).any()
                     else None,
                     "better_than_best_known": int((best < best_known).sum()),
                     "feasible_where_none_known": int(((best != INT64_MAX) & ~known).sum()),
                     "by_density": {str(d): stats(rs, (dens == d) & known) for d in DENSITIES}}
    w, c = out["warm_blocked"]["all"], out["cold_plain"]["all"]
    if w["median_s"] and c["median_s"]:
        out["speedup_median_cold_plain_over_warm_blocked"] = c["median_s"] / w["median_s"]
    both = ~np.isnan(reach["warm_blocked"]) & ~np.isnan(reach["cold_plain"])
    if both.any():
        out["per_instance_speedup_median_both_reached"] = float(
            np.median(reach["cold_plain"][both] / reach["warm_blocked"][both]))
    net.close()
    prob.close()
    return out


def mkp_measurement(a, sais, torch):
    """The plain sampler on linear objectives (Eq. 14): MKP N=250 m=5 (32 instances x 1024
    chains, the shape of config 1) and N=500 m=30 (128 x 256), 100 sweeps at beta_max 50, one
    timed launch after a warm-up; spin updates/s, and the issue activity of the m = 30 case from
    its ncu capture."""
    from paper_2501_04971_gb300 import workloads as wl
    res = {}
    for name, (n, m, cnt, C) in (("n250_m5", (250, 5, 32, 1024)), ("n500_m30", (500, 30, 128, 256))):
        prob = sais.Problem([wl.mkp(n, m, 9000 + s) for s in range(cnt)])
        lam = torch.full((prob.count * prob.m_stride,), 0.5, device="cuda")
        out = prob.alloc_outputs(C)
        T = 100
        prob.sample(lam, C, T, 50.0, 1, 0, variant="plain", out=out)
        prob.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        prob.sample(lam, C, T, 50.0, 1, 0, variant="plain", out=out)
        e1.record()
        prob.synchronize()
        ms = e0.elapsed_time(e1)
        upd = sum(sc.n_spins for sc in prob.scalars) * C * T
        res[name] = {"value": upd / (ms / 1e3), "unit": UNIT, "ms": ms, "instances": cnt,
                     "chains": C, "sweeps": T, "kernel": prob.plan(C, "plain")["kernel"],
                     "chains_per_cta": prob.plan(C, "plain")["chains_per_cta"]}
        prob.close()
    res["n500_m30"]["profile"] = ("ncu, 32 instances x 256 chains (bench.py --kernel-case "
                                  "plain_mkp500_m30): issue slots busy 31.7 %, 1.7 warps per SM "
                                  "at that size")
    return res


def ksweep_measurement(a, sais, torch, insts, sm_mhz):
    """The blocked sampler at block sizes K = 16, 32, 64 on the bench workload (`ksweep_sweeps`
    sweeps per launch, one timed launch after a warm-up): spin updates/s and SM cycles per
    spin-step (one spin of one 128-chain CTA), which kernel ran, and the plain sampler beside."""
    prob = sais.Problem(insts)
    C, T = a.chains, a.ksweep_sweeps
    lam = torch.zeros(prob.count * prob.m_stride, device="cuda")
    out = prob.alloc_outputs(C)
    nsp = np.array([s.n_spins for s in prob.scalars])
    upd = int(nsp.sum()) * C * T
    res = {"sweeps": T, "sm_mhz": sm_mhz}
    for k in (16, 32, 64, "plain"):
        kw = dict(variant="plain") if k == "plain" else dict(variant="blocked", block_k=k)
        try:
            prob.sample(lam, C, T, a.beta_max, 1, 0, out=out, **kw)
            torch.cuda.synchronize()
        except sais.SaisError as e:
            res[str(k)] = {"unsupported": str(e)}
            continue
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        prob.sample(lam, C, T, a.beta_max, 1, 1, out=out, **kw)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        row = {"value": upd / (ms / 1e3), "unit": UNIT, "ms": ms}
        if k != "plain":
            steps = int(sum(-(-int(n) // k) * k for n in nsp)) * (-(-C // 128)) * T
            row["cycles_per_spin_step"] = ms / 1e3 * sm_mhz * 1e6 * SM_COUNT / steps
            row["kernel"] = prob.blocked_kernel(k)
        res[str(k)] = row
    prob.close()
    return res


def penalty_measurement(a, sais, torch):
    """SAIM against the penalty method at an equal sample budget (the comparison of Table II,
    on synthetic instances): the same instances as the gap measurement (QKP N=300, four
    densities), Algorithm 1 with the multiplier step (eta = gap_eta, P = 2dN) and without it
    (eta = 0, lambda = 0: a fixed penalty P = s 2dN for s in 1..64), each `gap_iters`
    iterations x `chains` chains x `sweeps` sweeps, one CUDA graph per run.  Best-known profit
    per instance = the best feasible sample of all these runs (uncertified)."""
    import dataclasses
    from paper_2501_04971_gb300 import workloads as wl
    per = a.gap_instances
    base = [wl.qkp(300, d, 5000 + 100 * q + i) for q, d in enumerate(DENSITIES)
            for i in range(per)]
    C, T, beta, K = a.chains, a.sweeps, a.beta_max, a.gap_iters
    runs = {}
    for name, scale, eta in [("saim", 1.0, a.gap_eta)] + \
            [("penalty_x%d" % s_, float(s_), 0.0) for s_ in (1, 2, 4, 8, 16, 32, 64)]:
        insts = [dataclasses.replace(i, alpha=i.alpha * scale) for i in base]
        prob = sais.Problem(insts)
        r = prob.solve(K, C, T, beta, eta, 31337, variant="auto", use_graph=True)
        runs[name] = (r["best_cost"].copy(), r["feasible_count"].copy(), r["elapsed_ms"])
        prob.close()
    none = np.iinfo(np.int64).max
    best = np.min(np.stack([v[0] for v in runs.values()]), axis=0)
    samples = K * C
    out = {"instances": len(base), "budget": "%d iterations x %d chains x %d sweeps" % (K, C, T),
           "best_known": "best feasible sample over all runs below (uncertified)"}
    for name, (bc, fc, ms) in runs.items():
        feas = bc != none
        gap = np.where(feas & (best != none), (bc - best) / np.abs(best.astype(np.float64)), 1.0)
        out[name] = {"within_1pct": int(((gap <= 0.01) & feas).sum()),
                     "any_feasible": int(feas.sum()),
                     "median_gap": float(np.median(gap)),
                     "feasible_sample_fraction": float(fc.sum() / (samples * len(base))),
                     "device_ms": ms}
    return out


def run_best_measurement(a, sais, torch):
    """Best-in-run tracking and capacity tightening (Sec. IV-B) on the case the paper finds
    hard to make feasible, MKP N=250 m=5 (`rb_instances` instances, profits and weights of the
    MKP generator): Algorithm 1 storing each run's last sample (the paper's reading), storing
    its best feasible sweep-end state, and the latter with capacities tightened to 0.95 B and
    0.9 B, each `rb_iters` iterations x `chains` chains x `sweeps` sweeps with Table I's MKP
    settings (P = 5dN, beta_max = 50, eta = 20 in normalised units), one CUDA graph per run.  Best-known profit per instance = the best feasible sample of all
    these runs (uncertified).  Feasible fraction = stored feasible samples / (iterations x
    chains)."""
    import dataclasses
    from paper_2501_04971_gb300 import workloads as wl
    base = [wl.mkp(250, 5, 7000 + i) for i in range(a.rb_instances)]
    C, T, beta, K = a.chains, a.sweeps, a.rb_beta_max, a.rb_iters
    runs = {}
    for name, frac, rb in [("last_sample", 1.0, False), ("run_best", 1.0, True),
                           ("run_best_tight_0.95", 0.95, True), ("run_best_tight_0.9", 0.9, True)]:
        insts = [dataclasses.replace(i) for i in base]
        if frac < 1.0:
            for j in insts:
                j.b_tight = np.maximum(1, np.floor(np.asarray(j.b) * frac)).astype(np.int64)
        prob = sais.Problem(insts)
        r = prob.solve(K, C, T, beta, a.rb_eta, 4242, variant="auto", use_graph=True,
                       run_best=rb)
        runs[name] = (r["best_cost"].copy(), r["feasible_count"].copy(), r["elapsed_ms"])
        prob.close()
    none = np.iinfo(np.int64).max
    best = np.min(np.stack([v[0] for v in runs.values()]), axis=0)
    out = {"instances": len(base), "workload": "MKP N=250 m=5",
           "budget": "%d iterations x %d chains x %d sweeps" % (K, C, T),
           "beta_max": beta, "eta": a.rb_eta,
           "best_known": "best feasible sample over all runs below (uncertified)"}
    for name, (bc, fc, ms) in runs.items():
        feas = bc != none
        gap = np.where(feas & (best != none), (bc - best) / np.abs(best.astype(np.float64)), 1.0)
        out[name] = {"within_1pct": int(((gap <= 0.01) & feas).sum()),
                     "any_feasible": int(feas.sum()),
                     "median_gap": float(np.median(gap)),
                     "feasible_sample_fraction": float(fc.sum() / (K * C * len(base))),
                     "device_ms": ms}
    return out


def paper_scale_measurement(a, sais, torch):
    """The paper's own budget (Table I, QKP: 2000 runs of 1000 MCS, one sample per run,
    beta_max 10, P = 2dN) on synthetic QKP instances of the paper's sizes, N in {100, 200, 300}
    x d in {0.25, 0.5, 0.75, 1} (`ps_per_class` each): Algorithm 1 with one chain per instance
    for `ps_iters` iterations at Table I's eta = 20 (normalised units), against the batched
    form with the same number of samples per instance (`ps_iters` / 128 iterations x 128
    chains) and with the same number of iterations (`ps_iters` x 128 chains).  Accuracy of an
    instance = its best feasible profit / the best known (the best feasible sample of the three
    runs, uncertified), reported per size as the median and interquartile range the paper
    quotes (Sec. IV-A: median above 99.2 %, IQR below 0.8 %).  The single-chain sampler is
    latency-bound, so a one-chain iteration costs about as long as a 128-chain one."""
    from paper_2501_04971_gb300 import workloads as wl
    sizes = (100, 200, 300)
    insts = [wl.qkp(n, d, 8000 + 1000 * si + 100 * q + i) for si, n in enumerate(sizes)
             for q, d in enumerate(DENSITIES) for i in range(a.ps_per_class)]
    size_of = np.array([i.n for i in insts])
    K1, T, beta = a.ps_iters, a.sweeps, a.beta_max
    Kb = max(1, K1 // 128)
    prob = sais.Problem(insts)
    runs = {}
    for name, K, C, seed in [("paper_single_chain", K1, 1, 11),
                             ("batched_equal_samples", Kb, 128, 11),
                             ("batched_equal_iterations", K1, 128, 11)]:
        r = prob.solve(K, C, T, beta, a.ps_eta, seed, variant="auto", use_graph=True)
        runs[name] = (r["best_cost"].copy(), r["feasible_count"].copy(), r["elapsed_ms"], K, C)
    prob.close()
    none = np.iinfo(np.int64).max
    best = np.min(np.stack([v[0] for v in runs.values()]), axis=0)
    out = {"instances": len(insts), "sizes": list(sizes), "per_class": a.ps_per_class,
           "sweeps": T, "eta": a.ps_eta,
           "best_known": "best feasible sample over the three runs (uncertified)"}
    for name, (bc, fc, ms, K, C) in runs.items():
        feas = (bc != none) & (best != none)
        acc = np.where(feas, bc.astype(np.float64) / np.where(best != 0, best, 1), 0.0) * 100.0
        per = {}
        for n in sizes:
            v = acc[size_of == n]
            q1, med, q3 = np.percentile(v, [25, 50, 75])
            per[str(n)] = {"median_accuracy_pct": float(med), "iqr_pct": float(q3 - q1),
                           "min_accuracy_pct": float(v.min())}
        out[name] = {"iterations": K, "chains": C, "samples_per_instance": K * C,
                     "device_s": ms / 1e3,
                     "feasible_sample_fraction": float(fc.sum() / (K * C * len(insts))),
                     "accuracy_by_size": per}
    return out


def ragged_measurement(a, sais, torch):
    """The ragged batch: 384 QKP (N uniform in [100, 1000], profits up to 10^4) + 128 MKP
    (N in {250, 500}, m in {5, 10, 30}) with 64..256 chains each, in one SAIS_AUTO problem.
    The autotuner picks each launch group's sampler and CTA shape (its timing launches also
    give per-class rates) and then between one persistent launch over the batch's items and the
    concurrent group launches; Algorithm 1 runs `ragged_iters` iterations of `sweeps` sweeps as
    one captured CUDA graph (sais_solve, use_graph) in both modes; rate = spin updates / solve
    device time of the mode the autotuner kept."""
    from paper_2501_04971_gb300 import workloads as wl
    insts = wl.ragged_batch()
    prob = sais.Problem(insts)
    counts = np.random.default_rng(0x524147).integers(64, 257, prob.count).astype(np.int32)
    prob.set_instance_chains(counts)
    C = 256
    tune = prob.autotune(C, a.ragged_tune_sweeps)
    names = {0: "plain", 1: "blocked"}
    groups = []
    for g in range(tune["groups"]):
        groups.append({"variant": names[tune["variant"][g]], "instances": tune["size"][g],
                       "block_k": tune["block_k"][g], "chains_per_cta": tune["chains_per_cta"][g],
                       "spin_updates_per_s": tune["spin_updates"][g] / (tune["ms"][g] / 1e3),
                       "tune_launch_ms": tune["ms"][g],
                       "tune_launch_spin_updates": int(tune["spin_updates"][g])})
    # Both SAIS_AUTO modes on the same solve (identical samples); the headline is the one the
    # autotuner kept.
    modes = {}
    for mode in (("persistent", "groups") if tune["persistent_ok"] else ("groups",)):
        prob.set_auto_mode(mode)
        prob.solve(1, C, a.sweeps, a.beta_max, a.gap_eta, 99, variant="auto", use_graph=True)
        rm = prob.solve(a.ragged_iters, C, a.sweeps, a.beta_max, a.gap_eta, 100, variant="auto",
                        use_graph=True)
        modes[mode] = {"value": rm["spin_updates"] / (rm["elapsed_ms"] / 1e3),
                       "elapsed_ms": rm["elapsed_ms"], "result": rm}
        if mode == "persistent":   # the last iteration's launch: how evenly the SMs were busy
            st = prob.persistent_stats()
            bf = st["busy_fraction"]
            modes[mode]["last_launch"] = {
                "ctas": st["ctas"], "span_ms": st["span_ns"] / 1e6,
                "busy_fraction_mean": float(bf.mean()), "busy_fraction_min": float(bf.min()),
                "busy_fraction_p10": float(np.percentile(bf, 10)),
                "items_per_cta_max": int(st["items"].max()),
                "items_per_cta_min": int(st["items"].min()),
                "tail_ms": float((st["end_ns"].max() - np.median(st["end_ns"])) / 1e6)}
    kept = "persistent" if tune["persistent"] else "groups"
    r = modes[kept]["result"]
    nsp = np.array([s.n_spins for s in prob.scalars])
    out = {"workload": "384 QKP N~U[100,1000] (profits <= 1e4) + 128 MKP N in {250,500}, "
                       "m in {5,10,30}; chains U[64,256] per instance; %d sweeps; %d graph-"
                       "captured iterations of Algorithm 1" % (a.sweeps, a.ragged_iters),
           "value": r["spin_updates"] / (r["elapsed_ms"] / 1e3), "unit": UNIT,
           "elapsed_ms": r["elapsed_ms"], "spin_updates": int(r["spin_updates"]),
           "max_spins": int(nsp.max()), "groups": groups, "mode": kept,
           "modes": {k: {kk: vv for kk, vv in dict(v, unit=UNIT).items() if kk != "result"}
                     for k, v in modes.items()},
           "autotune_launch_ms": {"persistent": tune["persistent_ms"],
                                  "groups": tune["groups_ms"]},
           "feasible_instances": int((r["best_cost"] != np.iinfo(np.int64).max).sum())}
    prob.close()
    return out


def warmstart_measurement(a, sais, torch):
    """Learned warm start: `ws_train` seeded QKP/MKP instances (N in [100, 500]) labelled by the
    multipliers Algorithm 1 converges to (30 iterations x 128 chains x 200 sweeps, SAIS_AUTO,
    graph-captured), the network trained on 90 % of the instances by the project's kernels and
    checked on the other 10 %, then samples to a 1 % gap, warm against cold, on QKP N=500 d=0.5
    and MKP N=500 m=10 (`ws_eval` instances each).  Also the device time of the training step
    and of inference, with their tensor-core flops against the bf16 peak."""
    from paper_2501_04971_gb300 import warmstart as ws, workloads as wl
    t0 = time.perf_counter()
    insts = ws.training_instances(a.ws_train)
    t_gen = time.perf_counter() - t0
    bud = ws.SolveBudget(iters=30, chains=128, sweeps=200, beta_max=a.beta_max, eta=a.gap_eta)
    X, y, t_lab, upd = ws.label(insts, bud)
    rows = np.cumsum([0] + [i.m for i in insts])
    cut = int(rows[int(0.9 * len(insts))])
    net, losses, t_train = ws.train(X[:cut], y[:cut], epochs=a.ws_epochs)
    pred = ws.predict(net, X[cut:])
    mse_w = float(np.mean((np.maximum(pred, 0) - y[cut:]) ** 2))
    mse_c = float(np.mean(y[cut:] ** 2))
    # kernel timing on 4096 rows (one minibatch): training step (forward, backward, Adam
    # update) and inference
    B = min(4096, X.shape[0])
    Xd, yd = torch.tensor(X[:B], device="cuda"), torch.tensor(y[:B], device="cuda")
    out = torch.empty(B, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = {}
    for name, fn in (("train_step", lambda: net.train_step(Xd, yd, 1e-6)),
                     ("forward", lambda: net.forward(Xd, out=out))):
        for _ in range(5):
            fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(50):
            fn()
        e1.record()
        torch.cuda.synchronize()
        times[name] = e0.elapsed_time(e1) / 50
    flops_row = {"train_step": 2 * 128 * (16 + 144 + 128 + 144 + 16), "forward": 2 * 128 * (16 + 144)}
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = peaks.get("bf16_tflops", 1900.0)
    kern = {k: {"ms": v, "rows": B, "tflops": flops_row[k] * B / (v / 1e3) / 1e12,
                "frac_of_bf16_peak": flops_row[k] * B / (v / 1e3) / 1e12 / peak}
            for k, v in times.items()}
    ev_res = {}
    for name, ev in (("qkp_n500_d0.5", [wl.qkp(500, 0.5, 7000 + i) for i in range(a.ws_eval)]),
                     ("mkp_n500_m10", [wl.mkp(500, 10, 8000 + i) for i in range(a.ws_eval)])):
        t1 = time.perf_counter()
        r = ws.evaluate(net, ev, bud, best_seeds=2)
        ev_res[name] = {"cold": {k: v for k, v in r["cold"].items() if k != "per_instance"},
                        "warm": {k: v for k, v in r["warm"].items() if k != "per_instance"},
                        "best_known_feasible": r["best_known_feasible"],
                        "seconds": time.perf_counter() - t1}
    net.close()
    return {"train_instances": len(insts), "rows": int(X.shape[0]), "label_seconds": t_lab,
            "label_spin_updates_per_s": upd / t_lab, "generate_seconds": t_gen,
            "label_budget": "30 iterations x 128 chains x 200 sweeps, eta %g, lambda label = "
                            "mean of the second half" % bud.eta,
            "epochs": a.ws_epochs, "train_device_seconds": t_train,
            "loss_first_last": [losses[0], losses[-1]],
            "heldout_mse_warm": mse_w, "heldout_mse_lambda0": mse_c, "kernels": kern,
            "samples_to_1pct_gap": ev_res,
            "samples_unit": "chains x iterations (each sample = one anneal of 200 sweeps)"}


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------

def main():
    a = parse()
    if a.impl == "reference":
        return reference_arm(a)
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__
    # one rank compiles (concurrent builds would write the same objects); the others load
    if dist and rank != 0:
        dist.barrier()
    __graft_entry__.build()
    if dist and rank == 0:
        dist.barrier()
    from paper_2501_04971_gb300 import sais

    if a.make_best_known:
        return make_best_known(a, sais, torch)
    if a.kernel_case:
        return kernel_case(a, sais, torch)
    insts = workload(a.per_density, rank)
    prob = sais.Problem(insts, device=local)
    nspins = np.array([s.n_spins for s in prob.scalars], dtype=np.int64)
    upd_step = int(nspins.sum()) * a.chains * a.sweeps
    variant = a.variant
    if variant == "auto":
        variant = "plain"
        try:
            lam_probe = torch.zeros(prob.count * prob.m_stride, device="cuda")
            prob.sample(lam_probe, 32, 1, a.beta_max, 0, 0, variant="blocked")
            variant = "blocked"
        except sais.SaisError:
            pass

    stream = torch.cuda.current_stream()
    lam = torch.zeros(prob.count * prob.m_stride, device="cuda", dtype=torch.float32)
    out = prob.alloc_outputs(a.chains)
    best = prob.alloc_best()

    def step(k):
        prob.sample(lam, a.chains, a.sweeps, a.beta_max, 1234, k, variant=variant,
                    block_k=a.block_k, out=out, stream=stream)
        prob.track_best(out, a.chains, k, best, stream=stream)
        prob.update_lambda(out["g"], a.chains, a.eta, True, lam, stream=stream)

    for k in range(a.warmup):
        step(k)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(a.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_start.record(stream)
        for k in range(a.steps):
            ev[k][0].record(stream)
            prob.sample(lam, a.chains, a.sweeps, a.beta_max, 1234, a.warmup + k,
                        variant=variant, block_k=a.block_k, out=out, stream=stream)
            ev[k][1].record(stream)
            prob.track_best(out, a.chains, a.warmup + k, best, stream=stream)
            prob.update_lambda(out["g"], a.chains, a.eta, True, lam, stream=stream)
        t_end.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = t_start.elapsed_time(t_end)
    kern_ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    ms = over_ranks(ms, dist, "cuda", "max")
    # each rank's instances have their own N' (slack bits depend on the capacities)
    upd_all = over_ranks(upd_step, dist, "cuda", "sum")
    value = upd_all * a.steps / (ms / 1e3)

    # roofline of the dominant kernel (the sampler), per launch
    kmean = statistics.mean(kern_ms) / 1e3
    if variant == "blocked":
        npad = ((nspins + 63) // 64) * 64
        flops = float((2 * npad * nspins).sum()) * a.chains * a.sweeps
        # DRAM bytes (read + write) per instance of one launch of this kernel, measured with ncu
        # on a 152-instance, 200-sweep launch (bench.py --kernel-case rankk_qkp300): W is read
        # once per CTA, so the traffic scales with instances, not sweeps
        traffic = 212512.0 * prob.count if (a.chains == 128 and a.block_k in (0, 16)) else None
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
            if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
        peak = peaks.get("bf16_tflops", 1900.0) * 1e12
        roof = {"bound": "tensor", "achieved": flops / kmean / 1e12, "peak": peak / 1e12,
                "unit": "TFLOP/s", "frac": flops / kmean / peak, "traffic": traffic,
                "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst)" if peaks else
                "fallback 1.9 PFLOP/s"}
    else:
        flops = float((2 * nspins * nspins).sum()) * a.chains * a.sweeps
        peak = SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6
        roof = {"bound": "alu", "achieved": flops / kmean / 1e12, "peak": peak / 1e12,
                "unit": "TFLOP/s", "frac": flops / kmean / peak, "traffic": None,
                "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
                "per_update": "2 N' flops (Eq. 9 field, dense)"}
    roof["kernel_ms"] = kmean * 1e3

    # end to end through sais_solve with pinned host buffers, one iteration per step
    e2e = None
    if not a.no_e2e:
        M, Wd, cnt = prob.m_stride, prob.words, prob.count
        lam_h = torch.zeros(cnt * M, dtype=torch.float32).pin_memory()
        pinned = {"best_cost": torch.zeros(cnt, dtype=torch.int64).pin_memory(),
                  "best_x": torch.zeros(cnt * Wd, dtype=torch.int32).pin_memory(),
                  "best_iter": torch.zeros(cnt, dtype=torch.int32).pin_memory(),
                  "best_chain": torch.zeros(cnt, dtype=torch.int32).pin_memory(),
                  "feasible_count": torch.zeros(cnt, dtype=torch.int64).pin_memory(),
                  "lambda_final": torch.zeros(cnt * M, dtype=torch.float32).pin_memory(),
                  "lambda_trace": torch.zeros(cnt * M, dtype=torch.float32).pin_memory()}
        prm = sais.sais_solve_params()
        prm.iters, prm.chains, prm.sweeps, prm.beta_max = 1, a.chains, a.sweeps, a.beta_max
        prm.eta, prm.seed, prm.project_nonneg = a.eta, 1234, 1
        prm.variant = sais._VARIANTS[variant]
        prm.block_k = a.block_k
        prm.lambda0 = sais._P(lam_h.data_ptr())
        res = sais.sais_solve_result()
        for k_, v_ in pinned.items():
            setattr(res, k_, sais._P(v_.data_ptr()))
        sp = sais._P(stream.cuda_stream)
        prm.iter0 = 0
        sais.sais_solve(prob.handle, prm, res, sp)     # warm
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for k in range(a.steps):
            prm.iter0 = k
            sais.sais_solve(prob.handle, prm, res, sp)
            lam_h.copy_(pinned["lambda_final"])
        dt = time.perf_counter() - t0
        dt = over_ranks(dt, dist, "cuda", "max")
        h2d = cnt * M * 4 + cnt * (8 + 4 + 4) + 4
        d2h = cnt * (8 + Wd * 4 + 4 + 4 + 8 + M * 4 + M * 4)
        e2e = {"value": upd_all * a.steps / dt, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "api": "sais_solve(iters=1), pinned host lambda0 and results"}

    plain_cmp = None
    if variant == "blocked" and not a.no_plain:
        # the same workload on the plain sampler: identical samples, per-step time only
        for k in range(1):
            prob.sample(lam, a.chains, a.sweeps, a.beta_max, 1234, k, variant="plain", out=out,
                        stream=stream)
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        np_steps = max(1, min(2, a.steps))
        p0.record(stream)
        for k in range(np_steps):
            prob.sample(lam, a.chains, a.sweeps, a.beta_max, 1234, k, variant="plain", out=out,
                        stream=stream)
        p1.record(stream)
        torch.cuda.synchronize()
        pms = over_ranks(p0.elapsed_time(p1) / np_steps, dist, "cuda", "max")
        pval = upd_all / (pms / 1e3)
        plain_cmp = {"value": pval, "unit": UNIT, "sampler_ms_per_step": pms,
                     "blocked_over_plain": value / pval}
    mkp = None
    if not a.no_ksweep and world == 1:
        mkp = mkp_measurement(a, sais, torch)
    ksweep = None
    if not a.no_ksweep and world == 1 and variant == "blocked":
        ksweep = ksweep_measurement(a, sais, torch, insts, clk.summary().get("sm_mhz") or SM_MAX_MHZ)
    gap = None
    if not (a.no_target or a.no_gap) and world == 1 and os.path.exists(a.best_known):
        gap = target_measurement(a, sais, torch)
    ragged = None
    if not a.no_ragged and world == 1:
        ragged = ragged_measurement(a, sais, torch)
    pen = None
    if a.penalty and world == 1:
        pen = penalty_measurement(a, sais, torch)
    rbm = None
    if a.run_best and world == 1:
        rbm = run_best_measurement(a, sais, torch)
    psm = None
    if a.paper_scale and world == 1:
        psm = paper_scale_measurement(a, sais, torch)
    warm = None
    if a.warmstart and world == 1:
        warm = warmstart_measurement(a, sais, torch)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    if world == 1 and not a.no_cpu:
        cpu = cpu_baseline_line(insts, a.cpu_seconds)
    clocks = clk.summary()
    if variant == "blocked":
        # The sampler is bound by the latency of each chain's sequential decisions, not by a
        # pipe: SM cycles per spin-step of a 128-chain CTA (live, at the sampled clock), and the
        # issue and tensor-pipe activity of the same kernel from its ncu capture.
        mhz = clocks.get("sm_mhz") or SM_MAX_MHZ
        steps = float(((nspins + 15) // 16 * 16).sum()) * (-(-a.chains // 128)) * a.sweeps
        roof["latency"] = {
            "cycles_per_spin_step": kmean * mhz * 1e6 * SM_COUNT / steps,
            "smsp_issue_active": 0.473, "tensor_pipe_active": 0.056,
            "source": "ncu --set full of bench.py --kernel-case rankk_qkp300: issue slots "
                      "busy 47 %, tensor pipe 5.6 %"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16" if variant == "blocked" else "fp32",
            "data": "synthetic",
            "config": {"workload": workload_name(a), "instances": prob.count,
                       "chains": a.chains, "sweeps": a.sweeps, "spins_total": int(nspins.sum()),
                       "variant": variant, "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (W int16 + bf16 of 1024 instances, "
                             f"{prob.count * 2 * 2 * 320 * 320 / 1e6:.0f} MB)"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": 3 * a.steps, "clocks": clocks,
            "updates_per_step": upd_step, "plain": plain_cmp, "blocked_k": ksweep,
            "plain_mkp": mkp,
            "gap_1pct": gap,
            "ragged": ragged}
    if pen is not None:
        line["penalty_vs_saim"] = pen
    if rbm is not None:
        line["run_best_mkp"] = rbm
    if psm is not None:
        line["paper_scale_qkp"] = psm
    if warm is not None:
        line["warmstart"] = warm
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
