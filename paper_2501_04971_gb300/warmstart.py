"""Learned multiplier warm start: labels from the method's own runs, training, evaluation.

The paper starts Algorithm 1 from lambda = 0 (Sec. III-A).  Here a small network predicts, for
each constraint, the multiplier the method converges to, from features of the instance
(``sais_constraint_features``), and Algorithm 1 starts from that prediction instead
(``sais_warm_start``).  Everything that computes runs in libsais kernels: the labels come from
``sais_solve`` (SAIS_AUTO over ragged batches), training is ``sais_mlp_train_step`` (tcgen05
forward/backward + Adam), evaluation is the sampler loop; this module only prepares host arrays
and schedules the calls.

Label of constraint k of an instance: the mean of lambda_k over the second half of a run of
``iters`` iterations (the subgradient iterates oscillate around the dual optimum).
"""
from __future__ import annotations

import time
from dataclasses import dataclass
import numpy as np

from . import sais
from . import workloads as wl


def training_instances(count: int, seed0: int = 10 ** 6, n_lo: int = 100, n_hi: int = 500):
    """`count` instances, seeds seed0 + i: even i QKP (N uniform in [n_lo, n_hi], density in
    {0.25, 0.5, 0.75, 1}), odd i MKP (N uniform in [n_lo, n_hi], m in {5, 10})."""
    out = []
    for i in range(count):
        r = np.random.default_rng(seed0 + i)
        n = int(r.integers(n_lo, n_hi + 1))
        if i % 2 == 0:
            out.append(wl.qkp(n, float(r.choice([0.25, 0.5, 0.75, 1.0])), seed0 + i))
        else:
            out.append(wl.mkp(n, int(r.choice([5, 10])), seed0 + i))
    return out


@dataclass
class SolveBudget:
    iters: int = 30
    chains: int = 128
    sweeps: int = 200
    beta_max: float = 10.0
    eta: float = 2000.0


def label(instances, budget: SolveBudget, seed: int = 7, batch: int = 2048, device: int = 0):
    """Features (rows x 8) and converged-multiplier labels (rows) of every constraint, from
    Algorithm 1 started at lambda = 0 on batches of `batch` instances (SAIS_AUTO, one CUDA graph
    per batch).  Returns (X, y, seconds, spin_updates)."""
    Xs, ys = [], []
    t0, upd = time.perf_counter(), 0
    for b0 in range(0, len(instances), batch):
        part = instances[b0:b0 + batch]
        prob = sais.Problem(part, device=device)
        r = prob.solve(budget.iters, budget.chains, budget.sweeps, budget.beta_max, budget.eta,
                       seed + b0, variant="auto", use_graph=True)
        upd += int(r["spin_updates"])
        tr = r["lambda_trace"]                       # iters x count x m_stride
        half = tr[budget.iters // 2:].mean(axis=0)
        Xs.append(prob.features())
        ys.append(np.concatenate([half[j, :inst.m] for j, inst in enumerate(part)]))
        prob.close()
    return (np.concatenate(Xs).astype(np.float32), np.concatenate(ys).astype(np.float32),
            time.perf_counter() - t0, upd)


def train(X, y, epochs: int = 200, batch_rows: int = 4096, lr: float = 2e-3, seed: int = 0,
          device: int = 0, log_every: int = 0):
    """Adam on the mean squared error (normalised targets), minibatches of a fresh host
    permutation each epoch uploaded as one contiguous block.  Returns (net, losses per epoch,
    seconds of device time)."""
    import torch
    net = sais.MLP(seed, device)
    net.fit_normalization(X, y)
    rng = np.random.default_rng(seed)
    dev = torch.device("cuda", device)
    rows = X.shape[0]
    Xd = torch.empty((rows, 8), dtype=torch.float32, device=dev)
    yd = torch.empty(rows, dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    losses, t_dev = [], 0.0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for ep in range(epochs):
        perm = rng.permutation(rows)
        Xd.copy_(torch.from_numpy(np.ascontiguousarray(X[perm])))
        yd.copy_(torch.from_numpy(np.ascontiguousarray(y[perm])))
        ev0.record()
        for b0 in range(0, rows, batch_rows):
            b1 = min(rows, b0 + batch_rows)
            net.train_step(Xd[b0:b1], yd[b0:b1], lr, loss=loss)
        ev1.record()
        torch.cuda.synchronize()
        t_dev += ev0.elapsed_time(ev1) / 1e3
        losses.append(float(loss.item()))
        if log_every and ep % log_every == 0:
            print(f"epoch {ep}: last minibatch loss {losses[-1]:.4f}", flush=True)
    net.status()
    return net, losses, t_dev


def predict(net, X, device: int = 0) -> np.ndarray:
    import torch
    Xd = torch.tensor(np.ascontiguousarray(X, np.float32), device=torch.device("cuda", device))
    y = net.forward(Xd).cpu().numpy()
    return y


def best_history(prob, lam0, budget: SolveBudget, seed: int):
    """Algorithm 1 from lam0 (device tensor, count x m_stride), one iteration at a time through
    the C-ABI; returns the best feasible cost of every instance after each iteration
    (iters x count, INT64_MAX while none is feasible)."""
    import torch
    C, T = budget.chains, budget.sweeps
    lam = lam0.clone()
    o = prob.alloc_outputs(C)
    best = prob.alloc_best()
    hist = np.zeros((budget.iters, prob.count), np.int64)
    stream = torch.cuda.current_stream()
    for k in range(budget.iters):
        prob.sample(lam, C, T, budget.beta_max, seed, k, variant="auto", out=o, stream=stream)
        prob.track_best(o, C, k, best, stream=stream)
        prob.update_lambda(o["g"], C, budget.eta, True, lam, stream=stream)
        hist[k] = best["best_cost"].cpu().numpy()
    return hist


def samples_to_gap(hist, best_known, chains: int, gap: float = 0.01):
    """Samples (chains x iterations) until the best feasible profit reaches (1 - gap) x
    best-known, per instance (nan if never).  Costs are negative profits."""
    none = np.iinfo(np.int64).max
    hit = (hist != none) & (-hist >= (1 - gap) * (-best_known)[None, :])
    first = np.where(hit.any(axis=0), hit.argmax(axis=0) + 1.0, np.nan)
    return first * chains


def evaluate(net, instances, budget: SolveBudget, seed: int = 4242, best_seeds: int = 2,
             device: int = 0):
    """Samples to a 1 % gap, cold (lambda = 0, Algorithm 1 as in the paper) against warm
    (lambda = the network's prediction), on the same sampler seed.  Best-known per instance:
    the best feasible profit of `best_seeds` extra cold runs and of both evaluated runs
    (uncertified)."""
    import torch
    prob = sais.Problem(instances, device=device)
    dev = torch.device("cuda", device)
    cold = torch.zeros(prob.count * prob.m_stride, dtype=torch.float32, device=dev)
    warm = torch.zeros_like(cold)
    prob.warm_start(net, warm)
    best = np.full(prob.count, np.iinfo(np.int64).max, np.int64)
    for s in range(best_seeds):
        r = prob.solve(budget.iters, budget.chains, budget.sweeps, budget.beta_max, budget.eta,
                       90000 + s, variant="auto", use_graph=True)
        best = np.minimum(best, r["best_cost"])
    hist = {name: best_history(prob, lam0, budget, seed)
            for name, lam0 in (("cold", cold), ("warm", warm))}
    for h in hist.values():
        best = np.minimum(best, h[-1])
    res = {"best_known_feasible": int((best != np.iinfo(np.int64).max).sum())}
    for name, h in hist.items():
        reached = samples_to_gap(h, best, budget.chains)
        ok = ~np.isnan(reached)
        res[name] = {"reached": int(ok.sum()), "of": prob.count,
                     "median_samples": float(np.median(reached[ok])) if ok.any() else None,
                     "mean_samples_unreached_as_budget": float(
                         np.where(ok, reached, budget.iters * budget.chains).mean()),
                     "per_instance": reached}
    res["lambda0_warm"] = warm.cpu().numpy().reshape(prob.count, prob.m_stride)
    prob.close()
    return res
