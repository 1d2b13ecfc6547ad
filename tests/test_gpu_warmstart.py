"""The learned warm start end to end, at a small scale: labels from the method's own runs,
training by the project's kernels, and what the trained network gains over the cold start.

Gains checked: on held-out instances the predicted multipliers are far closer to the converged
ones than lambda = 0 (the cold start of Algorithm 1), and started from them the method reaches a
1 % gap to the best-known profit on at least as many evaluation instances, in no more samples
in total (unreached instances counted at the full budget).
"""
import numpy as np
import pytest

from paper_2501_04971_gb300 import warmstart as ws, workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.fixture(scope="module")
def trained():
    insts = ws.training_instances(600, seed0=2_000_000, n_lo=60, n_hi=160)
    bud = ws.SolveBudget(iters=20, chains=64, sweeps=100)
    X, y, _, _ = ws.label(insts, bud)
    rows = np.cumsum([0] + [i.m for i in insts])
    cut = rows[480]                       # the last 120 instances are held out
    net, losses, _ = ws.train(X[:cut], y[:cut], epochs=150)
    return net, X[cut:], y[cut:], losses


def test_training_converges(trained):
    _, _, _, losses = trained
    assert losses[-1] < 0.1 * losses[0]


def test_predictions_beat_the_cold_start_on_held_out_instances(trained):
    net, X, y, _ = trained
    pred = ws.predict(net, X)
    mse_warm = float(np.mean((np.maximum(pred, 0) - y) ** 2))
    mse_cold = float(np.mean(y ** 2))
    assert mse_warm < 0.25 * mse_cold, (mse_warm, mse_cold)


def test_warm_start_reaches_the_gap_in_fewer_samples(trained):
    net = trained[0]
    ev = [wl.mkp(150, 10, 3_000_000 + i) for i in range(8)] + \
         [wl.qkp(150, 0.5, 3_100_000 + i) for i in range(8)]
    bud = ws.SolveBudget(iters=20, chains=64, sweeps=100)
    r = ws.evaluate(net, ev, bud, best_seeds=1)
    assert r["warm"]["reached"] >= r["cold"]["reached"]
    assert r["warm"]["mean_samples_unreached_as_budget"] <= \
        r["cold"]["mean_samples_unreached_as_budget"]
