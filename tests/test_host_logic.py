"""Host-side logic that needs no GPU: the seeded instance generators (the shapes of the
paper's workloads, Sec. IV-A and IV-B) and the warm-start evaluation's bookkeeping."""
import numpy as np

from paper_2501_04971_gb300 import workloads as wl
from paper_2501_04971_gb300 import warmstart as ws


def test_qkp_generator_shape_and_determinism():
    for n, d, s in [(100, 0.25, 0), (300, 1.0, 3), (57, 0.5, 9)]:
        a, b = wl.qkp(n, d, s), wl.qkp(n, d, s)
        assert a.n == n and a.m == 1 and a.alpha == 2.0 and a.density == d
        assert np.array_equal(a.W, b.W) and np.array_equal(a.b, b.b)     # seeded
        assert np.array_equal(a.W, a.W.T) and not np.diag(a.W).any()     # symmetric, W_ii = 0
        assert a.W.min() >= 0 and a.W.max() <= 100 and a.h.max() <= 100
        w = a.A[0]
        assert w.min() >= 1 and w.max() <= 50
        assert 50 <= a.b[0] <= max(50, int(w.sum()))
        # pair density close to d over the upper triangle
        nz = np.count_nonzero(np.triu(a.W, 1)) + np.count_nonzero(a.h)
        assert abs(nz / (n * (n + 1) / 2) - d) < 0.08
    assert not np.array_equal(wl.qkp(100, 0.5, 1).W, wl.qkp(100, 0.5, 2).W)


def test_mkp_generator_shape():
    for n, m, s in [(250, 5, 0), (100, 10, 4), (500, 30, 2)]:
        a = wl.mkp(n, m, s)
        assert a.W is None and a.A.shape == (m, n) and a.alpha == 5.0 and a.density == -1.0
        assert a.A.min() >= 0 and a.A.max() <= 1000
        assert np.array_equal(a.b, np.maximum(1, np.floor(0.25 * a.A.sum(axis=1))).astype(np.int64))
        assert np.all(a.h >= np.floor(a.A.sum(axis=0) / m)) and np.all(a.h <= a.A.sum(axis=0) / m + 501)


def test_ragged_batch_mix():
    batch = wl.ragged_batch(40, 12, seed=5)
    q, k = batch[:40], batch[40:]
    assert all(i.m == 1 and 100 <= i.n <= 1000 for i in q)
    assert all(i.W is None and i.n in (250, 500) and i.m in (5, 10, 30) for i in k)


def test_training_instances_alternate_qkp_and_mkp():
    insts = ws.training_instances(10, seed0=77, n_lo=50, n_hi=80)
    assert len(insts) == 10
    for i, inst in enumerate(insts):
        assert 50 <= inst.n <= 80
        if i % 2 == 0:
            assert inst.W is not None and inst.density in (0.25, 0.5, 0.75, 1.0)
        else:
            assert inst.W is None and inst.m in (5, 10)
    again = ws.training_instances(10, seed0=77, n_lo=50, n_hi=80)
    assert all(np.array_equal(a.A, b.A) for a, b in zip(insts, again))


def test_samples_to_gap():
    none = np.iinfo(np.int64).max
    # 4 iterations x 3 instances of best-so-far costs (negative profits)
    hist = np.array([[none, -50, none],
                     [-95, -50, none],
                     [-99, -80, none],
                     [-100, -100, none]], np.int64)
    best = np.array([-100, -100, -10], np.int64)
    got = ws.samples_to_gap(hist, best, chains=8, gap=0.01)
    assert got[0] == 3 * 8            # -99 reaches 99 % at the third iteration
    assert got[1] == 4 * 8            # only the exact optimum at the fourth
    assert np.isnan(got[2])           # never feasible
    loose = ws.samples_to_gap(hist, best, chains=8, gap=0.06)
    assert loose[0] == 2 * 8          # -95 is within 6 %
