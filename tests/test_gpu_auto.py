"""Ragged batches: SAIS_AUTO (one persistent launch, or launch groups), per-instance chain
counts and the autotuner.

A batch that mixes quadratic and linear objectives, resident and streamed W, pair values that
need the BF16 hi/lo split, many constraints and an N' beyond the rank-k kernels' TMEM budget
runs under SAIS_AUTO as one persistent launch over a list of (instance, chain group) items, or
as several launch groups over one work list.  Every decision of every chain
depends only on (seed, instance, chain, sweep, spin), so the result must be identical, element by
element, to the plain sampler on the same batch, and a chain of an instance with fewer chains
must equal the same chain of the uniform run.  Sampled chains are checked against the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2501_04971_gb300 import sais, workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _mixed():
    return [wl.qkp(100, 0.5, 31),                     # blocked, W resident
            wl.qkp(400, 0.5, 32),                     # blocked, W streamed
            wl.qkp(150, 0.5, 33, profit_max=10000),   # blocked, streamed hi/lo
            wl.mkp(60, 3, 34),                        # linear objective: plain
            wl.qkp(600, 0.25, 35),                    # N' beyond 496: block fields
            wl.mkp(80, 10, 36),                       # m = 10: plain
            wl.qkp(60, 0.75, 37)]                     # blocked, W resident


def _with_constraints(inst, m, seed):
    """The QKP objective of `inst` with m random knapsack constraints instead of one."""
    import dataclasses
    r = np.random.default_rng(seed)
    A = r.integers(0, 50, (m, inst.n)).astype(np.int32)
    b = np.maximum(1, (A.sum(axis=1) // 3)).astype(np.int64)
    return dataclasses.replace(inst, m=m, A=A, b=b)


def _lam(prob, insts, seed=0):
    r = np.random.default_rng(seed)
    a = np.zeros((prob.count, prob.m_stride), np.float32)
    for j, inst in enumerate(insts):
        a[j, :inst.m] = r.uniform(0.0, 2.0, inst.m).astype(np.float32)
    return a


SENT = {"x": -1431655766, "cost": -7, "g": -9, "feasible": 0xAB}


def _filled(prob, C):
    o = prob.alloc_outputs(C)
    for k, v in SENT.items():
        o[k].fill_(v)
    return o


def _sample(prob, lam_h, C, T, seed, it, variant, **kw):
    lam = torch.tensor(lam_h.reshape(-1), device="cuda:0")
    out = prob.sample(lam, C, T, 10.0, seed, it, variant=variant, out=_filled(prob, C), **kw)
    prob.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _assert_same(a, b, what):
    for k in a:
        if not np.array_equal(a[k], b[k]):
            d = np.argwhere(a[k] != b[k])
            raise AssertionError(f"{what}: {k} differs at {len(d)} places, first {d[:4].tolist()}")


def _oracle_check(insts, lam_h, out, T, seed, it, js, nc=2):
    for j in js:
        inst = insts[j]
        ref = oracle.Problem(inst.n, inst.m, inst.W, inst.h, inst.A, inst.b, alpha=inst.alpha,
                             density=inst.density)
        J, hI, _ = ref.ising(lam_h[j, :inst.m])
        want = oracle.anneal(J, hI, 10.0, T, seed + j, it, nc)
        got = sais.unpack_bits(out["x"][j], ref.nprime)[:nc]
        assert np.array_equal(got, want), f"instance {j}: states differ from the oracle"
        for c in range(nc):
            assert out["cost"][j, c] == ref.cost(got[c])
            assert np.array_equal(out["g"][j, c, :inst.m], ref.constraints(got[c]))


def test_auto_groups_equal_plain_on_mixed_batch():
    insts = _mixed()
    prob = sais.Problem(insts)
    lam = _lam(prob, insts, 1)
    assert prob.plan(160, "auto")["kernel"] == "persistent"
    a = _sample(prob, lam, 160, 100, 21, 2, "auto")
    prob.set_auto_mode("groups")
    assert prob.plan(160, "auto")["kernel"] == "launch groups"
    g = _sample(prob, lam, 160, 100, 21, 2, "auto")
    p = _sample(prob, lam, 160, 100, 21, 2, "plain")
    _assert_same(a, p, "persistent vs plain")
    _assert_same(g, p, "groups vs plain")
    _oracle_check(insts, lam, a, 100, 21, 2, js=range(len(insts)))
    prob.close()


@pytest.mark.parametrize("case", ["qkp_sizes", "hilo_m8", "linear_only", "one_instance"])
def test_persistent_launch_equals_plain(case):
    """The persistent launch on batches of each item kind: block fields with m <= 1 and
    m <= 8 (with and without the hi/lo split, n up to 1000 with state chunks in shared memory),
    the plain sampler on 256 chains with m <= 8 and m <= 32, and a batch of one instance."""
    if case == "qkp_sizes":
        insts = [wl.qkp(n, d, 70 + i) for i, (n, d) in
                 enumerate([(1000, 0.5), (30, 1.0), (300, 0.25), (700, 0.75), (120, 0.5)])]
        C, T = 256, 12
    elif case == "hilo_m8":
        insts = [wl.qkp(200, 0.5, 80, profit_max=10000), _with_constraints(wl.qkp(90, 0.5, 81), 8, 3),
                 wl.qkp(500, 0.25, 82), wl.mkp(40, 20, 83)]
        C, T = 200, 16
    elif case == "linear_only":
        insts = [wl.mkp(70, 5, 90), wl.mkp(50, 30, 91), wl.mkp(120, 8, 92)]
        C, T = 300, 30
    else:
        insts = [wl.qkp(260, 0.5, 95)]
        C, T = 130, 20
    prob = sais.Problem(insts)
    assert prob.plan(C, "auto")["kernel"] == "persistent"
    lam = _lam(prob, insts, 7)
    a = _sample(prob, lam, C, T, 33, 1, "auto")
    st = prob.persistent_stats()
    # items: 128 chains per quadratic item, 256 per linear one
    n_items = sum(-(-C // (128 if inst.W is not None else 256)) for inst in insts)
    assert st["ctas"] == min(n_items, torch.cuda.get_device_properties(0).multi_processor_count)
    assert int(st["items"].sum()) == n_items and (st["items"] >= 1).all()
    assert (st["end_ns"] >= st["start_ns"]).all() and (st["busy_ns"] > 0).all()
    assert (st["busy_ns"] <= st["end_ns"] - st["start_ns"]).all()
    p = _sample(prob, lam, C, T, 33, 1, "plain")
    _assert_same(a, p, "persistent vs plain")
    _oracle_check(insts, lam, a, T, 33, 1, js=range(min(len(insts), 2)), nc=1)
    prob.close()


def test_persistent_launch_forced_timeout_reports_and_recovers():
    """A wait bound of one poll inside the persistent launch: its block-field items give up and
    record SAIS_ETIMEOUT, each CTA that gave up takes no further item and frees its TMEM, the
    context stays usable and the next launch is correct."""
    insts = [wl.qkp(300, 0.5, 96), wl.qkp(800, 0.5, 97), wl.mkp(50, 3, 98)]
    prob = sais.Problem(insts)
    assert prob.plan(128, "auto")["kernel"] == "persistent"
    lam_h = _lam(prob, insts, 8)
    lam = torch.tensor(lam_h.reshape(-1), device="cuda:0")
    prob.sample(lam, 128, 20, 10.0, 1, 0, variant="auto", debug_wait_polls=1)
    with pytest.raises(sais.SaisError) as e:
        prob.synchronize()
    assert e.value.status == sais.SAIS_ETIMEOUT
    prob.synchronize()   # the status word was reset
    a = _sample(prob, lam_h, 128, 20, 1, 0, "auto")
    p = _sample(prob, lam_h, 128, 20, 1, 0, "plain")
    _assert_same(a, p, "persistent vs plain after a timeout")
    prob.close()


def test_groups_mode_block_size_fits_the_group():
    """A block-field group whose largest member (n = 1000, hi/lo) does not fit the default K = 32
    in shared memory runs at K = 16 (it once launched at K = 32 and failed)."""
    insts = [wl.qkp(100, 0.5, 1), wl.qkp(600, 0.5, 2), wl.qkp(1000, 0.25, 3, profit_max=10000),
             wl.mkp(60, 12, 4), wl.qkp(300, 0.75, 5)]
    prob = sais.Problem(insts)
    prob.set_auto_mode("groups")
    lam = _lam(prob, insts, 10)
    g = _sample(prob, lam, 160, 12, 3, 1, "auto")
    p = _sample(prob, lam, 160, 12, 3, 1, "plain")
    _assert_same(g, p, "groups vs plain")
    prob.close()


@pytest.mark.parametrize("mode", ["persistent", "groups"])
def test_auto_trace_equals_plain(mode):
    """sais_sample_trace through SAIS_AUTO: every chain's state at every sweep end equals the
    plain sampler's, for each item kind of the batch (block fields, rank-k, plain)."""
    insts = [wl.qkp(120, 0.5, 21), wl.qkp(560, 0.5, 22), wl.mkp(50, 4, 23)]
    prob = sais.Problem(insts)
    prob.set_auto_mode(mode)
    lam = torch.tensor(_lam(prob, insts, 11).reshape(-1), device="cuda:0")
    a = prob.sample(lam, 128, 9, 10.0, 5, 2, variant="auto", trace=True)
    p = prob.sample(lam, 128, 9, 10.0, 5, 2, variant="plain", trace=True)
    prob.synchronize()
    for k in a:
        assert torch.equal(a[k], p[k]), k
    prob.close()


def test_auto_mode_rejects_unknown_mode():
    prob = sais.Problem([wl.qkp(40, 0.5, 1)])
    with pytest.raises(sais.SaisError) as e:
        sais.sais_set_auto_mode(prob.handle, 7)
    assert e.value.status == sais.SAIS_EINVAL
    prob.close()


def test_batch_beyond_persistent_launch_runs_groups():
    """An instance with m > 8 and a quadratic objective has no item kind of the persistent
    launch: SAIS_AUTO runs the batch as launch groups whatever the mode."""
    from test_gpu_blocked import _with_constraints
    insts = [_with_constraints(wl.qkp(80, 0.5, 99), 10, 4), wl.qkp(100, 0.5, 100)]
    prob = sais.Problem(insts)
    assert prob.plan(128, "auto")["kernel"] == "launch groups"
    lam = _lam(prob, insts, 9)
    a = _sample(prob, lam, 128, 20, 3, 0, "auto")
    p = _sample(prob, lam, 128, 20, 3, 0, "plain")
    _assert_same(a, p, "groups vs plain")
    prob.close()


def test_per_instance_chains_match_uniform_rows():
    insts = _mixed()
    counts = np.array([64, 200, 17, 129, 256, 1, 99], np.int32)
    C = 256
    prob = sais.Problem(insts)
    lam = _lam(prob, insts, 2)
    uni = _sample(prob, lam, C, 80, 5, 1, "plain")
    prob.set_instance_chains(counts)
    runs = {v: _sample(prob, lam, C, 80, 5, 1, v) for v in ("auto", "plain")}
    _assert_same(runs["auto"], runs["plain"], "auto vs plain, ragged chains")
    prob.set_auto_mode("groups")
    _assert_same(_sample(prob, lam, C, 80, 5, 1, "auto"), runs["plain"],
                 "groups vs plain, ragged chains")
    r = runs["auto"]
    for j, cj in enumerate(counts):
        for k in r:
            assert np.array_equal(r[k][j, :cj], uni[k][j, :cj]), (j, k)
            tail = r[k][j, cj:]
            assert (tail == np.array(SENT[k]).astype(tail.dtype)).all(), \
                f"instance {j}: {k} rows past its {cj} chains were written"
    prob.close()


def test_per_instance_chains_blocked_variant():
    insts = [wl.qkp(100, 0.5, 41), wl.qkp(60, 0.25, 42), wl.qkp(120, 1.0, 43)]
    counts = np.array([128, 40, 200], np.int32)
    prob = sais.Problem(insts)
    lam = _lam(prob, insts, 3)
    prob.set_instance_chains(counts)
    b = _sample(prob, lam, 256, 60, 8, 0, "blocked")
    p = _sample(prob, lam, 256, 60, 8, 0, "plain")
    _assert_same(b, p, "blocked vs plain, ragged chains")
    prob.close()


def test_ragged_multiplier_step_and_best_tracking():
    """The multiplier step averages over each instance's own chains, the best tracker looks at
    those chains only: both against the oracle's step and an argmin on the host."""
    insts = [wl.mkp(60, 3, 51), wl.qkp(100, 0.5, 52), wl.mkp(50, 5, 53)]
    counts = np.array([37, 128, 5], np.int32)
    C = 128
    prob = sais.Problem(insts)
    prob.set_instance_chains(counts)
    lam_h = _lam(prob, insts, 4)
    lam = torch.tensor(lam_h.reshape(-1), device="cuda:0")
    out = prob.sample(lam, C, 60, 10.0, 3, 0, variant="auto", out=_filled(prob, C))
    best = prob.alloc_best()
    prob.track_best(out, C, 0, best)
    prob.update_lambda(out["g"], C, 20.0, True, lam)
    prob.synchronize()
    g = out["g"].cpu().numpy()
    cost, feas = out["cost"].cpu().numpy(), out["feasible"].cpu().numpy()
    lam_new = lam.cpu().numpy().reshape(prob.count, prob.m_stride)
    bc = best["best_cost"].cpu().numpy()
    fc = best["feasible_count"].cpu().numpy()
    for j, inst in enumerate(insts):
        cj, m = int(counts[j]), inst.m
        ref = oracle.Problem(inst.n, inst.m, inst.W, inst.h, inst.A, inst.b, alpha=inst.alpha,
                             density=inst.density)
        gsum = g[j, :cj, :m].sum(axis=0)
        want = oracle.lambda_update(gsum, cj, 20.0, True, ref.sigma_g, lam_h[j, :m])
        assert np.array_equal(lam_new[j, :m], want), j
        f = feas[j, :cj].astype(bool)
        assert fc[j] == f.sum()
        if f.any():
            assert bc[j] == cost[j, :cj][f].min()
        else:
            assert bc[j] == np.iinfo(np.int64).max
    prob.close()


@pytest.mark.parametrize("ragged", [False, True])
@pytest.mark.parametrize("mode", ["persistent", "groups"])
def test_auto_solve_with_graph_equals_plain_solve(ragged, mode):
    insts = _mixed()[:4] + [wl.qkp(80, 0.5, 61)]
    prob = sais.Problem(insts)
    prob.set_auto_mode(mode)
    if ragged:
        prob.set_instance_chains(np.array([128, 50, 77, 128, 3], np.int32))
    a = prob.solve(5, 128, 120, 10.0, 20.0, 19, variant="plain")
    b = prob.solve(5, 128, 120, 10.0, 20.0, 19, variant="auto", use_graph=True)
    for k in ("best_cost", "best_x", "best_iter", "best_chain", "feasible_count",
              "lambda_trace", "lambda_final"):
        assert np.array_equal(a[k], b[k]), k
    assert a["spin_updates"] == b["spin_updates"]
    prob.close()


def test_autotune_keeps_results():
    insts = _mixed()
    prob = sais.Problem(insts)
    lam = _lam(prob, insts, 5)
    before = _sample(prob, lam, 128, 60, 4, 0, "auto")
    t = prob.autotune(128, 10)
    assert t["groups"] == len(t["variant"]) >= 2
    assert t["persistent_ok"] and t["persistent_ms"] > 0 and t["groups_ms"] > 0
    assert t["persistent"] == (t["persistent_ms"] < t["groups_ms"])
    assert prob.plan(128, "auto")["kernel"] == ("persistent" if t["persistent"]
                                                 else "launch groups")
    assert t["blocked_instances"] + t["plain_instances"] == len(insts)
    assert sum(t["size"]) == len(insts)
    assert all(ms > 0 for ms in t["ms"])
    after = _sample(prob, lam, 128, 60, 4, 0, "auto")
    _assert_same(before, after, "auto before vs after autotune")
    prob.close()


def test_set_instance_chains_rejects_and_resets():
    prob = sais.Problem([wl.qkp(40, 0.5, 1), wl.qkp(30, 0.5, 2)])
    with pytest.raises(sais.SaisError) as e:
        prob.set_instance_chains(np.array([4, 0], np.int32))
    assert e.value.status == sais.SAIS_EINVAL
    prob.set_instance_chains(np.array([64, 200], np.int32))
    lam = torch.zeros(prob.count * prob.m_stride, device="cuda:0")
    with pytest.raises(sais.SaisError) as e:   # stride below an instance's count
        prob.sample(lam, 128, 10, 10.0, 1, 0, variant="auto")
    assert e.value.status == sais.SAIS_EINVAL
    prob.set_instance_chains(None)
    prob.sample(lam, 128, 10, 10.0, 1, 0, variant="auto")
    prob.synchronize()
    prob.close()
