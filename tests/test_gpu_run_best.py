"""GPU parity of the best-in-run option and of capacity tightening (needs an sm_103a GPU).

* sais_sample_run_best: per chain, the best feasible sweep-end state, its cost, its sweep and
  the number of feasible sweep ends equal the oracle's (or_run_best over the oracle's own
  sweep trace), for the plain sampler, the single-CTA blocked sampler (W resident and
  streamed hi/lo), the block-field sampler and SAIS_AUTO over a ragged batch;
* capacity tightening B' < B (Sec. IV-B): the sampled problem is built from B', feasibility and
  the kept best use B, identical to the oracle; Algorithm 1 with both options matches the
  oracle's solve bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_2501_04971_gb300 import sais, workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

I64MAX = np.iinfo(np.int64).max


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _tighten(inst, frac):
    inst.b_tight = np.maximum(1, (np.asarray(inst.b, np.int64) * frac).astype(np.int64))
    return inst


def _ref(inst):
    bt = getattr(inst, "b_tight", None)
    return oracle.Problem(inst.n, inst.m, inst.W, inst.h, inst.A,
                          inst.b if bt is None else bt, alpha=inst.alpha, density=inst.density,
                          penalty=getattr(inst, "penalty", 0.0) or 0.0, b_check=inst.b)


def _lam_dev(lams, m_stride):
    a = np.zeros((len(lams), m_stride), np.float32)
    for j, l in enumerate(lams):
        a[j, :len(l)] = l
    return torch.tensor(a.reshape(-1), device="cuda:0")


def _run_best_vs_oracle(insts, lams, C, T, beta_max, seed, it, variant, **kw):
    prob = sais.Problem(insts)
    out = prob.sample_run_best(_lam_dev(lams, prob.m_stride), C, T, beta_max, seed, it,
                               variant=variant, **kw)
    torch.cuda.synchronize()
    prob.synchronize()
    x = out["x"].cpu().numpy()
    feas = out["feasible"].cpu().numpy()
    run = {k: v.cpu().numpy() for k, v in out["run"].items()}
    found = 0
    for j, inst in enumerate(insts):
        ref = _ref(inst)
        J, hI, _ = ref.ising(np.asarray(lams[j], np.float32))
        last, tr = oracle.anneal(J, hI, beta_max, T, seed + j, it, C, trace=True)
        cost, rx, sweep, nfeas = oracle.run_best(ref, tr)
        assert np.array_equal(sais.unpack_bits(x[j], ref.nprime), last), f"instance {j}: last"
        for c in range(C):
            assert bool(feas[j, c]) == ref.feasible(last[c]), (j, c)
        assert np.array_equal(run["cost"][j], cost), f"instance {j}: run cost"
        assert np.array_equal(run["sweep"][j], sweep), f"instance {j}: run sweep"
        assert np.array_equal(run["nfeas"][j], nfeas), f"instance {j}: feasible sweep ends"
        assert np.array_equal(sais.unpack_bits(run["x"][j], ref.nprime), rx), f"instance {j}"
        found += int((cost != I64MAX).sum())
    prob.close()
    return found


@pytest.mark.parametrize("variant", ["plain", "blocked"])
def test_run_best_qkp(variant):
    """QKP N=120 (W resident in the blocked sampler), 128 chains x 150 sweeps."""
    insts = [wl.qkp(120, 0.5, 3), wl.qkp(100, 0.75, 4)]
    assert _run_best_vs_oracle(insts, [[0.4], [0.8]], 128, 150, 10.0, 7, 2, variant) > 0


@pytest.mark.parametrize("variant,kw", [("blocked", {"block_k": 32}),
                                        ("plain", {"chains_per_cta": 128}),
                                        ("plain", {"chains_per_cta": 64})])
def test_run_best_launch_shapes(variant, kw):
    """Other launch shapes: 32-spin blocks, 64 and 128 chains per CTA (100 chains: a ragged
    last CTA)."""
    insts = [wl.qkp(90, 0.5, 21), wl.qkp(70, 0.75, 22)]
    assert _run_best_vs_oracle(insts, [[0.6], [0.9]], 100, 120, 10.0, 4, 3, variant, **kw) > 0


def test_run_best_per_instance_chains():
    """Per-instance chain counts (SAIS_AUTO work lists): chains past an instance's count are
    neither sampled into the outputs nor tracked; the others equal the plain sampler's."""
    insts = [wl.qkp(100, 0.5, 31), wl.mkp(60, 3, 32), wl.qkp(200, 0.25, 33)]
    lams = [[0.5], [1.0] * 3, [0.7]]
    prob = sais.Problem(insts)
    counts = np.array([128, 37, 200], np.int32)
    prob.set_instance_chains(counts)
    lam = _lam_dev(lams, prob.m_stride)
    a = prob.sample_run_best(lam, 256, 60, 10.0, 6, 0, variant="auto")
    torch.cuda.synchronize()
    prob.synchronize()
    run = {k: v.cpu().numpy() for k, v in a["run"].items()}
    for j, inst in enumerate(insts):
        ref = _ref(inst)
        J, hI, _ = ref.ising(np.asarray(lams[j], np.float32))
        _, tr = oracle.anneal(J, hI, 10.0, 60, 6 + j, 0, int(counts[j]), trace=True)
        cost, rx, sweep, nfeas = oracle.run_best(ref, tr)
        c = int(counts[j])
        assert np.array_equal(run["cost"][j, :c], cost), j
        assert np.array_equal(run["sweep"][j, :c], sweep), j
        assert np.array_equal(run["nfeas"][j, :c], nfeas), j
        assert np.array_equal(sais.unpack_bits(run["x"][j, :c], ref.nprime), rx), j
    prob.close()


def test_run_best_mkp_plain():
    """MKP N=80, m=5 (plain sampler, linear objective), tightened to 0.9 B."""
    insts = [_tighten(wl.mkp(80, 5, 2), 0.9)]
    assert _run_best_vs_oracle(insts, [[1.0] * 5], 64, 200, 10.0, 3, 1, "plain") > 0


def test_run_best_blocked_hilo_tightened():
    """Pair values up to 3000 (streamed hi/lo W), 2 constraints tightened to 0.8 B, at
    multipliers where every last state is infeasible but many runs pass a feasible state."""
    inst = wl.qkp(150, 0.25, 9, profit_max=3000)
    r = np.random.default_rng(1)
    inst.A = np.vstack([np.asarray(inst.A).reshape(1, -1), r.integers(1, 50, (1, inst.n))])
    inst.b = np.array([int(inst.b[0]), int(inst.A[1].sum() // 3)], np.int64)
    inst.m = 2
    _tighten(inst, 0.8)
    assert _run_best_vs_oracle([inst], [[150.0, 150.0]], 128, 120, 10.0, 5, 0, "blocked") > 20


@pytest.mark.parametrize("n", [500, 1010])
def test_run_best_large(n):
    """The block-field kernel (n = 500; n = 1010 with state chunks in shared memory), 128
    chains x 16 sweeps: the cost follows every flip and each sweep end is checked."""
    insts = [wl.qkp(n, 0.5, 11)]
    _run_best_vs_oracle(insts, [[1.0]], 128, 16, 10.0, 2, 0, "blocked")


@pytest.mark.parametrize("mode", ["persistent", "groups"])
def test_run_best_auto_ragged(mode):
    """SAIS_AUTO over a ragged batch (rank-k, block-field and plain work; one persistent launch
    or launch groups) equals the plain sampler's run-best outputs, and the plain sampler equals
    the oracle on two members."""
    insts = [wl.qkp(150, 0.5, 1), wl.qkp(520, 0.25, 2), _tighten(wl.mkp(90, 5, 3), 0.85),
             wl.qkp(60, 1.0, 4)]
    lams = [[0.5], [1.0], [1.0] * 5, [0.3]]
    prob = sais.Problem(insts)
    prob.set_auto_mode(mode)
    assert prob.plan(128, "auto")["kernel"] == ("persistent" if mode == "persistent"
                                                 else "launch groups")
    lam = _lam_dev(lams, prob.m_stride)
    a = prob.sample_run_best(lam, 128, 40, 10.0, 9, 1, variant="auto")
    b = prob.sample_run_best(lam, 128, 40, 10.0, 9, 1, variant="plain")
    torch.cuda.synchronize()
    prob.synchronize()
    for k in a["run"]:
        assert torch.equal(a["run"][k], b["run"][k]), k
    for k in ("x", "cost", "g", "feasible"):
        assert torch.equal(a[k], b[k]), k
    prob.close()
    _run_best_vs_oracle([insts[2], insts[3]], [lams[2], lams[3]], 128, 40, 10.0, 9, 1, "plain")


@pytest.mark.parametrize("variant,run_best", [("plain", True), ("plain", False),
                                              ("blocked", True)])
def test_solve_tightened_matches_oracle(variant, run_best):
    """Algorithm 1 on a tightened instance (B' = 0.85 B): multipliers, kept best (checked
    against B) and the stored-feasible count equal the oracle's solve."""
    inst = _tighten(wl.qkp(60, 0.5, 5), 0.85)
    prob = sais.Problem(inst)
    got = prob.solve(8, 64, 120, 10.0, 20.0, 4, variant=variant, run_best=run_best,
                     use_graph=variant == "blocked")
    prob.close()
    ref = _ref(inst)
    want = oracle.solve(ref, K=8, C=64, T=120, beta_max=10.0, eta=20.0, seed=4,
                        run_best=run_best)
    assert np.array_equal(got["lambda_trace"][:, 0, :ref.m], want.lambda_trace)
    assert got["feasible_count"][0] == want.feasible_count
    assert want.best_cost is not None
    assert got["best_cost"][0] == want.best_cost
    assert (got["best_iter"][0], got["best_chain"][0]) == (want.best_iter, want.best_chain)
    x = sais.unpack_bits(got["best_x"][0], ref.nprime)
    assert np.array_equal(x, want.best_x)
    A = np.asarray(inst.A, np.int64).reshape(inst.m, inst.n)
    assert (A @ x[:inst.n].astype(np.int64) <= np.asarray(inst.b)).all()


def test_tightening_rejects_bad_capacities():
    inst = wl.qkp(40, 0.5, 1)
    inst.b_tight = np.array([int(inst.b[0]) + 1], np.int64)
    with pytest.raises(sais.SaisError) as e:
        sais.Problem(inst)
    assert e.value.status == sais.SAIS_EINVAL
