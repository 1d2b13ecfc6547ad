"""GPU parity: the CUDA path through the C-ABI against the CPU oracle (needs an sm_103a GPU).

Bars (integer work bit-exact; decisions identical up to FP64 ties):
* returned states, their costs c(x), constraint values g(x) and feasibility are identical;
* teacher-forced sweep decisions agree on >= 99.99 % of updates, and any disagreement sits
  at a tie |tanh(beta I) + rho| < 1e-9;
* Algorithm 1 gives the same best objective, feasible count and multiplier trajectory on
  every seed of the N=100 QKP parity set;
* the multiplier step is bit-exact.
"""
import numpy as np
import pytest

import oracle
from paper_2501_04971_gb300 import sais, workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# Parity configuration: QKP N=100, d=0.25, 64 chains, beta 0 -> 10 over 1000 sweeps,
# 20 multiplier iterations, eta = 0.1, penalty 0.01 (in normalised units).
CFG0 = dict(chains=64, sweeps=1000, beta_max=10.0, iters=20, eta=0.1, penalty=0.01)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _ref(inst):
    return oracle.Problem(inst.n, inst.m, inst.W, inst.h, inst.A, inst.b, alpha=inst.alpha,
                          density=inst.density, penalty=getattr(inst, "penalty", 0.0) or 0.0)


def _lam_dev(lams, m_stride):
    a = np.zeros((len(lams), m_stride), np.float32)
    for j, l in enumerate(lams):
        a[j, :len(l)] = l
    return torch.tensor(a.reshape(-1), device="cuda:0")


def _check_outputs(ref, x, cost, g, feas, nchk=None):
    """Every returned state: cost, g and feasibility recomputed by the oracle in int64."""
    C = x.shape[0] if nchk is None else nchk
    for c in range(C):
        assert cost[c] == ref.cost(x[c]), c
        gg = ref.constraints(x[c])
        assert np.array_equal(g[c, :ref.m], gg), c
        assert np.all(g[c, ref.m:] == 0)
        assert bool(feas[c]) == ref.feasible(x[c]), c


def _sample_and_compare(insts, lams, C, T, beta_max, seed, it, variant="plain", chain_sel=None,
                        **kw):
    prob = sais.Problem(insts)
    out = prob.sample(_lam_dev(lams, prob.m_stride), C, T, beta_max, seed, it, variant=variant,
                      **kw)
    torch.cuda.synchronize()
    X = out["x"].cpu().numpy()
    cost, g, feas = (out[k].cpu().numpy() for k in ("cost", "g", "feasible"))
    for j, inst in enumerate(insts):
        ref = _ref(inst)
        assert prob.scalars[j].n_spins == ref.nprime
        x = sais.unpack_bits(X[j], ref.nprime)
        assert np.all(sais.unpack_bits(X[j], prob.words * 32)[:, ref.nprime:] == 0)
        J, hI, _ = ref.ising(np.asarray(lams[j], np.float32))
        sel = chain_sel or [(0, C)]
        for c0, nc in sel:
            want = oracle.anneal(J, hI, beta_max, T, seed + j, it, nc, chain0=c0)
            got = x[c0:c0 + nc]
            if not np.array_equal(got, want):
                bad = np.argwhere(got != want)
                raise AssertionError(f"instance {j}: {len(bad)} spins differ, first {bad[:5]}")
        _check_outputs(ref, x, cost[j], g[j], feas[j])
    prob.close()


def test_noise_stream_at_beta_zero():
    """With one sweep at beta = 0 every decision is the sign of the noise: the states expose
    the Philox stream (key seed + j, counter (i/4, t, c, k), word i%4) spin by spin."""
    insts = [wl.qkp(50, 0.5, 1), wl.mkp(61, 3, 2), wl.qkp(10, 1.0, 3)]
    lams = [[0.3], [0.1, 0.2, 0.0], [1.0]]
    _sample_and_compare(insts, lams, C=40, T=1, beta_max=0.0, seed=2**40 + 5, it=7)


def test_states_match_oracle_qkp_n100():
    inst = wl.qkp(100, 0.25, 0)
    _sample_and_compare([inst], [[0.5]], C=64, T=300, beta_max=10.0, seed=11, it=3)


@pytest.mark.parametrize("case", ["unconstrained", "mkp", "ragged_chains", "one_sweep",
                                  "mixed_batch", "table1_qkp", "negative_lambda", "big_profits",
                                  "max_constraints", "single_item", "one_chain", "beta_zero"])
def test_states_match_oracle_edge_cases(case):
    if case == "unconstrained":
        inst = wl.qkp(33, 0.5, 4)
        inst.m, inst.A, inst.b = 0, np.zeros((0, 33), np.int32), np.zeros(0, np.int64)
        _sample_and_compare([inst], [[]], C=32, T=50, beta_max=5.0, seed=1, it=0)
    elif case == "mkp":
        _sample_and_compare([wl.mkp(37, 3, 2)], [[0.2, 1.0, 0.0]], C=64, T=80, beta_max=50.0,
                            seed=3, it=1)
    elif case == "ragged_chains":
        _sample_and_compare([wl.qkp(45, 0.5, 5)], [[0.4]], C=37, T=60, beta_max=10.0, seed=4,
                            it=2)
    elif case == "one_sweep":
        _sample_and_compare([wl.qkp(70, 0.75, 6)], [[0.4]], C=64, T=1, beta_max=5.0, seed=5,
                            it=0)
    elif case == "mixed_batch":
        insts = [wl.qkp(45, 0.5, 7), wl.mkp(60, 4, 8), wl.qkp(100, 0.25, 9), wl.mkp(20, 1, 3)]
        lams = [[0.2], [0.5, 0.1, 0.0, 0.3], [2.0], [0.7]]
        _sample_and_compare(insts, lams, C=48, T=40, beta_max=10.0, seed=6, it=5)
    elif case == "table1_qkp":
        _sample_and_compare([wl.qkp(100, 0.5, 10)], [[3.5]], C=64, T=200, beta_max=10.0,
                            seed=7, it=9)
    elif case == "negative_lambda":
        _sample_and_compare([wl.mkp(40, 2, 11)], [[-0.5, 2.5]], C=32, T=60, beta_max=20.0,
                            seed=8, it=0)
    elif case == "big_profits":
        _sample_and_compare([wl.qkp(120, 0.5, 12, profit_max=10000)], [[1.5]], C=32, T=60,
                            beta_max=10.0, seed=9, it=0)
    elif case == "max_constraints":   # m = 32, the most the samplers keep in registers
        lam = list(np.linspace(0.0, 1.5, 32))
        _sample_and_compare([wl.mkp(50, 32, 13)], [lam], C=32, T=30, beta_max=10.0, seed=10,
                            it=1)
    elif case == "single_item":
        inst = wl.qkp(1, 1.0, 14)
        _sample_and_compare([inst], [[0.3]], C=32, T=20, beta_max=10.0, seed=11, it=0)
    elif case == "one_chain":
        _sample_and_compare([wl.qkp(80, 0.5, 15)], [[0.6]], C=1, T=100, beta_max=10.0, seed=12,
                            it=3)
    else:   # beta_max = 0: every sweep samples the uniform distribution
        _sample_and_compare([wl.qkp(60, 0.5, 16)], [[0.6]], C=64, T=5, beta_max=0.0, seed=13,
                            it=0)


def test_teacher_forced_decisions_config0():
    """Replay every recorded sweep of the parity configuration (QKP N=100, 64 chains, 1000
    sweeps) decision by decision in the oracle from the GPU's own states."""
    inst = wl.qkp(100, 0.25, 0)
    inst.penalty = CFG0["penalty"]
    ref = _ref(inst)
    lam = np.array([0.8], np.float32)
    C, T, seed, it = CFG0["chains"], CFG0["sweeps"], 77, 4
    prob = sais.Problem(inst)
    out = prob.sample(_lam_dev([lam], prob.m_stride), C, T, CFG0["beta_max"], seed, it,
                      trace=True)
    torch.cuda.synchronize()
    tr = sais.unpack_bits(out["trace"].cpu().numpy()[0], ref.nprime)   # C x T x N'
    J, hI, _ = ref.ising(lam)
    total, bad, worst = 0, 0, 0.0
    for c in range(C):
        prev = np.zeros(ref.nprime, np.uint8)
        for t in range(T):
            b = float(oracle.beta(CFG0["beta_max"], t, T))
            nb, _, margins = oracle.replay_sweep(J, hI, b, seed, it, c, t, prev, tr[c, t])
            total += ref.nprime
            bad += nb
            if nb:
                worst = max(worst, float(np.abs(margins).max()))
            prev = tr[c, t]
    agree = 1.0 - bad / total
    print(f"teacher-forced: {total} updates, {bad} disagreements, agreement {agree:.8f}")
    assert agree >= 0.9999
    assert worst < 1e-9
    prob.close()


def _solve_both(inst, seed, iters, chains, sweeps, beta_max, eta, project=True, **kw):
    prob = sais.Problem(inst)
    got = prob.solve(iters, chains, sweeps, beta_max, eta, seed, project=project, **kw)
    prob.close()
    ref = _ref(inst)
    want = oracle.solve(ref, K=iters, C=chains, T=sweeps, beta_max=beta_max, eta=eta,
                        seed=seed, project=project)
    return ref, got, want


def _assert_solve_equal(ref, got, want, tag=""):
    assert np.array_equal(got["lambda_trace"][:, 0, :ref.m], want.lambda_trace), tag
    assert got["feasible_count"][0] == want.feasible_count, tag
    if want.best_cost is None:
        assert got["best_cost"][0] == np.iinfo(np.int64).max, tag
        assert got["best_iter"][0] == -1, tag
    else:
        assert got["best_cost"][0] == want.best_cost, tag
        assert got["best_iter"][0] == want.best_iter and got["best_chain"][0] == want.best_chain
        x = sais.unpack_bits(got["best_x"][0], ref.nprime)
        assert np.array_equal(x, want.best_x), tag


@pytest.mark.parametrize("iseed", range(10))
def test_config0_best_found_every_seed(iseed):
    """Algorithm 1 on the parity set: instance seeds 0-9 x sampler seeds 0-7."""
    inst = wl.qkp(100, 0.25, iseed)
    inst.penalty = CFG0["penalty"]
    for s in range(8):
        ref, got, want = _solve_both(inst, s, CFG0["iters"], CFG0["chains"], CFG0["sweeps"],
                                     CFG0["beta_max"], CFG0["eta"])
        _assert_solve_equal(ref, got, want, f"instance {iseed} seed {s}")


def test_table1_qkp_solve_parity_and_graph():
    """Table I parameters (P = 2dN, eta = 20, beta_max = 10) on a QKP N=100, d=0.5; the
    captured-graph loop gives the same result as the stream loop."""
    inst = wl.qkp(100, 0.5, 3)
    ref, got, want = _solve_both(inst, 5, 12, 32, 300, 10.0, 20.0)
    _assert_solve_equal(ref, got, want, "table1")
    prob = sais.Problem(inst)
    g2 = prob.solve(12, 32, 300, 10.0, 20.0, 5, use_graph=True)
    prob.close()
    for k in ("best_cost", "best_x", "best_iter", "best_chain", "feasible_count",
              "lambda_trace", "lambda_final"):
        assert np.array_equal(got[k], g2[k]), k


def test_solve_resumes_bit_exactly():
    inst = wl.mkp(60, 3, 4)
    prob = sais.Problem(inst)
    full = prob.solve(10, 32, 100, 50.0, 2.5, 9)
    a = prob.solve(5, 32, 100, 50.0, 2.5, 9)
    b = prob.solve(5, 32, 100, 50.0, 2.5, 9, iter0=5, lambda0=a["lambda_final"])
    prob.close()
    assert np.array_equal(full["lambda_trace"], np.concatenate([a["lambda_trace"],
                                                                b["lambda_trace"]]))
    assert full["feasible_count"][0] == a["feasible_count"][0] + b["feasible_count"][0]


def test_update_lambda_bit_exact():
    insts = [wl.qkp(30, 0.5, 1), wl.mkp(40, 5, 2), wl.mkp(25, 3, 3)]
    prob = sais.Problem(insts)
    r = np.random.default_rng(0)
    C = 50
    for eta, project in ((0.1, True), (20.0, True), (0.05, False), (3.0, False)):
        g = r.integers(-40000, 40000, size=(len(insts), C, prob.m_stride)).astype(np.int64)
        lam0 = r.normal(0, 1, size=(len(insts), prob.m_stride)).astype(np.float32)
        d_g = torch.tensor(g.reshape(-1), device="cuda:0")
        d_l = torch.tensor(lam0.reshape(-1), device="cuda:0")
        prob.update_lambda(d_g, C, eta, project, d_l)
        got = d_l.cpu().numpy().reshape(len(insts), prob.m_stride)
        for j, inst in enumerate(insts):
            ref = _ref(inst)
            want = oracle.lambda_update(g[j, :, :inst.m].sum(axis=0), C, eta, project,
                                        ref.sigma_g, lam0[j, :inst.m])
            assert np.array_equal(got[j, :inst.m], want), (eta, project, j)
            assert np.array_equal(got[j, inst.m:], lam0[j, inst.m:])
    prob.close()


def test_mkp_full_size_sampled_chains():
    """MKP N=250, m=5 at its full launch (1024 chains, 2000 sweeps): states of sampled chains
    against the oracle, cost/constraints/feasibility of every chain."""
    inst = wl.mkp(250, 5, 0)
    _sample_and_compare([inst], [[0.3, 0.1, 0.6, 0.0, 0.2]], C=1024, T=2000, beta_max=50.0,
                        seed=21, it=3, chain_sel=[(0, 4), (509, 3), (1020, 4)])


def test_qkp300_full_size_sampled_chains():
    """QKP N=300 at the four densities, 128 chains x 1000 sweeps: sampled chains' states
    against the oracle, every chain's outputs recomputed."""
    insts = [wl.qkp(300, d, s) for d in (0.25, 0.5, 0.75, 1.0) for s in range(2)]
    lams = [[1.0 + 0.3 * j] for j in range(len(insts))]
    _sample_and_compare(insts, lams, C=128, T=1000, beta_max=10.0, seed=31, it=0,
                        chain_sel=[(0, 2), (127, 1)])
