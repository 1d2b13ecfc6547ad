"""Blocked samplers (tcgen05) against the plain sampler and the oracle.

Two kernels: rank-k updates of fields resident in TMEM (N'_pad + K <= 512), and block fields
from a GEMM over the chain states (up to n = 1024 items, the states past 496 TMEM columns in
shared memory; and K = 32 streamed or hi/lo, K = 64).  Both are exact (integer products and
sums below 2^24 in FP32), so every blocked sampler must make every decision the plain sampler
makes: identical states after every sweep, identical costs, constraint values and feasibility,
and all identical to the CPU oracle.
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


def _lam(prob, lams):
    a = np.zeros((prob.count, prob.m_stride), np.float32)
    for j, l in enumerate(lams):
        a[j, :len(l)] = l
    return torch.tensor(a.reshape(-1), device="cuda:0")


def _run(prob, lam, C, T, beta, seed, it, variant, block_k=0, trace=False):
    out = prob.sample(lam, C, T, beta, seed, it, variant=variant, block_k=block_k, trace=trace)
    prob.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _compare(insts, lams, C, T, beta, seed, it, block_k, trace=False, oracle_chains=None):
    prob = sais.Problem(insts)
    lam = _lam(prob, lams)
    p = _run(prob, lam, C, T, beta, seed, it, "plain", trace=trace)
    b = _run(prob, lam, C, T, beta, seed, it, "blocked", block_k=block_k, trace=trace)
    for k in p:
        if not np.array_equal(p[k], b[k]):
            diff = np.argwhere(p[k] != b[k])
            raise AssertionError(f"{k}: blocked differs from plain at {len(diff)} places, "
                                 f"first {diff[:4].tolist()}")
    for j, inst in enumerate(insts):
        ref = oracle.Problem(inst.n, inst.m, inst.W, inst.h, inst.A, inst.b, alpha=inst.alpha,
                             density=inst.density)
        J, hI, _ = ref.ising(np.asarray(lams[j], np.float32))
        c0, nc = oracle_chains or (0, C)
        want = oracle.anneal(J, hI, beta, T, seed + j, it, nc, chain0=c0)
        got = sais.unpack_bits(b["x"][j], ref.nprime)[c0:c0 + nc]
        assert np.array_equal(got, want), f"instance {j}: blocked states differ from the oracle"
        x = sais.unpack_bits(b["x"][j], ref.nprime)
        for c in range(0, C, max(1, C // 16)):
            assert b["cost"][j, c] == ref.cost(x[c])
            assert np.array_equal(b["g"][j, c, :ref.m], ref.constraints(x[c]))
            assert bool(b["feasible"][j, c]) == ref.feasible(x[c])
    prob.close()


@pytest.mark.parametrize("block_k", [16, 32, 64])
def test_blocked_equals_plain_qkp_n100(block_k):
    _compare([wl.qkp(100, 0.25, 0)], [[0.5]], C=128, T=200, beta=10.0, seed=3, it=1,
             block_k=block_k)


@pytest.mark.parametrize("block_k", [32, 64])
def test_blocked_fewer_chains_than_lanes(block_k):
    _compare([wl.qkp(100, 0.25, 1)], [[0.9]], C=64, T=150, beta=10.0, seed=4, it=0,
             block_k=block_k)


@pytest.mark.parametrize("block_k", [16, 32, 64])
def test_blocked_ragged_chain_groups_and_spins(block_k):
    """200 chains (two CTAs, the second ragged) on an instance whose N' is not a multiple of
    the block size, and whose items end inside a block of 32 or 64 (n = 45: 48 state
    columns)."""
    inst = wl.qkp(45, 0.5, 5)
    _compare([inst], [[0.4]], C=200, T=120, beta=10.0, seed=5, it=2, block_k=block_k)


@pytest.mark.parametrize("block_k", [32, 64])
def test_blocked_wide_blocks_full_size_and_two_constraints(block_k):
    """K = 32 and 64 at QKP N=300 over 1000 sweeps, and with two constraints."""
    insts = [wl.qkp(300, 0.5, 60), _with_constraints(wl.qkp(300, 0.75, 61), 2, 61)]
    _compare(insts, [[1.0], [0.4, 0.9]], C=128, T=1000, beta=10.0, seed=25, it=0,
             block_k=block_k, oracle_chains=(0, 2))


def test_blocked_mixed_batch_sizes():
    """Instances of different N' (N'_pad 64 .. 320) in one launch."""
    insts = [wl.qkp(50, 0.5, 6), wl.qkp(120, 0.75, 7), wl.qkp(300, 0.25, 8), wl.qkp(200, 1.0, 9)]
    _compare(insts, [[0.3], [1.1], [2.0], [0.0]], C=128, T=100, beta=10.0, seed=6, it=4,
             block_k=16, oracle_chains=(0, 8))


def test_blocked_trace_every_sweep_equals_plain():
    _compare([wl.qkp(80, 0.5, 10)], [[0.6]], C=128, T=60, beta=10.0, seed=7, it=3, block_k=32,
             trace=True)


def test_blocked_full_size_qkp300():
    """QKP N=300 at the four densities, 128 chains, 1000 sweeps: blocked == plain everywhere,
    sampled chains against the oracle."""
    insts = [wl.qkp(300, d, s) for d in (0.25, 0.5, 0.75, 1.0) for s in range(2)]
    lams = [[0.5 + 0.4 * j] for j in range(len(insts))]
    _compare(insts, lams, C=128, T=1000, beta=10.0, seed=8, it=0, block_k=16,
             oracle_chains=(0, 2))


def test_blocked_solve_equals_plain_solve():
    inst = wl.qkp(100, 0.5, 11)
    prob = sais.Problem(inst)
    a = prob.solve(6, 128, 200, 10.0, 20.0, 13, variant="plain")
    b = prob.solve(6, 128, 200, 10.0, 20.0, 13, variant="blocked", use_graph=True)
    prob.close()
    for k in ("best_cost", "best_x", "best_iter", "best_chain", "feasible_count",
              "lambda_trace", "lambda_final"):
        assert np.array_equal(a[k], b[k]), k


def test_blocked_timeout_path_reports_and_recovers():
    """A wait bound of one poll makes the decision warps give up: the kernel records
    SAIS_ETIMEOUT, drains its copies and MMAs, frees TMEM and exits; the context stays usable
    and the next launch is correct."""
    inst = wl.qkp(60, 0.5, 12)
    prob = sais.Problem(inst)
    lam = _lam(prob, [[0.5]])
    prob.sample(lam, 128, 50, 10.0, 1, 0, variant="blocked", debug_wait_polls=1)
    with pytest.raises(sais.SaisError) as e:
        prob.synchronize()
    assert e.value.status == sais.SAIS_ETIMEOUT
    prob.synchronize()  # status word was reset
    p = _run(prob, lam, 128, 50, 10.0, 1, 0, "plain")
    b = _run(prob, lam, 128, 50, 10.0, 1, 0, "blocked")
    assert np.array_equal(p["x"], b["x"])
    prob.close()


@pytest.mark.parametrize("block_k", [32, 64])
def test_blocked_wide_blocks_hilo(block_k):
    """K = 32 and 64 with the BF16 hi/lo split (pair values up to 10^4)."""
    _compare([wl.qkp(200, 0.5, 62, profit_max=10000), wl.qkp(90, 0.25, 63)], [[3.0], [0.5]],
             C=128, T=80, beta=10.0, seed=26, it=1, block_k=block_k, oracle_chains=(0, 2))


@pytest.mark.parametrize("case", ["hilo_n100", "hilo_n300", "stream_n400", "hilo_stream_mixed"])
def test_blocked_streamed_and_hilo(case):
    """W streamed through the shared-memory tile ring, and the BF16 hi/lo split for pair
    values above 256 (profits up to 10^4): still identical to the plain sampler and the oracle."""
    if case == "hilo_n100":
        _compare([wl.qkp(100, 0.5, 21, profit_max=10000)], [[0.7]], C=128, T=150, beta=10.0,
                 seed=9, it=1, block_k=16)
    elif case == "hilo_n300":
        _compare([wl.qkp(300, 0.75, 22, profit_max=10000)], [[1.5]], C=128, T=200, beta=10.0,
                 seed=10, it=0, block_k=16, oracle_chains=(0, 2))
    elif case == "stream_n400":
        _compare([wl.qkp(400, 0.5, 23)], [[2.0]], C=128, T=120, beta=10.0, seed=11, it=2,
                 block_k=16, oracle_chains=(0, 2))
    else:
        insts = [wl.qkp(150, 0.5, 24), wl.qkp(420, 0.25, 25, profit_max=5000),
                 wl.qkp(60, 1.0, 26, profit_max=300)]
        _compare(insts, [[0.2], [3.0], [0.9]], C=160, T=80, beta=10.0, seed=12, it=3,
                 block_k=16, oracle_chains=(0, 3))


@pytest.mark.parametrize("case", ["n500", "n1000_hilo", "mixed_ragged", "n640_trace", "n1020",
                                  "n990_tail", "n1000_mixed", "n700_default_k"])
def test_large_instances_equal_plain_and_oracle(case):
    """Large instances on the block-field kernel (one CTA per SM): up to n = 992 items (960 with
    the hi/lo split, whose accumulator takes 2K columns) the state columns fit TMEM beside the
    fields; beyond, the last 16-spin chunks live in shared memory as the MMA's A operand
    (n1000_hilo, n1020, n1000_mixed).  All identical to the plain sampler and the oracle."""
    if case == "n500":
        _compare([wl.qkp(500, 0.5, 31)], [[1.0]], C=128, T=60, beta=10.0, seed=13, it=1,
                 block_k=16, oracle_chains=(0, 2))
    elif case == "n1000_hilo":
        _compare([wl.qkp(1000, 0.25, 32, profit_max=10000)], [[2.0]], C=128, T=24, beta=10.0,
                 seed=14, it=0, block_k=16, oracle_chains=(0, 1))
    elif case == "mixed_ragged":
        insts = [wl.qkp(700, 0.5, 33), wl.qkp(200, 0.75, 34), wl.qkp(960, 1.0, 35)]
        _compare(insts, [[0.5], [1.5], [3.0]], C=160, T=30, beta=10.0, seed=15, it=2,
                 block_k=16, oracle_chains=(0, 1))
    elif case == "n640_trace":
        _compare([wl.qkp(640, 0.5, 36)], [[0.8]], C=128, T=20, beta=10.0, seed=16, it=3,
                 block_k=16, trace=True, oracle_chains=(0, 1))
    elif case == "n1020":   # two state chunks in shared memory
        _compare([wl.qkp(1020, 0.5, 38)], [[1.2]], C=128, T=12, beta=10.0, seed=17, it=0,
                 block_k=16, oracle_chains=(0, 1))
    elif case == "n990_tail":   # n = 990: 496 state columns and 16 fields, all of TMEM
        _compare([wl.qkp(990, 0.75, 39), wl.qkp(250, 0.5, 40)], [[0.6], [1.0]], C=128, T=12,
                 beta=10.0, seed=18, it=1, block_k=16, oracle_chains=(0, 1))
    elif case == "n1000_mixed":   # a batch whose largest instance needs state chunks in SMEM
        _compare([wl.qkp(1000, 0.5, 44), wl.qkp(200, 0.5, 45)], [[1.0], [0.7]], C=128, T=12,
                 beta=10.0, seed=27, it=2, block_k=16, oracle_chains=(0, 1))
    else:                   # the library's block size (K = 32 for the block-field kernel)
        _compare([wl.qkp(700, 0.5, 46), wl.qkp(460, 0.25, 47)], [[0.9], [0.4]], C=160, T=20,
                 beta=10.0, seed=28, it=0, block_k=0, oracle_chains=(0, 1))


@pytest.mark.parametrize("n", [600, 1000])
def test_large_timeout_path_reports_and_recovers(n):
    """The timeout path of the block-field kernel, states in TMEM (n = 600) and partly in
    shared memory (n = 1000)."""
    inst = wl.qkp(n, 0.5, 37)
    prob = sais.Problem(inst)
    lam = _lam(prob, [[0.5]])
    prob.sample(lam, 128, 10, 10.0, 1, 0, variant="blocked", debug_wait_polls=1)
    with pytest.raises(sais.SaisError) as e:
        prob.synchronize()
    assert e.value.status == sais.SAIS_ETIMEOUT
    prob.synchronize()
    p = _run(prob, lam, 128, 10, 10.0, 1, 0, "plain")
    b = _run(prob, lam, 128, 10, 10.0, 1, 0, "blocked")
    assert np.array_equal(p["x"], b["x"]) and np.array_equal(p["cost"], b["cost"])
    prob.close()


def _with_constraints(inst, m, seed):
    """The QKP objective of `inst` with m random knapsack constraints instead of one."""
    import dataclasses
    r = np.random.default_rng(seed)
    A = r.integers(0, 50, (m, inst.n)).astype(np.int32)
    b = np.maximum(1, (A.sum(axis=1) // 3)).astype(np.int64)
    return dataclasses.replace(inst, m=m, A=A, b=b)


@pytest.mark.parametrize("case", ["unconstrained", "m8", "m3_streamed"])
def test_blocked_constraint_counts(case):
    """Blocked sampler at its constraint extremes: no constraint (m = 0) and m = 8 (its limit),
    resident and streamed W."""
    if case == "unconstrained":
        inst = wl.qkp(90, 0.5, 41)
        import dataclasses
        inst = dataclasses.replace(inst, m=0, A=np.zeros((0, 90), np.int32),
                                   b=np.zeros(0, np.int64))
        _compare([inst], [[]], C=128, T=60, beta=10.0, seed=19, it=0, block_k=16)
    elif case == "m8":
        inst = _with_constraints(wl.qkp(120, 0.5, 42), 8, 42)
        _compare([inst], [list(np.linspace(0.1, 2.0, 8))], C=128, T=60, beta=10.0, seed=20,
                 it=1, block_k=16)
    else:
        inst = _with_constraints(wl.qkp(380, 0.5, 43), 3, 43)
        _compare([inst], [[0.5, 1.0, 1.5]], C=128, T=30, beta=10.0, seed=21, it=2, block_k=16,
                 oracle_chains=(0, 2))


@pytest.mark.parametrize("n", [520, 1000])
@pytest.mark.parametrize("case", ["one_chain", "m8", "three_clusters"])
def test_large_instance_extremes(case, n):
    """The block-field kernel at n = 520 and n = 1000 (state chunks in shared memory), each with
    a single valid chain, with 8 constraints, and with 300 chains (three CTAs per instance, the
    last one ragged)."""
    if case == "one_chain":
        _compare([wl.qkp(n, 0.5, 51)], [[1.0]], C=1, T=20, beta=10.0, seed=22, it=0,
                 block_k=16)
    elif case == "m8":
        inst = _with_constraints(wl.qkp(n, 0.5, 52), 8, 52)
        _compare([inst], [list(np.linspace(0.2, 1.6, 8))], C=128, T=16, beta=10.0, seed=23,
                 it=1, block_k=16, oracle_chains=(0, 1))
    else:
        _compare([wl.qkp(n, 0.75, 53)], [[0.9]], C=300, T=16, beta=10.0, seed=24, it=2,
                 block_k=16, oracle_chains=(290, 2))


def test_blocked_unsupported_cases():
    cases = ([([wl.mkp(40, 3, 1)], 16), ([wl.qkp(1100, 0.25, 2)], 16),
              ([wl.qkp(1030, 0.5, 3), wl.qkp(40, 0.5, 4)], 16),
              ([_with_constraints(wl.qkp(100, 0.5, 5), 3, 5)], 64),
              ([wl.qkp(1000, 0.5, 6)], 64)])
    for insts, k in cases:
        prob = sais.Problem(insts)
        lam = torch.zeros(prob.count * prob.m_stride, device="cuda:0")
        with pytest.raises(sais.SaisError) as e:
            prob.sample(lam, 128, 10, 10.0, 1, 0, variant="blocked", block_k=k)
        assert e.value.status == sais.SAIS_EUNSUPPORTED
        prob.close()
