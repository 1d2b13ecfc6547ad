"""Pins of the CPU oracle against things other than itself (CPU only).

Each test ties one part of the oracle to the paper's printed numbers, a closed form, an
invariant, brute force on tiny inputs, or an independent library routine, so that a plausible
mistake (a dropped term, a wrong sign, a wrong index) fails at least one of them.
``test_oracle_mutants.py`` plants such mistakes and checks that they are caught.
"""
import ctypes
import ctypes.util
import math
import os

import numpy as np
import pytest

import oracle
from paper_2501_04971_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, *v = line.split()
            vals[k] = v if len(v) > 1 else v[0]
    return vals


def _problem(inst, **kw):
    args = dict(alpha=inst.alpha, density=inst.density)
    args.update(kw)
    return oracle.Problem(inst.n, inst.m, inst.W, inst.h, inst.A, inst.b, **args)


def _tiny_qkp(n=5, b=7, seed=3, dens=0.6, wmax=4, pmax=9):
    r = np.random.default_rng(seed)
    p = np.triu(np.where(r.random((n, n)) < dens, r.integers(1, pmax + 1, (n, n)), 0))
    W = p + p.T
    np.fill_diagonal(W, 0)
    h = np.diag(p).copy()
    A = r.integers(1, wmax + 1, (1, n))
    return W, h, A, np.array([b])


# --------------------------------------------------------------------------------------
# Slack encoding and problem scalars (Sec. III-A, Sec. IV-A/B, Table I)
# --------------------------------------------------------------------------------------

def test_slack_bits_closed_form():
    """Q = floor(log2 b) + 1 (Sec. IV-A): 2^(Q-1) <= b < 2^Q, checked in exact integers."""
    lib = oracle.load()
    r = np.random.default_rng(0)
    bs = list(range(1, 5000)) + [int(v) for v in r.integers(1, 2**62, 2000)]
    bs += [2**k for k in range(62)] + [2**k - 1 for k in range(1, 62)]
    for b in bs:
        q = lib.or_slack_bits(b)
        assert 2 ** (q - 1) <= b < 2 ** q, (b, q)


def test_paper_qkp_300_50_8_penalty():
    """P = 2dN = 313 for a 300-item, d = 0.5 instance (Sec. IV-A): N counts 13 slack spins."""
    g = _golden("paper_qkp_300_50_8.txt")
    n, d, alpha = int(g["n"]), float(g["density"]), float(g["alpha"])
    for b in (int(g["b_min"]), 6000, int(g["b_max"])):
        inst = wl.qkp(n, d, 8)
        inst.b = np.array([b])
        p = _problem(inst, alpha=alpha, density=d)
        assert p.nprime == int(g["nprime"])
        assert int(p.Q[0]) == int(g["Q"])
        assert float(p.P) == float(g["P"])
    inst = wl.qkp(n, d, 8)
    inst.b = np.array([int(g["b_max"]) + 1])
    assert _problem(inst, alpha=alpha, density=d).nprime == int(g["nprime"]) + 1


def test_paper_mkp_penalty_about_10():
    """MKP, 250 items, 5 knapsacks: P = 5 d N with d = 2/(N+1) is the P = 10 of Fig. 5."""
    g = _golden("paper_mkp_250_5_penalty.txt")
    inst = wl.mkp(int(g["n"]), int(g["m"]), 0)
    p = _problem(inst, alpha=float(g["alpha"]), density=-1.0)
    assert abs(float(p.P) - float(g["P"])) <= float(g["rel_tol"]) * float(g["P"])
    # exact closed form 10 N'/(N'+1) rounded once to FP32
    assert float(p.P) == float(np.float32(5.0 * (2.0 / (p.nprime + 1.0)) * p.nprime))


def test_table1_parameters_golden():
    """Table I as transcribed: QKP alpha=2, beta_max=10, eta=20; MKP alpha=5, 50, 0.05."""
    rows = {}
    with open(os.path.join(GOLDEN, "table1_parameters.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, *v = line.split()
                rows[k] = [float(x) for x in v]
    assert rows["QKP"] == [2, 1000, 2000, 10, 20]
    assert rows["MKP"] == [5, 1000, 5000, 50, 0.05]
    assert wl.qkp(10, 0.5, 0).alpha == rows["QKP"][0] and wl.mkp(10, 2, 0).alpha == rows["MKP"][0]


def test_normalisation_scales():
    """sigma_f = 1/max(|W|,|h|), sigma_g = 1/max(|A|,|b|) (Sec. IV-A), rounded once to FP32."""
    W, h, A, b = _tiny_qkp()
    W[0, 1] = W[1, 0] = 37
    p = oracle.Problem(5, 1, W, h, A, b, alpha=2.0, density=0.5)
    assert p.sigma_f == np.float32(1.0 / 37.0)
    assert p.sigma_g == np.float32(1.0 / max(A.max(), 7))
    assert p.P == np.float32(2.0 * 0.5 * p.nprime)
    p2 = oracle.Problem(5, 1, W, h, A, b, alpha=2.0, density=0.5, penalty=3.25)
    assert p2.P == np.float32(3.25)


def test_slack_extension_reaches_equality():
    """For every feasible x the slack bits can absorb b - A x exactly: A_ext [x; bits] = b.
    For an infeasible x no slack setting reaches g = 0 (slack spins are non-negative)."""
    inst = wl.mkp(12, 3, 5, a_max=20)
    p = _problem(inst)
    r = np.random.default_rng(1)
    n = inst.n
    offs = n + np.concatenate([[0], np.cumsum(p.Q)[:-1]])
    for _ in range(300):
        x = np.zeros(p.nprime, dtype=np.uint8)
        x[:n] = r.random(n) < 0.3
        load = inst.A.astype(np.int64) @ x[:n]
        feas = bool(np.all(load <= inst.b))
        assert p.feasible(x) == feas
        if feas:
            for k in range(inst.m):
                s = int(inst.b[k] - load[k])
                for q in range(int(p.Q[k])):
                    x[offs[k] + q] = (s >> q) & 1
            assert np.all(p.constraints(x) == 0)
            assert p.feasible(x)  # slack bits never change feasibility
        else:
            # the items alone already exceed some capacity: g_k > 0 whatever the slack bits
            k = int(np.argmax(load - inst.b))
            assert p.constraints(x)[k] > 0


def test_cost_closed_forms():
    """c(x) = -x^T W x/2 - h^T x (Eq. 12): single items give -h_i, pairs add -W_ij."""
    inst = wl.qkp(30, 0.5, 2)
    p = _problem(inst)
    h, W = inst.h.astype(np.int64), inst.W.astype(np.int64)
    x = np.zeros(p.nprime, dtype=np.uint8)
    assert p.cost(x) == 0
    for i in range(inst.n):
        x[:] = 0
        x[i] = 1
        assert p.cost(x) == -h[i]
        for j in range(i + 1, inst.n, 7):
            x[j] = 1
            assert p.cost(x) == -h[i] - h[j] - W[i, j]
            x[j] = 0
    x[:] = 0
    x[:inst.n] = 1  # all items: every pair once
    assert p.cost(x) == -h.sum() - np.triu(W, 1).sum()
    # slack spins carry no profit
    x[:] = 0
    x[inst.n:] = 1
    assert p.cost(x) == 0


# --------------------------------------------------------------------------------------
# Ising form: energy identity and flip identity (Eq. 1, 5, 9)
# --------------------------------------------------------------------------------------

def _all_states(N):
    s = np.arange(1 << N, dtype=np.int64)
    return ((s[:, None] >> np.arange(N)) & 1).astype(np.uint8)


@pytest.mark.parametrize("kind", ["qkp", "mkp"])
def test_energy_identity_exhaustive(kind):
    """L(x) - H(2x-1) is the same constant for every state (Eq. 1 vs Eq. 5), N' <= 12."""
    if kind == "qkp":
        W, h, A, b = _tiny_qkp(n=6, b=11, seed=7)
        p = oracle.Problem(6, 1, W, h, A, b, alpha=2.0, density=0.5)
        lam = np.array([0.7], dtype=np.float32)
    else:
        inst = wl.mkp(5, 2, 3, a_max=6)
        p = _problem(inst)
        lam = np.array([0.4, -0.3], dtype=np.float32)
    assert p.nprime <= 12
    J, hI, cst = p.ising(lam)
    assert np.allclose(J, J.T, rtol=0, atol=0) and np.all(np.diag(J) == 0)
    L = p.enumerate_lagrangian(lam)
    X = _all_states(p.nprime)
    H = np.array([oracle.ising_energy(J, hI, x) for x in X])
    scale = np.abs(L).max() + 1.0
    assert np.max(np.abs((L - H) - cst)) <= 1e-12 * scale


def test_flip_identity_random_states():
    """L(x|x_i=1) - L(x|x_i=0) = -2 I_i with I_i = sum_j J_ij m_j + h_i (Eq. 9-11), N' = 112."""
    inst = wl.qkp(100, 0.25, 4)
    p = _problem(inst, penalty=0.8)
    r = np.random.default_rng(5)
    lam = np.array([1.3], dtype=np.float32)
    J, hI, _ = p.ising(lam)
    for _ in range(5):
        x = (r.random(p.nprime) < 0.4).astype(np.uint8)
        m = 2.0 * x - 1.0
        I = J @ m + hI
        for i in range(0, p.nprime, 3):
            x1 = x.copy(); x1[i] = 1
            x0 = x.copy(); x0[i] = 0
            dL = p.lagrangian(x1, lam) - p.lagrangian(x0, lam)
            assert abs(dL + 2.0 * I[i]) <= 1e-11 * (1.0 + abs(dL)), (i, dL, I[i])


# --------------------------------------------------------------------------------------
# Boltzmann law of the p-bit machine (Eq. 11)
# --------------------------------------------------------------------------------------

def _tv_setup():
    W, h, A, b = _tiny_qkp(n=5, b=6, seed=11, wmax=3, pmax=6)
    p = oracle.Problem(5, 1, W, h, A, b, alpha=2.0, density=0.5, penalty=0.9)
    lam = np.array([0.35], dtype=np.float32)
    return p, lam


@pytest.mark.slow
def test_boltzmann_total_variation():
    """Final states of 10^6 independent chains (60 sweeps at fixed beta) follow
    exp(-beta L)/Z (Eq. 11) with total-variation distance < 0.01.  The expected TV of an
    exact sampler, sum_x sqrt(p_x (1-p_x) / (2 pi n)), is printed beside it."""
    p, lam = _tv_setup()
    beta = np.float32(2.5)
    J, hI, _ = p.ising(lam)
    L = p.enumerate_lagrangian(lam)
    w = np.exp(-float(beta) * (L - L.min()))
    prob = w / w.sum()
    nsamp = 1_000_000
    states = oracle.gibbs_fixed(J, hI, float(beta), 60, seed=1234, nchains=nsamp)
    freq = np.bincount(states, minlength=len(prob)) / nsamp
    tv = 0.5 * np.abs(freq - prob).sum()
    floor = np.sum(np.sqrt(prob * (1 - prob) / (2 * np.pi * nsamp)))
    print(f"N'={p.nprime} states={len(prob)} TV={tv:.5f} noise floor={floor:.5f}")
    assert floor < 0.006, "test has too little power: distribution too flat"
    assert tv < 0.01
    assert tv < 3.0 * floor


def test_beta_zero_is_uniform():
    """At beta = 0, tanh(0) = 0 and each spin is set by the sign of the noise: every state is
    equally likely, each marginal exactly 1/2 in law."""
    p, lam = _tv_setup()
    J, hI, _ = p.ising(lam)
    nsamp = 200_000
    states = oracle.gibbs_fixed(J, hI, 0.0, 1, seed=99, nchains=nsamp)
    bits = ((states[:, None] >> np.arange(p.nprime)) & 1).astype(np.float64)
    marg = bits.mean(axis=0)
    assert np.all(np.abs(marg - 0.5) < 5 * 0.5 / math.sqrt(nsamp))
    counts = np.bincount(states, minlength=1 << p.nprime)
    e = nsamp / len(counts)
    chi2 = ((counts - e) ** 2 / e).sum()
    dof = len(counts) - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof)


def test_large_beta_finds_ground_state():
    """At large beta the most frequent final state is the argmin of L (brute force)."""
    p, lam = _tv_setup()
    J, hI, _ = p.ising(lam)
    L = p.enumerate_lagrangian(lam)
    states = oracle.gibbs_fixed(J, hI, 40.0, 200, seed=7, nchains=4000)
    mode = np.bincount(states, minlength=len(L)).argmax()
    assert mode == int(np.argmin(L))


def test_infinite_beta_is_greedy_descent():
    """At beta -> infinity each update sets m_i = sign(I_i): after a sweep with no change the
    state is a local minimum of L under single flips."""
    inst = wl.qkp(40, 0.5, 9)
    p = _problem(inst, penalty=1.0)
    lam = np.array([0.2], dtype=np.float32)
    J, hI, _ = p.ising(lam)
    x = oracle.anneal(J, hI, 1e30, 40, seed=3, it=0, nchains=4)
    for c in range(4):
        L0 = p.lagrangian(x[c], lam)
        for i in range(p.nprime):
            y = x[c].copy(); y[i] ^= 1
            assert p.lagrangian(y, lam) >= L0 - 1e-12


# --------------------------------------------------------------------------------------
# Teacher-forced replay of recorded sweeps (Eq. 10, Sec. III-B)
# --------------------------------------------------------------------------------------

def _replay_setup():
    inst = wl.qkp(24, 0.5, 6)
    p = _problem(inst, penalty=0.7)
    lam = np.array([0.45], dtype=np.float32)
    J, hI, _ = p.ising(lam)
    return p, lam, J, hI


def test_replay_sweep_reproduces_the_oracles_own_trace():
    """Replaying every recorded sweep of the oracle's own annealing runs from the recorded start
    state gives no disagreement; changing one recorded decision (the sweep's last spin, so no
    later decision depends on it) gives exactly one, at that spin, with the oracle's margin on
    the side of the original bit."""
    p, lam, J, hI = _replay_setup()
    T, C, seed, it, bmax = 40, 3, 21, 2, 6.0
    _, tr = oracle.anneal(J, hI, bmax, T, seed=seed, it=it, nchains=C, trace=True)
    N = p.nprime
    last = N - 1
    for c in range(C):
        for t in range(T):
            x0 = tr[c, t - 1] if t > 0 else np.zeros(N, np.uint8)
            b = float(oracle.beta(bmax, t, T))
            nbad, _, _ = oracle.replay_sweep(J, hI, b, seed, it, c, t, x0, tr[c, t])
            assert nbad == 0, (c, t)
            if t % 7 == 3:
                x1 = tr[c, t].copy()
                x1[last] ^= 1
                nbad, spins, margins = oracle.replay_sweep(J, hI, b, seed, it, c, t, x0, x1)
                assert nbad == 1 and spins[0] == last, (c, t, nbad, spins)
                assert (margins[0] > 0) == bool(tr[c, t, last]), (c, t, margins)


def test_replay_sweep_margins_from_the_lagrangian():
    """For an arbitrary recorded path x1 (random bits, so nearly every spin disagrees), the
    replay reports exactly the spins where Eq. 10 on the current state differs from x1, and its
    margin tanh(beta I_i) + rho there, with I_i = -(L(x|x_i=1) - L(x|x_i=0))/2 (Eq. 5, 9) and
    rho the noise word of (seed, k, chain, t, i); the state before spin i is x1 on spins < i and
    x0 on the rest."""
    p, lam, J, hI = _replay_setup()
    N = p.nprime
    r = np.random.default_rng(8)
    seed, it = 33, 5
    for trial in range(6):
        x0 = (r.random(N) < 0.5).astype(np.uint8)
        x1 = (r.random(N) < 0.5).astype(np.uint8)
        beta = float(np.float32(0.5 + 1.5 * trial))
        chain, t = 3 + trial, 7 * trial
        want_spins, want_margins = [], []
        x = x0.copy()
        for i in range(N):
            hi = x.copy(); hi[i] = 1
            lo = x.copy(); lo[i] = 0
            I = -(p.lagrangian(hi, lam) - p.lagrangian(lo, lam)) / 2.0
            v = math.tanh(beta * I) + oracle.pbit_noise(seed, it, chain, t, i)
            if (v > 0) != bool(x1[i]):
                want_spins.append(i)
                want_margins.append(v)
            x[i] = x1[i]
        nbad, spins, margins = oracle.replay_sweep(J, hI, beta, seed, it, chain, t, x0, x1,
                                                   max_out=N)
        assert nbad == len(want_spins) and list(spins) == want_spins, trial
        assert np.allclose(margins, want_margins, rtol=0, atol=1e-10), trial


# --------------------------------------------------------------------------------------
# Noise: Philox4x32-10 and rand(-1,1)
# --------------------------------------------------------------------------------------

def _curand():
    names = [ctypes.util.find_library("curand"), "libcurand.so", "libcurand.so.10"]
    for d in ("/usr/local/cuda/lib64", "/usr/local/cuda/targets/sbsa-linux/lib",
              "/usr/local/cuda/targets/x86_64-linux/lib"):
        names += [os.path.join(d, "libcurand.so")]
    for nm in names:
        if not nm:
            continue
        try:
            return ctypes.CDLL(nm)
        except OSError:
            continue
    return None


def test_philox_matches_curand_host_generator():
    """The oracle's Philox4x32-10 against cuRAND's host Philox4_32_10 generator (a library
    routine run on the CPU): output group g of seed s is Philox(counter=(g>>16, 0, g&0xFFFF, 0),
    key=(s_lo, s_hi))."""
    cr = _curand()
    if cr is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    if cr.curandCreateGeneratorHost(ctypes.byref(gen), 161) != 0:  # CURAND_RNG_PSEUDO_PHILOX4_32_10
        pytest.skip("cuRAND host generator unavailable")
    try:
        for seed in (0x0123456789ABCDEF, 42, 0xFFFFFFFF00000001):
            assert cr.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
            assert cr.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(0)) == 0
            ngroups = 65536 + 512
            buf = np.zeros(4 * ngroups, dtype=np.uint32)
            assert cr.curandGenerate(gen, buf.ctypes.data_as(ctypes.c_void_p),
                                     ctypes.c_size_t(buf.size)) == 0
            key = [seed & 0xFFFFFFFF, seed >> 32]
            for g in list(range(0, 512)) + list(range(65536, 65536 + 512)) + [4097, 30001]:
                want = buf[4 * g:4 * g + 4]
                got = oracle.philox4x32_10([g >> 16, 0, g & 0xFFFF, 0], key)
                assert np.array_equal(got, want), (seed, g)
    finally:
        cr.curandDestroyGenerator(gen)


def test_rand_pm1_grid():
    """rho is an odd multiple of 2^-24 inside (-1, 1), symmetric under word complement."""
    assert oracle.rand_pm1(0) == -1.0 + 2.0 ** -24
    assert oracle.rand_pm1(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    assert oracle.rand_pm1(0x80000000) == 2.0 ** -24
    r = np.random.default_rng(2)
    for w in r.integers(0, 2**32, 2000, dtype=np.uint64):
        w = int(w)
        v = oracle.rand_pm1(w)
        k = (v + 1.0) * 2**24
        assert k == int(k) and int(k) % 2 == 1 and -1 < v < 1
        assert oracle.rand_pm1(~w & 0xFFFFFFFF) == -v


def test_noise_stream_statistics():
    """rho over (spin, sweep, chain) is uniform on (-1,1): mean ~ 0, variance ~ 1/3, and the
    four words of one Philox block are used by four consecutive spins."""
    vals = np.array([oracle.pbit_noise(77, 3, c, t, i)
                     for c in range(4) for t in range(25) for i in range(100)])
    n = len(vals)
    assert abs(vals.mean()) < 5 * math.sqrt(1 / 3 / n)
    assert abs(vals.var() - 1 / 3) < 0.03
    out = oracle.philox4x32_10([5, 9, 2, 3], [77, 0])
    for w in range(4):
        assert oracle.pbit_noise(77, 3, 2, 9, 20 + w) == oracle.rand_pm1(int(out[w]))


def test_beta_schedule():
    """Linear schedule from 0 to beta_max (Sec. III-B), one FP32 value per sweep."""
    T = 1000
    bs = [float(oracle.beta(10.0, t, T)) for t in range(T)]
    assert bs[0] == 0.0 and bs[-1] == 10.0
    assert all(b1 > b0 for b0, b1 in zip(bs, bs[1:]))
    assert abs(bs[500] - 10.0 * 500 / 999) < 1e-6
    assert float(oracle.beta(3.0, 0, 1)) == 3.0


# --------------------------------------------------------------------------------------
# Multiplier step and Algorithm 1
# --------------------------------------------------------------------------------------

def test_lambda_invariants():
    """Projection keeps lambda >= 0; a zero mean subgradient leaves lambda unchanged; all-positive
    constraint values raise every lambda (Sec. IV-B: lambda grows while A x - B >= 0)."""
    r = np.random.default_rng(3)
    sg = np.float32(1 / 3000)
    lam = np.zeros(5, dtype=np.float32)
    for _ in range(200):
        gs = r.integers(-5000, 5000, 5) * 64
        lam = oracle.lambda_update(gs, 64, 0.5, True, sg, lam)
        assert np.all(lam >= 0)
    lam0 = np.array([0.3, 1.5, 0.0, 2.0, 7.0], dtype=np.float32)
    assert np.array_equal(oracle.lambda_update(np.zeros(5), 64, 20.0, True, sg, lam0), lam0)
    up = oracle.lambda_update(np.full(5, 64 * 10), 64, 20.0, True, sg, lam0)
    assert np.all(up > lam0)
    down = oracle.lambda_update(np.full(5, -64 * 10), 64, 20.0, False, sg, lam0)
    assert np.all(down < lam0)
    # the step uses the mean over the C chains: C equal samples step like one sample
    g1 = np.array([7, -3, 120, 0, -55])
    assert np.array_equal(oracle.lambda_update(g1 * 64, 64, 20.0, False, sg, lam0),
                          oracle.lambda_update(g1, 1, 20.0, False, sg, lam0))


def test_step_rule_reduces_to_algorithm1():
    """With no decay and no averaging the step-size rule is Algorithm 1's constant step, bit
    for bit, at any iteration index."""
    r = np.random.default_rng(9)
    sg = np.float32(1 / 3000)
    lam = r.random(6).astype(np.float32)
    for it in range(40):
        gs = r.integers(-4000, 4000, 6) * 16
        want = oracle.lambda_update(gs, 16, 20.0, True, sg, lam)
        got = oracle.lambda_update_rule(gs, 16, 20.0, True, sg, lam, it)
        assert np.array_equal(got, want)
        lam = want


@pytest.mark.parametrize("eta_sqrt", [False, True])
def test_step_rule_closed_forms(eta_sqrt):
    """A constant subgradient mean gbar from iteration it0 on: the average after j steps is
    (1 - mu^j) gbar, and lambda moves by the sum of eta/(1 + c it) (or its square root)
    sigma_g (1 - mu^(j+1)) gbar; checked against the closed sums in exact rationals (the
    decay) and FP64, within the FP32 rounding of lambda at each step."""
    from fractions import Fraction as Fr
    C, gbar, eta, c, mu, sg, it0, K = 16, 7, 3000.0, 0.5, 0.75, np.float32(2.0 ** -12), 5, 30
    lam = np.array([0.5], np.float32)
    avg = np.zeros(1, np.float64)
    for j in range(K):
        lam = oracle.lambda_update_rule(np.array([gbar * C]), C, eta, False, sg, lam, it0 + j,
                                        decay=c, eta_sqrt=eta_sqrt, mu=mu, avg=avg)
    assert abs(avg[0] - (1 - mu ** K) * gbar) <= 1e-12 * gbar
    total = 0.0
    for j in range(K):
        den = Fr(1) + Fr(c) * (it0 + j)
        step = float(Fr(eta) / den) if not eta_sqrt else eta / math.sqrt(float(den))
        total += step * float(sg) * (1 - mu ** (j + 1)) * gbar
    want = 0.5 + total
    assert abs(float(lam[0]) - want) <= K * float(np.spacing(np.float32(want)))
    # the two rules differ by far more than that tolerance
    other = 0.0
    for j in range(K):
        den = 1.0 + c * (it0 + j)
        step = eta / (math.sqrt(den) if not eta_sqrt else den)
        other += step * float(sg) * (1 - mu ** (j + 1)) * gbar
    assert abs(other - total) > 100 * K * float(np.spacing(np.float32(want)))


def test_solve_step_rule_matches_the_step_function():
    """Algorithm 1 with the step-size rule equals the rule applied to the oracle's own last
    samples (decay on the absolute iteration index, the average starting at 0)."""
    inst = wl.qkp(30, 0.5, 6)
    p = _problem(inst)
    kw = dict(K=10, C=8, T=60, beta_max=10.0, eta=200.0, seed=9, iter0=3, keep_samples=True)
    res = oracle.solve(p, eta_decay=0.3, eta_sqrt=True, momentum=0.6, **kw)
    lam = np.zeros(1, np.float32)
    avg = np.zeros(1, np.float64)
    for k in range(10):
        lam = oracle.lambda_update_rule(res.g[k].sum(axis=0), 8, 200.0, True, p.sigma_g, lam,
                                        3 + k, decay=0.3, eta_sqrt=True, mu=0.6, avg=avg)
        assert np.array_equal(res.lambda_trace[k], lam)


def test_algorithm1_single_chain_no_projection():
    """With C = 1 and no projection the batch step is Algorithm 1's lambda <- lambda + eta g(x_k)
    applied to the last sample of each run, and the returned solution is the best stored
    feasible sample."""
    inst = wl.qkp(20, 0.5, 1)
    p = _problem(inst)
    res = oracle.solve(p, K=12, C=1, T=60, beta_max=10.0, eta=20.0, seed=5, project=False,
                       keep_samples=True)
    lam = np.zeros(1, dtype=np.float64)
    for k in range(12):
        lam = lam + 20.0 * (float(p.sigma_g) * res.g[k, 0, 0])
        lam = lam.astype(np.float32).astype(np.float64)
        assert res.lambda_trace[k, 0] == np.float32(lam[0])
    if res.best_cost is not None:
        assert p.feasible(res.best_x)
        assert res.costs[res.best_iter, res.best_chain] == res.best_cost == p.cost(res.best_x)


def test_solve_stores_best_feasible_and_resumes_bit_exactly():
    """Alg. 1 keeps the best feasible last sample (first achiever on ties) and a run of 20
    iterations equals two runs of 10 chained through lambda and the iteration index."""
    inst = wl.qkp(40, 0.5, 3)
    p = _problem(inst)
    kw = dict(C=8, T=80, beta_max=10.0, eta=20.0, seed=11)
    full = oracle.solve(p, K=20, keep_samples=True, **kw)
    a = oracle.solve(p, K=10, keep_samples=True, **kw)
    b = oracle.solve(p, K=10, iter0=10, lambda0=a.lambda_trace[-1], keep_samples=True, **kw)
    assert np.array_equal(full.lambda_trace, np.concatenate([a.lambda_trace, b.lambda_trace]))
    assert np.array_equal(full.costs, np.concatenate([a.costs, b.costs]))
    assert full.feasible_count == a.feasible_count + b.feasible_count
    if full.best_cost is not None:
        assert p.feasible(full.best_x) and p.cost(full.best_x) == full.best_cost
        assert full.costs[full.best_iter, full.best_chain] == full.best_cost
        cand = [a.best_cost, b.best_cost]
        assert full.best_cost == min(c for c in cand if c is not None)


def _np_cost(inst, X):
    """c(x) = -x^T W x / 2 - h^T x (Sec. IV-A) of every row of X (items first), int64 numpy."""
    Xi = X[:, :inst.n].astype(np.int64)
    lin = Xi @ np.asarray(inst.h, np.int64)
    if inst.W is None:
        return -lin
    W = np.asarray(inst.W, np.int64)
    return -np.einsum("ci,ij,cj->c", Xi, W, Xi) // 2 - lin


def _np_feasible(inst, X, cap):
    """A x <= cap on the items (Sec. IV-A), every row of X, numpy."""
    A = np.asarray(inst.A, np.int64).reshape(inst.m, inst.n)
    return ((X[:, :inst.n].astype(np.int64) @ A.T) <= np.asarray(cap, np.int64)[None, :]).all(1)


@pytest.mark.parametrize("kind", ["qkp", "mkp", "qkp_tight"])
def test_run_best_is_the_best_feasible_sweep_end_state(kind):
    """The best-in-run option stores, per chain, the least-cost state feasible under the true
    capacities among the states at the ends of the sweeps, the earliest sweep on ties: checked
    against numpy evaluations of the cost and the items' loads of every traced state."""
    if kind == "mkp":
        inst = wl.mkp(30, 3, 5)
    else:
        inst = wl.qkp(30, 0.5, 4)
    if kind == "qkp_tight":
        bt = np.maximum(1, (np.asarray(inst.b) * 4) // 5)
        p = oracle.Problem(inst.n, inst.m, inst.W, inst.h, inst.A, bt, alpha=inst.alpha,
                           density=inst.density, b_check=inst.b)
    else:
        p = _problem(inst)
    lam = np.full(inst.m, 0.5, np.float32)
    J, hI, _ = p.ising(lam)
    C, T = 12, 150
    _, tr = oracle.anneal(J, hI, 10.0, T, 21, 3, C, trace=True)
    cost, x, sweep, nfeas = oracle.run_best(p, tr)
    some = False
    for c in range(C):
        X = tr[c]
        feas = _np_feasible(inst, X, inst.b)
        assert nfeas[c] == int(feas.sum())
        if not feas.any():
            assert cost[c] == np.iinfo(np.int64).max and sweep[c] == -1 and not x[c].any()
            continue
        some = True
        cs = np.where(feas, _np_cost(inst, X), np.iinfo(np.int64).max)
        t = int(np.argmin(cs))      # numpy's argmin takes the first minimiser
        assert sweep[c] == t and cost[c] == cs[t]
        assert np.array_equal(x[c], X[t])
    assert some
    # a made-up trace with repeated states: the earliest sweep of the least-cost feasible state
    r = np.random.default_rng(6)
    pool = r.integers(0, 2, (6, p.nprime)).astype(np.uint8)
    idx = r.integers(0, 6, (4, 40))
    fake = pool[idx]
    cost2, _, sweep2, nfeas2 = oracle.run_best(p, fake)
    feas = _np_feasible(inst, pool, inst.b)
    cs = np.where(feas, _np_cost(inst, pool), np.iinfo(np.int64).max)
    for c in range(4):
        ok = feas[idx[c]]
        assert nfeas2[c] == int(ok.sum())
        if ok.any():
            best = cs[idx[c]].min()
            assert cost2[c] == best and sweep2[c] == int(np.flatnonzero(cs[idx[c]] == best)[0])
    if kind == "qkp_tight":
        # states between B' and B count as feasible: some sweep-end state exceeds B' but not B
        A = np.asarray(inst.A, np.int64).reshape(inst.m, inst.n)
        loads = tr[:, :, :inst.n].reshape(-1, inst.n).astype(np.int64) @ A.T
        assert ((loads > bt[None, :]) & (loads <= np.asarray(inst.b)[None, :])).any()


def test_solve_run_best_keeps_the_multiplier_path():
    """With the best-in-run option the multipliers still step on the last samples (the same
    lambda trace and last-sample costs as without it), every stored sample is a sweep-end
    state, so the best cost can only improve and the stored-feasible count can only grow."""
    inst = wl.mkp(40, 3, 8)
    p = _problem(inst)
    kw = dict(K=8, C=16, T=100, beta_max=10.0, eta=20.0, seed=3, keep_samples=True)
    last = oracle.solve(p, **kw)
    rb = oracle.solve(p, run_best=True, **kw)
    assert np.array_equal(last.lambda_trace, rb.lambda_trace)
    assert np.array_equal(last.costs, rb.costs) and np.array_equal(last.g, rb.g)
    assert rb.feasible_count >= last.feasible_count
    assert rb.best_cost is not None
    if last.best_cost is not None:
        assert rb.best_cost <= last.best_cost
    assert _np_feasible(inst, rb.best_x[None, :], inst.b)[0]
    assert _np_cost(inst, rb.best_x[None, :])[0] == rb.best_cost


def test_solve_run_best_stores_each_chains_best_sweep_end():
    """Algorithm 1 with the best-in-run option, rebuilt from its parts: per iteration the
    annealing traces at that iteration's multipliers, each chain's best feasible sweep end
    (or_run_best), the first least-cost one in (iteration, chain) order, and the count of
    chains with one."""
    inst = wl.mkp(30, 3, 11)
    p = _problem(inst)
    lam0 = np.full(3, 2.0, np.float32)
    K, C, T, seed = 3, 6, 80, 13
    res = oracle.solve(p, K=K, C=C, T=T, beta_max=20.0, eta=50.0, seed=seed, lambda0=lam0,
                       run_best=True)
    lams = [lam0] + [res.lambda_trace[k] for k in range(K - 1)]
    best, where, bx, count = None, None, None, 0
    for k in range(K):
        J, hI, _ = p.ising(lams[k])
        _, tr = oracle.anneal(J, hI, 20.0, T, seed, k, C, trace=True)
        cost, x, sweep, _ = oracle.run_best(p, tr)
        for c in range(C):
            if sweep[c] < 0:
                continue
            count += 1
            if best is None or cost[c] < best:
                best, where, bx = int(cost[c]), (k, c), x[c]
    assert count > 0 and best is not None
    assert res.feasible_count == count
    assert res.best_cost == best and (res.best_iter, res.best_chain) == where
    assert np.array_equal(res.best_x, bx)


def test_capacity_tightening_checks_the_true_capacities():
    """B' < B (Sec. IV-B): the sampled problem is the one built from B' (its slack bits,
    scales and penalty), feasibility uses B, and a long run on a tiny instance reaches the
    brute-force optimum under B, never a state beyond B."""
    W, h, A, b = _tiny_qkp(n=9, b=17, seed=8)
    bt = np.array([12])
    base = oracle.Problem(9, 1, W, h, A, bt, alpha=2.0, density=0.5)
    p = oracle.Problem(9, 1, W, h, A, bt, alpha=2.0, density=0.5, b_check=b)
    assert p.nprime == base.nprime == 9 + 4            # Q = floor(log2 12) + 1
    assert (p.sigma_g, p.P) == (base.sigma_g, base.P)
    r = np.random.default_rng(1)
    X = r.integers(0, 2, (400, p.nprime)).astype(np.uint8)
    loads = X[:, :9].astype(np.int64) @ A[0]
    for x, ld in zip(X, loads):
        assert p.feasible(x) == (ld <= 17) and base.feasible(x) == (ld <= 12)
    # brute-force optimum under B (numpy enumeration of the 2^9 item states)
    S = ((np.arange(1 << 9)[:, None] >> np.arange(9)) & 1).astype(np.int64)
    c_all = -np.einsum("si,ij,sj->s", S, W, S) // 2 - S @ h
    opt = c_all[(S @ A[0]) <= 17].min()
    res = oracle.solve(p, K=30, C=16, T=200, beta_max=10.0, eta=2.0, seed=2, run_best=True)
    assert res.best_cost == opt
    assert int(res.best_x[:9].astype(np.int64) @ A[0]) <= 17


def _dual_reachable(p, inst, lam_grid):
    """Costs of the feasible ground states of L(., lambda) over a grid of lambda (one
    constraint), by enumeration: L is affine in lambda, L = L0 + lambda (L1 - L0)."""
    N = p.nprime
    X = ((np.arange(1 << N)[:, None] >> np.arange(N)) & 1).astype(np.uint8)
    L0 = p.enumerate_lagrangian(np.zeros(1, np.float32))
    L1 = p.enumerate_lagrangian(np.ones(1, np.float32))
    feas = np.all(X[:, :inst.n].astype(np.int64) @ inst.A.T.astype(np.int64) <= inst.b, axis=1)
    out = set()
    for lam in lam_grid:
        a = int(np.argmin(L0 + lam * (L1 - L0)))
        if feas[a]:
            out.add(p.cost(X[a]))
    return out


def test_tiny_instances_against_brute_force():
    """Algorithm 1 on tiny QKPs (N' <= 18) with Table I parameters, against enumeration:
    the best stored sample is feasible, never better than OPT (Eq. 2), at least as good as every
    feasible ground state of L that the multiplier ascent passes through, and equal to OPT
    whenever OPT is such a ground state (no duality gap at P)."""
    hits = 0
    for seed in range(6):
        inst = wl.qkp(12, 0.5, 100 + seed, weight_max=9)
        inst.b = np.array([max(5, int(inst.A.sum()) // 2)])
        p = _problem(inst)
        opt, _ = p.brute_force_opt()
        reach = _dual_reachable(p, inst, np.linspace(0.0, 40.0, 801))
        res = oracle.solve(p, K=60, C=16, T=150, beta_max=10.0, eta=20.0, seed=seed)
        assert res.best_cost is not None and p.feasible(res.best_x)
        assert p.cost(res.best_x) == res.best_cost
        assert opt <= res.best_cost <= min(reach), (seed, res.best_cost, opt, sorted(reach))
        if opt in reach:
            assert res.best_cost == opt, (seed, res.best_cost, opt)
        hits += res.best_cost == opt
    assert hits >= 4


def test_tiny_mkp_reaches_optimum():
    """A small MKP (two knapsacks, N' = 24) reaches its enumerated optimum."""
    inst = wl.mkp(14, 2, 7, a_max=30)
    p = _problem(inst)
    opt, _ = p.brute_force_opt()
    res = oracle.solve(p, K=60, C=16, T=150, beta_max=50.0, eta=2.5, seed=1)
    assert res.best_cost == opt
