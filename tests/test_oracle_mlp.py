"""Pins of the oracle's learned warm start (features, MLP forward/backward, Adam).

Each check ties the oracle to something other than itself: a hand-computed feature example,
a network whose output has a closed form, central finite differences of the loss for the
backward pass, the BF16 rounding of a library routine, and Adam's closed form for constant and
hand-worked gradients (Kingma & Ba, Algorithm 1).
"""
import numpy as np
import pytest

import oracle

P, H = oracle.MLP_PARAMS, oracle.MLP_HIDDEN
W1, W2, W3, B3 = oracle.MLP_OFF_W1, oracle.MLP_OFF_W2, oracle.MLP_OFF_W3, oracle.MLP_OFF_B3
K1, K2 = 16, 144


def _norm(mu=None, sd=None, y_mu=0.0, y_sd=1.0):
    n = np.zeros(16, np.float32)
    n[:7] = 0.0 if mu is None else mu
    n[7:14] = 1.0 if sd is None else sd
    n[14], n[15] = y_mu, y_sd
    return n


def _rand_params(seed, scale=0.3):
    r = np.random.default_rng(seed)
    p = np.zeros(P, np.float32)
    w1 = r.normal(0, scale, (H, K1)).astype(np.float32)
    w1[:, 8:] = 0
    w2 = r.normal(0, scale / 4, (H, K2)).astype(np.float32)
    w2[:, 129:] = 0
    p[W1:W1 + H * K1] = w1.reshape(-1)
    p[W2:W2 + H * K2] = w2.reshape(-1)
    p[W3:W3 + H] = r.normal(0, scale, H)
    p[B3] = 0.25
    return p


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    r = np.random.default_rng(0)
    v = np.concatenate([r.normal(0, 1, 4000), r.normal(0, 1e4, 2000), r.normal(0, 1e-4, 2000)])
    v = v.astype(np.float32)
    # exact ties (lower 16 bits 0x8000) with both parities of the kept bit
    ties = (np.arange(1000, dtype=np.uint32) << 16) | 0x3F800000 | 0x8000
    v = np.concatenate([v, ties.view(np.float32)])
    want = torch.tensor(v).to(torch.bfloat16).to(torch.float32).numpy()
    got = np.array([oracle.bf16_round(x) for x in v], np.float32)
    assert np.array_equal(got, want)


def test_features_hand_example():
    W = np.array([[0, 4, 0], [4, 0, 2], [0, 2, 0]], np.int64)
    pr = oracle.Problem(3, 1, W, np.array([1, 0, 3]), np.array([[2, 3, 5]]), np.array([6]),
                        alpha=2.0, density=0.5)
    f = oracle.features(pr)[0]
    sg, sf = 1 / 6, 1 / 4            # 1/max(A, b), 1/max(|W|, |h|)
    a = np.array([2, 3, 5.0])
    prof = np.array([1, 3, 4, 2.0])  # nonzero h_i and W_ij (i < j)
    want = [min(1, 6 / 10), sg * a.mean(), sg * a.std(), sf * prof.mean(), sf * prof.std(),
            3 / 1000, 0.5, 0.0]
    assert np.allclose(f, want, rtol=1e-6, atol=1e-7), (f, want)


def test_features_mkp_rows_and_density():
    A = np.array([[1, 2, 3, 4], [0, 0, 0, 0], [5, 5, 5, 5]])
    pr = oracle.Problem(4, 3, None, np.array([3, 0, 7, 2]), A, np.array([5, 9, 100]), alpha=5.0)
    f = oracle.features(pr)
    assert f.shape == (3, 8)
    assert f[0, 0] == np.float32(0.5) and f[1, 0] == 1.0 and f[2, 0] == 1.0   # min(1, b/sum)
    assert f[1, 1] == 0 and f[1, 2] == 0
    assert np.allclose(f[:, 3], (12 / 3) / 7) and np.allclose(f[:, 5], 0.004)
    # MKP density reading d = 2/(N'+1) enters P and the features alike
    assert np.allclose(f[:, 6], pr.d_used)


def test_forward_closed_form():
    """W1 picks feature perm[o] into unit o (scale s_o, bias c_o), W2 is the identity on those
    units plus a bias, w3 weights them: u = b3 + sum_o w3_o relu(relu(s_o x'_perm(o) + c_o) + e_o)."""
    perm = [3, 0, 6, 1, 5, 2, 4]
    s = np.array([1.5, -2.0, 0.5, 1.0, -1.0, 3.0, 0.25])
    c = np.array([0.1, 0.2, -0.3, 0.0, 0.5, -1.0, 0.05])
    e = np.array([0.0, -0.1, 0.2, 0.3, 0.0, 0.1, -0.2])
    w3 = np.arange(1, 8) / 4.0
    p = np.zeros(P, np.float32)
    w1 = np.zeros((H, K1)); w2 = np.zeros((H, K2))
    for o in range(7):
        w1[o, perm[o]] = s[o]
        w1[o, 7] = c[o]
        w2[o, o] = 1.0
        w2[o, 128] = e[o]
    p[W1:W1 + H * K1] = w1.reshape(-1)
    p[W2:W2 + H * K2] = w2.reshape(-1)
    p[W3:W3 + 7] = w3
    p[B3] = 0.5
    mu = np.array([0.1, -0.2, 0.3, 0.0, 0.5, 1.0, -1.0], np.float32)
    sd = np.array([1.0, 2.0, 0.5, 4.0, 1.0, 0.25, 2.0], np.float32)
    norm = _norm(mu, sd, y_mu=3.0, y_sd=2.0)
    X = np.random.default_rng(1).normal(0, 1, (50, 8)).astype(np.float32)
    y = oracle.mlp_forward(p, norm, X)
    xp = (X[:, :7].astype(np.float64) - mu) / sd
    relu = lambda v: np.maximum(v, 0)
    s, c, e = (v.astype(np.float32).astype(np.float64) for v in (s, c, e))
    u = 0.5 + sum(w3[o] * relu(relu(s[o] * xp[:, perm[o]] + c[o]) + e[o]) for o in range(7))
    assert np.allclose(y, 3.0 + 2.0 * u, rtol=1e-12, atol=1e-12)


def test_backward_matches_central_differences():
    p = _rand_params(2)
    norm = _norm(np.full(7, 0.1), np.full(7, 1.3), y_mu=0.5, y_sd=2.0)
    r = np.random.default_rng(3)
    X = r.normal(0, 1, (24, 8)).astype(np.float32)
    t = r.normal(0.5, 2, 24).astype(np.float32)
    loss, g = oracle.mlp_grad(p, norm, X, t)
    u = (oracle.mlp_forward(p, norm, X) - 0.5) / 2.0
    assert np.isclose(loss, np.mean((u - (t - 0.5) / 2.0) ** 2), rtol=1e-12)
    idx = np.concatenate([r.choice(np.arange(W1, W1 + H * K1).reshape(H, K1)[:, :8].ravel(), 60),
                          r.choice(np.arange(W2, W2 + H * K2).reshape(H, K2)[:, :129].ravel(), 80),
                          r.choice(np.arange(W3, W3 + H), 30), [B3]])
    h = np.float32(2.0 ** -12)
    worst = 0.0
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (oracle.mlp_grad(pp, norm, X, t)[0] - oracle.mlp_grad(pm, norm, X, t)[0]) / \
            (float(pp[i]) - float(pm[i]))
        worst = max(worst, abs(fd - g[i]) / (abs(g[i]) + 1e-6))
    assert worst < 1e-5, worst
    # padding columns carry no gradient
    assert not g[W1:W1 + H * K1].reshape(H, K1)[:, 8:].any()
    assert not g[W2:W2 + H * K2].reshape(H, K2)[:, 129:].any()


def test_bf16_mode_is_exact_on_representable_values():
    """With weights, inputs and every intermediate sum of the forward pass representable in
    BF16 the BF16 mode rounds nothing there and equals the FP64 mode; in the backward pass the
    rounded dz2 and dz1 (each within 2^-9 relative) keep every gradient entry within 2^-7 of
    the magnitude bound of the ABS mode."""
    r = np.random.default_rng(4)
    p = np.zeros(P, np.float32)
    w1 = np.zeros((H, K1)); w1[:, :8] = r.integers(-2, 3, (H, 8)) * 0.5
    w2 = np.zeros((H, K2)); w2[:16, :16] = r.integers(-1, 2, (16, 16)) * 0.25
    w2[:16, 128] = 0.5
    p[W1:W1 + H * K1] = w1.reshape(-1)
    p[W2:W2 + H * K2] = w2.reshape(-1)
    p[W3:W3 + 16] = r.integers(-2, 3, 16) * 0.5
    p[B3] = 1.0
    X = r.integers(0, 3, (16, 8)).astype(np.float32)
    X[:, 7] = 0
    t = r.integers(-3, 4, 16).astype(np.float32)
    norm = _norm()
    assert np.array_equal(oracle.mlp_forward(p, norm, X, oracle.MLP_BF16),
                          oracle.mlp_forward(p, norm, X, 0))
    l0, g0 = oracle.mlp_grad(p, norm, X, t, 0)
    l1, g1 = oracle.mlp_grad(p, norm, X, t, oracle.MLP_BF16)
    _, ga = oracle.mlp_grad(p, norm, X, t, oracle.MLP_ABS)
    assert l0 == l1
    assert (np.abs(g1 - g0) <= 2.0 ** -7 * ga).all()
    assert np.array_equal(g0[W3:], g1[W3:])       # w3, b3: no rounded operand
    assert not np.array_equal(g0, g1)             # but dz2 / dz1 were rounded somewhere


def test_abs_mode_bounds_values():
    p = _rand_params(5)
    norm = _norm(np.full(7, -0.2), np.full(7, 0.7), y_mu=1.0, y_sd=3.0)
    r = np.random.default_rng(6)
    X = r.normal(0, 1, (32, 8)).astype(np.float32)
    t = r.normal(1, 3, 32).astype(np.float32)
    y = oracle.mlp_forward(p, norm, X)
    ya = oracle.mlp_forward(p, norm, X, oracle.MLP_ABS)
    assert (ya >= np.abs(y) - 1e-12).all()
    _, g = oracle.mlp_grad(p, norm, X, t)
    _, ga = oracle.mlp_grad(p, norm, X, t, oracle.MLP_ABS)
    assert (ga >= np.abs(g) - 1e-12).all()


def test_adam_closed_forms():
    lr = 1e-2
    th = np.array([1.0, -2.0, 0.5]); m = np.zeros(3); v = np.zeros(3)
    g = np.array([0.3, -4.0, 0.0])
    for t in range(1, 6):
        oracle.adam_step(th, m, v, g, t, lr)
        # constant gradient: m_hat = g, v_hat = g^2 at every step
        want = np.array([1.0, -2.0, 0.5]) - t * lr * g / (np.abs(g) + 1e-8)
        assert np.allclose(th, want, rtol=0, atol=1e-12)
    # gradients +1 then -1 (beta1 0.9, beta2 0.999): steps -lr, then +lr * (0.01 / 0.19)
    th = np.zeros(1); m = np.zeros(1); v = np.zeros(1)
    oracle.adam_step(th, m, v, np.ones(1), 1, lr)
    assert np.isclose(th[0], -lr / (1 + 1e-8), rtol=1e-12)
    oracle.adam_step(th, m, v, -np.ones(1), 2, lr)
    assert np.isclose(th[0], -lr / (1 + 1e-8) + lr * (0.01 / 0.19) / (1 + 1e-8), rtol=1e-12)
