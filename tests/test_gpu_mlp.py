"""The warm-start network's CUDA kernels (tcgen05 forward/backward, Adam) against the oracle.

The oracle runs the same network in FP64 with BF16 rounding at the points where the kernels
feed the tensor cores (weights, x', h1, dz2, dz1), so the remaining differences are FP32
accumulation (about K 2^-24 of the magnitude sums) and, rarely, a BF16 rounding that lands on
the other side of a tie.  Both are bounded by a small multiple of the oracle's magnitude-bound
mode (every term replaced by its absolute value, every mask by 1); the tests use 2^-7 of that
bound element by element and a much tighter aggregate bound.
"""
import numpy as np
import pytest

import oracle
from paper_2501_04971_gb300 import sais, workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P = oracle.MLP_PARAMS
W1, W2, W3, B3 = oracle.MLP_OFF_W1, oracle.MLP_OFF_W2, oracle.MLP_OFF_W3, oracle.MLP_OFF_B3


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _params(seed):
    r = np.random.default_rng(seed)
    p = np.zeros(P, np.float32)
    w1 = r.normal(0, 0.5, (128, 16)); w1[:, 8:] = 0
    w2 = r.normal(0, 0.12, (128, 144)); w2[:, 129:] = 0
    p[W1:W1 + 2048] = w1.reshape(-1)
    p[W2:W2 + 18432] = w2.reshape(-1)
    p[W3:W3 + 128] = r.normal(0, 0.2, 128)
    p[B3] = 0.3
    return p


def _norm(seed):
    r = np.random.default_rng(seed)
    n = np.zeros(16, np.float32)
    n[:7] = r.normal(0, 0.5, 7)
    n[7:14] = r.uniform(0.5, 2.0, 7)
    n[14], n[15] = 1.5, 2.5
    return n


def _data(rows, seed):
    r = np.random.default_rng(seed)
    X = r.normal(0, 1, (rows, 8)).astype(np.float32)
    X[:, 7] = 0
    t = r.normal(1.5, 3, rows).astype(np.float32)
    return X, t


def _dev(a):
    return torch.tensor(a, device="cuda:0")


@pytest.mark.parametrize("rows", [1, 128, 300])
def test_forward_matches_oracle(rows):
    p, n = _params(1), _norm(2)
    X, _ = _data(rows, 3)
    net = sais.MLP(0)
    net.set_params(p, n)
    y = net.forward(_dev(X)).cpu().numpy().astype(np.float64)
    net.status()
    ref = oracle.mlp_forward(p, n, X, oracle.MLP_BF16)
    bound = oracle.mlp_forward(p, n, X, oracle.MLP_ABS) - abs(n[14])
    assert (np.abs(y - ref) <= 2.0 ** -7 * bound + 1e-6).all()
    assert np.linalg.norm(y - ref) <= 1e-4 * np.linalg.norm(bound)
    net.close()


@pytest.mark.parametrize("rows", [128, 300])
def test_gradient_matches_oracle(rows):
    p, n = _params(4), _norm(5)
    X, t = _data(rows, 6)
    net = sais.MLP(0)
    net.set_params(p, n)
    g, loss = net.gradient(_dev(X), _dev(t))
    g = g.cpu().numpy().astype(np.float64)
    net.status()
    lref, gref = oracle.mlp_grad(p, n, X, t, oracle.MLP_BF16)
    _, gabs = oracle.mlp_grad(p, n, X, t, oracle.MLP_ABS)
    assert abs(float(loss.item()) - lref) <= 1e-4 * lref
    bad = np.abs(g - gref) > 2.0 ** -7 * gabs + 1e-7
    assert not bad.any(), f"{bad.sum()} entries, first {np.argwhere(bad)[:5].ravel().tolist()}"
    assert np.linalg.norm(g - gref) <= 2.0 ** -10 * np.linalg.norm(gabs)
    # the padding columns and the unused tail get exactly zero
    assert not g[B3 + 1:].any()
    assert not g[W1:W1 + 2048].reshape(128, 16)[:, 8:].any()
    assert not g[W2:W2 + 18432].reshape(128, 144)[:, 129:].any()
    net.close()


def test_adam_step_matches_oracle():
    """Three training steps: each equals the oracle's Adam step applied to the kernel's own
    gradient (itself checked against the oracle above) with the same moment history and the
    FP32 values of beta1 = 0.9 and beta2 = 0.999 that the kernel uses."""
    p, n = _params(7), _norm(8)
    X, t = _data(256, 9)
    net = sais.MLP(0)
    net.set_params(p, n)
    lr = 1e-3
    Xd, td = _dev(X), _dev(t)
    loss = torch.zeros(1, device="cuda:0")
    th_gpu, mom, vel = p.astype(np.float64), np.zeros(P), np.zeros(P)
    for step in range(1, 4):
        # the kernel's own gradient at the current parameters, then one Adam step on both sides
        g_gpu = net.gradient(Xd, td)[0].cpu().numpy().astype(np.float64)
        net.train_step(Xd, td, lr, loss=loss)
        p1, _ = net.get_params()
        oracle.adam_step(th_gpu, mom, vel, g_gpu, step, lr, b1=float(np.float32(0.9)),
                         b2=float(np.float32(0.999)))
        assert np.allclose(p1, th_gpu, rtol=1e-6, atol=1e-8), step
        th_gpu = p1.astype(np.float64)
    net.status()
    assert float(loss.item()) > 0
    net.close()


def test_training_reduces_loss_and_keeps_padding_zero():
    r = np.random.default_rng(10)
    X = r.uniform(-1, 1, (4096, 8)).astype(np.float32)
    X[:, 7] = 0
    t = (2 * X[:, 0] + np.sin(3 * X[:, 1]) + np.abs(X[:, 2]) * X[:, 3]).astype(np.float32)
    net = sais.MLP(11)
    net.fit_normalization(X, t)
    Xd, td = _dev(X), _dev(t)
    loss = torch.zeros(1, device="cuda:0")
    net.train_step(Xd, td, 3e-3, loss=loss)
    first = float(loss.item())
    for _ in range(400):
        net.train_step(Xd, td, 3e-3, loss=loss)
    last = float(loss.item())
    net.status()
    assert last < 0.05 * first, (first, last)
    p, _ = net.get_params()
    assert not p[W1:W1 + 2048].reshape(128, 16)[:, 8:].any()
    assert not p[W2:W2 + 18432].reshape(128, 144)[:, 129:].any()
    assert not p[B3 + 1:].any()
    net.close()


def test_features_match_oracle():
    insts = [wl.qkp(100, 0.5, 1), wl.mkp(60, 5, 2), wl.qkp(40, 1.0, 3, profit_max=5000),
             wl.mkp(90, 10, 4)]
    prob = sais.Problem(insts)
    f = prob.features()
    r = 0
    for inst in insts:
        ref = oracle.Problem(inst.n, inst.m, inst.W, inst.h, inst.A, inst.b, alpha=inst.alpha,
                             density=inst.density)
        want = oracle.features(ref)
        assert np.allclose(f[r:r + inst.m], want, rtol=2e-7, atol=0), (r, f[r:r + inst.m], want)
        r += inst.m
    assert r == f.shape[0]
    prob.close()


def test_warm_start_scatters_clamped_predictions():
    insts = [wl.mkp(60, 5, 5), wl.qkp(80, 0.5, 6), wl.mkp(70, 3, 7)]
    prob = sais.Problem(insts)
    net = sais.MLP(12)
    p, n = _params(13), _norm(14)
    n[14] = -0.5   # some predictions negative -> clamped to 0
    net.set_params(p, n)
    lam = torch.full((prob.count * prob.m_stride,), -7.0, device="cuda:0")
    prob.warm_start(net, lam)
    F = prob.features()
    y = net.forward(_dev(F)).cpu().numpy()
    got = lam.cpu().numpy().reshape(prob.count, prob.m_stride)
    r = 0
    for j, inst in enumerate(insts):
        assert np.array_equal(got[j, :inst.m], np.maximum(y[r:r + inst.m], 0))
        assert (got[j, inst.m:] == -7.0).all()
        r += inst.m
    assert (y < 0).any() and (y > 0).any()
    net.close()
    prob.close()


def test_set_params_roundtrip_and_validation():
    net = sais.MLP(0)
    p = _params(15)
    p[W1 + 9] = 5.0          # a padding column entry: zeroed on set
    n = _norm(16)
    net.set_params(p, n)
    q, m = net.get_params()
    assert q[W1 + 9] == 0.0
    p[W1 + 9] = 0.0
    assert np.array_equal(q, p) and np.array_equal(m, n)
    bad = n.copy()
    bad[8] = 0.0
    with pytest.raises(sais.SaisError) as e:
        net.set_params(p, bad)
    assert e.value.status == sais.SAIS_EINVAL
    net.close()
