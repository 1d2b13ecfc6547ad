"""GPU parity of the multiplier step's step-size rule (needs an sm_103a GPU).

sais_update_lambda_rule and sais_solve with a decaying eta (1/(1 + c k) or 1/sqrt(1 + c k))
and an exponentially averaged subgradient equal the oracle's or_lambda_update_rule and solve
bit for bit: the multipliers (FP32) and the running averages (FP64) are exactly rounded
quantities of one fixed evaluation order.
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


@pytest.mark.parametrize("decay,eta_sqrt,mu", [(0.0, False, 0.0), (0.25, False, 0.0),
                                               (0.25, True, 0.0), (0.0, False, 0.7),
                                               (1.5, True, 0.9)])
def test_update_rule_bit_exact(decay, eta_sqrt, mu):
    insts = [wl.qkp(50, 0.5, 1), wl.mkp(40, 5, 2), wl.mkp(30, 3, 3)]
    prob = sais.Problem(insts)
    C, M = 32, prob.m_stride
    refs = [oracle.Problem(i.n, i.m, i.W, i.h, i.A, i.b, alpha=i.alpha, density=i.density)
            for i in insts]
    r = np.random.default_rng(4)
    lam_h = np.zeros((prob.count, M), np.float32)
    for j, i in enumerate(insts):
        lam_h[j, :i.m] = r.random(i.m) * 0.5
    lam = torch.tensor(lam_h.reshape(-1), device="cuda:0")
    avg = torch.zeros(prob.count * M, dtype=torch.float64, device="cuda:0")
    avg_h = [np.zeros(i.m, np.float64) for i in insts]
    for step in range(20):
        it = 7 + step
        g = np.zeros((prob.count, C, M), np.int64)
        for j, i in enumerate(insts):
            g[j, :, :i.m] = r.integers(-3000, 3000, (C, i.m))
        prob.update_lambda_rule(torch.tensor(g.reshape(-1), device="cuda:0"), C, 900.0, True,
                                lam, it, decay, eta_sqrt, mu, avg if mu else None)
        for j, (i, ref) in enumerate(zip(insts, refs)):
            lam_h[j, :i.m] = oracle.lambda_update_rule(g[j, :, :i.m].sum(axis=0), C, 900.0, True,
                                                       ref.sigma_g, lam_h[j, :i.m], it,
                                                       decay=decay, eta_sqrt=eta_sqrt, mu=mu,
                                                       avg=avg_h[j])
        got = lam.cpu().numpy().reshape(prob.count, M)
        assert np.array_equal(got.view(np.uint32), lam_h.view(np.uint32)), step
        if mu:
            ga = avg.cpu().numpy().reshape(prob.count, M)
            for j, i in enumerate(insts):
                assert np.array_equal(ga[j, :i.m].view(np.uint64), avg_h[j].view(np.uint64))
    prob.close()


@pytest.mark.parametrize("variant", ["plain", "blocked"])
def test_solve_with_rule_matches_oracle(variant):
    inst = wl.qkp(60, 0.5, 12)
    prob = sais.Problem(inst)
    kw = dict(eta_decay=0.2, eta_sqrt=True, momentum=0.5)
    got = prob.solve(10, 64, 100, 10.0, 400.0, 6, iter0=4, variant=variant,
                     use_graph=variant == "blocked", **kw)
    prob.close()
    ref = oracle.Problem(inst.n, inst.m, inst.W, inst.h, inst.A, inst.b, alpha=inst.alpha,
                         density=inst.density)
    want = oracle.solve(ref, K=10, C=64, T=100, beta_max=10.0, eta=400.0, seed=6, iter0=4, **kw)
    assert np.array_equal(got["lambda_trace"][:, 0, :1], want.lambda_trace)
    assert got["feasible_count"][0] == want.feasible_count
    if want.best_cost is None:
        assert got["best_cost"][0] == np.iinfo(np.int64).max
    else:
        assert got["best_cost"][0] == want.best_cost
        assert (got["best_iter"][0], got["best_chain"][0]) == (want.best_iter, want.best_chain)


def test_rule_rejects_bad_parameters():
    prob = sais.Problem(wl.qkp(30, 0.5, 1))
    with pytest.raises(sais.SaisError) as e:
        prob.solve(2, 32, 10, 10.0, 20.0, 1, momentum=1.0)
    assert e.value.status == sais.SAIS_EINVAL
    with pytest.raises(sais.SaisError) as e:
        prob.solve(2, 32, 10, 10.0, 20.0, 1, eta_decay=-0.5)
    assert e.value.status == sais.SAIS_EINVAL
    g = torch.zeros(32 * prob.m_stride, dtype=torch.int64, device="cuda:0")
    lam = torch.zeros(prob.m_stride, device="cuda:0")
    with pytest.raises(sais.SaisError) as e:
        prob.update_lambda_rule(g, 32, 20.0, True, lam, 0, momentum=0.5, avg=None)
    assert e.value.status == sais.SAIS_EINVAL
    prob.close()
