"""The library's device allocations through a caller's allocator (needs a GPU).

sais_set_device_allocator routes every device buffer the library owns (problem data, sais_solve
and sais_autotune scratch, SAIS_AUTO work lists, per-instance chain counts, the warm-start
network) through the caller's pair.  Failure detection: an allocator that refuses makes the
entry points return SAIS_ENOMEM and leaves the process usable.  Accounting: a counting allocator
on top of PyTorch's caching allocator sees every block come back, and the results equal those
of the default cudaMalloc / cudaFree path bit for bit.
"""
import numpy as np
import pytest

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
    yield
    sais.sais_set_device_allocator()


def _workload():
    """A ragged batch through SAIS_AUTO (work list, chain counts), a solve (scratch), the
    autotuner (scratch) and the network (buffers, partial gradients); returns the results."""
    insts = [wl.qkp(120, 0.5, 1), wl.qkp(60, 0.25, 2), wl.mkp(50, 3, 3)]
    prob = sais.Problem(insts)
    prob.set_instance_chains(np.array([64, 40, 30], np.int32))
    lam = torch.zeros(prob.count * prob.m_stride, device="cuda")
    out = prob.sample(lam, 64, 30, 10.0, 5, 0, variant="auto")
    prob.synchronize()
    res = {k: v.cpu().numpy().copy() for k, v in out.items()}
    sol = prob.solve(3, 64, 30, 10.0, 20.0, 6, variant="auto")
    prob.autotune(64, 5)
    prob.set_instance_chains(None)
    net = sais.MLP(3)
    gen = torch.Generator(device="cuda").manual_seed(0)
    X = torch.rand(300, 8, device="cuda", generator=gen)
    y = torch.rand(300, device="cuda", generator=gen)
    net.train_step(X, y, 1e-3)
    torch.cuda.synchronize()
    params = net.get_params()[0].copy()
    net.close()
    prob.close()
    return res, sol, params


def test_refusing_allocator_gives_enomem_and_recovers():
    calls = []
    sais.sais_set_device_allocator(lambda n, dev: calls.append(n) or 0,
                                   lambda p, n, dev: None)
    try:
        with pytest.raises(sais.SaisError) as e:
            sais.Problem([wl.qkp(50, 0.5, 9)])
        assert e.value.status == sais.SAIS_ENOMEM
        with pytest.raises(sais.SaisError) as e:
            sais.MLP(1)
        assert e.value.status == sais.SAIS_ENOMEM
        assert calls, "the library did not ask the installed allocator"
    finally:
        sais.sais_set_device_allocator()
    prob = sais.Problem([wl.qkp(50, 0.5, 9)])   # the default path works again
    prob.close()


def test_counting_allocator_balances_and_matches_default():
    want = _workload()
    live, stats = {}, {"allocs": 0, "frees": 0}

    def alloc(n, dev):
        p = torch.cuda.caching_allocator_alloc(n, dev)
        live[p] = n
        stats["allocs"] += 1
        return p

    def free(p, n, dev):
        assert live.pop(p) == n
        stats["frees"] += 1
        torch.cuda.caching_allocator_delete(p)

    sais.sais_set_device_allocator(alloc, free)
    try:
        got = _workload()
    finally:
        sais.sais_set_device_allocator()
    assert stats["allocs"] >= 6 and stats["frees"] == stats["allocs"] and not live, stats
    for k in want[0]:
        assert np.array_equal(want[0][k], got[0][k]), k
    for k in ("best_cost", "best_x", "lambda_trace", "feasible_count"):
        assert np.array_equal(want[1][k], got[1][k]), k
    assert np.array_equal(want[2], got[2])


def test_allocator_arguments():
    with pytest.raises(sais.SaisError) as e:
        sais._check(sais.lib().sais_set_device_allocator(
            sais.DEVICE_ALLOC_FN(lambda n, d, c: None), sais.DEVICE_FREE_FN(), None), "set")
    assert e.value.status == sais.SAIS_EINVAL
