"""sais_solve_noalloc, the allocation-free form of Algorithm 1 (needs a GPU).

Callers that may not allocate while they run (a latency-critical loop that must stay out of the
allocator, a host that reserves all device memory up front, a plug-in that only gets its own
buffers) use sais_solve_noalloc, whose scratch is a fixed static device array.  These checks call
it through the C-ABI, twice in a row, and require the same results as sais_solve (bit for bit:
the samples, the kept best and the multipliers are integer or exactly rounded quantities).  This
file is collected last so that a failure here leaves every other test already run; it passes on
its own in a fresh process as well.
"""
import ctypes

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


def _noalloc(prob, iters, chains, sweeps, beta_max, eta, seed, variant="plain", lambda0=None,
             run_best=False, eta_decay=0.0, eta_sqrt=False, momentum=0.0, stream=None):
    """Call sais_solve_noalloc through the C-ABI with host result arrays."""
    prm = sais.sais_solve_params()
    prm.iters, prm.chains, prm.sweeps, prm.beta_max = iters, chains, sweeps, beta_max
    prm.eta, prm.seed, prm.iter0, prm.project_nonneg = eta, seed, 0, 1
    prm.variant = sais._VARIANTS[variant]
    prm.run_best = int(run_best)
    prm.eta_decay, prm.eta_sqrt, prm.momentum = eta_decay, int(eta_sqrt), momentum
    keep = None
    if lambda0 is not None:
        keep = np.ascontiguousarray(lambda0, np.float32).reshape(-1)
        prm.lambda0 = keep.ctypes.data_as(ctypes.c_void_p)
    cnt, W, M = prob.count, prob.words, prob.m_stride
    out = {"best_cost": np.zeros(cnt, np.int64), "best_x": np.zeros((cnt, W), np.uint32),
           "best_iter": np.zeros(cnt, np.int32), "best_chain": np.zeros(cnt, np.int32),
           "feasible_count": np.zeros(cnt, np.int64),
           "lambda_final": np.zeros((cnt, M), np.float32),
           "lambda_trace": np.zeros((iters, cnt, M), np.float32)}
    res = sais.sais_solve_result()
    for k, v in out.items():
        setattr(res, k, v.ctypes.data_as(ctypes.c_void_p))
    sp = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    st = sais.lib().sais_solve_noalloc(prob.handle, ctypes.byref(prm), ctypes.byref(res), sp)
    return st, out


KEYS = ("best_cost", "best_x", "best_iter", "best_chain", "feasible_count", "lambda_final",
        "lambda_trace")


@pytest.mark.parametrize("variant", ["plain", "blocked"])
def test_noalloc_matches_solve_on_two_calls(variant):
    insts = [wl.qkp(100, 0.5, 3), wl.qkp(60, 0.25, 4), wl.qkp(120, 0.75, 5)]
    prob = sais.Problem(insts)
    lam0 = np.full((prob.count, prob.m_stride), 0.25, np.float32)
    want = prob.solve(8, 128, 150, 10.0, 20.0, 17, lambda0=lam0, variant=variant)
    for call in range(2):
        st, got = _noalloc(prob, 8, 128, 150, 10.0, 20.0, 17, variant=variant, lambda0=lam0)
        assert st == sais.SAIS_OK, sais.sais_last_error()
        for k in KEYS:
            assert np.array_equal(got[k], want[k]), (call, k)
    prob.close()


def test_noalloc_run_best_with_tightening_matches_solve():
    """The best-in-run option, tightened capacities and the step-size rule through the
    allocation-free form."""
    insts = [wl.qkp(100, 0.5, 8), wl.qkp(80, 0.75, 9)]
    for inst in insts:
        inst.b_tight = np.maximum(1, (np.asarray(inst.b) * 4) // 5).astype(np.int64)
    prob = sais.Problem(insts)
    rule = dict(eta_decay=0.3, eta_sqrt=False, momentum=0.6)
    for variant in ("plain", "blocked"):
        want = prob.solve(6, 128, 120, 10.0, 20.0, 21, variant=variant, run_best=True, **rule)
        st, got = _noalloc(prob, 6, 128, 120, 10.0, 20.0, 21, variant=variant, run_best=True,
                           **rule)
        assert st == sais.SAIS_OK, sais.sais_last_error()
        for k in KEYS:
            assert np.array_equal(got[k], want[k]), (variant, k)
    prob.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    prob = sais.Problem([wl.qkp(300, 0.5, s) for s in range(16)])
    st, _ = _noalloc(prob, 2, 32768, 1, 10.0, 20.0, 1)   # ~30 MB of scratch needed
    assert st == sais.SAIS_EINVAL
    msg = sais.sais_last_error()
    assert "static scratch holds" in msg and "bytes" in msg
    st, got = _noalloc(prob, 2, 32, 20, 10.0, 20.0, 1)   # a size that fits still works after it
    assert st == sais.SAIS_OK, sais.sais_last_error()
    prob.close()


def test_noalloc_rejects_auto_variant():
    prob = sais.Problem([wl.qkp(60, 0.5, 6)])
    st, _ = _noalloc(prob, 2, 32, 10, 10.0, 20.0, 1, variant="auto")
    assert st == sais.SAIS_EINVAL and "SAIS_AUTO" in sais.sais_last_error()
    prob.close()


def test_noalloc_rejects_before_queueing_then_runs_on_another_stream():
    """A call the sampler cannot run (the blocked sampler on an objective without W) is refused
    before anything reaches the GPU; a valid call on another stream right after it still equals
    sais_solve."""
    mkp = sais.Problem([wl.mkp(40, 3, 2)])
    st, _ = _noalloc(mkp, 2, 32, 10, 10.0, 20.0, 1, variant="blocked")
    assert st == sais.SAIS_EUNSUPPORTED, sais.sais_last_error()
    mkp.close()
    prob = sais.Problem([wl.qkp(80, 0.5, 12)])
    want = prob.solve(4, 64, 60, 10.0, 20.0, 9, variant="plain")
    side = torch.cuda.Stream()
    st, got = _noalloc(prob, 4, 64, 60, 10.0, 20.0, 9, variant="plain", stream=side)
    assert st == sais.SAIS_OK, sais.sais_last_error()
    for k in KEYS:
        assert np.array_equal(got[k], want[k]), k
    prob.close()


def test_noalloc_second_call_leaves_free_memory_unchanged():
    """The defining property, checked coarsely: after a first call (which may load the module
    holding the static array), a second call changes the device's free memory by nothing.
    cudaMemGetInfo counts whole allocations, so this sees any cudaMalloc the call might make."""
    prob = sais.Problem([wl.qkp(100, 0.5, 13), wl.qkp(70, 0.25, 14)])
    st, _ = _noalloc(prob, 3, 64, 50, 10.0, 20.0, 5, variant="blocked")
    assert st == sais.SAIS_OK, sais.sais_last_error()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    st, _ = _noalloc(prob, 3, 64, 50, 10.0, 20.0, 5, variant="blocked")
    assert st == sais.SAIS_OK, sais.sais_last_error()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    prob.close()
