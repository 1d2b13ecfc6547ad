"""The C-ABI library loads, exports every symbol include/sais.h declares, and its host-side
problem scalars (slack extension, normalisation, penalty; no GPU involved) agree bit-for-bit
with the independently written CPU oracle.  CPU only: no compute call touches a GPU."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_2501_04971_gb300 import build as libbuild
from paper_2501_04971_gb300 import sais, workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    libbuild.build()
    return sais.lib()


def _declared():
    text = open(os.path.join(ROOT, "include", "sais.h")).read()
    return sorted(set(re.findall(r"SAIS_API\s+[\w\s\*]+?\b(sais_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("sais_create_problem", "sais_sample", "sais_update_lambda", "sais_solve"):
        assert want in names
    assert set(names) == set(sais.EXPORTS)


def test_library_exports_every_declared_symbol(L):
    for name in _declared():
        assert hasattr(L, name), name


def test_status_strings(L):
    for s in range(7):
        assert sais.sais_status_string(s)
    assert sais.sais_status_string(99) == "unknown status"


def _pairs():
    out = [wl.qkp(100, 0.25, s) for s in range(5)]
    out += [wl.qkp(300, d, s) for d in (0.25, 0.5, 0.75, 1.0) for s in range(3)]
    out += [wl.mkp(250, 5, s) for s in range(3)] + [wl.mkp(500, 30, 1), wl.mkp(37, 3, 2)]
    out += [wl.qkp(700, 0.5, 4, profit_max=10000)]
    return out


@pytest.mark.parametrize("idx", range(len(_pairs())))
def test_describe_matches_oracle_scalars(L, idx):
    inst = _pairs()[idx]
    s = sais.describe(inst)
    ref = oracle.Problem(inst.n, inst.m, inst.W, inst.h, inst.A, inst.b, alpha=inst.alpha,
                         density=inst.density)
    assert s.n_spins == ref.nprime
    assert s.words == (ref.nprime + 31) // 32
    assert np.float32(s.sigma_f) == ref.sigma_f
    assert np.float32(s.sigma_g) == ref.sigma_g
    assert np.float32(s.penalty) == ref.P
    assert s.density == ref.d_used


def test_describe_measured_density_and_override(L):
    inst = wl.qkp(50, 0.5, 3)
    inst.density = -1.0
    s = sais.describe(inst)
    ref = oracle.Problem(inst.n, inst.m, inst.W, inst.h, inst.A, inst.b, alpha=2.0, density=-1.0)
    assert s.density == ref.d_used and np.float32(s.penalty) == ref.P
    inst.penalty = 7.5
    assert sais.describe(inst).penalty == 7.5


def _bad(inst, status):
    with pytest.raises(sais.SaisError) as e:
        sais.describe(inst)
    assert e.value.status == status, str(e.value)


def test_describe_rejects_invalid_instances(L):
    base = wl.qkp(20, 0.5, 1)
    x = wl.qkp(20, 0.5, 1); x.W = x.W.copy(); x.W[0, 1] += 1
    _bad(x, sais.SAIS_EINVAL)                       # not symmetric
    x = wl.qkp(20, 0.5, 1); x.W = x.W.copy(); x.W[3, 3] = 5
    _bad(x, sais.SAIS_EINVAL)                       # nonzero diagonal
    x = wl.qkp(20, 0.5, 1); x.b = np.array([0])
    _bad(x, sais.SAIS_EINVAL)                       # capacity < 1
    x = wl.qkp(20, 0.5, 1); x.A = -base.A
    _bad(x, sais.SAIS_EINVAL)                       # negative weight
    x = wl.qkp(20, 0.5, 1); x.W = x.W.copy(); x.W[0, 1] = x.W[1, 0] = 40000
    _bad(x, sais.SAIS_EOVERFLOW)                    # int16 range
    x = wl.qkp(1200, 1.0, 1, profit_max=30000)
    _bad(x, sais.SAIS_EOVERFLOW)                    # |F| >= 2^24
    x = wl.mkp(20, 2, 1); x.b = np.array([2**24, 5])
    _bad(x, sais.SAIS_EOVERFLOW)                    # constraint range >= 2^24
    x = wl.mkp(20, 2, 1); x.m = 33
    with pytest.raises(Exception):
        sais.describe(x)
    x = wl.qkp(20, 0.5, 1); x.alpha = float("nan")
    _bad(x, sais.SAIS_EINVAL)


@pytest.mark.parametrize("frac", [1.0, 0.8, 0.5, 0.01])
def test_describe_tightened_capacities_match_oracle(L, frac):
    """Capacity tightening (Sec. IV-B): the sampled problem is the one built from B' -- slack
    bits, sigma_g and the penalty rule on that N' -- bit for bit the oracle's problem with
    b = B'; b_tight = b leaves the scalars unchanged."""
    for inst in (wl.qkp(120, 0.5, 2), wl.mkp(90, 5, 3), wl.qkp(300, 0.25, 1)):
        bt = np.maximum(1, np.floor(np.asarray(inst.b) * frac)).astype(np.int64)
        inst.b_tight = bt
        s = sais.describe(inst)
        ref = oracle.Problem(inst.n, inst.m, inst.W, inst.h, inst.A, bt, alpha=inst.alpha,
                             density=inst.density, b_check=inst.b)
        assert s.n_spins == ref.nprime
        assert np.float32(s.sigma_g) == ref.sigma_g
        assert np.float32(s.penalty) == ref.P
        assert s.density == ref.d_used
        if frac == 1.0:
            inst.b_tight = None
            plain = sais.describe(inst)
            assert (plain.n_spins, plain.sigma_g, plain.penalty) == \
                (s.n_spins, s.sigma_g, s.penalty)


def test_describe_rejects_bad_tightened_capacities(L):
    x = wl.mkp(30, 3, 1)
    x.b_tight = np.asarray(x.b, np.int64) + np.array([0, 1, 0])
    _bad(x, sais.SAIS_EINVAL)                       # B' > B
    x.b_tight = np.array([1, 0, 1], np.int64)
    _bad(x, sais.SAIS_EINVAL)                       # B' < 1


def test_last_error_message(L):
    x = wl.qkp(20, 0.5, 1); x.b = np.array([-3])
    with pytest.raises(sais.SaisError):
        sais.describe(x)
    assert "b[0]" in sais.sais_last_error()


def test_no_cpu_fallback(L, tmp_path):
    """The product path fails loudly: a missing library raises, and without an sm_103 device
    creating a problem returns SAIS_EUNSUPPORTED or SAIS_ECUDA instead of computing anywhere
    else."""
    with pytest.raises(RuntimeError):
        sais.lib(str(tmp_path / "libsais_missing.so"))
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except ImportError:
        has_gpu = False
    if has_gpu:
        pytest.skip("a CUDA device is present")
    with pytest.raises(sais.SaisError) as e:
        sais.Problem(wl.qkp(20, 0.5, 1))
    assert e.value.status in (sais.SAIS_EUNSUPPORTED, sais.SAIS_ECUDA)
