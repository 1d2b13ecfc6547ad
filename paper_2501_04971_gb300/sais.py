"""Thin ctypes binding of libsais (include/sais.h).

Argument marshalling only: every step of the sampling path runs in the library's CUDA kernels.
PyTorch provides device memory and streams.  The raw entry points keep the C names
(``sais_create_problem``, ``sais_sample``, ...); :class:`Problem` wraps a handle for tests and
benchmarks.  There is no CPU fallback: a missing library raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import List, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# SAIS_DEBUG=1 in the environment loads the build with the device-side checks
# (paper_2501_04971_gb300.build.build(debug=True)).
LIB_PATH = os.path.join(HERE, "_build_debug" if os.environ.get("SAIS_DEBUG") == "1" else "_build",
                        "libsais.so")

_i32, _i64, _u32, _u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
_f32, _f64, _P = ctypes.c_float, ctypes.c_double, ctypes.c_void_p

SAIS_OK, SAIS_EINVAL, SAIS_ENOMEM, SAIS_ECUDA, SAIS_EOVERFLOW, SAIS_ETIMEOUT, \
    SAIS_EUNSUPPORTED, SAIS_EBOUNDS = range(8)
SAIS_PLAIN, SAIS_BLOCKED, SAIS_AUTO = 0, 1, 2
SAIS_AUTO_PERSISTENT, SAIS_AUTO_GROUPS = 0, 1
_VARIANTS = {"plain": SAIS_PLAIN, "blocked": SAIS_BLOCKED, "auto": SAIS_AUTO}


class sais_problem_desc(ctypes.Structure):
    _fields_ = [("n", _i32), ("m", _i32), ("W", _P), ("h", _P), ("A", _P), ("b", _P),
                ("alpha", _f32), ("density", _f32), ("penalty", _f32), ("b_tight", _P)]


class sais_problem_scalars(ctypes.Structure):
    _fields_ = [("n", _i32), ("m", _i32), ("n_spins", _i32), ("words", _i32),
                ("sigma_f", _f32), ("sigma_g", _f32), ("penalty", _f32), ("reserved", _f32),
                ("density", _f64)]


class sais_layout(ctypes.Structure):
    _fields_ = [("count", _i32), ("max_spins", _i32), ("words", _i32), ("m_stride", _i32),
                ("device", _i32), ("has_quadratic", _i32)]


class sais_sample_params(ctypes.Structure):
    _fields_ = [("chains", _i32), ("sweeps", _i32), ("beta_max", _f32), ("iter", _u32),
                ("seed", _u64), ("variant", _i32), ("block_k", _i32),
                ("chains_per_cta", _i32), ("debug_wait_polls", _i32)]


class sais_solve_params(ctypes.Structure):
    _fields_ = [("iters", _i32), ("chains", _i32), ("sweeps", _i32), ("beta_max", _f32),
                ("eta", _f64), ("seed", _u64), ("iter0", _u32), ("project_nonneg", _i32),
                ("variant", _i32), ("block_k", _i32), ("chains_per_cta", _i32),
                ("use_graph", _i32), ("lambda0", _P), ("run_best", _i32),
                ("eta_decay", _f64), ("eta_sqrt", _i32), ("momentum", _f64)]


class sais_plan(ctypes.Structure):
    _fields_ = [("kernel", _i32), ("block_k", _i32), ("chains_per_cta", _i32), ("hilo", _i32)]


KERNEL_NAMES = {0: "plain", 1: "rank-k, W resident", 2: "rank-k, W streamed",
                3: "block fields by GEMM", 4: "launch groups", 5: "persistent"}


class sais_tuning(ctypes.Structure):
    _fields_ = [("groups", _i32), ("blocked_instances", _i32), ("plain_instances", _i32),
                ("reserved", _i32), ("group_variant", _i32 * 16), ("group_block_k", _i32 * 16),
                ("group_chains_per_cta", _i32 * 16), ("group_size", _i32 * 16),
                ("group_ms", _f64 * 16), ("group_spin_updates", _i64 * 16),
                ("persistent_ok", _i32), ("persistent", _i32), ("persistent_ms", _f64),
                ("groups_ms", _f64)]


class sais_solve_result(ctypes.Structure):
    _fields_ = [("best_cost", _P), ("best_x", _P), ("best_iter", _P), ("best_chain", _P),
                ("feasible_count", _P), ("lambda_final", _P), ("lambda_trace", _P),
                ("elapsed_ms", _f64), ("spin_updates", _i64)]


DEVICE_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, _i32, ctypes.c_void_p)
DEVICE_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, _i32, ctypes.c_void_p)

_SIGS = {
    "sais_describe": [ctypes.POINTER(sais_problem_desc), ctypes.POINTER(sais_problem_scalars)],
    "sais_create_problem": [ctypes.POINTER(sais_problem_desc), _i32, ctypes.POINTER(_P)],
    "sais_create_batch": [ctypes.POINTER(sais_problem_desc), _i32, _i32, ctypes.POINTER(_P)],
    "sais_destroy_problem": [_P],
    "sais_problem_info": [_P, ctypes.POINTER(sais_layout)],
    "sais_instance_scalars": [_P, _i32, ctypes.POINTER(sais_problem_scalars)],
    "sais_sample": [_P, ctypes.POINTER(sais_sample_params), _P, _P, _P, _P, _P, _P],
    "sais_sample_trace": [_P, ctypes.POINTER(sais_sample_params), _P, _P, _P, _P, _P, _P, _P],
    "sais_sample_run_best": [_P, ctypes.POINTER(sais_sample_params), _P, _P, _P, _P, _P, _P, _P,
                             _P, _P, _P],
    "sais_update_lambda": [_P, _P, _i32, _f64, _i32, _P, _P],
    "sais_update_lambda_rule": [_P, _P, _i32, _f64, _i32, _u32, _f64, _i32, _f64, _P, _P, _P],
    "sais_track_best": [_P, _P, _P, _P, _i32, _u32, _P, _P, _P, _P, _P, _P],
    "sais_solve": [_P, ctypes.POINTER(sais_solve_params), ctypes.POINTER(sais_solve_result), _P],
    "sais_synchronize": [_P, _P],
    "sais_sample_plan": [_P, ctypes.POINTER(sais_sample_params), ctypes.POINTER(sais_plan)],
    "sais_set_auto_mode": [_P, ctypes.c_int32],
    "sais_debug_check_selftest": [_P, _P],
    "sais_persistent_stats": [_P, _P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), _P],
    "sais_set_instance_chains": [_P, _P],
    "sais_autotune": [_P, _i32, _i32, ctypes.POINTER(sais_tuning), _P],
    "sais_solve_noalloc": [_P, ctypes.POINTER(sais_solve_params),
                           ctypes.POINTER(sais_solve_result), _P],
    "sais_constraint_features": [_P, _P, _i32, ctypes.POINTER(_i32)],
    "sais_mlp_create": [_i32, _u64, ctypes.POINTER(_P)],
    "sais_mlp_destroy": [_P],
    "sais_mlp_set_params": [_P, _P, _P],
    "sais_mlp_get_params": [_P, _P, _P],
    "sais_mlp_fit_normalization": [_P, _P, _P, _i32],
    "sais_mlp_forward": [_P, _P, _i32, _P, _P],
    "sais_mlp_gradient": [_P, _P, _P, _i32, _P, _P, _P],
    "sais_mlp_train_step": [_P, _P, _P, _i32, _f32, _P, _P],
    "sais_mlp_status": [_P],
    "sais_warm_start": [_P, _P, _P, _P],
    "sais_set_device_allocator": [DEVICE_ALLOC_FN, DEVICE_FREE_FN, _P],
}
MLP_PARAMS, MLP_FEATURES = 20612, 8
EXPORTS = list(_SIGS) + ["sais_status_string", "sais_last_error"]

_lib = None
_lock = threading.Lock()


class SaisError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: status {status}: {msg}")
        self.status = status


def lib(path: Optional[str] = None):
    """Open libsais.so (built by ``paper_2501_04971_gb300.build``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libsais is not built ({p} missing): run "
                               "paper_2501_04971_gb300.build.build() first")
        L = ctypes.CDLL(p)
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = _i32
        L.sais_status_string.argtypes = [_i32]
        L.sais_status_string.restype = ctypes.c_char_p
        L.sais_last_error.argtypes = []
        L.sais_last_error.restype = ctypes.c_char_p
        if path is None:
            _lib = L
        return L


def _check(st: int, where: str):
    if st != SAIS_OK:
        raise SaisError(st, where, lib().sais_last_error().decode())


# --- raw entry points, same names as the C-ABI ----------------------------------------------

def sais_describe(desc):
    out = sais_problem_scalars()
    _check(lib().sais_describe(ctypes.byref(desc), ctypes.byref(out)), "sais_describe")
    return out


def sais_create_problem(desc, device: int = 0):
    h = _P()
    _check(lib().sais_create_problem(ctypes.byref(desc), device, ctypes.byref(h)),
           "sais_create_problem")
    return h


def sais_create_batch(descs, device: int = 0):
    arr = (sais_problem_desc * len(descs))(*descs)
    h = _P()
    _check(lib().sais_create_batch(arr, len(descs), device, ctypes.byref(h)), "sais_create_batch")
    return h


def sais_destroy_problem(h):
    _check(lib().sais_destroy_problem(h), "sais_destroy_problem")


def sais_problem_info(h):
    out = sais_layout()
    _check(lib().sais_problem_info(h, ctypes.byref(out)), "sais_problem_info")
    return out


def sais_instance_scalars(h, index: int):
    out = sais_problem_scalars()
    _check(lib().sais_instance_scalars(h, index, ctypes.byref(out)), "sais_instance_scalars")
    return out


def sais_sample(h, prm, lam_ptr, x_ptr, cost_ptr, g_ptr, feas_ptr, stream_ptr):
    _check(lib().sais_sample(h, ctypes.byref(prm), lam_ptr, x_ptr, cost_ptr, g_ptr, feas_ptr,
                             stream_ptr), "sais_sample")


def sais_sample_trace(h, prm, lam_ptr, x_ptr, cost_ptr, g_ptr, feas_ptr, trace_ptr, stream_ptr):
    _check(lib().sais_sample_trace(h, ctypes.byref(prm), lam_ptr, x_ptr, cost_ptr, g_ptr,
                                   feas_ptr, trace_ptr, stream_ptr), "sais_sample_trace")


def sais_sample_run_best(h, prm, lam_ptr, x_ptr, cost_ptr, g_ptr, feas_ptr, run_x_ptr,
                         run_cost_ptr, run_sweep_ptr, run_nfeas_ptr, stream_ptr):
    _check(lib().sais_sample_run_best(h, ctypes.byref(prm), lam_ptr, x_ptr, cost_ptr, g_ptr,
                                      feas_ptr, run_x_ptr, run_cost_ptr, run_sweep_ptr,
                                      run_nfeas_ptr, stream_ptr), "sais_sample_run_best")


def sais_update_lambda(h, g_ptr, chains: int, eta: float, project: int, lam_ptr, stream_ptr):
    _check(lib().sais_update_lambda(h, g_ptr, chains, eta, project, lam_ptr, stream_ptr),
           "sais_update_lambda")


def sais_update_lambda_rule(h, g_ptr, chains: int, eta: float, project: int, it: int,
                            eta_decay: float, eta_sqrt: int, momentum: float, avg_ptr, lam_ptr,
                            stream_ptr):
    _check(lib().sais_update_lambda_rule(h, g_ptr, chains, eta, project, it, eta_decay,
                                         eta_sqrt, momentum, avg_ptr, lam_ptr, stream_ptr),
           "sais_update_lambda_rule")


def sais_track_best(h, x_ptr, cost_ptr, feas_ptr, chains: int, it: int, best_cost_ptr,
                    best_x_ptr, best_iter_ptr, best_chain_ptr, feas_count_ptr, stream_ptr):
    _check(lib().sais_track_best(h, x_ptr, cost_ptr, feas_ptr, chains, it, best_cost_ptr,
                                 best_x_ptr, best_iter_ptr, best_chain_ptr, feas_count_ptr,
                                 stream_ptr), "sais_track_best")


def sais_solve(h, prm, res, stream_ptr):
    _check(lib().sais_solve(h, ctypes.byref(prm), ctypes.byref(res), stream_ptr), "sais_solve")


def sais_solve_noalloc(h, prm, res, stream_ptr):
    _check(lib().sais_solve_noalloc(h, ctypes.byref(prm), ctypes.byref(res), stream_ptr),
           "sais_solve_noalloc")


def sais_sample_plan(h, prm) -> sais_plan:
    out = sais_plan()
    _check(lib().sais_sample_plan(h, ctypes.byref(prm), ctypes.byref(out)), "sais_sample_plan")
    return out


def sais_set_auto_mode(h, mode: int):
    _check(lib().sais_set_auto_mode(h, mode), "sais_set_auto_mode")


def sais_persistent_stats(h, cap: int, stream_ptr) -> np.ndarray:
    out = np.zeros((cap, 4), np.uint64)
    n = ctypes.c_int32(0)
    _check(lib().sais_persistent_stats(h, out.ctypes.data_as(_P), cap, ctypes.byref(n),
                                       stream_ptr), "sais_persistent_stats")
    return out[:min(cap, n.value)]


_allocator_keep: list = []


def sais_set_device_allocator(alloc=None, free=None):
    """Install Python callables alloc(bytes, device) -> int pointer (0 on failure) and
    free(ptr, bytes, device) as the library's device allocator; no arguments restores
    cudaMalloc / cudaFree.  The callables are kept alive here."""
    if alloc is None and free is None:
        _check(lib().sais_set_device_allocator(DEVICE_ALLOC_FN(), DEVICE_FREE_FN(), None),
               "sais_set_device_allocator")
        return
    fa = DEVICE_ALLOC_FN(lambda n, dev, ctx: alloc(n, dev) or None)
    ff = DEVICE_FREE_FN(lambda p, n, dev, ctx: free(p, n, dev))
    _allocator_keep.append((fa, ff))
    _check(lib().sais_set_device_allocator(fa, ff, None), "sais_set_device_allocator")


def sais_set_instance_chains(h, counts_ptr):
    _check(lib().sais_set_instance_chains(h, counts_ptr), "sais_set_instance_chains")


def sais_autotune(h, chains: int, sweeps: int, stream_ptr):
    out = sais_tuning()
    _check(lib().sais_autotune(h, chains, sweeps, ctypes.byref(out), stream_ptr), "sais_autotune")
    return out


def sais_constraint_features(h, rows_cap: int) -> np.ndarray:
    out = np.zeros((max(rows_cap, 1), MLP_FEATURES), np.float32)
    rows = _i32(0)
    _check(lib().sais_constraint_features(h, out.ctypes.data_as(_P), rows_cap,
                                          ctypes.byref(rows)), "sais_constraint_features")
    return out[:rows.value]


def sais_warm_start(h, mlp_h, lam_ptr, stream_ptr):
    _check(lib().sais_warm_start(h, mlp_h, lam_ptr, stream_ptr), "sais_warm_start")


def sais_synchronize(h, stream_ptr):
    _check(lib().sais_synchronize(h, stream_ptr), "sais_synchronize")


def sais_status_string(st: int) -> str:
    return lib().sais_status_string(st).decode()


def sais_last_error() -> str:
    return lib().sais_last_error().decode()


# --- convenience wrapper ------------------------------------------------------------------

def _desc(inst, keep: list) -> sais_problem_desc:
    """sais_problem_desc for an object with n, m, W, h, A, b, alpha, density (+ penalty, and
    b_tight: reduced capacities B' for capacity tightening)."""
    def arr(a, dt):
        if a is None:
            return None
        c = np.ascontiguousarray(a, dtype=dt)
        keep.append(c)
        return c.ctypes.data_as(_P)
    d = sais_problem_desc()
    d.n, d.m = int(inst.n), int(inst.m)
    d.W = arr(inst.W, np.int32)
    d.h = arr(inst.h, np.int32)
    d.A = arr(np.asarray(inst.A).reshape(inst.m, inst.n) if inst.m else None, np.int32)
    d.b = arr(inst.b if inst.m else None, np.int64)
    d.alpha = float(inst.alpha)
    d.density = float(inst.density)
    d.penalty = float(getattr(inst, "penalty", 0.0) or 0.0)
    bt = getattr(inst, "b_tight", None)
    d.b_tight = arr(bt if (bt is not None and inst.m) else None, np.int64)
    return d


def describe(inst) -> sais_problem_scalars:
    keep = []
    return sais_describe(_desc(inst, keep))


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return _P(s.cuda_stream)


class Problem:
    """A handle over one or more instances (``workloads.Instance``-like objects)."""

    def __init__(self, instances, device: int = 0):
        if not isinstance(instances, (list, tuple)):
            instances = [instances]
        keep: list = []
        descs = [_desc(i, keep) for i in instances]
        self.handle = sais_create_batch(descs, device)
        self.device = device
        self.layout = sais_problem_info(self.handle)
        self.count = self.layout.count
        self.words = self.layout.words
        self.m_stride = self.layout.m_stride
        self.scalars = [sais_instance_scalars(self.handle, j) for j in range(self.count)]

    def close(self):
        if self.handle:
            sais_destroy_problem(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _params(self, chains, sweeps, beta_max, seed, it, variant, block_k, chains_per_cta,
                debug_wait_polls=0):
        p = sais_sample_params()
        p.chains, p.sweeps, p.beta_max, p.iter, p.seed = chains, sweeps, beta_max, it, seed
        p.variant = _VARIANTS[variant] if isinstance(variant, str) else int(variant)
        p.block_k, p.chains_per_cta = block_k, chains_per_cta
        p.debug_wait_polls = debug_wait_polls
        return p

    def plan(self, chains: int, variant="blocked", block_k: int = 0,
             chains_per_cta: int = 0) -> dict:
        """The launch sais_sample would make (sais_sample_plan): kernel name, block size, CTA
        shape, hi/lo split."""
        pl = sais_sample_plan(self.handle, self._params(chains, 1, 1.0, 0, 0, variant, block_k,
                                                        chains_per_cta))
        return {"kernel": KERNEL_NAMES.get(pl.kernel, str(pl.kernel)), "block_k": pl.block_k,
                "chains_per_cta": pl.chains_per_cta, "hilo": bool(pl.hilo)}

    def set_auto_mode(self, mode: str):
        """sais_set_auto_mode: "persistent" (one launch when the batch fits it) or "groups"."""
        sais_set_auto_mode(self.handle, {"persistent": SAIS_AUTO_PERSISTENT,
                                         "groups": SAIS_AUTO_GROUPS}[mode])

    def persistent_stats(self, stream=None) -> dict:
        """sais_persistent_stats of the last persistent launch: per CTA start / end (global timer,
        ns), busy ns and items, plus the busy fraction of each CTA over the launch's span."""
        r = sais_persistent_stats(self.handle, 1024, _stream_ptr(stream)).astype(np.int64)
        span = int(r[:, 1].max() - r[:, 0].min()) if len(r) else 0
        busy = r[:, 2] / span if span > 0 else np.zeros(len(r))
        return {"ctas": len(r), "start_ns": r[:, 0], "end_ns": r[:, 1], "busy_ns": r[:, 2],
                "items": r[:, 3], "span_ns": span, "busy_fraction": busy}

    def blocked_kernel(self, block_k: int, chains: int = 128) -> str:
        """Name of the kernel the blocked sampler runs at this block size."""
        return self.plan(chains, "blocked", block_k)["kernel"]

    def set_instance_chains(self, counts=None):
        """sais_set_instance_chains: per-instance chain counts (None: one count for all)."""
        if counts is None:
            sais_set_instance_chains(self.handle, None)
            self.inst_chains = None
            return
        c = np.ascontiguousarray(counts, dtype=np.int32)
        assert c.size == self.count
        sais_set_instance_chains(self.handle, c.ctypes.data_as(_P))
        self.inst_chains = c

    def autotune(self, chains: int, sweeps: int = 20, stream=None):
        """sais_autotune: returns a dict of the per-group choices."""
        t = sais_autotune(self.handle, chains, sweeps, _stream_ptr(stream))
        g = t.groups
        return {"groups": g, "blocked_instances": t.blocked_instances,
                "plain_instances": t.plain_instances,
                "variant": list(t.group_variant)[:g], "block_k": list(t.group_block_k)[:g],
                "chains_per_cta": list(t.group_chains_per_cta)[:g],
                "size": list(t.group_size)[:g], "ms": list(t.group_ms)[:g],
                "spin_updates": list(t.group_spin_updates)[:g],
                "persistent_ok": bool(t.persistent_ok), "persistent": bool(t.persistent),
                "persistent_ms": t.persistent_ms, "groups_ms": t.groups_ms}

    @property
    def feature_rows(self) -> int:
        return int(sum(s.m for s in self.scalars))

    def features(self) -> np.ndarray:
        """sais_constraint_features: (sum_j m_j) x 8 host array."""
        return sais_constraint_features(self.handle, self.feature_rows)

    def warm_start(self, mlp: "MLP", lam, stream=None):
        """sais_warm_start: lam[j*m_stride + k] = max(0, network prediction)."""
        sais_warm_start(self.handle, mlp.handle, _P(lam.data_ptr()), _stream_ptr(stream))

    def synchronize(self, stream=None):
        """sais_synchronize: wait for the stream, raise SaisError on a device-side timeout."""
        sais_synchronize(self.handle, _stream_ptr(stream))

    def debug_check_selftest(self, stream=None):
        """sais_debug_check_selftest: queue a failing device-side check (debug builds)."""
        _check(lib().sais_debug_check_selftest(self.handle, _stream_ptr(stream)),
               "sais_debug_check_selftest")

    def alloc_outputs(self, chains: int, trace_sweeps: int = 0):
        import torch
        dev = torch.device("cuda", self.device)
        n = self.count * chains
        out = {
            "x": torch.empty(n * self.words, dtype=torch.int32, device=dev),
            "cost": torch.empty(n, dtype=torch.int64, device=dev),
            "g": torch.empty(n * self.m_stride, dtype=torch.int64, device=dev),
            "feasible": torch.empty(n, dtype=torch.uint8, device=dev),
        }
        if trace_sweeps:
            out["trace"] = torch.empty(n * trace_sweeps * self.words, dtype=torch.int32, device=dev)
        return out

    def alloc_run_best(self, chains: int):
        """Device outputs of sais_sample_run_best's best-in-run part."""
        import torch
        dev = torch.device("cuda", self.device)
        n = self.count * chains
        return {"x": torch.empty(n * self.words, dtype=torch.int32, device=dev),
                "cost": torch.empty(n, dtype=torch.int64, device=dev),
                "sweep": torch.empty(n, dtype=torch.int32, device=dev),
                "nfeas": torch.empty(n, dtype=torch.int32, device=dev)}

    def sample_run_best(self, lam, chains: int, sweeps: int, beta_max: float, seed: int,
                        it: int = 0, variant="plain", block_k: int = 0, chains_per_cta: int = 0,
                        out=None, run=None, stream=None):
        """sais_sample_run_best: the last samples as sample() returns them, plus "run": each
        chain's best feasible sweep-end state x [count, chains, words], its cost (INT64_MAX if
        none), sweep (-1 if none) and the number of feasible sweep ends."""
        prm = self._params(chains, sweeps, beta_max, seed, it, variant, block_k, chains_per_cta)
        o = out or self.alloc_outputs(chains)
        r = run or self.alloc_run_best(chains)
        sais_sample_run_best(self.handle, prm, _P(lam.data_ptr()), _P(o["x"].data_ptr()),
                             _P(o["cost"].data_ptr()), _P(o["g"].data_ptr()),
                             _P(o["feasible"].data_ptr()), _P(r["x"].data_ptr()),
                             _P(r["cost"].data_ptr()), _P(r["sweep"].data_ptr()),
                             _P(r["nfeas"].data_ptr()), _stream_ptr(stream))
        C = chains
        return {"x": o["x"].view(self.count, C, self.words),
                "cost": o["cost"].view(self.count, C),
                "g": o["g"].view(self.count, C, self.m_stride),
                "feasible": o["feasible"].view(self.count, C),
                "run": {"x": r["x"].view(self.count, C, self.words),
                        "cost": r["cost"].view(self.count, C),
                        "sweep": r["sweep"].view(self.count, C),
                        "nfeas": r["nfeas"].view(self.count, C)}}

    def sample(self, lam, chains: int, sweeps: int, beta_max: float, seed: int, it: int = 0,
               variant="plain", block_k: int = 0, chains_per_cta: int = 0, trace: bool = False,
               out=None, stream=None, debug_wait_polls: int = 0):
        """One annealing run per chain (sais_sample / sais_sample_trace); returns device tensors
        x [count, chains, words] (int32 bit patterns), cost [count, chains],
        g [count, chains, m_stride], feasible [count, chains] (and trace)."""
        prm = self._params(chains, sweeps, beta_max, seed, it, variant, block_k, chains_per_cta,
                           debug_wait_polls)
        o = out or self.alloc_outputs(chains, sweeps if trace else 0)
        sp = _stream_ptr(stream)
        args = (_P(lam.data_ptr()), _P(o["x"].data_ptr()), _P(o["cost"].data_ptr()),
                _P(o["g"].data_ptr()), _P(o["feasible"].data_ptr()))
        if trace:
            sais_sample_trace(self.handle, prm, *args, _P(o["trace"].data_ptr()), sp)
        else:
            sais_sample(self.handle, prm, *args, sp)
        C = chains
        res = {"x": o["x"].view(self.count, C, self.words),
               "cost": o["cost"].view(self.count, C),
               "g": o["g"].view(self.count, C, self.m_stride),
               "feasible": o["feasible"].view(self.count, C)}
        if trace:
            res["trace"] = o["trace"].view(self.count, C, sweeps, self.words)
        return res

    def update_lambda(self, g, chains: int, eta: float, project: bool, lam, stream=None):
        sais_update_lambda(self.handle, _P(g.data_ptr()), chains, eta, int(project),
                           _P(lam.data_ptr()), _stream_ptr(stream))

    def update_lambda_rule(self, g, chains: int, eta: float, project: bool, lam, it: int,
                           eta_decay: float = 0.0, eta_sqrt: bool = False,
                           momentum: float = 0.0, avg=None, stream=None):
        """sais_update_lambda_rule: the step with a decaying eta and an averaged subgradient
        (avg: FP64 device tensor [count*m_stride], zero before the first step)."""
        sais_update_lambda_rule(self.handle, _P(g.data_ptr()), chains, eta, int(project), it,
                                eta_decay, int(eta_sqrt), momentum,
                                _P(avg.data_ptr()) if avg is not None else None,
                                _P(lam.data_ptr()), _stream_ptr(stream))

    def alloc_best(self):
        """Device state of sais_track_best, initialised (best_cost INT64_MAX, indices -1)."""
        import torch
        dev = torch.device("cuda", self.device)
        return {"best_cost": torch.full((self.count,), np.iinfo(np.int64).max, dtype=torch.int64,
                                        device=dev),
                "best_x": torch.zeros(self.count * self.words, dtype=torch.int32, device=dev),
                "best_iter": torch.full((self.count,), -1, dtype=torch.int32, device=dev),
                "best_chain": torch.full((self.count,), -1, dtype=torch.int32, device=dev),
                "feasible_count": torch.zeros(self.count, dtype=torch.int64, device=dev)}

    def track_best(self, out: dict, chains: int, it: int, best: dict, stream=None):
        """The "store feasible x_k" step (sais_track_best) for samples `out` of sample(), or for
        the "run" part of sample_run_best() (no "feasible": a set cost marks a feasible one)."""
        feas = out.get("feasible")
        sais_track_best(self.handle, _P(out["x"].data_ptr()), _P(out["cost"].data_ptr()),
                        _P(feas.data_ptr()) if feas is not None else None, chains, it,
                        _P(best["best_cost"].data_ptr()), _P(best["best_x"].data_ptr()),
                        _P(best["best_iter"].data_ptr()), _P(best["best_chain"].data_ptr()),
                        _P(best["feasible_count"].data_ptr()), _stream_ptr(stream))

    def solve(self, iters: int, chains: int, sweeps: int, beta_max: float, eta: float,
              seed: int, iter0: int = 0, project: bool = True, lambda0=None, variant="plain",
              block_k: int = 0, chains_per_cta: int = 0, use_graph: bool = False,
              run_best: bool = False, eta_decay: float = 0.0, eta_sqrt: bool = False,
              momentum: float = 0.0, stream=None) -> dict:
        """Algorithm 1 on every instance (sais_solve); returns host numpy arrays.  run_best:
        keep each chain's best feasible sweep-end state instead of its last state; eta_decay,
        eta_sqrt, momentum: the step-size rule of sais_update_lambda_rule."""
        prm = sais_solve_params()
        prm.iters, prm.chains, prm.sweeps, prm.beta_max = iters, chains, sweeps, beta_max
        prm.eta, prm.seed, prm.iter0, prm.project_nonneg = eta, seed, iter0, int(project)
        prm.variant = _VARIANTS[variant] if isinstance(variant, str) else int(variant)
        prm.block_k, prm.chains_per_cta, prm.use_graph = block_k, chains_per_cta, int(use_graph)
        prm.run_best = int(run_best)
        prm.eta_decay, prm.eta_sqrt, prm.momentum = eta_decay, int(eta_sqrt), momentum
        l0 = None
        if lambda0 is not None:
            l0 = np.ascontiguousarray(np.asarray(lambda0, dtype=np.float32).reshape(-1))
            assert l0.size == self.count * self.m_stride
            prm.lambda0 = l0.ctypes.data_as(_P)
        cnt, W, M = self.count, self.words, self.m_stride
        out = {"best_cost": np.zeros(cnt, np.int64), "best_x": np.zeros((cnt, W), np.uint32),
               "best_iter": np.zeros(cnt, np.int32), "best_chain": np.zeros(cnt, np.int32),
               "feasible_count": np.zeros(cnt, np.int64),
               "lambda_final": np.zeros((cnt, M), np.float32),
               "lambda_trace": np.zeros((iters, cnt, M), np.float32)}
        res = sais_solve_result()
        for k, v in out.items():
            setattr(res, k, v.ctypes.data_as(_P))
        sais_solve(self.handle, prm, res, _stream_ptr(stream) if stream is not None else None)
        out["elapsed_ms"] = res.elapsed_ms
        out["spin_updates"] = res.spin_updates
        return out


def unpack_bits(words: np.ndarray, nspins: int) -> np.ndarray:
    """Bit-packed states [..., words] (spin i = bit i%32 of word i/32) -> uint8 [..., nspins]."""
    w = np.ascontiguousarray(words).view(np.uint32)
    bits = (w[..., :, None] >> np.arange(32, dtype=np.uint32)) & 1
    return bits.reshape(*w.shape[:-1], -1)[..., :nspins].astype(np.uint8)


class MLP:
    """The warm-start network (sais_mlp_*): device-resident BF16/FP32 parameters, Adam state."""

    def __init__(self, seed: int = 0, device: int = 0):
        h = _P()
        _check(lib().sais_mlp_create(device, seed, ctypes.byref(h)), "sais_mlp_create")
        self.handle, self.device = h, device

    def close(self):
        if self.handle:
            lib().sais_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        p = np.zeros(MLP_PARAMS, np.float32)
        n = np.zeros(16, np.float32)
        _check(lib().sais_mlp_get_params(self.handle, p.ctypes.data_as(_P), n.ctypes.data_as(_P)),
               "sais_mlp_get_params")
        return p, n

    def set_params(self, params, norm=None):
        p = np.ascontiguousarray(params, np.float32)
        assert p.size == MLP_PARAMS
        n = None if norm is None else np.ascontiguousarray(norm, np.float32)
        _check(lib().sais_mlp_set_params(self.handle, p.ctypes.data_as(_P),
                                         None if n is None else n.ctypes.data_as(_P)),
               "sais_mlp_set_params")

    def fit_normalization(self, X, y):
        X = np.ascontiguousarray(X, np.float32)
        y = np.ascontiguousarray(y, np.float32)
        _check(lib().sais_mlp_fit_normalization(self.handle, X.ctypes.data_as(_P),
                                                y.ctypes.data_as(_P), X.shape[0]),
               "sais_mlp_fit_normalization")

    def forward(self, X, out=None, stream=None):
        """X: device float32 tensor (rows x 8); returns the device predictions (rows)."""
        import torch
        y = out if out is not None else torch.empty(X.shape[0], dtype=torch.float32,
                                                    device=X.device)
        _check(lib().sais_mlp_forward(self.handle, _P(X.data_ptr()), X.shape[0],
                                      _P(y.data_ptr()), _stream_ptr(stream)), "sais_mlp_forward")
        return y

    def gradient(self, X, t, stream=None):
        import torch
        g = torch.empty(MLP_PARAMS, dtype=torch.float32, device=X.device)
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        _check(lib().sais_mlp_gradient(self.handle, _P(X.data_ptr()), _P(t.data_ptr()),
                                       X.shape[0], _P(g.data_ptr()), _P(loss.data_ptr()),
                                       _stream_ptr(stream)), "sais_mlp_gradient")
        return g, loss

    def train_step(self, X, t, lr: float, loss=None, stream=None):
        _check(lib().sais_mlp_train_step(self.handle, _P(X.data_ptr()), _P(t.data_ptr()),
                                         X.shape[0], lr,
                                         None if loss is None else _P(loss.data_ptr()),
                                         _stream_ptr(stream)), "sais_mlp_train_step")

    def status(self):
        _check(lib().sais_mlp_status(self.handle), "sais_mlp_status")
