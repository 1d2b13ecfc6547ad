"""CPU oracle of the Self-Adaptive Ising Machine (SAIM), arXiv 2501.04971.

TEST INFRASTRUCTURE ONLY.  The tests, the smoke check of the package entry point and the
benchmark's CPU-baseline leg are the only users of this package.  It wraps ``saim_oracle.c``
(plain C, FP64 fields, int64 objective/constraint values, its own Philox4x32-10) through
ctypes; it shares no code with the GPU library and imports nothing from it.

Every function names the passage of the paper it follows (section, equation, algorithm, table).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "saim_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "mlp_oracle.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsaim_oracle.so")
_lock = threading.Lock()
_lib = None

# Flags: FP64 evaluated exactly as written (no fused multiply-add), no fast-math, OpenMP over
# chains.  Portable across x86-64 and aarch64 (no -march=native).
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
          "-fopenmp", "-Wall", "-Wextra", "-Wno-unused-parameter"]


def build(force: bool = False, src: Optional[str] = None, out: str = _LIB_PATH,
          extra_flags: Optional[list] = None) -> str:
    """Compile the oracle with gcc into ``out`` (default: oracle/_build/libsaim_oracle.so).
    ``src`` replaces saim_oracle.c (the mutation tests build altered copies of it)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    srcs = [src or _SRC] + _SRCS[1:]
    if (not force and os.path.exists(out)
            and all(os.path.getmtime(out) >= os.path.getmtime(f) for f in srcs)
            and not extra_flags):
        return out
    cmd = ["gcc", *CFLAGS, *(extra_flags or []), *srcs, "-o", out + ".tmp", "-lm"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    os.replace(out + ".tmp", out)
    return out


_P = ctypes.c_void_p
_i32, _i64, _u32, _u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
_f32, _f64 = ctypes.c_float, ctypes.c_double

_SIGS = {
    "or_slack_bits": (_i32, [_i64]),
    "or_num_spins": (_i32, [_i32, _i32, _P]),
    "or_extend": (None, [_i32, _i32, _P, _P, _i32, _P]),
    "or_scales": (None, [_i32, _i32, _P, _P, _P, _P, _i32, _f32, _f32, _f32, _P, _P]),
    "or_cost": (_i64, [_i32, _P, _P, _P]),
    "or_constraints": (None, [_i32, _i32, _P, _P, _P, _P]),
    "or_feasible": (_i32, [_i32, _i32, _P, _P, _P]),
    "or_lagrangian": (_f64, [_i32, _i32, _i32, _P, _P, _P, _P, _P, _f32, _f32, _f32, _P]),
    "or_ising": (_f64, [_i32, _i32, _i32, _P, _P, _P, _P, _P, _f32, _f32, _f32, _P, _P]),
    "or_ising_energy": (_f64, [_i32, _P, _P, _P]),
    "or_philox4x32_10": (None, [_P, _P, _P]),
    "or_rand_pm1": (_f64, [_u32]),
    "or_pbit_noise": (_f64, [_u64, _u32, _u32, _u32, _u32]),
    "or_beta": (_f32, [_f32, _i32, _i32]),
    "or_anneal": (None, [_i32, _P, _P, _f32, _i32, _u64, _u32, _i32, _i32, _P, _P]),
    "or_gibbs_fixed": (None, [_i32, _P, _P, _f32, _i32, _u64, _u32, _i64, _P]),
    "or_replay_sweep": (_i32, [_i32, _P, _P, _f32, _u64, _u32, _u32, _u32, _P, _P, _P, _P,
                               _i32]),
    "or_lambda_update": (None, [_i32, _P, _i64, _f64, _i32, _f32, _P]),
    "or_lambda_update_rule": (None, [_i32, _P, _i64, _f64, _i32, _f32, _u32, _f64, _i32, _f64,
                                     _P, _P]),
    "or_run_best": (None, [_i32, _i32, _i32, _P, _P, _P, _P, _i32, _i32, _P, _P, _P, _P, _P]),
    "or_solve": (None, [_i32, _i32, _P, _P, _P, _P, _P, _f32, _f32, _f32, _i32, _i32, _i32,
                        _f32, _f64, _u64, _u32, _i32, _i32, _f64, _i32, _f64, _P, _P, _P, _P,
                        _P, _P, _P, _P, _P]),
    "or_enumerate_lagrangian": (None, [_i32, _i32, _i32, _P, _P, _P, _P, _P, _f32, _f32, _f32,
                                       _P]),
    "or_brute_force_opt": (_i64, [_i32, _i32, _P, _P, _P, _P, _P]),
    "or_bf16_round": (_f32, [_f32]),
    "or_set_threads": (None, [_i32]),
    "or_max_threads": (_i32, []),
    "or_features": (None, [_i32, _i32, _P, _P, _P, _P, _f32, _f32, _f32, _P]),
    "or_mlp_forward": (None, [_P, _P, _P, _i32, _i32, _P]),
    "or_mlp_grad": (_f64, [_P, _P, _P, _P, _i32, _i32, _P]),
    "or_adam_step": (None, [_i32, _P, _P, _P, _P, _i32, _f64, _f64, _f64, _f64]),
}


def load(path: Optional[str] = None):
    """Load (building first if needed) the oracle shared library and declare its signatures."""
    global _lib
    with _lock:
        if path is None and _lib is not None:
            return _lib
        p = path or build()
        lib = ctypes.CDLL(p)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if path is None:
            _lib = lib
        return lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


@dataclass
class Problem:
    """An integer instance of Eq. 2 in the knapsack form of Sec. IV: minimise
    -x^T W x / 2 - h^T x subject to A x <= b (W None for the linear MKP objective), extended
    with binary slack spins (Sec. IV-A) and normalised (Sec. IV-A/B)."""
    n: int
    m: int
    W: Optional[np.ndarray]
    h: np.ndarray
    A: np.ndarray
    b: np.ndarray
    alpha: float = 2.0
    density: float = -1.0
    penalty: float = 0.0
    # Capacities that feasibility is checked against (None: b).  Capacity tightening B' < B
    # (Sec. IV-B): b holds the reduced B' that L is built from, b_check the true B.
    b_check: Optional[np.ndarray] = None

    def __post_init__(self):
        lib = load()
        self.W = _c(self.W, np.int64)
        self.h = _c(self.h, np.int64)
        self.A = _c(np.asarray(self.A).reshape(self.m, self.n), np.int64)
        self.b = _c(self.b, np.int64)
        self.b_check = _c(self.b if self.b_check is None else self.b_check, np.int64)
        self.nprime = int(lib.or_num_spins(self.n, self.m, _ptr(self.b)))
        self.Q = np.array([lib.or_slack_bits(int(v)) for v in self.b], dtype=np.int32)
        self.Aext = np.zeros((self.m, self.nprime), dtype=np.int64)
        lib.or_extend(self.n, self.m, _ptr(self.A), _ptr(self.b), self.nprime, _ptr(self.Aext))
        sc = np.zeros(3, dtype=np.float32)
        d = np.zeros(1, dtype=np.float64)
        lib.or_scales(self.n, self.m, _ptr(self.W), _ptr(self.h), _ptr(self.A), _ptr(self.b),
                      self.nprime, self.alpha, self.density, self.penalty, _ptr(sc), _ptr(d))
        self.sigma_f, self.sigma_g, self.P = (np.float32(v) for v in sc)
        self.d_used = float(d[0])

    # --- Sec. IV-A, Eq. 12-13 -------------------------------------------------------------
    def cost(self, x) -> int:
        x = _c(x, np.uint8)
        return int(load().or_cost(self.n, _ptr(self.W), _ptr(self.h), _ptr(x)))

    def constraints(self, x) -> np.ndarray:
        x = _c(x, np.uint8)
        g = np.zeros(self.m, dtype=np.int64)
        load().or_constraints(self.m, self.nprime, _ptr(self.Aext), _ptr(self.b), _ptr(x), _ptr(g))
        return g

    def feasible(self, x) -> bool:
        x = _c(x, np.uint8)
        return bool(load().or_feasible(self.n, self.m, _ptr(self.A), _ptr(self.b_check),
                                       _ptr(x)))

    # --- Eq. 3 and 5 ----------------------------------------------------------------------
    def lagrangian(self, x, lam) -> float:
        x = _c(x, np.uint8)
        lam = _c(lam, np.float32)
        return float(load().or_lagrangian(self.n, self.m, self.nprime, _ptr(self.W), _ptr(self.h),
                                          _ptr(self.Aext), _ptr(self.b), _ptr(lam),
                                          self.sigma_f, self.sigma_g, self.P, _ptr(x)))

    # --- Eq. 1 ----------------------------------------------------------------------------
    def ising(self, lam):
        """(J, h, const) with L(x) = H(2x-1) + const (Eq. 1 and 5)."""
        lam = _c(lam, np.float32)
        J = np.zeros((self.nprime, self.nprime), dtype=np.float64)
        hI = np.zeros(self.nprime, dtype=np.float64)
        cst = load().or_ising(self.n, self.m, self.nprime, _ptr(self.W), _ptr(self.h),
                              _ptr(self.Aext), _ptr(self.b), _ptr(lam), self.sigma_f,
                              self.sigma_g, self.P, _ptr(J), _ptr(hI))
        return J, hI, float(cst)

    def enumerate_lagrangian(self, lam) -> np.ndarray:
        """L(x) for every state (x_i = bit i of the index), N' <= 24."""
        assert self.nprime <= 24
        lam = _c(lam, np.float32)
        L = np.zeros(1 << self.nprime, dtype=np.float64)
        load().or_enumerate_lagrangian(self.n, self.m, self.nprime, _ptr(self.W), _ptr(self.h),
                                       _ptr(self.Aext), _ptr(self.b), _ptr(lam), self.sigma_f,
                                       self.sigma_g, self.P, _ptr(L))
        return L

    def brute_force_opt(self):
        """OPT of Eq. 2 by enumeration of the items (n <= 24): (cost, x) or (None, None)."""
        assert self.n <= 24
        x = np.zeros(self.n, dtype=np.uint8)
        v = load().or_brute_force_opt(self.n, self.m, _ptr(self.W), _ptr(self.h), _ptr(self.A),
                                      _ptr(self.b), _ptr(x))
        if v == np.iinfo(np.int64).max:
            return None, None
        return int(v), x


def ising_energy(J: np.ndarray, hI: np.ndarray, x) -> float:
    x = _c(x, np.uint8)
    return float(load().or_ising_energy(len(hI), _ptr(np.ascontiguousarray(J)),
                                        _ptr(np.ascontiguousarray(hI)), _ptr(x)))


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    load().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def rand_pm1(word: int) -> float:
    return float(load().or_rand_pm1(int(word) & 0xFFFFFFFF))


def pbit_noise(seed: int, it: int, chain: int, sweep: int, spin: int) -> float:
    return float(load().or_pbit_noise(seed, it, chain, sweep, spin))


def beta(beta_max: float, t: int, T: int) -> np.float32:
    return np.float32(load().or_beta(beta_max, t, T))


def anneal(J, hI, beta_max: float, T: int, seed: int, it: int, nchains: int, chain0: int = 0,
           trace: bool = False):
    """Annealing runs of Sec. III-B; returns x (nchains x N' uint8) and optionally the trace
    (nchains x T x N')."""
    N = len(hI)
    J = np.ascontiguousarray(J, dtype=np.float64)
    hI = np.ascontiguousarray(hI, dtype=np.float64)
    x = np.zeros((nchains, N), dtype=np.uint8)
    tr = np.zeros((nchains, T, N), dtype=np.uint8) if trace else None
    load().or_anneal(N, _ptr(J), _ptr(hI), beta_max, T, seed, it, chain0, nchains, _ptr(x),
                     _ptr(tr))
    return (x, tr) if trace else x


def gibbs_fixed(J, hI, beta_: float, sweeps: int, seed: int, nchains: int, it: int = 0):
    N = len(hI)
    assert N <= 32
    J = np.ascontiguousarray(J, dtype=np.float64)
    hI = np.ascontiguousarray(hI, dtype=np.float64)
    out = np.zeros(nchains, dtype=np.uint32)
    load().or_gibbs_fixed(N, _ptr(J), _ptr(hI), beta_, sweeps, seed, it, nchains, _ptr(out))
    return out


def replay_sweep(J, hI, beta_: float, seed: int, it: int, chain: int, t: int, x0, x1,
                 max_out: int = 64):
    """Teacher-forced replay (see saim_oracle.c): (n_disagree, spins, margins)."""
    N = len(hI)
    x0 = _c(x0, np.uint8)
    x1 = _c(x1, np.uint8)
    spins = np.zeros(max_out, dtype=np.int32)
    margins = np.zeros(max_out, dtype=np.float64)
    nbad = load().or_replay_sweep(N, _ptr(np.ascontiguousarray(J)), _ptr(np.ascontiguousarray(hI)),
                                  beta_, seed, it, chain, t, _ptr(x0), _ptr(x1), _ptr(spins),
                                  _ptr(margins), max_out)
    k = min(nbad, max_out)
    return int(nbad), spins[:k].copy(), margins[:k].copy()


def run_best(p: Problem, trace):
    """Best feasible sweep-end state of every run (see or_run_best in saim_oracle.c) from a
    trace (C x T x N' bytes, as returned by anneal): (cost C, states C x N', sweep C,
    feasible sweep-end states C); cost INT64_MAX, state 0 and sweep -1 where none."""
    tr = _c(trace, np.uint8)
    C, T, N = tr.shape
    assert N == p.nprime
    cost = np.zeros(C, np.int64)
    x = np.zeros((C, N), np.uint8)
    sweep = np.zeros(C, np.int32)
    nfeas = np.zeros(C, np.int32)
    load().or_run_best(p.n, p.m, N, _ptr(p.W), _ptr(p.h), _ptr(p.A), _ptr(p.b_check), C, T,
                       _ptr(tr), _ptr(cost), _ptr(x), _ptr(sweep), _ptr(nfeas))
    return cost, x, sweep, nfeas


def lambda_update(gsum, C: int, eta: float, project: bool, sigma_g, lam) -> np.ndarray:
    """Algorithm 1's multiplier step (batch mean, optional projection); returns the new lambda."""
    g = _c(gsum, np.int64)
    out = np.array(lam, dtype=np.float32, copy=True)
    load().or_lambda_update(len(out), _ptr(g), C, eta, int(project), np.float32(sigma_g),
                            _ptr(out))
    return out


def lambda_update_rule(gsum, C: int, eta: float, project: bool, sigma_g, lam, it: int,
                       decay: float = 0.0, eta_sqrt: bool = False, mu: float = 0.0, avg=None):
    """The multiplier step with a step-size rule (or_lambda_update_rule): returns the new
    lambda; `avg` (FP64 array, the averaged subgradient) is updated in place when mu != 0."""
    g = _c(gsum, np.int64)
    out = np.array(lam, dtype=np.float32, copy=True)
    if mu != 0.0:
        assert avg is not None and avg.dtype == np.float64 and avg.flags.c_contiguous
    load().or_lambda_update_rule(len(out), _ptr(g), C, eta, int(project), np.float32(sigma_g),
                                 it, decay, int(eta_sqrt), mu, _ptr(avg), _ptr(out))
    return out


@dataclass
class SolveResult:
    best_cost: Optional[int]
    best_x: Optional[np.ndarray]
    best_iter: int
    best_chain: int
    lambda_trace: np.ndarray
    feasible_count: int
    costs: Optional[np.ndarray]
    g: Optional[np.ndarray]


def solve(p: Problem, K: int, C: int, T: int, beta_max: float, eta: float, seed: int,
          iter0: int = 0, project: bool = True, lambda0=None, keep_samples: bool = False,
          run_best: bool = False, eta_decay: float = 0.0, eta_sqrt: bool = False,
          momentum: float = 0.0):
    """Algorithm 1 (Sec. III-A) with the p-bit machine of Sec. III-B as the minimiser.
    Feasibility is checked against p.b_check; run_best stores each chain's best feasible
    sweep-end state instead of its last state; eta_decay, eta_sqrt and momentum select the
    step-size rule of lambda_update_rule (the average starts at 0 in every call)."""
    lib = load()
    bc = np.zeros(1, dtype=np.int64)
    bx = np.zeros(p.nprime, dtype=np.uint8)
    bi = np.zeros(1, dtype=np.int32)
    bch = np.zeros(1, dtype=np.int32)
    lt = np.zeros((K, p.m), dtype=np.float32)
    fc = np.zeros(1, dtype=np.int64)
    costs = np.zeros((K, C), dtype=np.int64) if keep_samples else None
    gs = np.zeros((K, C, p.m), dtype=np.int64) if keep_samples else None
    l0 = _c(lambda0, np.float32)
    lib.or_solve(p.n, p.m, _ptr(p.W), _ptr(p.h), _ptr(p.A), _ptr(p.b), _ptr(p.b_check),
                 p.alpha, p.density, p.penalty, K, C, T, beta_max, eta, seed, iter0,
                 int(project), int(run_best), eta_decay, int(eta_sqrt), momentum, _ptr(l0),
                 _ptr(bc), _ptr(bx), _ptr(bi), _ptr(bch), _ptr(lt), _ptr(fc), _ptr(costs),
                 _ptr(gs))
    found = int(bc[0]) != np.iinfo(np.int64).max
    return SolveResult(int(bc[0]) if found else None, bx if found else None, int(bi[0]),
                       int(bch[0]), lt, int(fc[0]), costs, gs)


# --------------------------------------------------------------------------------------------
# Learned multiplier warm start (no counterpart in the paper; see mlp_oracle.c)
# --------------------------------------------------------------------------------------------
MLP_PARAMS, MLP_HIDDEN = 20612, 128
MLP_OFF_W1, MLP_OFF_W2, MLP_OFF_W3, MLP_OFF_B3 = 0, 2048, 20480, 20608
MLP_BF16, MLP_ABS = 1, 2


def set_threads(n: int) -> None:
    """Threads of the oracle's OpenMP loops (timing only; results do not depend on it)."""
    load().or_set_threads(int(n))


def max_threads() -> int:
    return int(load().or_max_threads())


def bf16_round(v: float) -> float:
    """FP32 -> BF16, round to nearest even (returned as FP32)."""
    return float(load().or_bf16_round(float(v)))


def features(p: "Problem") -> np.ndarray:
    """Per-constraint features (m x 8) of Sec. IV-A's normalised instance (mlp_oracle.c)."""
    out = np.zeros((p.m, 8), np.float32)
    load().or_features(p.n, p.m, _ptr(p.W), _ptr(p.h), _ptr(p.A), _ptr(p.b), p.alpha,
                       p.density, p.penalty, _ptr(out))
    return out


def mlp_forward(params, norm, X, flags: int = 0) -> np.ndarray:
    """lambda predicted for each row of X (rows x 8), FP64."""
    params, norm, X = _c(params, np.float32), _c(norm, np.float32), _c(X, np.float32)
    y = np.zeros(X.shape[0], np.float64)
    load().or_mlp_forward(_ptr(params), _ptr(norm), _ptr(X), X.shape[0], flags, _ptr(y))
    return y


def mlp_grad(params, norm, X, t, flags: int = 0):
    """(loss, gradient[MLP_PARAMS]) of the mean squared error on normalised targets, FP64."""
    params, norm, X, t = (_c(params, np.float32), _c(norm, np.float32), _c(X, np.float32),
                          _c(t, np.float32))
    g = np.zeros(MLP_PARAMS, np.float64)
    loss = load().or_mlp_grad(_ptr(params), _ptr(norm), _ptr(X), _ptr(t), X.shape[0], flags,
                              _ptr(g))
    return float(loss), g


def adam_step(theta, mom, vel, g, t: int, lr: float, b1: float = 0.9, b2: float = 0.999,
              eps: float = 1e-8):
    """One Adam step in place on FP64 arrays (Kingma & Ba, Algorithm 1)."""
    for a in (theta, mom, vel):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = _c(g, np.float64)
    load().or_adam_step(theta.size, _ptr(theta), _ptr(mom), _ptr(vel), _ptr(g), t, lr, b1, b2,
                        eps)
