"""Seeded synthetic instances shaped like the paper's knapsack workloads.

This module only draws integer data (profits, weights, capacities).  It holds none of the
method's arithmetic (no slack encoding, normalisation, penalty or sampling), so both the GPU
library's tests and the CPU oracle can be fed from it.

The paper benchmarks QKP instances with N in {100, 200, 300} and profit-matrix density
d in {0.25, 0.5, 0.75, 1} (Sec. IV-A) and MKP instances with N in {100, 250} items and
M in {5, 10} knapsacks (Sec. IV-B).  Those library instances are not available here; the
generators below produce random instances of the same shape:

* QKP: p_ij (i <= j) nonzero with probability d, uniform integer in [1, profit_max]; the
  diagonal gives the item values h_i = p_ii, the off-diagonal the symmetric pair values
  W_ij = W_ji = p_ij; weights w_i uniform in [1, 50]; capacity uniform in [50, sum w]; one
  constraint.
* MKP: a_ki uniform integer in [0, 1000], b_k = floor(0.25 sum_i a_ki) (at least 1),
  p_i = round(sum_k a_ki / m + 500 u_i) with u_i uniform in [0, 1).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional

import numpy as np


@dataclass
class Instance:
    """Integer knapsack instance: minimise -x^T W x / 2 - h^T x s.t. A x <= b."""
    n: int
    m: int
    W: Optional[np.ndarray]      # n x n int32 symmetric, zero diagonal; None = linear (MKP)
    h: np.ndarray                # n int32
    A: np.ndarray                # m x n int32
    b: np.ndarray                # m int64
    density: float               # generator density (QKP) or -1 (MKP: derived rule)
    alpha: float                 # penalty rule constant (QKP 2, MKP 5: Table I)
    name: str = ""


def _rng(*key: int) -> np.random.Generator:
    return np.random.default_rng([int(k) & 0xFFFFFFFF for k in key])


def qkp(n: int, density: float, seed: int, profit_max: int = 100, weight_max: int = 50,
        cap_min: int = 50) -> Instance:
    """QKP instance with n items, profit density `density` (see module doc)."""
    r = _rng(0x514B50, n, int(round(density * 1000)), profit_max, seed)
    mask = r.random((n, n)) < density
    vals = r.integers(1, profit_max + 1, size=(n, n))
    p = np.triu(np.where(mask, vals, 0))
    h = np.diag(p).astype(np.int32).copy()
    W = (p + p.T).astype(np.int32)
    np.fill_diagonal(W, 0)
    w = r.integers(1, weight_max + 1, size=n)
    hi = max(cap_min, int(w.sum()))
    cap = int(r.integers(min(cap_min, hi), hi + 1))
    return Instance(n=n, m=1, W=W, h=h, A=w.astype(np.int32)[None, :],
                    b=np.array([max(1, cap)], dtype=np.int64), density=float(density),
                    alpha=2.0, name=f"qkp-{n}-{int(round(density * 100))}-{seed}")


def mkp(n: int, m: int, seed: int, a_max: int = 1000, tightness: float = 0.25,
        bonus: float = 500.0) -> Instance:
    """MKP instance with n items and m knapsacks (see module doc)."""
    r = _rng(0x4D4B50, n, m, a_max, seed)
    a = r.integers(0, a_max + 1, size=(m, n))
    b = np.maximum(1, np.floor(tightness * a.sum(axis=1))).astype(np.int64)
    u = r.random(n)
    p = np.rint(a.sum(axis=0) / m + bonus * u).astype(np.int32)
    return Instance(n=n, m=m, W=None, h=p, A=a.astype(np.int32), b=b, density=-1.0,
                    alpha=5.0, name=f"mkp-{n}-{m}-{seed}")


# ---- the benchmark configurations -------------------------------------------------------

def qkp_n100_set(count: int = 10) -> List[Instance]:
    """QKP N=100, d=0.25 (parity configuration; instance seeds 0..count-1)."""
    return [qkp(100, 0.25, s) for s in range(count)]


def mkp_n250_m5(seed: int = 0) -> Instance:
    """MKP N=250, m=5 (parity configuration)."""
    return mkp(250, 5, seed)


def qkp_n300_batch(per_density: int = 256, densities=(0.25, 0.5, 0.75, 1.0)) -> List[Instance]:
    """QKP N=300 at the four densities, `per_density` instances each (throughput workload)."""
    return [qkp(300, d, s) for d in densities for s in range(per_density)]


def ragged_batch(n_qkp: int = 384, n_mkp: int = 128, seed: int = 0) -> List[Instance]:
    """Ragged mix: QKP with N uniform in [100, 1000] and profits up to 10^4, plus MKP with
    N in {250, 500} and m in {5, 10, 30}."""
    r = _rng(0x524147, n_qkp, n_mkp, seed)
    out = []
    for i in range(n_qkp):
        n = int(r.integers(100, 1001))
        d = float(r.choice([0.25, 0.5, 0.75, 1.0]))
        out.append(qkp(n, d, 1000 + i, profit_max=10000))
    for i in range(n_mkp):
        n = int(r.choice([250, 500]))
        m = int(r.choice([5, 10, 30]))
        out.append(mkp(n, m, 1000 + i))
    return out
