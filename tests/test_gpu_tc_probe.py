"""The tcgen05 MMA instruction-cost measurement behind the choice between the rank-k and the
block-field samplers (needs a GPU; a measurement, so the checks are on its form and on the
one property the dispatch relies on, not on exact cycle counts).

tests/cuda/mma_issue_cost.cu times chains of M = 128 MMAs for N = 16..256 and 19 MMAs spread
over independent accumulators.  The rank-k sampler updates 128 chains' fields with two wide
MMAs per block; the block-field sampler needs ceil(n/16) narrow ones.  That trade only favours
the rank-k update if a narrow MMA costs about as much as a wide one, which is checked here.
"""
import os
import re
import subprocess

import pytest

from paper_2501_04971_gb300 import build as libbuild

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_mma_issue_cost_probe(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    exe = str(tmp_path / "mma_issue_cost")
    cmd = [libbuild.nvcc(), *libbuild.ARCH, "-O3", "-std=c++17", "-I", libbuild.INCLUDE, "-I",
           libbuild.CSRC, os.path.join(HERE, "cuda", "mma_issue_cost.cu"), "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    chain = {(a, int(n), int(k)): int(c) for a, n, k, c in
             re.findall(r"chain A=(\w+) N=(\d+) R=(\d+) cycles=(\d+)", r.stdout)}
    split = {(int(n), int(p)): int(c) for n, p, c in
             re.findall(r"split N=(\d+) R=19 P=(\d+) cycles=(\d+)", r.stdout)}
    assert len(chain) == 60 and len(split) == 9
    # 19 narrow MMAs cost far more than one, whatever N: the instruction count dominates
    for n in (16, 32, 64, 128):
        assert chain[("tmem", n, 19)] > 3 * chain[("tmem", n, 1)]
    assert chain[("tmem", 16, 19)] > 0.5 * chain[("tmem", 128, 19)]
