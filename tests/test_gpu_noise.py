"""Exhaustive device check of the p-bit noise transform and its error bound (needs a GPU).

The samplers decide Eq. 10 as beta I + atanh(rho) > 0 with theta = atanh(rho) from a fast
hardware logarithm and a guard band; the guard is only rigorous if the bound on theta holds.
rho takes 2^24 values, so all of them are checked against FP64 atanh on the GPU itself.
"""
import os
import re
import subprocess

import pytest

from paper_2501_04971_gb300 import build as libbuild

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_noise_transform_bound_exhaustive(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    exe = str(tmp_path / "noise_bound")
    cmd = [libbuild.nvcc(), *libbuild.ARCH, "-O3", "-std=c++17", "-I", libbuild.INCLUDE, "-I",
           libbuild.CSRC, os.path.join(HERE, "cuda", "noise_bound.cu"), "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    print(r.stdout)
    m = re.search(r"values=(\d+) violations=(\d+) max_abs_err=(\S+) max_ratio=(\S+) "
                  r"rho_inexact=(\d+)", r.stdout)
    assert m, r.stdout + r.stderr
    assert int(m.group(1)) == 1 << 24
    assert int(m.group(2)) == 0, r.stdout
    assert int(m.group(5)) == 0, r.stdout
    assert float(m.group(4)) < 1.0
    assert r.returncode == 0
