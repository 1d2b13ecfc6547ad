"""The debug build (device-side index and size checks, SAIS_DEBUG=1): its checked translation units
compile for sm_103a (no GPU needed; the GPU test runs the debug library)."""
import concurrent.futures as cf
import os
import subprocess

import pytest

from paper_2501_04971_gb300 import build as libbuild


@pytest.mark.parametrize("debug", [True])
def test_checked_sources_compile_with_sais_debug(tmp_path, debug):
    try:
        cc = libbuild.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    srcs = ["sais_post.cu", "sais_field.cu"]

    def one(src):
        cmd = [cc, *libbuild.ARCH, *libbuild.FLAGS, "-DSAIS_DEBUG=1", "-c",
               os.path.join(libbuild.CSRC, src), "-o", str(tmp_path / (src + ".o"))]
        return subprocess.run(cmd, capture_output=True, text=True)

    with cf.ThreadPoolExecutor(len(srcs)) as ex:
        for src, r in zip(srcs, ex.map(one, srcs)):
            assert r.returncode == 0, f"{src}:\n{r.stderr[-3000:]}"
            assert os.path.getsize(tmp_path / (src + ".o")) > 0
