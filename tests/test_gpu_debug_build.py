"""The debug build (SAIS_DEBUG=1): device-side checks of indices and sizes in every sampler
kernel.  On valid inputs no check fires and every output equals the release build's; a check
that fails by construction (sais_debug_check_selftest) is reported by sais_synchronize as
SAIS_EBOUNDS with its source line and the status is reset.  The release build refuses the
self-test."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2501_04971_gb300 import build as libbuild, sais

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _run(tmp_path, debug):
    out = str(tmp_path / ("debug.npz" if debug else "release.npz"))
    env = dict(os.environ, SAIS_DEBUG="1" if debug else "0",
               PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, os.path.join(HERE, "gpu_debug_run.py"), out], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return dict(np.load(out))


def test_debug_build_matches_release_and_reports_checks(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    libbuild.build(debug=True)
    rel = _run(tmp_path, False)
    dbg = _run(tmp_path, True)
    assert int(rel["selftest"][0]) == -sais.SAIS_EUNSUPPORTED
    assert int(dbg["selftest"][0]) == sais.SAIS_EBOUNDS
    assert "check at line" in str(dbg["selftest_msg"][0])
    keys = [k for k in rel if not k.startswith("selftest")]
    assert keys
    for k in keys:
        assert np.array_equal(rel[k], dbg[k]), k
