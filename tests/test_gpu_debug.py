"""The BLS_DEBUG build against the regular one (marked gpu).

libbls_debug.so is the same library with device-side checks on every histogram bin,
shared-memory row and TMEM column index of the search kernels (and on the unbinned
search's sort and run ends): a failed check skips or redirects the access and records an
error that makes the call fail with ERR_INTERNAL.  On the parity cases (plain, batched in
both kernels and every sum, phase and sign mode, the survey shape at two tile widths,
nb = 400, unbinned, served requests, the allocation-free search) every call of the debug
build succeeds -- no check fired -- and its results equal the regular build's bit for bit
(the checks change no arithmetic)."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1112_1701_b300 import build

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(out, debug):
    env = dict(os.environ)
    env.pop("BLS_DEBUG", None)
    if debug:
        env["BLS_DEBUG"] = "1"
    r = subprocess.run([sys.executable, "-m", "tests.debug_cases", out], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return np.load(out)


def test_debug_build_runs_clean_and_matches(tmp_path):
    build.build()
    reg = _run(str(tmp_path / "regular.npz"), False)
    dbg = _run(str(tmp_path / "debug.npz"), True)
    assert str(reg["lib"]).endswith("libbls.so")
    assert str(dbg["lib"]).endswith("libbls_debug.so")
    keys = [k for k in reg.files if k != "lib"]
    assert set(keys) == set(dbg.files) - {"lib"}
    for k in keys:
        assert np.array_equal(reg[k], dbg[k]), k
