"""The bounds-checked library (``-DVOFP_CHECKED``) on the GPU: a stand-in for a device memory checker.

Its kernels test the index of every guarded global-memory access against the array's extent and count the
failures in device words instead of making the access (``csrc/checked.cuh``).  The sweep re-runs the parity
files -- every kernel against the CPU oracle, tiny odd sizes (1, 2, 3, 5, 7 cells on an axis), all boundary
conditions, three precisions, the TMA and batched passes, the VoF update -- in a child process that loads the
checked library; the conftest hook asserts after each test that no index test failed.  The self-test makes
one test fail by construction (no memory access) and checks that it is recorded with its site, index and
extent, so a clean sweep means the checks ran, not that they were compiled out.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INSIDE = os.environ.get("VOFP_CHECKED") == "1"
FILES = ["tests/test_gpu_checked.py", "tests/test_gpu_parity.py", "tests/test_gpu_vof.py", "tests/test_gpu_vd.py",
         "tests/test_gpu_batch.py", "tests/test_gpu_mixed.py"]


@pytest.mark.skipif(not INSIDE, reason="runs inside the bounds-checked sweep (VOFP_CHECKED=1)")
def test_selftest_failure_is_recorded():
    import torch
    from paper_1907_00890_gb300 import vofp
    assert vofp.CHECKED and vofp.LIB.endswith("libvofp_checked.so")
    st, w = vofp.vofp_debug_check_word(reset=True)
    assert st == 1 and w["count"] == 0
    assert vofp.vofp_debug_check_selftest() == 0
    torch.cuda.synchronize()
    st, w = vofp.vofp_debug_check_word(reset=True)
    assert st == 1 and w == {"count": 1, "site": 99, "index": 5, "extent": 4}
    st, w = vofp.vofp_debug_check_word()
    assert w["count"] == 0  # cleared


@pytest.mark.skipif(INSIDE, reason="the sweep itself")
def test_bounds_checked_sweep_of_the_parity_files():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_00890_gb300 import build
    build.build(checked=True)
    env = dict(os.environ, VOFP_CHECKED="1")
    # the 512^3 refinement cases repeat kernels the smaller cases already run, at a minute each
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-m", "gpu", "-p", "no:cacheprovider", "-k", "not 512"] + FILES
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1500)
    tail = "\n".join((r.stdout + r.stderr).splitlines()[-25:])
    assert r.returncode == 0, tail
    assert " passed" in tail and "failed" not in tail, tail
