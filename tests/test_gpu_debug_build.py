"""The bounds-checked debug build (compiled with HMI_DEBUG) on tiny and ragged
frames, with guard bands around every output buffer; run in a child process
so that the test process keeps the regular library.  See
tests/debug_build_check.py."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_debug_build_bounds_checks_and_guard_bands():
    env = dict(os.environ, HMI_DEBUG_BUILD="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "debug_build_check.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout[-2000:] + r.stderr[-2000:]
