"""The debug build (HSOLVE_DEBUG=1, -DHS_DEBUG) checks every global index its
tile engines form and reports ERR_BOUNDS instead of touching memory.  This
test builds it (into its own directory) and runs the tiny and ragged parity
cases of tests/debug_cases.py against it in a child process: every case must
match the oracle and no check may fire."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_debug_build_tiny_and_ragged_cases():
    pytest.importorskip("torch")
    env = dict(os.environ, HSOLVE_DEBUG="1")
    root = os.path.dirname(HERE)
    subprocess.run([sys.executable, "-c", "from paper_2305_05988_gb300 import _build; _build.build()"], cwd=root,
                   env=env, check=True, timeout=1200)
    out = subprocess.run([sys.executable, os.path.join(HERE, "debug_cases.py")], cwd=root, env=env,
                         capture_output=True, text=True, timeout=1200)
    assert out.returncode == 0, out.stdout[-2000:] + out.stderr[-4000:]
    assert "no bounds check fired" in out.stdout
