"""The bounds-checked build (RELO_CHECKED=1: guarded accesses check their index, count a failure
and skip the access; the stand-in for a device memory checker) runs the parity, fusion, limit,
global-rendering and fault tests, which must pass and leave zero failed checks."""
import os
import subprocess
import sys

import pytest

from paper_1801_08361_gb300 import build

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SUITES = ["tests/test_gpu_parity.py", "tests/test_gpu_fusion.py", "tests/test_gpu_limits.py",
          "tests/test_gpu_render_global.py", "tests/test_gpu_faults.py"]


def test_checked_build_runs_the_gpu_suites_without_a_failed_check(tmp_path):
    build.build_cuda(checked=True)
    report = tmp_path / "checks.txt"
    env = dict(os.environ, RELO_CHECKED="1", RELO_CHECK_REPORT=str(report))
    out = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider"] + SUITES,
                         cwd=ROOT, env=env, capture_output=True, text=True)
    assert out.returncode == 0, out.stdout[-3000:] + out.stderr[-2000:]
    assert report.read_text().strip() == "0"
