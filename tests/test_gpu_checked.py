"""The GPU parity tests again, on the bounds-checked build (libjpsi_checked.so:
every store whose index comes from data, a scan or a counter first tests the
index against its array, and a run whose kernels would have stored outside
an array fails with JPSI_ECUDA).  This stands in for a device memory checker:
the same oracle comparisons, on every tile, form and mode, run in a child
process that loads the checked library through JPSI_LIBRARY."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SUITES = ["tests/test_gpu_parity.py", "tests/test_gpu_paths.py", "tests/test_gpu_stream.py"]


def test_parity_suites_on_the_checked_build():
    import paper_1810_11966_gb300.build as b
    b.build()
    env = dict(os.environ, JPSI_LIBRARY=b.LIB_CHECKED)
    which = subprocess.run([sys.executable, "-c", "import paper_1810_11966_gb300 as jp; jp.load(); print(jp.LIB_PATH)"],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert which.returncode == 0 and which.stdout.strip() == b.LIB_CHECKED, which.stderr[-2000:]
    r = subprocess.run([sys.executable, "-m", "pytest", *SUITES, "-m", "gpu", "-q", "-x", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=3000)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    assert " passed" in r.stdout and "failed" not in r.stdout
