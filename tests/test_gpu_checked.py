"""Memory safety without a sanitizer: the parity cases of the ragged grids
(every tile shape, both precisions, grids from 3x3 up and smaller than a
tile), the wet/dry, periodic and inflow cases and a batch run on the
index-checked build, in a process of their own; every check word must stay
0 (no index out of range) and every result must still match the oracle."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_runs_the_parity_cases_with_no_index_out_of_range():
    lib = os.path.join(ROOT, "paper_2301_12010_gb300", "libswe_checked.so")
    assert os.path.exists(lib), "build the checked library first (__graft_entry__.build())"
    env = dict(os.environ, SWE_LIB_VARIANT="checked")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_cases.py")], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "CHECKED OK" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
