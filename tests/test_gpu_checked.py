"""The bounds-checked build (-DPPMLR_CHECK; compute-sanitizer is not
available here): every shared-memory, staged-box, geometry and state index of
the sweep kernels is tested against its array on the cases of
checked_cases.py -- all launch forms, chunked and ragged tiles, the options
and the ensemble -- in a separate process that loads the checked library."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_no_kernel_index_leaves_its_array():
    from paper_1607_02214_gb300 import build
    lib = build.build(check=True)
    env = dict(os.environ, PPMLR_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_cases.py")], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "all cases OK" in r.stdout
