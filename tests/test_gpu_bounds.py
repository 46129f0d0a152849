"""Bounds-checked run of the kernels (compute-sanitizer is not available
where this library is tested): the library built with -DWBLBE_DEBUG_BOUNDS
checks every global access of the step, moments and batched kernels, and the
run-time shared-memory slots, before making it.  A fresh process runs the
edge-case workloads of bounds_workload.py on that build; no access may fall
outside its buffer.  Collected before test_zz_no_alloc.py."""
import json
import os
import subprocess
import sys

import pytest

from paper_2012_11075_gb300 import _build, wblbe

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_regular_build_has_no_checks():
    from tests.gpu_helpers import need_gpu
    need_gpu()
    assert wblbe.debug_bounds_errors() == 0xFFFFFFFF


def test_edge_cases_stay_in_bounds():
    from tests.gpu_helpers import need_gpu
    need_gpu()
    lib = _build.build(debug_bounds=True)
    env = dict(os.environ, WBLBE_LIBRARY=str(lib),
               PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    out = subprocess.run([sys.executable, "-m", "tests.bounds_workload"], cwd=ROOT, env=env,
                         capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    res = json.loads(out.stdout.strip().splitlines()[-1])
    assert res["runs"] > 70
    assert res["errors"] == 0, res
