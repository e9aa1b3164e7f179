"""The index-checking build (libmhd_debug.so, MHD_BOUNDS_CHECK): every
computed global-memory index of the step kernels (neighbour and closure
loads, assembly over shared DOFs, loads and stores of the stage kernels, the
images of walled states) is checked against its array; a bad one is counted
and redirected to element 0 instead of being made.  compute-sanitizer is
closed on this pool; this build stands in for its memory check on the paths
the parity tests take.  The run covers every (p, k) on 1 x 1, 1 x 3, 3 x 1,
2 x 2 and 5 x 3 meshes with every map on (full and reduced 2D2V stage),
walled contexts and a batch; no index may leave its array."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.gpu
def test_no_index_leaves_its_array():
    env = dict(os.environ, MHD_DEBUG_BUILD="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "debug_bounds_run.py")], capture_output=True,
                         text=True, timeout=900, env=env, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-3000:]
    res = json.loads([ln for ln in out.stdout.splitlines() if ln.startswith("{")][-1])
    assert res["runs"] > 80 and res["oob"] == 0, res
