"""The debug build of the library: every kernel index checked on tiny boxes.

The library compiled with LBM_BOUNDS_CHECK replaces any index outside its
buffer by 0 and records it (lbm_check / lbm_batch_check return
LBM_ERR_BOUNDS); nothing traps.  tests/bounds_exercise.py runs every step kind
(two-pass, the single passes, the work list, batches, the no-alloc step, the
one-node kernels of an odd Nx) on 4^3 and 6 x 5 x 7 boxes, where every periodic
wrap is also a tile edge.  With the debug build every status must be LBM_OK,
and the results must equal the normal build's.
"""

import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _exercise(debug):
    env = dict(os.environ)
    env["LBM_DEBUG_LIBRARY"] = "1" if debug else "0"
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "bounds_exercise.py")], capture_output=True,
                       text=True, timeout=900, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads([line for line in r.stdout.splitlines() if line.startswith("{")][-1])


def test_debug_build_finds_no_index_outside_its_buffer():
    from paper_1805_08643_gb300 import _build

    _build.build()
    _build.build(debug=True)
    dbg = _exercise(True)
    ref = _exercise(False)
    assert set(dbg) == set(ref) and len(dbg) >= 55
    bad = {k: v["status"] for k, v in dbg.items() if any(s != 0 for s in v["status"])}
    assert not bad, f"statuses of the debug build (8 = LBM_ERR_BOUNDS): {bad}"
    for k in ref:
        a, b = dbg[k]["sum"], ref[k]["sum"]
        flat = lambda v: [x for y in v for x in (y if isinstance(y, list) else [y])]
        assert flat(a) == pytest.approx(flat(b), rel=1e-12, abs=1e-12), k
