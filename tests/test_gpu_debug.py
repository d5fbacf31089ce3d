"""The debug build on tiny lattices (GPU).

libxy_debug.so is the library compiled with -DXY_DEBUG: the two-pass sweep,
the layout conversions and the whole-lattice batch kernel check their index
arithmetic on the device, and a check that fails sets a bit of a device word
and skips the access instead of trapping (include/xy.h: xy_debug_checks).
A child process loads that build (XY_GB300_LIB) and runs the smallest sides,
where the index arithmetic has its edge cases (L = 2: each pair bonded twice;
L % 4 == 2: unpaired Philox draws): sweeps in lock step with the oracle,
batches bit-identical to single lattices, and no failed check.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0811_2111_gb300 import build as _build  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TESTS = os.path.join(ROOT, "tests")

CHILD = r"""
import ctypes as C, json, sys
import numpy as np
sys.path[:0] = [%(root)r, %(tests)r]
from paper_0811_2111_gb300 import _lib as X
from paper_0811_2111_gb300.lattice import Batch, Lattice
from gpu_util import ANGLE_TOL, lockstep_sweep

lib = X.lib()
assert lib.xy_debug_build() == 1, "not the debug build"
for L in (2, 4, 6, 10):
    with Lattice(L, 1.0, 3, algorithm="two_pass") as lat:
        before, t0 = lat.state()
        for i in range(3):
            lat.sweep(1)
            after, _ = lat.state()
            red, blk = lockstep_sweep(before, after, L, 1.0, 3, t0 + i)
            assert red.out_band_mismatch == 0 and blk.out_band_mismatch == 0, L
            assert max(red.max_angle_err, blk.max_angle_err) <= ANGLE_TOL, L
            before = after
Ls = [2, 4, 6, 10, 12, 16]
with Batch(Ls, [1.0] * len(Ls), 5, sweeps_per_round=3) as b:
    b.run(2)
    states = [b.state(i) for i in range(len(Ls))]
for i, L in enumerate(Ls):
    with Lattice(L, 1.0, 5, lattice_id=i, algorithm="two_pass") as lat:
        lat.sweep(6)
        s, _ = lat.state()
    assert np.array_equal(states[i], s), L
w = C.c_uint32(0xffffffff)
assert lib.xy_debug_checks(C.byref(w)) == 0
print(json.dumps({"failed_checks": w.value}))
"""


def test_debug_build_runs_tiny_lattices_without_a_failed_check():
    lib = _build.build(debug=True)
    env = dict(os.environ, XY_GB300_LIB=lib)
    r = subprocess.run([sys.executable, "-c", CHILD % {"root": ROOT, "tests": TESTS}],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["failed_checks"] == 0
