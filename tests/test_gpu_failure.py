"""Out-of-memory paths of every engine, provoked on the host (GPU).

xy_debug_fail_alloc(k) makes the k-th device allocation of the library fail
as if the device were out of memory, without reaching the driver.  For each
engine every allocation of its create call is made to fail in turn: the call
must return XY_ENOMEM, free what it had allocated (device memory back to
where it was) and leave the device usable: afterwards the same engine is
created normally and its sweep checked against the oracle in lock step.
Nothing here faults or exhausts the GPU.
"""
import ctypes as C
import math

import numpy as np
import pytest

from gpu_util import ANGLE_TOL, lockstep_sweep

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0811_2111_gb300 import build as _build  # noqa: E402

_build.build()
from paper_0811_2111_gb300 import _lib as X  # noqa: E402
from paper_0811_2111_gb300.hmc import HMC  # noqa: E402
from paper_0811_2111_gb300.lattice import Batch, Lattice, Quad  # noqa: E402


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _fail_each_allocation(make, max_allocs=40):
    """Make allocation 1, 2, ... of `make()` fail until it succeeds unarmed;
    returns the number of allocations the create call makes."""
    lib = X.lib()
    before = _free_bytes()
    for k in range(1, max_allocs + 1):
        assert lib.xy_debug_fail_alloc(k) == X.XY_OK
        try:
            obj = make()
        except X.XYError as e:
            assert e.status == X.XY_ENOMEM, (k, str(e))
            continue
        finally:
            lib.xy_debug_fail_alloc(0)
        # the k-th allocation was never reached: every earlier one was tried
        obj.close()
        after = _free_bytes()
        # what the failed calls allocated was freed (allow the driver's own
        # bookkeeping a few MiB)
        assert abs(after - before) <= 8 << 20, (before, after)
        return k - 1
    raise AssertionError("create still allocating after %d allocations" % max_allocs)


def test_allocation_hook_refuses_negative_counts():
    assert X.lib().xy_debug_fail_alloc(-1) == X.XY_EINVAL
    assert X.lib().xy_debug_fail_alloc(0) == X.XY_OK


@pytest.mark.parametrize("L,algorithm", [(32, "two_pass"), (256, "persistent"), (256, "fused")])
def test_lattice_create_reports_enomem_and_device_stays_usable(L, algorithm):
    n = _fail_each_allocation(lambda: Lattice(L, 1.0, 3, algorithm=algorithm))
    # the angles are the caller's (a torch buffer); the context allocates its
    # flag word, the one-launch sweeps the second buffer and a wait word, the
    # persistent sweep its tile counters
    assert n >= {"two_pass": 1, "fused": 3, "persistent": 4}[algorithm]
    # the device works: one sweep in lock step with the oracle
    with Lattice(L, 1.0, 3, algorithm=algorithm) as lat:
        before, t0 = lat.state()
        lat.sweep(1)
        after, _ = lat.state()
    red, blk = lockstep_sweep(before, after, L, 1.0, 3, t0)
    assert red.out_band_mismatch == 0 and blk.out_band_mismatch == 0
    assert max(red.max_angle_err, blk.max_angle_err) <= ANGLE_TOL


def test_record_growth_reports_enomem_and_keeps_the_context():
    """A sweep call that must grow the record buffer fails with XY_ENOMEM; the
    error is sticky in that context, and a fresh context works."""
    lib = X.lib()
    with Lattice(64, 1.0, 5) as lat:
        lat.sweep(1)
        assert lib.xy_debug_fail_alloc(1) == X.XY_OK
        try:
            with pytest.raises(X.XYError) as ei:
                lat.reserve(1 << 16)
        finally:
            lib.xy_debug_fail_alloc(0)
        assert ei.value.status == X.XY_ENOMEM
    with Lattice(64, 1.0, 5) as lat:
        lat.sweep(3)
        assert lat.observables()["accepted"].size == 3


def test_batch_hmc_and_quad_creates_report_enomem():
    n_b = _fail_each_allocation(lambda: Batch([16, 128, 100], [0.9, 1.0, 1.1], 7,
                                              sweeps_per_round=2))
    n_h = _fail_each_allocation(lambda: HMC(64, 1.0, 7, 0.1, 5))
    n_q = _fail_each_allocation(lambda: Quad(64, [1.0, 1.05, 1.1, 1.15], 7))
    assert min(n_b, n_h, n_q) >= 2
    with Batch([16, 128], [0.9, 1.0], 7, sweeps_per_round=2) as b:
        b.run(2)
        assert b.observables(0)["accepted"].size == 4
    with HMC(64, 1.0, 7, 0.1, 5) as h:
        h.run(2)
    with Quad(64, [1.0, 1.05, 1.1, 1.15], 7) as q:
        q.sweep(2)
        s, n = q.state(0)
        assert n == 2 and np.all(np.isfinite(s))
