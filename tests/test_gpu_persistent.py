"""The persistent fused sweep (XY_ALGO_PERSISTENT): every sweep of an xy_sweep
call in one cooperative launch, tiles ordered only by their neighbours'
per-tile sweep counters.  Each tile runs the fused kernel's arithmetic, so the
angles, the accept counts and the records (exact fixed-point sums of the same
per-tile partial sums) must equal those of one fused launch per sweep, bit for
bit, whatever the number of sweeps per call; and through the fused kernel it
inherits the lock-step parity with the oracle (checked directly at L = 4096 in
test_gpu_parity.py).
"""
import numpy as np
import pytest

from gpu_util import record_tolerance

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0811_2111_gb300 import build as _build  # noqa: E402

_build.build()
from paper_0811_2111_gb300 import _lib as X  # noqa: E402
from paper_0811_2111_gb300.lattice import Lattice  # noqa: E402

FIELDS = ("C", "Ix", "Iy", "Mx", "My", "accepted", "beta")


def _run(L, algorithm, calls, sincos="accurate", reduce="exact", beta=1.12, seed=31, lid=2,
         ctas_per_sm=0):
    with Lattice(L, beta, seed, sincos=sincos, reduce=reduce, lattice_id=lid,
                 algorithm=algorithm, ctas_per_sm=ctas_per_sm) as lat:
        for n in calls:
            lat.sweep(n)
        s, nxt = lat.state()
        obs = lat.observables()
    return s, nxt, obs


@pytest.mark.parametrize("L", [128, 256, 384, 512, 1024, 2048])
@pytest.mark.parametrize("sincos,reduce", [("accurate", "exact"), ("fast", "compensated"),
                                           ("libm", "exact")])
def test_persistent_equals_fused(L, sincos, reduce):
    """L = 128: one tile column (left and right neighbour are the tile itself);
    384: three tile columns and twelve rows; 512-2048: 64-1024 tiles, where
    fewer tiles than the CTAs' current and fetched items make tiles wait on
    their neighbours' and their own previous sweep, run on other CTAs."""
    n = 25
    sp, np_, op = _run(L, "persistent", (n,), sincos, reduce)
    sf, nf, of = _run(L, "fused", (n,), sincos, reduce)
    assert np_ == nf == n
    assert np.array_equal(sp, sf)
    for k in FIELDS:
        assert np.array_equal(op[k], of[k]), k


def test_more_tiles_than_resident_ctas():
    """L = 4096: 4096 tiles on at most 3 x 152 resident CTAs (about nine tiles
    per CTA per sweep); 12 sweeps in one launch, then 1 and 2 more."""
    sp, np_, op = _run(4096, "persistent", (12, 1, 2))
    sf, nf, of = _run(4096, "fused", (15,))
    assert np_ == nf == 15
    assert np.array_equal(sp, sf)
    for k in FIELDS:
        assert np.array_equal(op[k], of[k]), k


def test_bench_launch_configuration():
    """The throughput configuration as bench.py times it: L=4096, beta=1.12, seed 7,
    1000 sweeps in one persistent launch, against 1000 fused launches (whose
    sweeps are checked against the oracle in lock step in test_gpu_parity.py):
    the same final state, accept counts and records, bit for bit."""
    sp, np_, op = _run(4096, "persistent", (1000,), seed=7, lid=0)
    sf, nf, of = _run(4096, "fused", (1000,), seed=7, lid=0)
    assert np_ == nf == 1000
    assert np.array_equal(sp, sf)
    for k in FIELDS:
        assert np.array_equal(op[k], of[k]), k


@pytest.mark.parametrize("algorithm", ["persistent", "fused"])
@pytest.mark.parametrize("sincos,reduce", [("accurate", "exact"), ("fast", "compensated")])
def test_work_plans_are_bit_identical(algorithm, sincos, reduce):
    """The tile kernel compiled for 2 CTAs per SM (up to 128 registers), for 3
    (up to 80) and for 4 (up to 64): the same angles, accept counts and records;
    L = 4096, 20 sweeps."""
    s3, n3, o3 = _run(4096, algorithm, (20,), sincos, reduce, ctas_per_sm=3)
    assert n3 == 20
    for ctas in (2, 4):
        s, n, o = _run(4096, algorithm, (20,), sincos, reduce, ctas_per_sm=ctas)
        assert n == 20
        assert np.array_equal(s, s3), ctas
        for k in FIELDS:
            assert np.array_equal(o[k], o3[k]), (ctas, k)


@pytest.mark.parametrize("L", [128, 256, 512, 4096])
@pytest.mark.parametrize("sincos,reduce", [("accurate", "exact"), ("fast", "compensated"),
                                           ("libm", "exact")])
def test_two_sweep_launches_equal_one_sweep_launches(L, sincos, reduce):
    """Temporal blocking (XY_ALGO_FUSED2: a tile staged with a halo of four, both
    sweeps' half-sweeps in shared memory on shrinking regions): angles, accept
    counts and exact records bit for bit those of one launch per sweep (the
    compensated sums to their tolerance), for an even and an odd number of
    sweeps per call (the odd last one runs one-sweep).
    L = 128: the halo of one tile column wraps onto the tile itself."""
    s2, n2, o2 = _run(L, "fused2", (6, 3, 2), sincos, reduce)
    s1, n1, o1 = _run(L, "fused", (11,), sincos, reduce)
    assert n2 == n1 == 11
    assert np.array_equal(s2, s1)
    for k in FIELDS:
        if reduce == "exact" or k in ("accepted", "beta"):
            assert np.array_equal(o2[k], o1[k]), k
        else:   # compensated FP32 partial sums depend on which thread holds which site
            assert np.max(np.abs(o2[k] - o1[k])) <= record_tolerance(L * L, sincos=sincos,
                                                                      reduce=reduce), k


def test_calls_split_anywhere():
    """The state after odd and even sweep counts per call (the ping-pong buffer
    parity), and one sweep per call, equal one call for all sweeps."""
    ref, _, oref = _run(512, "persistent", (9,))
    for calls in ((1, 1, 1, 1, 1, 1, 1, 1, 1), (2, 3, 4), (5, 4)):
        s, n, o = _run(512, "persistent", calls)
        assert n == 9 and np.array_equal(s, ref), calls
        for k in FIELDS:
            assert np.array_equal(o[k], oref[k]), (calls, k)


def test_caller_owned_buffer():
    L, beta, seed = 256, 0.9, 17
    theta = torch.zeros(L * L, dtype=torch.float32, device="cuda")
    p = X.xy_params()
    p.L, p.start, p.beta, p.J, p.delta, p.seed = L, X.XY_START_HOT, beta, 1.0, np.pi, seed
    p.sincos_mode, p.reduce_mode, p.lattice_id = X.XY_SINCOS_ACCURATE, X.XY_REDUCE_EXACT, 0
    p.algorithm = X.XY_ALGO_PERSISTENT
    import ctypes as C
    stream = torch.cuda.current_stream()
    ctx = X.xy_create(p, C.c_void_p(stream.cuda_stream), C.c_void_p(theta.data_ptr()))
    try:
        X.check(X.lib().xy_sweep(ctx, 5), ctx)
        X.check(X.lib().xy_synchronize(ctx), ctx)
        host = np.empty(L * L, np.float32)
        nxt = C.c_uint64()
        X.check(X.lib().xy_get_state(ctx, host.ctypes.data_as(C.c_void_p), C.byref(nxt)), ctx)
    finally:
        X.check(X.lib().xy_destroy(ctx))
    sf, _, _ = _run(L, "fused", (5,), beta=beta, seed=seed, lid=0)
    assert nxt.value == 5 and np.array_equal(host.reshape(L, L), sf)


def test_algorithm_needs_l_multiple_of_128():
    with pytest.raises(X.XYError):
        Lattice(130, 1.0, 1, algorithm="persistent")


@pytest.mark.parametrize("L,expected", [(128, "persistent"), (4096, "persistent"),
                                        (8192, "fused"), (130, "two_pass")])
def test_auto_choice(L, expected):
    """AUTO: the persistent sweep for multiples of 128 up to 4096 (where a sweep
    is at most nine waves of tiles), one fused launch per sweep beyond,
    two-pass for other even sides."""
    with Lattice(L, 1.0, 1) as lat:
        assert lat.algorithm == expected
    for algo in ("fused", "persistent"):
        if L % 128 == 0:
            with Lattice(L, 1.0, 1, algorithm=algo) as lat:
                assert lat.algorithm == algo


def test_wait_runs_out_and_reports_timeout():
    """The failure path, made on purpose without a fault: a persistent launch
    whose first sweep is never handed out, so every wait of its second sweep
    runs out after 4096 polls; the kernel ends with its error word set and the
    call reports XY_ETIMEOUT.  The device stays usable: a persistent run right
    after is still bit for bit the fused one."""
    import ctypes as C
    stream = torch.cuda.current_stream()
    st = X.lib().xy_selftest_persistent_wait(C.c_void_p(stream.cuda_stream), 4096)
    assert st == X.XY_ETIMEOUT, X.xy_last_error(None)
    assert "ran out" in X.xy_last_error(None)
    sp, _, op = _run(256, "persistent", (5,))
    sf, _, of = _run(256, "fused", (5,))
    assert np.array_equal(sp, sf)
    for k in FIELDS:
        assert np.array_equal(op[k], of[k]), k
