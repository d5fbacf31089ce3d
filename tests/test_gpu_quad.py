"""Four replicas per site (the RGBA packing of Sec. 3.2) against single lattices.

Replica r of a quad context must be the single lattice with lattice id
lattice_id + r and beta betas[r], bit for bit in its angles and accept counts
(the same Philox counters and per-site arithmetic), with record sums equal to
the reduction's rounding; and, through that, it inherits the single lattice's
lock-step parity with the oracle (checked directly on a small case too).
"""
import numpy as np
import pytest

from gpu_util import ANGLE_TOL, lockstep_sweep, record_tolerance

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0811_2111_gb300 import build as _build  # noqa: E402

_build.build()
from paper_0811_2111_gb300 import _lib as X  # noqa: E402
from paper_0811_2111_gb300.lattice import Lattice, Quad  # noqa: E402

BETAS = [0.7, 1.0, 1.12, 1.4]


@pytest.mark.parametrize("L", [2, 6, 32, 34, 64, 96, 130, 256])
@pytest.mark.parametrize("sincos,reduce", [("accurate", "exact"), ("fast", "exact"),
                                           ("accurate", "compensated"), ("libm", "exact")])
def test_replicas_equal_single_lattices(L, sincos, reduce):
    """AUTO: the persistent sweep for L % 32 == 0 (32, 64, 96, 256), two-pass otherwise."""
    sweeps = 7
    with Quad(L, BETAS, 19, sincos=sincos, reduce=reduce, lattice_id=40) as q:
        assert q.algorithm == ("persistent" if L % 32 == 0 else "two_pass")
        q.sweep(sweeps)
        states = [q.state(r)[0] for r in range(4)]
        obs = [q.observables(r) for r in range(4)]
    for r, beta in enumerate(BETAS):
        with Lattice(L, beta, 19, sincos=sincos, reduce=reduce, lattice_id=40 + r,
                     algorithm="two_pass") as lat:
            lat.sweep(sweeps)
            s, _ = lat.state()
            o = lat.observables()
        assert np.array_equal(states[r], s), (L, r)
        assert np.array_equal(obs[r]["accepted"], o["accepted"]), (L, r)
        assert np.all(obs[r]["beta"] == beta)
        tol = record_tolerance(L * L, sincos=sincos, reduce=reduce)
        for k in ("C", "Ix", "Iy", "Mx", "My"):
            if reduce == "exact":       # the same per-site terms: the same record bits
                assert np.array_equal(obs[r][k], o[k]), (L, r, k)
            else:
                assert np.max(np.abs(obs[r][k] - o[k])) <= tol, (L, r, k)


def test_hot_start_and_cold_start():
    with Quad(64, BETAS, 5, lattice_id=3) as q:
        hot = [q.state(r)[0] for r in range(4)]
    for r in range(4):
        with Lattice(64, 1.0, 5, lattice_id=3 + r, algorithm="two_pass") as lat:
            assert np.array_equal(hot[r], lat.state()[0])
    with Quad(16, BETAS, 5, start="cold") as q:
        assert all(np.all(q.state(r)[0] == 0) for r in range(4))


def test_lockstep_with_oracle():
    L, seed = 32, 3
    with Quad(L, BETAS, seed, lattice_id=7) as q:
        before = [q.state(r)[0] for r in range(4)]
        for i in range(3):
            q.sweep(1)
            for r in range(4):
                after = q.state(r)[0]
                red, blk = lockstep_sweep(before[r], after, L, BETAS[r], seed, i, lattice_id=7 + r)
                assert red.out_band_mismatch == 0 and blk.out_band_mismatch == 0
                assert max(red.max_angle_err, blk.max_angle_err) <= ANGLE_TOL
                before[r] = after


def test_error_paths():
    with pytest.raises(X.XYError):
        Quad(15, BETAS, 1)
    with pytest.raises(X.XYError):
        Quad(16, [1.0, -1.0, 1.0, 1.0], 1)
    with Quad(16, BETAS, 1) as q:
        q.sweep(2)
        with pytest.raises(X.XYError):
            q.observables(4)
    with Quad(16, BETAS, 1) as q:
        with pytest.raises(X.XYError):
            q.sweep(-1)


@pytest.mark.parametrize("L", [32, 128, 512])
@pytest.mark.parametrize("sincos,reduce", [("accurate", "exact"), ("fast", "compensated")])
def test_fused_equals_two_pass(L, sincos, reduce):
    """The one-launch sweep (tiles of 32 rows x 16 sites, the red ring recomputed
    at the tile edges, several tiles per row and column from L = 64 on) and the
    two-pass kernels: the same angles and accept counts, sums to rounding."""
    sweeps = 5
    out = {}
    for algo in ("fused", "two_pass"):
        with Quad(L, BETAS, 23, sincos=sincos, reduce=reduce, lattice_id=5, algorithm=algo) as q:
            assert q.algorithm == algo
            q.sweep(sweeps)
            out[algo] = ([q.state(r)[0] for r in range(4)], [q.observables(r) for r in range(4)],
                         q.state(0)[1])
    (sf, of, nf), (st, ot, nt) = out["fused"], out["two_pass"]
    assert nf == nt == sweeps
    tol = record_tolerance(L * L, sincos=sincos, reduce=reduce)
    for r in range(4):
        assert np.array_equal(sf[r], st[r]), r
        assert np.array_equal(of[r]["accepted"], ot[r]["accepted"]), r
        assert np.all(of[r]["beta"] == BETAS[r])
        for k in ("C", "Ix", "Iy", "Mx", "My"):
            if reduce == "exact":
                assert np.array_equal(of[r][k], ot[r][k]), (r, k)
            else:
                assert np.max(np.abs(of[r][k] - ot[r][k])) <= tol, (r, k)


def test_fused_sweeps_in_pieces_equal_one_run():
    """The ping-pong buffer parity carries over between calls: 3 + 1 + 4 sweeps
    give the state of 8 sweeps in one call."""
    with Quad(64, BETAS, 29, algorithm="fused") as a, Quad(64, BETAS, 29, algorithm="fused") as b:
        for n in (3, 1, 4):
            a.sweep(n)
        b.sweep(8)
        for r in range(4):
            sa, na = a.state(r)
            sb, nb = b.state(r)
            assert na == nb == 8 and np.array_equal(sa, sb)


def test_fused_algorithm_needs_l_multiple_of_32():
    for algo in ("fused", "persistent"):
        with pytest.raises(X.XYError):
            Quad(34, BETAS, 1, algorithm=algo)
    with Quad(34, BETAS, 1) as q:
        assert q.algorithm == "two_pass"
    with Quad(1024, BETAS, 1) as q:
        assert q.algorithm == "persistent"
    with Quad(2048, BETAS, 1) as q:
        assert q.algorithm == "fused"


@pytest.mark.parametrize("L", [32, 64, 128, 512, 2048])
@pytest.mark.parametrize("sincos,reduce", [("accurate", "exact"), ("fast", "compensated"),
                                           ("libm", "exact")])
def test_persistent_equals_fused(L, sincos, reduce):
    """All sweeps of a call in one cooperative launch against one fused launch
    per sweep: angles, accept counts and records bit for bit (the same tile
    arithmetic and per-tile partial sums; L = 32: one tile, its own neighbour
    in every direction; 2048: 4096 tiles)."""
    n = 13
    out = {}
    for algo in ("persistent", "fused"):
        with Quad(L, BETAS, 37, sincos=sincos, reduce=reduce, lattice_id=3, algorithm=algo) as q:
            assert q.algorithm == algo
            q.sweep(n)
            out[algo] = ([q.state(r)[0] for r in range(4)], [q.observables(r) for r in range(4)])
    (sp, op), (sf, of) = out["persistent"], out["fused"]
    for r in range(4):
        assert np.array_equal(sp[r], sf[r]), r
        for k in ("C", "Ix", "Iy", "Mx", "My", "accepted", "beta"):
            assert np.array_equal(op[r][k], of[r][k]), (r, k)


def test_persistent_calls_split_anywhere():
    with Quad(128, BETAS, 41, algorithm="persistent") as a, \
            Quad(128, BETAS, 41, algorithm="persistent") as b:
        for n in (1, 4, 3, 1):
            a.sweep(n)
        b.sweep(9)
        for r in range(4):
            sa, na = a.state(r)
            sb, nb = b.state(r)
            assert na == nb == 9 and np.array_equal(sa, sb)


def test_throughput_configuration_replicas_equal_single_lattices():
    """The four-replica throughput configuration as bench.py times it: L = 4096,
    betas 1.00, 1.06, 1.12, 1.18, seed 7, AUTO (one fused launch per sweep,
    16384 tiles).  Each replica is the single lattice with lattice id r (the
    persistent single-lattice sweep, itself in lock step with the oracle at this
    size): angles, accept counts and exact record sums bit for bit."""
    L, betas, seed, sweeps = 4096, [1.0, 1.06, 1.12, 1.18], 7, 3
    with Quad(L, betas, seed) as q:
        assert q.algorithm == "fused"
        q.sweep(sweeps)
        states = [q.state(r)[0] for r in range(4)]
        obs = [q.observables(r) for r in range(4)]
    for r, beta in enumerate(betas):
        with Lattice(L, beta, seed, lattice_id=r) as lat:
            assert lat.algorithm == "persistent"
            lat.sweep(sweeps)
            s, n = lat.state()
            o = lat.observables()
        assert n == sweeps
        assert np.array_equal(states[r], s), r
        for k in ("C", "Ix", "Iy", "Mx", "My", "accepted", "beta"):
            assert np.array_equal(obs[r][k], o[k]), (r, k)


def test_library_max_side_replicas_equal_single_lattices():
    """The library's largest side, XY_MAX_L = 32768 (2^30 sites, four replicas
    a site: 16 GiB a buffer), two sweeps by AUTO's fused launch: each replica's
    exact record sums and accept counts equal, bit for bit, those of the
    single lattice with lattice id r at that side (itself checked across its
    three sweep kernels and against oracle statistics there)."""
    L, betas, seed, sweeps = X.XY_MAX_L, [1.0, 1.06, 1.12, 1.18], 7, 2
    with Quad(L, betas, seed) as q:
        assert q.algorithm == "fused"
        q.sweep(sweeps)
        obs = [q.observables(r) for r in range(4)]
    for r, beta in enumerate(betas):
        with Lattice(L, beta, seed, lattice_id=r) as lat:
            lat.sweep(sweeps)
            o = lat.observables()
        for k in ("C", "Ix", "Iy", "Mx", "My", "accepted", "beta"):
            assert np.array_equal(obs[r][k], o[k]), (r, k)
