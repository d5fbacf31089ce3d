"""CUDA path vs FP64 oracle, element by element (needs a GB300).

Everything goes through the C ABI (``libxy.so`` via the ctypes binding).
Tolerances (each follows from the FP32 arithmetic of the kernels):
  * Philox words and hot-start counters: bit-exact;
  * accept decisions: identical outside |u - exp(-beta dE)| < 1e-6 (accurate
    path); the in-band count is reported;
  * post-sweep angles: within 1e-5 rad of the oracle's choice;
  * per-sweep sums: ``gpu_util.record_tolerance``;
  * long runs: observables within 3 sigma (binned jackknife).
"""
import json
import os

import numpy as np
import pytest

import oracle
from gpu_util import (ANGLE_TOL, BAND_ACCURATE, circ, compare_record, lockstep_sweep,
                      record_tolerance)

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0811_2111_gb300 import build as _build  # noqa: E402

_build.build()
from paper_0811_2111_gb300 import lattice as LT  # noqa: E402
from paper_0811_2111_gb300 import workloads as WL  # noqa: E402
from paper_0811_2111_gb300 import _lib as X  # noqa: E402


def run_lockstep(lat, n, beta, seed, J=1.0, delta=np.pi, band=BAND_ACCURATE, lattice_id=0,
                 fast=False, sincos=None):
    """n GPU sweeps, each checked in lock-step; returns summary dict."""
    L = lat.L
    tol = record_tolerance(L * L, fast, sincos=sincos)
    n0, _ = lat.info()
    s_before, t0 = lat.state()
    worst = dict(in_band=0, out_band=0, angle=0.0, rec=0.0, acc_mismatch=0,
                 rec_abs=np.zeros(5))
    for i in range(n):
        lat.sweep(1)
        s_after, _ = lat.state()
        red, blk = lockstep_sweep(s_before, s_after, L, beta, seed, t0 + i, J, delta, band,
                                  lattice_id)
        obs = lat.observables(n0 + i, 1)
        row = {k: obs[k][0] for k in obs}
        diff, _ = compare_record(row, s_after, L, J)
        worst["in_band"] += red.in_band + blk.in_band
        worst["out_band"] += red.out_band_mismatch + blk.out_band_mismatch
        worst["angle"] = max(worst["angle"], red.max_angle_err, blk.max_angle_err)
        worst["rec"] = max(worst["rec"], float(diff.max()) / tol)
        worst["rec_abs"] = np.maximum(worst["rec_abs"], diff)
        worst["acc_mismatch"] += int(row["accepted"]) != red.accepted + blk.accepted
        s_before = s_after
    return worst


# ---------------------------------------------------------------------------
# Philox and start configurations
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed,sweep,lid,dom,first,n", [
    (1, 0, 0, 1, 0, 1024),
    (7, 999, 0, 1, 0, 1 << 20),
    (0xFFFFFFFFFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF, 2, 0xFFFFFFFF - 4095, 4096),
    (0x243F6A8885A308D3, 12345, 17, 0, 16777216 - 100000, 100000),
])
def test_philox_words_bit_exact(seed, sweep, lid, dom, first, n):
    gpu = LT.philox_words(seed, sweep, lid, dom, first, n)
    ref = oracle.philox_words(seed, sweep, lid, dom, first, n)
    assert np.array_equal(gpu, ref)


@pytest.mark.parametrize("seed", [0x123456789ABCDEF, 1, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand(seed):
    """An independent Philox4x32-10: cuRAND's host generator.  With seed s its
    key is (s_lo, s_hi) and output 4 i + j is word j of counter (0, 0, i, 0)
    (established on this GPU: the first outputs of the default ordering).  The
    same counters from the GPU kernels (site 0, sweep 0, lattice id i, domain 0)
    and from the oracle must give the same words."""
    import ctypes as C
    import ctypes.util
    path = "/usr/local/cuda/lib64/libcurand.so"
    if not os.path.exists(path):
        path = ctypes.util.find_library("curand")
    if not path:
        pytest.skip("libcurand not found")
    cur = C.CDLL(path)
    n_ctr = 256
    gen = C.c_void_p()
    assert cur.curandCreateGenerator(C.byref(gen), 161) == 0        # PHILOX4_32_10
    try:
        assert cur.curandSetPseudoRandomGeneratorSeed(gen, C.c_ulonglong(seed)) == 0
        out = torch.zeros(4 * n_ctr, dtype=torch.int32, device="cuda")
        assert cur.curandGenerate(gen, C.c_void_p(out.data_ptr()), C.c_size_t(4 * n_ctr)) == 0
        torch.cuda.synchronize()
    finally:
        cur.curandDestroyGenerator(gen)
    lib = out.cpu().numpy().view(np.uint32).reshape(n_ctr, 4)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    ref = np.stack([oracle.philox4x32_10([0, 0, i, 0], key) for i in range(n_ctr)])
    assert np.array_equal(lib, ref)
    gpu = np.concatenate([LT.philox_words(seed, 0, i, 0, 0, 1) for i in range(0, n_ctr, 17)])
    assert np.array_equal(gpu, ref[::17])


@pytest.mark.parametrize("L,seed,lid", [(32, 1, 0), (4096, 7, 0), (64, 5, 3)])
def test_hot_start_matches_oracle(L, seed, lid):
    with LT.Lattice(L, 1.0, seed, lattice_id=lid) as lat:
        s, nxt = lat.state()
    assert nxt == 0
    ref = oracle.start(L, L, seed, lid)
    assert circ(s.reshape(-1), ref).max() < 1e-6
    assert s.min() >= 0 and s.max() < np.float32(2 * np.pi)


def test_cold_start_is_zero():
    with LT.Lattice(16, 1.0, 3, start="cold") as lat:
        s, _ = lat.state()
    assert np.all(s == 0)


# ---------------------------------------------------------------------------
# Lock-step parity
# ---------------------------------------------------------------------------

def test_lockstep_small_config_accurate():
    """L=32, beta=1, seed 1, 1000 sweeps, accurate path: the small configuration."""
    w = WL.SMALL
    with LT.Lattice(w.L, w.beta, w.seed) as lat:
        r = run_lockstep(lat, w.sweeps, w.beta, w.seed)
    print("lockstep L=32:", r)
    assert r["out_band"] == 0
    assert r["angle"] <= ANGLE_TOL
    assert r["rec"] <= 1.0
    assert r["acc_mismatch"] == 0


@pytest.mark.parametrize("L", [2, 4, 6, 10, 34, 130, 258])
def test_lockstep_edge_sizes(L):
    """Degenerate and ragged sides: L=2 (double bonds), odd plane widths, partial tiles."""
    with LT.Lattice(L, 0.9, 100 + L) as lat:
        r = run_lockstep(lat, 30, 0.9, 100 + L)
    assert r["out_band"] == 0 and r["angle"] <= ANGLE_TOL
    assert r["rec"] <= 1.0 and r["acc_mismatch"] == 0


@pytest.mark.parametrize("L,algorithm", [(128, "fused"), (256, "fused"), (384, "fused")])
def test_lockstep_fused_sizes(L, algorithm):
    """Fused single-pass kernels: one tile wide (L=128 wraps onto itself), several tiles."""
    with LT.Lattice(L, 1.05, 300 + L, algorithm=algorithm) as lat:
        r = run_lockstep(lat, 25, 1.05, 300 + L)
    assert r["out_band"] == 0 and r["angle"] <= ANGLE_TOL
    assert r["rec"] <= 1.0 and r["acc_mismatch"] == 0


@pytest.mark.parametrize("sincos", ["accurate", "fast", "libm"])
def test_fused_and_two_pass_are_bit_identical(sincos):
    """Same decisions bit for bit (shared pinned-rounding site update) for the fused
    and two-pass kernels; the odd sweep count exercises the copy back into the
    caller's buffer, and a reset/set_state in between the state round trip."""
    out = {}
    for algo in ("fused", "two_pass"):
        with LT.Lattice(256, 1.12, 41, sincos=sincos, algorithm=algo) as lat:
            lat.sweep(13)
            mid, nxt = lat.state()
            lat.reset(99)
            lat.set_state(mid, nxt)
            lat.sweep(12)
            out[algo] = (lat.state(), lat.observables())
    (st, nt), ot = out["two_pass"]
    assert nt == 25
    for algo in ("fused",):
        (sf, nf), of = out[algo]
        assert nf == nt
        assert np.array_equal(sf, st), algo
        assert np.array_equal(of["accepted"], ot["accepted"]), algo
        # exact sums: the fused and two-pass kernels form the same per-site
        # terms, so the records are identical
        for k in ("C", "Ix", "Iy", "Mx", "My"):
            assert np.array_equal(of[k], ot[k]), (algo, k)


def test_unit_vector_accuracy():
    """The kernels' sincos against FP64 on [0, 2 pi]: the polynomial path is at most
    ~1 ulp (<= 1.2e-7 absolute), CUDA's sincosf at most 2 ulp, the SFU path a few 1e-7."""
    rng = np.random.default_rng(2)
    t = np.concatenate([rng.random(1 << 22) * 2 * np.pi,
                        np.arange(0, 6.2831855, np.pi / 4)]).astype(np.float32)
    t = np.clip(t, 0, np.float32(2 * np.pi))
    ref_c, ref_s = np.cos(t.astype(np.float64)), np.sin(t.astype(np.float64))
    bounds = {"accurate": 1.2e-7, "libm": 2.4e-7, "fast": 2e-6}
    for mode, bound in bounds.items():
        c, s = LT.unit_vectors(t, mode)
        ec, es = c - ref_c, s - ref_s
        norm = (c.astype(np.float64) ** 2 + s.astype(np.float64) ** 2 - 1).mean()
        print(f"{mode}: max|dc| {np.abs(ec).max():.3e} max|ds| {np.abs(es).max():.3e} "
              f"mean dc {ec.mean():.2e} mean ds {es.mean():.2e} mean(|v|^2-1) {norm:.2e}")
        assert np.abs(ec).max() <= bound and np.abs(es).max() <= bound


@pytest.mark.parametrize("beta,J,delta", [(0.0, 1.0, np.pi), (2.5, 1.0, 0.7), (0.6, -1.3, 2.0)])
def test_lockstep_parameters(beta, J, delta):
    with LT.Lattice(128, beta, 21, J=J, delta=delta) as lat:
        r = run_lockstep(lat, 20, beta, 21, J=J, delta=delta)
    assert r["out_band"] == 0 and r["angle"] <= ANGLE_TOL
    assert r["rec"] <= 1.0 and r["acc_mismatch"] == 0


@pytest.mark.parametrize("algorithm", ["fused", "two_pass", "persistent"])
def test_lockstep_large_config_full_size(algorithm):
    """L=4096, beta=1.12, seed 7 (the throughput configuration; AUTO runs it with the
    persistent sweep): sweeps 0, 1 and 20 checked over all 16.8M sites, sweeps
    2-18 in one launch in between."""
    w = WL.LARGE
    with LT.Lattice(w.L, w.beta, w.seed, algorithm=algorithm) as lat:
        r0 = run_lockstep(lat, 2, w.beta, w.seed)
        lat.sweep(17)
        r1 = run_lockstep(lat, 1, w.beta, w.seed)
    for r in (r0, r1):
        print("lockstep L=4096:", r, "tolerance", record_tolerance(w.L * w.L))
        assert r["out_band"] == 0
        assert r["angle"] <= ANGLE_TOL
        assert r["rec"] <= 1.0 and r["acc_mismatch"] == 0


def test_record_check_catches_one_wrong_bond_at_full_size():
    """L=4096: the GPU record of a sweep is within record_tolerance of the oracle's
    sums on the same state, and an oracle with one wrong bond (the x bond of one site
    taken to its y neighbour instead, the change of C and of Ix at least 0.5) falls
    outside it."""
    w = WL.LARGE
    L = w.L
    tol = record_tolerance(L * L)
    with LT.Lattice(L, w.beta, w.seed) as lat:
        lat.sweep(3)
        state, _ = lat.state()
        obs = lat.observables(2, 1)
    got = np.array([obs[k][0] for k in ("C", "Ix", "Iy", "Mx", "My")])
    th = state.reshape(-1).astype(np.float64)
    ref = oracle.measure(th, L, L)
    assert np.max(np.abs(got - ref)) <= tol
    s = np.arange(L * L)
    right = (s // L) * L + (s + 1) % L
    down = (s + L) % (L * L)
    dC = np.cos(th - th[down]) - np.cos(th - th[right])
    dI = np.sin(th - th[down]) - np.sin(th - th[right])
    site = int(np.flatnonzero((np.abs(dC) >= 0.5) & (np.abs(dI) >= 0.5))[0])
    planted = ref.copy()
    planted[0] += dC[site]
    planted[1] += dI[site]
    print(f"L=4096 record vs oracle: max |diff| {np.max(np.abs(got - ref)):.3e}, tolerance "
          f"{tol:.3e}; one wrong bond moves C by {dC[site]:+.3f}, Ix by {dI[site]:+.3f}")
    assert abs(got[0] - planted[0]) > tol and abs(got[1] - planted[1]) > tol


def test_fast_path_error_is_bounded():
    """__sincosf/__expf path: decisions may differ in a wider band, stated and bounded."""
    w = WL.SMALL
    with LT.Lattice(w.L, w.beta, w.seed, sincos="fast") as lat:
        r_wide = run_lockstep(lat, 300, w.beta, w.seed, band=2e-5, fast=True)
    print("fast path, band 2e-5:", r_wide)
    assert r_wide["out_band"] == 0
    assert r_wide["angle"] <= ANGLE_TOL and r_wide["rec"] <= 1.0


def test_compensated_reduction_matches_exact():
    w = WL.SMALL
    outs = []
    for red in ("exact", "compensated"):
        with LT.Lattice(128, 1.1, 9, reduce=red) as lat:
            lat.sweep(50)
            outs.append((lat.state()[0], lat.observables()))
    assert np.array_equal(outs[0][0], outs[1][0])      # the chain does not depend on it
    tol = record_tolerance(128 * 128, reduce="compensated")
    for k in ("C", "Ix", "Iy", "Mx", "My"):
        assert np.max(np.abs(outs[0][1][k] - outs[1][1][k])) <= tol


# ---------------------------------------------------------------------------
# Statistics, resume, determinism
# ---------------------------------------------------------------------------

def test_long_run_observables_agree_with_oracle_ensemble():
    """16 independent GPU chains vs the stored ensemble of 64 oracle chains.

    The error of each mean is the chain-to-chain spread of the oracle
    ensemble (tests/golden/ensemble_L32_beta1.0.json, written by
    tests/golden/make_golden.py from the oracle only); single-chain
    jackknife errors underestimate it near the BKT region."""
    gold = json.load(open(os.path.join(GOLDEN, "ensemble_L32_beta1.0.json")))
    ref = np.array(gold["chains"])
    L, beta, n, cut = gold["L"], gold["beta"], gold["sweeps"], gold["discard"]
    chains = 16
    rows = []
    for c in range(chains):
        with LT.Lattice(L, beta, 1, lattice_id=c) as lat:
            lat.sweep(n)
            r = lat.observables()
        rows.append([r["e"][cut:].mean(), r["abs_m"][cut:].mean(), r["upsilon"][cut:].mean(),
                     r["accepted"][cut:].astype(np.float64).mean() / (L * L)])
    g = np.array(rows)
    sd = ref.std(axis=0, ddof=1)
    err = sd * np.sqrt(1.0 / chains + 1.0 / ref.shape[0])
    for i, k in enumerate(gold["columns"]):
        print(f"{k}: gpu {g[:, i].mean():.5f} oracle {ref[:, i].mean():.5f} +- {err[i]:.5f}")
        assert abs(g[:, i].mean() - ref[:, i].mean()) <= 3.5 * err[i]


def test_resume_is_bit_exact_and_runs_are_deterministic():
    L, beta, seed = 64, 1.05, 17
    with LT.Lattice(L, beta, seed) as a:
        a.sweep(20)
        sa, _ = a.state()
        oa = a.observables()
    with LT.Lattice(L, beta, seed) as b:
        b.sweep(10)
        mid, nxt = b.state()
        ob1 = b.observables()
    with LT.Lattice(L, beta, seed) as c:
        c.set_state(mid, nxt)
        c.sweep(10)
        sc, nxt2 = c.state()
        oc = c.observables()
    assert nxt2 == 20
    assert np.array_equal(sa, sc)
    for k in ("C", "Ix", "Iy", "Mx", "My", "accepted"):
        assert np.array_equal(oa[k][:10], ob1[k])
        assert np.array_equal(oa[k][10:], oc[k])


def test_max_side_runs():
    """Largest configured side (1 GiB of angles): sampled sites checked against the oracle."""
    w = WL.HUGE
    with LT.Lattice(w.L, w.beta, w.seed) as lat:
        s0, _ = lat.state()
        lat.sweep(1)
        s1, _ = lat.state()
        obs = lat.observables()
    L = w.L
    rng = np.random.default_rng(0)
    y = rng.integers(0, L, 20000)
    x = rng.integers(0, L, 20000)
    red = ((x + y) & 1) == 0
    sites = (y * L + x)[red]
    tp, u1, p, acc = oracle.attempt_sites(s0.reshape(-1).astype(np.float64), L, L, sites,
                                          w.beta, w.seed, 0)
    b = s0.reshape(-1)[sites]
    a = s1.reshape(-1)[sites]
    changed = a != b
    unobs = circ(tp, b) < 2e-6
    band = np.abs(u1 - p) < BAND_ACCURATE
    assert np.count_nonzero((changed != acc) & ~unobs & ~band) == 0
    assert np.isfinite(obs["e"]).all() and -2.0 < obs["e"][0] < 0.0


def test_library_max_side_algorithms_agree_and_match_oracle_statistics():
    """The library's largest side, XY_MAX_L = 32768 (2^30 sites, 4 GiB of angles a
    buffer), where the state is too large to hand to the oracle whole.

    Two sweeps from the seed-7 hot start by the per-sweep fused, the
    persistent and the two-pass kernels give bit-identical records (exact
    fixed-point sums and accept counts).  Their energy per site and acceptance
    after each sweep are averages over 2^30 sites of quantities that, starting
    from i.i.d. uniform angles, depend only on a neighbourhood of a few sites,
    so they match the oracle's on sixteen L = 512 lattices with their own hot
    starts to within the sampling error of those (5 sigma)."""
    L, beta, seed, n = X.XY_MAX_L, 1.12, 7, 2
    recs = {}
    for algo in ("fused", "persistent", "two_pass"):
        with LT.Lattice(L, beta, seed, algorithm=algo) as lat:
            assert lat.algorithm == algo
            lat.sweep(n)
            recs[algo] = lat.observables()
    ref = recs["fused"]
    for algo in ("persistent", "two_pass"):
        for k in ref:
            assert np.array_equal(recs[algo][k], ref[k]), (algo, k)
    g_e = ref["e"]
    g_acc = ref["accepted"].astype(np.float64) / float(L * L)

    Lo, chains = 512, 16
    rows = []
    for c in range(chains):
        rec, _ = oracle.run(Lo, Lo, beta, n, 100 + c, nthreads=oracle.max_threads())
        e, _, _ = oracle.observables(rec[:, :5], Lo * Lo, beta)
        rows.append(np.concatenate([e, rec[:, 5] / (Lo * Lo)]))
    o = np.array(rows)
    err = o.std(axis=0, ddof=1) * np.sqrt(1.0 / chains + (Lo / L) ** 2)
    got = np.concatenate([g_e, g_acc])
    print("L=32768 e, acceptance:", got, "oracle L=512:", o.mean(axis=0), "+-", err)
    assert np.all(np.abs(got - o.mean(axis=0)) <= 5.0 * err)


# ---------------------------------------------------------------------------
# Error paths through the ABI
# ---------------------------------------------------------------------------

def test_error_paths_on_device():
    lat = LT.Lattice(16, 1.0, 1)
    lat.sweep(0)                                        # empty request is a no-op
    assert lat.info() == (0, 0)
    bad = np.zeros((16, 16), np.float32)
    bad[3, 4] = np.nan
    with pytest.raises(X.XYError) as ei:
        lat.set_state(bad, 0)
    assert ei.value.status == X.XY_EINVAL
    lat.sweep(2)                                        # not sticky: still usable
    assert lat.info()[0] == 2
    with pytest.raises(X.XYError) as ei:
        X.xy_measure(lat.ctx, 1, 5)
    assert ei.value.status == X.XY_EINVAL
    with pytest.raises(X.XYError) as ei:                # sticky from now on
        lat.sweep(1)
    assert ei.value.status == X.XY_EINVAL
    ctx = lat.ctx
    lat.close()
    assert X.lib().xy_destroy(ctx) == X.XY_ESTATE       # double destroy refused
    assert X.lib().xy_sweep(ctx, 1) == X.XY_ESTATE      # use after destroy refused


def test_sweep_counter_limit():
    with LT.Lattice(8, 1.0, 1) as lat:
        s, _ = lat.state()
        lat.set_state(s, 0xFFFFFFFF - 2)
        lat.sweep(2)
        with pytest.raises(X.XYError) as ei:
            lat.sweep(2)
        assert ei.value.status == X.XY_EINVAL
