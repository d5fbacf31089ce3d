"""Hybrid Monte Carlo on the GPU against the FP64 oracle (Sec. 1.2).

* The hot start equals the Metropolis engine's; the momenta equal the
  oracle's Box-Muller of the same Philox words to FP32 accuracy.
* Leap-frog in lock step: from the same FP32 state, one GPU step equals one
  FP64 oracle step to FP32 rounding, and n steps to the FP32 error amplified
  by the dynamics.
* The tiled kernel and the one-thread-per-site kernel agree bit for bit.
* Whole trajectories: dH equals the oracle's dH from the same start within
  the FP32 integration error, decisions agree outside the rounding band, the
  record sums equal the oracle's sums of the GPU state, a rejected trajectory
  leaves the state untouched bit for bit.
* Ensembles: exact 2x2 energies, <exp(-dH)> = 1.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
import exact_small as ex
from gpu_util import record_tolerance
from stats_util import jackknife_mean

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0811_2111_gb300 import build as _build  # noqa: E402

_build.build()
from paper_0811_2111_gb300 import _lib as X  # noqa: E402
from paper_0811_2111_gb300.hmc import HMC  # noqa: E402
from paper_0811_2111_gb300.lattice import Lattice  # noqa: E402

TWO_PI = 2 * np.pi
ANGLE_STEP_TOL = 2e-6     # one leap-frog step: FP32 rounding of theta + eps p and of F


def circ(a, b):
    d = np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)) % TWO_PI
    return np.minimum(d, TWO_PI - d)


def random_state(L, seed, p_scale=1.0):
    rng = np.random.default_rng(seed)
    th = rng.uniform(0, TWO_PI, L * L).astype(np.float32)
    p = (p_scale * rng.normal(size=L * L)).astype(np.float32)
    return th, p


def test_hot_start_equals_metropolis_start():
    for L in (6, 128):
        with HMC(L, 1.0, 77, 0.1, 5, lattice_id=3) as h:
            th, p, t = h.state()
        with Lattice(L, 1.0, 77, lattice_id=3, algorithm="two_pass") as lat:
            ref, _ = lat.state()
        assert np.array_equal(th, ref)
        assert np.all(p == 0) and t == 0


@pytest.mark.parametrize("L", [2, 6, 130, 256])
def test_momenta_match_oracle(L):
    with HMC(L, 1.0, 12345, 0.1, 5, lattice_id=9) as h:
        th, _, _ = h.state()
        h.set_state(th, None, next_traj=41)
        h.refresh()
        _, p, _ = h.state()
    want = oracle.hmc_momenta(L, L, 12345, 41, 9)
    err = np.abs(p.reshape(-1).astype(np.float64) - want)
    assert np.all(err <= 1e-6 * np.maximum(1.0, np.abs(want))), err.max()


@pytest.mark.parametrize("L,kernel", [(2, "site"), (6, "site"), (34, "site"), (128, "tiled"),
                                      (128, "site"), (256, "tiled")])
@pytest.mark.parametrize("sincos", ["accurate", "fast"])
def test_one_leapfrog_step_matches_oracle(L, kernel, sincos):
    beta, eps = 1.1, 0.08
    th, p = random_state(L, L + 5)
    with HMC(L, beta, 3, eps, 1, sincos=sincos, kernel=kernel) as h:
        h.set_state(th, p, 0)
        h.integrate(1)
        g_th, g_p, _ = h.state()
    o_th, o_p = oracle.hmc_leapfrog(th, p, L, L, beta, eps, 1)
    tol = ANGLE_STEP_TOL if sincos == "accurate" else 2e-5
    assert np.max(circ(g_th.reshape(-1), o_th)) <= tol
    dp = np.abs(g_p.reshape(-1) - o_p)
    assert np.all(dp <= tol * (1.0 + np.abs(o_p))), dp.max()


@pytest.mark.parametrize("L", [6, 128])
def test_n_steps_match_oracle(L):
    """Steps 2.. use the full-kick kernel; the FP32 error grows with the dynamics."""
    beta, eps, n = 1.0, 0.05, 8
    th, p = random_state(L, 99)
    with HMC(L, beta, 3, eps, n) as h:
        h.set_state(th, p, 0)
        h.integrate(n)
        g_th, g_p, _ = h.state()
        sums = h.last_sums()
    o_th, o_p = oracle.hmc_leapfrog(th, p, L, L, beta, eps, n)
    assert np.max(circ(g_th.reshape(-1), o_th)) <= 2e-5
    assert np.max(np.abs(g_p.reshape(-1) - o_p)) <= 2e-5 * (1 + np.abs(o_p).max())
    K0, V0 = oracle.hmc_hamiltonian(th, p, L, L, beta)
    K1, V1 = oracle.hmc_hamiltonian(o_th, o_p, L, L, beta)
    N = L * L
    assert abs(sums["start"]["K"] - K0) <= 1e-6 * N
    assert abs(-beta * sums["start"]["C"] - V0) <= 1e-6 * N
    assert abs(sums["end"]["K"] - K1) <= 2e-5 * N
    assert abs(-beta * sums["end"]["C"] - V1) <= 2e-5 * N


@pytest.mark.parametrize("L,n_md", [(128, 7), (256, 7), (128, 1), (128, 2), (128, 4), (256, 5),
                                    (16, 3), (32, 4), (48, 4), (64, 7)])
def test_kernels_are_bit_identical(L, n_md):
    """The tiled kernel (one step per launch), the two-step kernel (full steps
    two per launch, odd remainders singly), the TMA-fed kernel, the persistent
    TMA kernel (a trajectory's steps in one launch), the cluster kernel (a
    whole trajectory per launch) and the per-site kernel: same bits."""
    kernels = ["site"]
    if L % 128 == 0:
        kernels += ["tiled", "tiled2", "tiled_tma", "persistent"]
    if L in (16, 32, 64, 128, 256):
        kernels += ["cluster"]
    out = {}
    for kernel in kernels:
        with HMC(L, 1.05, 8, 0.1, n_md, kernel=kernel, lattice_id=2) as h:
            h.run(6)
            th, p, _ = h.state()
            o = h.observables()
            h.integrate(3)
            th2, p2, _ = h.state()
            out[kernel] = (th, p, o, th2, p2, h.last_sums())
    b = out["site"]
    for name in kernels[1:]:
        a = out[name]
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), name
        for k in ("C", "Ix", "Iy", "Mx", "My", "dH"):
            assert np.array_equal(a[2][k], b[2][k]), (name, k)
        assert np.array_equal(a[2]["accepted"], b[2]["accepted"]), name
        assert np.array_equal(a[3], b[3]) and np.array_equal(a[4], b[4]), name
        assert a[5] == b[5], name


@pytest.mark.parametrize("L,n_md", [(512, 4), (512, 5), (1024, 8), (1024, 3), (4096, 6),
                                    (4096, 5)])
def test_auto_kernel_equals_one_step_launches(L, n_md):
    """AUTO at sides the tiled kernels take: the full steps two per launch
    (momenta ping-ponged between two buffers; one tile per CTA at L = 512 and
    1024, resident CTAs walking the tiles with the next tile's loads copied in
    ahead at L = 4096) with an odd remaining step on the TMA or the plain
    tiled kernel, against one tiled launch per step: angles, momenta, records
    and sums bit for bit, over trajectories with an even and an odd number of
    full steps and a plain integration."""
    out = {}
    for kernel in ("tiled", "auto"):
        with HMC(L, 1.1, 17, 0.5 / n_md, n_md, kernel=kernel, lattice_id=3) as h:
            h.run(5)
            th, p, _ = h.state()
            o = h.observables()
            h.integrate(n_md + 1)
            th2, p2, _ = h.state()
            out[kernel] = (th, p, o, th2, p2, h.last_sums())
    a, b = out["auto"], out["tiled"]
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    for k in ("C", "Ix", "Iy", "Mx", "My", "dH", "accepted"):
        assert np.array_equal(a[2][k], b[2][k]), k
    assert np.all(np.isfinite(a[2]["dH"]))
    assert np.array_equal(a[3], b[3]) and np.array_equal(a[4], b[4])
    assert a[5] == b[5]


def test_library_max_side_kernels_agree_and_match_oracle_statistics():
    """The library's largest side, XY_MAX_L = 32768 (2^30 sites), where the
    state is too large to hand to the oracle whole.

    One trajectory of six leap-frog steps from the seed-17 hot start by one
    tiled launch per step and by AUTO (two full steps per launch, resident
    CTAs walking the tiles): records and start/end sums bit for bit.  The
    kinetic and bond sums per site at the trajectory's start and end (before
    the accept test) and dH per site are averages over 2^30 sites of
    quantities that, from i.i.d. angles and momenta, depend only on a
    neighbourhood of a few sites, so they match the oracle's trajectories on
    sixteen L = 256 lattices to within the sampling error of those (5 sigma)."""
    L, beta, n_md = X.XY_MAX_L, 1.1, 6
    eps = 0.5 / n_md
    out = {}
    for kernel in ("tiled", "auto"):
        with HMC(L, beta, 17, eps, n_md, kernel=kernel) as h:
            h.run(1)
            out[kernel] = (h.observables(), h.last_sums())
    (oa, sa), (ob, sb) = out["auto"], out["tiled"]
    for k in ("C", "Ix", "Iy", "Mx", "My", "dH", "accepted"):
        assert np.array_equal(oa[k], ob[k]), k
    assert sa == sb
    N = float(L) * L
    got = np.array([sa["start"]["K"] / N, sa["end"]["K"] / N, sa["start"]["C"] / N,
                    sa["end"]["C"] / N, oa["dH"][0] / N])

    Lo, chains = 256, 16
    rows = []
    for c in range(chains):
        th0 = oracle.start(Lo, Lo, 100 + c)
        _, _, d = oracle.hmc_trajectory(th0, Lo, Lo, beta, eps, n_md, 100 + c, 0)
        No = float(Lo * Lo)
        rows.append([d["K0"] / No, d["K1"] / No, -d["V0"] / beta / No, -d["V1"] / beta / No,
                     d["dH"] / No])
    o = np.array(rows)
    err = o.std(axis=0, ddof=1) * np.sqrt(1.0 / chains + (Lo / L) ** 2)
    print("L=32768 K0, K1, C0, C1, dH per site:", got, "oracle L=256:", o.mean(axis=0), "+-",
          err)
    assert np.all(np.abs(got - o.mean(axis=0)) <= 5.0 * err)


@pytest.mark.parametrize("L,eps,n_md", [(8, 0.2, 5), (32, 0.1, 10), (128, 0.05, 12)])
def test_trajectories_match_oracle_step_by_step(L, eps, n_md):
    """Each trajectory from the GPU's FP32 state: dH, decision and final state."""
    beta, seed, lid = 1.0, 21, 4
    N = L * L
    dh_tol = 2e-6 * N ** 0.5 * n_md + 1e-5
    band = 2 * dh_tol
    mismatches = 0
    with HMC(L, beta, seed, eps, n_md, lattice_id=lid) as h:
        th, _, _ = h.state()
        for t in range(12):
            h.run(1)
            g_th, _, _ = h.state()
            o = h.observables(t, 1)
            o_th, o_pend, info = oracle.hmc_trajectory(th, L, L, beta, eps, n_md, seed, t, lid)
            assert abs(o["dH"][0] - info["dH"]) <= dh_tol, (t, o["dH"][0], info["dH"])
            u = oracle.philox_words(seed, t, lid, 4, 0, 1)[0, 0] >> 8
            u = u / 2.0 ** 24
            gpu_acc = bool(o["accepted"][0])
            if gpu_acc != info["accepted"]:
                assert abs(u - np.exp(-info["dH"])) <= band, t
                mismatches += 1
            if gpu_acc:
                if info["accepted"]:
                    assert np.max(circ(g_th.reshape(-1), o_th)) <= 5e-5
            else:
                assert np.array_equal(g_th.reshape(-1), th.reshape(-1))
            sums = oracle.measure(g_th.reshape(-1).astype(np.float64), L, L)
            tol = record_tolerance(N)
            for k, v in zip(("C", "Ix", "Iy", "Mx", "My"), sums):
                assert abs(o[k][0] - v) <= tol, (t, k)
            th = g_th
    assert mismatches <= 1


def test_rejection_leaves_state_untouched():
    L = 64
    with HMC(L, 1.0, 5, 0.9, 6) as h:
        rejected = 0
        for t in range(10):
            before, _, _ = h.state()
            h.run(1)
            after, _, _ = h.state()
            if not h.observables(t, 1)["accepted"][0]:
                rejected += 1
                assert np.array_equal(before, after)
        _, _, acc = h.info()
    assert rejected >= 5 and acc == 10 - rejected


def test_reversibility_in_fp32():
    L, beta, eps, n = 128, 1.0, 0.05, 20
    th, p = random_state(L, 7)
    with HMC(L, beta, 3, eps, n) as h:
        h.set_state(th, p, 0)
        h.integrate(n)
        t1, p1, _ = h.state()
        h.set_state(t1, -p1, 0)
        h.integrate(n)
        t2, p2, _ = h.state()
    assert np.max(circ(t1.reshape(-1), th)) > 0.1
    err_t = np.max(circ(t2.reshape(-1), th))
    err_p = np.max(np.abs(-p2.reshape(-1) - p))
    print(f"FP32 reversibility violation after {n}+{n} steps: angle {err_t:.2e}, momentum {err_p:.2e}")
    assert err_t < 1e-4 and err_p < 1e-4


@pytest.mark.parametrize("beta", [0.5, 1.0, 2.0])
def test_hmc_samples_exact_2x2_energy(beta):
    with HMC(2, beta, 31, 0.3, 4) as h:
        h.run(20000)
        e = h.observables()["e"]
    m, err = jackknife_mean(e[2000:])
    print(f"beta {beta}: gpu {m:.5f} +- {err:.5f} exact {ex.e_2x2_bessel(beta):.5f}")
    assert abs(m - ex.e_2x2_bessel(beta)) <= 3.5 * err + 1e-6


def test_creutz_equality_on_gpu():
    with HMC(64, 1.0, 13, 0.1, 10) as h:
        h.run(3000)
        o = h.observables()
    w = np.exp(-o["dH"][300:])
    m, err = jackknife_mean(w)
    rate = o["accepted"].mean()
    print(f"<exp(-dH)> = {m:.4f} +- {err:.4f}, acceptance {rate:.3f}")
    assert abs(m - 1.0) <= 3.5 * err
    assert 0.3 < rate < 0.999


def test_beta_zero_is_free_motion():
    L, eps, n = 128, 0.25, 4
    with HMC(L, 0.0, 3, eps, n) as h:
        th0, _, _ = h.state()
        h.run(5)
        o = h.observables()
    assert np.all(o["accepted"] == 1)
    assert np.max(np.abs(o["dH"])) < 1e-6


def test_large_lattice_one_step_matches_oracle():
    """L = 4096 (the throughput size): one step from a random FP32 state."""
    L, beta, eps = 4096, 1.12, 0.03
    th, p = random_state(L, 5)
    with HMC(L, beta, 7, eps, 1) as h:
        h.set_state(th, p, 0)
        h.integrate(1)
        g_th, g_p, _ = h.state()
    o_th, o_p = oracle.hmc_leapfrog(th, p, L, L, beta, eps, 1)
    assert np.max(circ(g_th.reshape(-1), o_th)) <= ANGLE_STEP_TOL
    assert np.max(np.abs(g_p.reshape(-1) - o_p) / (1 + np.abs(o_p))) <= ANGLE_STEP_TOL


def test_error_paths():
    """Refused arguments raise; as everywhere in the ABI the first error is
    sticky in its context, so each case gets a fresh context."""
    with HMC(16, 1.0, 1, 0.1, 3) as h:
        with pytest.raises(X.XYError):
            h.integrate(0)
        with pytest.raises(X.XYError):
            h.run(1)                                # sticky
    with HMC(16, 1.0, 1, 0.1, 3) as h:
        bad = np.zeros(256, np.float32)
        bad[5] = np.nan
        with pytest.raises(X.XYError):
            h.set_state(bad)                        # refused before any work: not sticky
        h.run(2)
        assert h.info()[0] == 2
    with HMC(16, 1.0, 1, 0.1, 3) as h:
        with pytest.raises(X.XYError):
            h.set_step(-1.0, 3)
    for kernel in ("tiled", "tiled2", "tiled_tma"):
        with pytest.raises(X.XYError):
            HMC(96, 1.0, 1, 0.1, 3, kernel=kernel)
    for L in (8, 48, 512):
        with pytest.raises(X.XYError):
            HMC(L, 1.0, 1, 0.1, 3, kernel="cluster")


def test_caller_owned_angle_buffer_holds_the_state():
    """With d_angles given, the state is back in that buffer after every call
    (the trajectory moves it between three buffers on the device)."""
    import ctypes as C
    L = 128
    dev = torch.device("cuda")
    buf = torch.empty(L * L, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    p = X.xy_hmc_params()
    p.L, p.start, p.beta, p.J, p.eps, p.n_md = L, X.XY_START_COLD, 1.0, 1.0, 0.001, 1
    p.sincos_mode, p.seed, p.lattice_id, p.kernel = 0, 11, 0, 0
    h = X.xy_hmc_create(p, C.c_void_p(stream.cuda_stream), C.c_void_p(buf.data_ptr()))
    try:
        moved = rejected = 0
        for t in range(40):
            # tiny steps are accepted (the state moves), huge ones are often rejected
            X.xy_hmc_set_step(h, 0.001 if t % 2 == 0 else 2.0, 1 if t % 2 == 0 else 5)
            before = buf.cpu().numpy().copy()
            X.xy_hmc_run(h, 1)
            th = np.empty(L * L, np.float32)
            X.xy_hmc_get_state(h, th.ctypes.data_as(C.c_void_p))
            after = buf.cpu().numpy()
            assert np.array_equal(after, th)
            if np.array_equal(after, before):
                rejected += 1
            else:
                moved += 1
            if moved > 2 and rejected > 2:
                break
        assert moved > 0 and rejected > 0          # both buffer paths exercised
    finally:
        X.xy_hmc_destroy(h)
    assert torch.isfinite(buf).all()                 # still the caller's, still valid


def test_bounded_wait_runs_out_and_reports_timeout():
    """The failure path of the device waits, without a fault: a wait on an
    mbarrier that nothing completes runs out after its bound, the error word
    reaches the host as XY_ETIMEOUT, and the GPU stays usable."""
    stream = torch.cuda.current_stream()
    st = X.lib().xy_selftest_bounded_wait(C.c_void_p(stream.cuda_stream), 4096)
    assert st == X.XY_ETIMEOUT, X.xy_hmc_last_error(None)
    assert X.lib().xy_selftest_bounded_wait(None, 0) == X.XY_EINVAL
    with HMC(128, 1.0, 3, 0.05, 4, kernel="tiled_tma") as h:   # still usable afterwards
        h.run(2)
        assert h.info()[0] == 2


@pytest.mark.parametrize("L,n_md", [(512, 9), (1024, 20), (4096, 12)])
def test_persistent_steps_equal_tma_steps(L, n_md):
    """The trajectory-long persistent launch against one TMA step launch per
    step, at sides where tiles wait on each other (L = 512: 64 tiles on 64
    CTAs) and where they never do (L = 4096: 4096 tiles on 304 CTAs): angles,
    momenta, records and sums bit for bit, over accepted and rejected
    trajectories and a plain integration."""
    out = {}
    for kernel in ("tiled_tma", "persistent"):
        with HMC(L, 1.1, 13, 0.6 / n_md, n_md, kernel=kernel, lattice_id=1) as h:
            h.run(4)
            th, p, _ = h.state()
            o = h.observables()
            h.integrate(n_md + 1)
            th2, p2, _ = h.state()
            out[kernel] = (th, p, o, th2, p2, h.last_sums())
    a, b = out["persistent"], out["tiled_tma"]
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    for k in ("C", "Ix", "Iy", "Mx", "My", "dH", "accepted"):
        assert np.array_equal(a[2][k], b[2][k]), k
    assert np.array_equal(a[3], b[3]) and np.array_equal(a[4], b[4])
    assert a[5] == b[5]
