"""Pins of the FP64 oracle against facts fixed outside it (CPU only).

Each test checks the oracle against something it cannot produce itself: a
library implementation of Philox, closed forms of the bond sums, exact
partition functions of tiny tori, the leading high- and low-temperature
expansions, and the energy bookkeeping of single-site moves.  Between them
they fail on a dropped neighbour, a wrong sign, a swapped x/y index, a wrong
counter word or a wrong helicity term.
"""
import json
import math
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
from scipy.special import i0, i1

import oracle
from stats_util import jackknife_mean
import exact_small as ex

TWO_PI = 2 * np.pi


def chain(Lx, Ly, beta, n, seed, order=0, delta=np.pi, start=1, J=1.0, therm=0.1):
    rec, _ = oracle.run(Lx, Ly, beta, n, seed=seed, order=order, delta=delta, start=start,
                        J=J)
    rec = rec[int(therm * n):]
    e, m, u = oracle.observables(rec[:, :5], Lx * Ly, beta, J)
    return rec, e, m, u


def within(x, err, ref, extra=0.0, k=3.0):
    return abs(x - ref) <= k * err + extra


# ---------------------------------------------------------------------------
# Philox4x32-10
# ---------------------------------------------------------------------------

TRITON_SCRIPT = textwrap.dedent("""
    import os, sys, json
    os.environ["TRITON_INTERPRET"] = "1"
    import torch, triton, triton.language as tl

    @triton.jit
    def _k(out, c0p, c1p, c2p, c3p, seed, n: tl.constexpr):
        i = tl.arange(0, n)
        a, b, c, d = tl.philox(seed, tl.load(c0p + i), tl.load(c1p + i),
                               tl.load(c2p + i), tl.load(c3p + i))
        tl.store(out + 4 * i + 0, a)
        tl.store(out + 4 * i + 1, b)
        tl.store(out + 4 * i + 2, c)
        tl.store(out + 4 * i + 3, d)

    cases = json.loads(sys.stdin.read())
    res = []
    for seed, ctrs in cases:
        n = len(ctrs)
        cols = [torch.tensor([c[k] for c in ctrs], dtype=torch.int64).to(torch.uint32)
                for k in range(4)]
        out = torch.zeros(4 * n, dtype=torch.uint32)
        _k[(1,)](out, *cols, seed, n)
        res.append([int(v) & 0xffffffff for v in out.view(torch.int32).tolist()])
    print(json.dumps(res))
""")


def test_philox_matches_library_implementation():
    """Oracle Philox == Triton's Philox4x32-10 (run on the CPU interpreter)."""
    pytest.importorskip("triton")
    pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    cases = []
    for seed in (0, 1, 7, 0xFFFFFFFFFFFFFFFF, 0x243F6A8885A308D3):
        ctrs = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 2, 3, 4]]
        ctrs += rng.integers(0, 2 ** 32, size=(5, 4), dtype=np.uint64).tolist()
        cases.append([int(seed), [[int(v) for v in c] for c in ctrs]])
    env = dict(os.environ, TRITON_INTERPRET="1")
    r = subprocess.run([sys.executable, "-c", TRITON_SCRIPT], input=json.dumps(cases),
                       capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lib_out = json.loads(r.stdout.strip().splitlines()[-1])
    for (seed, ctrs), ref in zip(cases, lib_out):
        key = [seed & 0xFFFFFFFF, seed >> 32]
        mine = np.concatenate([oracle.philox4x32_10(c, key) for c in ctrs])
        assert mine.tolist() == ref, f"seed {seed:#x}"


def test_philox_every_counter_and_key_word_matters():
    base = oracle.philox4x32_10([11, 22, 33, 44], [55, 66])
    for k in range(4):
        ctr = [11, 22, 33, 44]
        ctr[k] ^= 1
        assert not np.array_equal(oracle.philox4x32_10(ctr, [55, 66]), base)
    for k in range(2):
        key = [55, 66]
        key[k] ^= 1
        assert not np.array_equal(oracle.philox4x32_10([11, 22, 33, 44], key), base)


def test_philox_words_layout():
    w = oracle.philox_words(seed=0x1234567890, sweep=9, lattice_id=3, domain=1, first=100, n=3)
    for i in range(3):
        ref = oracle.philox4x32_10([100 + i, 9, 3, 1], [0x34567890, 0x12])
        assert np.array_equal(w[i], ref)


@pytest.mark.parametrize("L", [8, 6])
def test_metropolis_words_pair_sites_and_are_never_reused(L):
    """A sweep's Metropolis draws: the sites x and x + 2 of a row (x & 2 == 0)
    share one block, the first taking words 0/1, the second 2/3; so every
    word of the generator is used at most once per sweep, every site reads
    its accept uniform from that position and its proposal is
    theta + delta (2 u0 - 1) with u0 the word before it (L = 6: the pair
    x = 4, 6 is cut by the edge and x = 4 takes the lower words alone)."""
    seed, sweep, lid, delta = 0xABCDEF12345, 5, 2, 2.0
    theta = oracle.start(L, L, seed=seed, lattice_id=lid)
    sites = np.arange(L * L)
    tp, u1, p, acc = oracle.attempt_sites(theta, L, L, sites, 1.0, seed, sweep, lattice_id=lid,
                                          delta=delta)
    used = set()
    for s in sites:
        y, x = divmod(int(s), L)
        base, upper = y * L + (x & ~2), (x >> 1) & 1
        w = oracle.philox_words(seed, sweep, lid, 1, base, 1)[0]
        assert (base, upper) not in used
        used.add((base, upper))
        u = (w >> 8) * 2.0 ** -24
        assert u1[s] == u[2 * upper + 1]
        want = (theta[s] + delta * (2.0 * u[2 * upper] - 1.0)) % TWO_PI
        assert abs(tp[s] - want) < 1e-12
    assert len(used) == L * L


# ---------------------------------------------------------------------------
# Start configurations
# ---------------------------------------------------------------------------

def test_hot_start_is_uniform_and_seeded():
    from scipy.stats import kstest
    L = 128
    th = oracle.start(L, L, seed=7)
    assert th.min() >= 0.0 and th.max() < TWO_PI
    assert kstest(th / TWO_PI, "uniform").pvalue > 1e-3
    # uniform angles: |M|^2 / N has mean 1 (Rayleigh); loose check
    M = np.hypot(np.cos(th).sum(), np.sin(th).sum())
    assert M ** 2 / th.size < 20
    # multiples of 2 pi / 2^24 exactly (24-bit uniforms)
    k = th / TWO_PI * 2 ** 24
    assert np.allclose(k, np.round(k), atol=1e-6)
    assert not np.array_equal(th, oracle.start(L, L, seed=8))
    assert not np.array_equal(th, oracle.start(L, L, seed=7, lattice_id=1))
    assert np.all(oracle.start(8, 8, seed=7, hot=False) == 0.0)


# ---------------------------------------------------------------------------
# Bond and spin sums: closed forms
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("Lx,Ly", [(2, 2), (4, 6), (8, 8), (6, 4)])
def test_measure_uniform_configuration(Lx, Ly):
    N = Lx * Ly
    a = 0.7
    C, Ix, Iy, Mx, My = oracle.measure(np.full(N, a), Lx, Ly)
    assert C == pytest.approx(2 * N, abs=1e-12)
    assert abs(Ix) < 1e-12 and abs(Iy) < 1e-12
    assert Mx == pytest.approx(N * math.cos(a), abs=1e-12)
    assert My == pytest.approx(N * math.sin(a), abs=1e-12)


@pytest.mark.parametrize("Lx,Ly,k", [(8, 8, 1), (8, 6, 3), (4, 8, 1), (6, 10, 2)])
def test_measure_twisted_configurations(Lx, Ly, k):
    N = Lx * Ly
    y, x = np.divmod(np.arange(N), Lx)
    # twist along x: theta = 2 pi k x / Lx
    q = 2 * np.pi * k / Lx
    C, Ix, Iy, Mx, My = oracle.measure(q * x, Lx, Ly)
    assert C == pytest.approx(N * math.cos(q) + N, abs=1e-9)
    assert Ix == pytest.approx(-N * math.sin(q), abs=1e-9)
    assert abs(Iy) < 1e-9
    assert abs(Mx) < 1e-9 and abs(My) < 1e-9
    # twist along y
    q = 2 * np.pi * k / Ly
    C, Ix, Iy, Mx, My = oracle.measure(q * y, Lx, Ly)
    assert C == pytest.approx(N * math.cos(q) + N, abs=1e-9)
    assert Iy == pytest.approx(-N * math.sin(q), abs=1e-9)
    assert abs(Ix) < 1e-9


@pytest.mark.parametrize("Lx,Ly", [(2, 2), (2, 4), (4, 2), (6, 4), (8, 8), (3, 5)])
def test_delta_energy_matches_total_energy_difference(Lx, Ly):
    """dE of a single-site move == E(after) - E(before), E = -J C."""
    rng = np.random.default_rng(Lx * 100 + Ly)
    N = Lx * Ly
    J = 1.3
    for _ in range(20):
        th = rng.uniform(0, TWO_PI, N)
        s = int(rng.integers(N))
        new = rng.uniform(0, TWO_PI)
        e0 = -J * oracle.measure(th, Lx, Ly)[0]
        th2 = th.copy()
        th2[s] = new
        e1 = -J * oracle.measure(th2, Lx, Ly)[0]
        assert oracle.delta_energy(th, Lx, Ly, s, new, J) == pytest.approx(e1 - e0, abs=1e-11)


# ---------------------------------------------------------------------------
# Sweep structure
# ---------------------------------------------------------------------------

def test_sweep_is_two_half_sweeps_and_attempts_agree():
    L, beta, seed = 8, 1.1, 3
    th0 = oracle.start(L, L, seed)
    th = th0.copy()
    acc = oracle.sweep(th, L, L, beta, seed, 5)
    a, tp, u1, p, z = oracle.half_sweep(th0, L, L, 0, beta, seed, 5)
    b, tp1, u11, p1, z1 = oracle.half_sweep(a, L, L, 1, beta, seed, 5)
    assert np.array_equal(b, th)
    assert acc == z.sum() + z1.sum()
    red = np.flatnonzero((np.arange(L * L) % L + np.arange(L * L) // L) % 2 == 0)
    tpa, u1a, pa, za = oracle.attempt_sites(th0, L, L, red, beta, seed, 5)
    assert np.array_equal(tpa, tp[red]) and np.array_equal(za, z[red])
    assert np.array_equal(u1a, u1[red]) and np.array_equal(pa, p[red])
    # Sec. 3.2 select: accepted sites take the proposal, others keep the old angle
    assert np.array_equal(a[red], np.where(z[red], tp[red], th0[red]))
    # proposals lie in [0, 2 pi) and within delta of the old angle (circularly)
    d = np.abs(tp[red] - th0[red])
    d = np.minimum(d, TWO_PI - d)
    assert np.all((tp[red] >= 0) & (tp[red] < TWO_PI)) and np.all(d <= np.pi + 1e-12)


def test_checkerboard_rejects_odd_sides():
    th = np.zeros(9)
    with pytest.raises(ValueError):
        oracle.sweep(th, 3, 3, 1.0, 1, 0, order=0)
    oracle.sweep(th, 3, 3, 1.0, 1, 0, order=1)


def test_openmp_half_sweep_is_identical():
    L = 32
    th = oracle.start(L, L, 11)
    a = oracle.half_sweep(th, L, L, 0, 1.0, 11, 2, nthreads=1)[0]
    b = oracle.half_sweep(th, L, L, 0, 1.0, 11, 2, nthreads=4)[0]
    assert np.array_equal(a, b)


# ---------------------------------------------------------------------------
# Physics pins
# ---------------------------------------------------------------------------

def test_beta_zero_limit():
    """beta = 0: every proposal accepted, <e> = <Upsilon> = 0, <m^2> = 1/N."""
    L, n = 8, 20000
    rec, e, m, u = chain(L, L, 0.0, n, seed=21, therm=0.0)
    assert np.all(rec[:, 5] == L * L)
    me, ee = jackknife_mean(e)
    mu, eu = jackknife_mean(u)
    m2, em2 = jackknife_mean(m * m)
    assert within(me, ee, 0.0)
    assert within(mu, eu, 0.0)
    assert within(m2, em2, 1.0 / (L * L))


@pytest.mark.parametrize("beta", [0.5, 1.0, 2.0])
def test_2x2_torus_exact(beta):
    """The 2x2 torus is a 4-ring with coupling 2 beta: Bessel-sum partition function."""
    rec, e, m, u = chain(2, 2, beta, 200000, seed=31)
    me, ee = jackknife_mean(e)
    assert within(me, ee, ex.e_2x2_bessel(beta))
    # on a side of 2 the currents vanish identically, so Upsilon_s = -e_s / 2
    assert np.max(np.abs(rec[:, 1:3])) < 1e-12
    assert np.allclose(u, -e / 2, atol=1e-12)
    mm, em = jackknife_mean(m)
    assert within(mm, em, ex.mean_abs_m_grid(2, 2, beta, M=24), extra=1e-5)


@pytest.mark.parametrize("Lx,Ly,order", [(2, 4, 0), (4, 2, 0), (2, 3, 1)])
def test_small_tori_exact(Lx, Ly, order):
    """Energy and helicity modulus vs the transfer-matrix partition function.

    Upsilon comes from the curvature of the free energy under a boundary
    twist, so the oracle's (C - beta (Ix^2 + Iy^2)) / 2N estimator is checked
    against its definition, not against itself."""
    beta = 1.0
    rec, e, m, u = chain(Lx, Ly, beta, 200000, seed=41 + Lx, order=order)
    e_ex, u_ex = ex.exact_observables(Lx, Ly, beta)
    me, ee = jackknife_mean(e)
    mu, eu = jackknife_mean(u)
    assert within(me, ee, e_ex, extra=1e-6)
    assert within(mu, eu, u_ex, extra=1e-5)
    if (Lx, Ly) == (2, 3):
        mm, em = jackknife_mean(m)
        assert within(mm, em, ex.mean_abs_m_grid(2, 3, beta, M=16), extra=1e-4)


@pytest.mark.parametrize("beta", [0.05, 0.1])
def test_high_temperature_limit(beta):
    """<cos bond> = I1(beta)/I0(beta) + O(beta^3) at high temperature."""
    L = 8
    rec, e, m, u = chain(L, L, beta, 40000, seed=51)
    me, ee = jackknife_mean(e)
    assert within(me, ee, -2 * i1(beta) / i0(beta), extra=2 * beta ** 3)


@pytest.mark.parametrize("beta", [10.0, 20.0])
def test_spin_wave_limit(beta):
    """Low temperature: e = -2 + (1 - 1/N) / (2 beta) + O(beta^-2) (equipartition)."""
    L = 16
    N = L * L
    rec, e, m, u = chain(L, L, beta, 20000, seed=61, start=0, delta=0.5, therm=0.2)
    me, ee = jackknife_mean(e)
    assert within(me, ee, -2 + (1 - 1 / N) / (2 * beta), extra=2 / beta ** 2)
    # acceptance neither frozen nor trivial with the small window
    acc = rec[:, 5].mean() / N
    assert 0.2 < acc < 0.95


def test_coupling_scales_temperature():
    """Same seed: (J, beta) and (1, beta J) give identical decisions and e/J."""
    L = 8
    r1, _ = oracle.run(L, L, 0.8, 200, seed=71, J=1.5)
    r2, _ = oracle.run(L, L, 1.2, 200, seed=71, J=1.0)
    assert np.array_equal(r1[:, 5], r2[:, 5])
    assert np.allclose(r1[:, :5], r2[:, :5], atol=1e-9)


# ---------------------------------------------------------------------------
# Replica exchange
# ---------------------------------------------------------------------------

def test_exchange_rule_reduces_to_metropolis_on_two_replicas():
    """Swap iff u < exp((b_p - b_q)(E_p - E_q)): with equal energies every pair swaps,
    and a pair whose swap would lower the joint weight swaps at that rate."""
    ls = [0]
    pos = [0, 1, 2, 3]
    betas = [0.5, 0.7, 0.9, 1.1]
    bl = list(betas)
    pl, bl2, sw = oracle.exchange(ls, pos, betas, bl, [-3.0, -3.0, -3.0, -3.0], 0, seed=9)
    assert sw[0] and sw[2] and not sw[1] and not sw[3]          # round 0 pairs (0,1), (2,3)
    assert list(pl) == [1, 0, 3, 2] and list(bl2) == [0.7, 0.5, 1.1, 0.9]
    # round 1 pairs (1,2) only
    pl, bl3, sw = oracle.exchange(ls, pos, betas, bl, [-3.0] * 4, 1, seed=9)
    assert list(sw) == [False, True, False, False]
    # acceptance frequency of a disfavoured swap: exp((0.5-0.7)(-1-(-6))) = exp(-1)
    acc = np.mean([oracle.exchange([0], [0, 1], [0.5, 0.7], [0.5, 0.7], [-1.0, -6.0], 2 * r,
                                   seed=11)[2][0] for r in range(20000)])
    assert abs(acc - math.exp(-1.0)) < 4 * math.sqrt(math.exp(-1) * (1 - math.exp(-1)) / 20000)


def test_parallel_tempering_samples_each_temperature_exactly():
    """A 3-temperature ladder of 2x2 tori: the energy series at each temperature
    label must match that temperature's exact Bessel-sum value."""
    betas = [0.5, 1.0, 2.0]
    rec = oracle.pt_run(2, 2, betas, rounds=40000, sweeps_per_round=2, seed=3)
    e = -rec[:, :, 0] / 4
    b = rec[:, :, 6]
    for beta in betas:
        series = np.array([e[:, t][b[:, t] == beta][0] for t in range(e.shape[1])])
        m, err = jackknife_mean(series[2000:])
        assert within(m, err, ex.e_2x2_bessel(beta), extra=1e-6, k=3.5)
    # every sweep carries each temperature exactly once
    assert np.all(np.sort(b, axis=0) == np.array(betas)[:, None])


# ---------------------------------------------------------------------------
# Statistics helper
# ---------------------------------------------------------------------------

def test_jackknife_on_ar1_series():
    """Error of the mean of an AR(1) series vs its closed form."""
    rng = np.random.default_rng(3)
    rho, n = 0.9, 400000
    z = rng.standard_normal(n)
    x = np.empty(n)
    x[0] = z[0] / math.sqrt(1 - rho ** 2)
    for i in range(1, n):
        x[i] = rho * x[i - 1] + z[i]
    mean, err = jackknife_mean(x, n_bins=100)
    sigma2 = 1.0 / (1 - rho ** 2)
    expected = math.sqrt(sigma2 / n * (1 + rho) / (1 - rho))
    assert 0.7 * expected < err < 1.3 * expected
    assert abs(mean) < 4 * expected


def test_transfer_matrix_quadrature_converges():
    """The trapezoid rule behind the exact small-torus pins converges spectrally:
    from 8 to 16 grid points the energy moves by ~5e-4, beyond 16 only by the
    finite-difference noise (~1e-11)."""
    e = {M: ex.exact_observables(2, 3, 1.0, M=M) for M in (8, 16, 24, 48)}
    assert abs(e[8][0] - e[16][0]) > 1e-4
    assert abs(e[24][0] - e[16][0]) < 1e-9 and abs(e[48][0] - e[24][0]) < 1e-9
    assert abs(e[24][1] - e[16][1]) < 1e-8 and abs(e[48][1] - e[24][1]) < 1e-8
