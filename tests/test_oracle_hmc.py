"""Pins of the FP64 oracle's Hybrid Monte Carlo (Sec. 1.2) against what the
mathematics fixes, independently of the oracle's own formulas:

* the force is minus the gradient of the potential (central differences of
  the potential, which is computed from cosines of bonds, not from the sines
  the force uses);
* leap-frog is time-reversible, preserves phase-space volume (finite-difference
  Jacobian determinant 1) and has an O(eps^2) energy error at fixed
  trajectory length;
* at beta = 0 the motion is free and every trajectory is accepted;
* the momenta are standard normal and independent;
* <exp(-dH)> = 1 at equilibrium, and the acceptance of a trajectory with
  energy change dH is min(1, exp(-dH));
* the chain samples the exact energies of the 2x2 torus (Bessel closed form)
  and of the 2x3 and 2x4 tori (transfer-matrix partition function).
"""
import math

import numpy as np
import pytest

import oracle
import exact_small as ex
from stats_util import jackknife_mean

TWO_PI = 2 * np.pi


def circ(a, b):
    d = np.abs(np.asarray(a) - np.asarray(b)) % TWO_PI
    return np.minimum(d, TWO_PI - d)


def random_state(L_x, L_y, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0, TWO_PI, L_x * L_y), rng.normal(size=L_x * L_y)


@pytest.mark.parametrize("Lx,Ly", [(2, 2), (4, 6), (3, 5), (8, 8)])
def test_force_is_minus_gradient_of_potential(Lx, Ly):
    beta = 1.3
    th, p = random_state(Lx, Ly, 7 + Lx)
    F = oracle.hmc_force(th, Lx, Ly, beta)
    h = 1e-5
    fd = np.zeros_like(F)
    for s in range(Lx * Ly):
        a, b = th.copy(), th.copy()
        a[s] += h
        b[s] -= h
        fd[s] = -(oracle.hmc_hamiltonian(a, p, Lx, Ly, beta)[1]
                  - oracle.hmc_hamiltonian(b, p, Lx, Ly, beta)[1]) / (2 * h)
    assert np.max(np.abs(F - fd)) < 1e-7


def test_kinetic_and_potential_parts():
    """K is sum p^2/2; V = beta H: the ferromagnetic ground state has V = -2 beta J N."""
    Lx, Ly, beta, J = 4, 6, 0.7, 1.5
    th = np.full(Lx * Ly, 1.234)
    p = np.arange(Lx * Ly, dtype=np.float64) / 10
    K, V = oracle.hmc_hamiltonian(th, p, Lx, Ly, beta, J)
    assert K == pytest.approx(float(np.sum(p * p)) / 2, rel=1e-14)
    assert V == pytest.approx(-2 * beta * J * Lx * Ly, rel=1e-14)


def test_free_motion_at_beta_zero():
    Lx, Ly, eps, n = 4, 4, 0.3, 7
    th, p = random_state(Lx, Ly, 3)
    t2, p2 = oracle.hmc_leapfrog(th, p, Lx, Ly, 0.0, eps, n)
    assert np.array_equal(p2, p)
    assert np.max(circ(t2, th + n * eps * p)) < 1e-12
    rec, _ = oracle.hmc_run(Lx, Ly, 0.0, eps, n, 50, seed=5)
    assert np.all(rec[:, 6] == 1.0) and np.all(rec[:, 5] == 0.0)


@pytest.mark.parametrize("Lx,Ly", [(4, 4), (6, 2), (5, 3)])
def test_leapfrog_is_reversible(Lx, Ly):
    th, p = random_state(Lx, Ly, 11)
    t1, p1 = oracle.hmc_leapfrog(th, p, Lx, Ly, 1.1, 0.1, 20)
    assert np.max(circ(t1, th)) > 0.1                   # it moved
    t2, p2 = oracle.hmc_leapfrog(t1, -p1, Lx, Ly, 1.1, 0.1, 20)
    assert np.max(circ(t2, th)) < 1e-11
    assert np.max(np.abs(-p2 - p)) < 1e-11


def test_leapfrog_preserves_phase_space_volume():
    """|det J| = 1 for the map (theta, p) -> leap-frog(theta, p) on the 2x2 torus
    (8 dimensions), from a central-difference Jacobian."""
    Lx = Ly = 2
    n = Lx * Ly
    th, p = random_state(Lx, Ly, 2)
    th = th * 0.5 + 1.0                                  # away from the wrap point
    x0 = np.concatenate([th, p])
    h = 1e-6

    def f(x):
        t, q = oracle.hmc_leapfrog(x[:n], x[n:], Lx, Ly, 1.0, 0.15, 8)
        return np.concatenate([t, q])

    ref = f(x0)
    jac = np.zeros((2 * n, 2 * n))
    for k in range(2 * n):
        a, b = x0.copy(), x0.copy()
        a[k] += h
        b[k] -= h
        fa, fb = f(a), f(b)
        d = fa - fb
        d[:n] = (d[:n] + np.pi) % TWO_PI - np.pi         # angles across the wrap
        jac[:, k] = d / (2 * h)
    assert np.all(np.isfinite(ref))
    assert abs(np.linalg.det(jac) - 1.0) < 1e-6


def test_energy_error_is_second_order():
    """At fixed trajectory length the leap-frog energy error scales as eps^2."""
    Lx = Ly = 4
    th, p = random_state(Lx, Ly, 19)
    H0 = sum(oracle.hmc_hamiltonian(th, p, Lx, Ly, 1.0))
    dh = []
    for eps, n in ((0.1, 10), (0.05, 20), (0.025, 40)):
        t, q = oracle.hmc_leapfrog(th, p, Lx, Ly, 1.0, eps, n)
        dh.append(sum(oracle.hmc_hamiltonian(t, q, Lx, Ly, 1.0)) - H0)
    r1, r2 = dh[0] / dh[1], dh[1] / dh[2]
    assert 3.6 < r1 < 4.4 and 3.9 < r2 < 4.1, dh


def test_momenta_are_standard_normal_and_independent():
    stats = pytest.importorskip("scipy.stats")
    L = 64
    p = np.concatenate([oracle.hmc_momenta(L, L, 17, t, 3) for t in range(8)])
    assert abs(p.mean()) < 4 / math.sqrt(p.size)
    assert abs(p.var() - 1.0) < 4 * math.sqrt(2.0 / p.size)
    assert stats.kstest(p, "norm").pvalue > 1e-3
    a, b = oracle.hmc_momenta(L, L, 17, 0, 3), oracle.hmc_momenta(L, L, 17, 1, 3)
    assert abs(np.corrcoef(a, b)[0, 1]) < 4 / L
    assert abs(np.corrcoef(a[:-1], a[1:])[0, 1]) < 4 / L
    c = oracle.hmc_momenta(L, L, 17, 0, 4)               # another lattice id
    assert abs(np.corrcoef(a, c)[0, 1]) < 4 / L


def test_creutz_equality():
    """<exp(-dH)> = 1 for an area-preserving reversible integrator at equilibrium."""
    rec, _ = oracle.hmc_run(8, 8, 1.0, 0.25, 4, 6000, seed=3)
    w = np.exp(-rec[500:, 5])
    m, err = jackknife_mean(w)
    assert abs(m - 1.0) < 3.5 * err
    assert 0.5 < rec[:, 6].mean() < 0.99


def test_acceptance_is_min_one_exp_minus_dH():
    """Accept rate of trajectories binned by dH follows min(1, exp(-dH))."""
    rec, _ = oracle.hmc_run(8, 8, 1.0, 0.45, 3, 20000, seed=8)
    dH, acc = rec[:, 5], rec[:, 6]
    checked = 0
    for lo, hi in ((-2.0, -0.2), (0.2, 0.6), (0.6, 1.2), (1.2, 2.5)):
        sel = (dH >= lo) & (dH < hi)
        if sel.sum() < 200:
            continue
        want = np.minimum(1.0, np.exp(-dH[sel])).mean()
        got = acc[sel].mean()
        err = math.sqrt(max(want * (1 - want), 1e-4) / sel.sum())
        assert abs(got - want) < 4 * err + 1e-9, (lo, hi, got, want)
        checked += 1
    assert checked >= 3


@pytest.mark.parametrize("beta", [0.5, 1.0, 2.0])
def test_hmc_samples_exact_2x2_energy(beta):
    rec, _ = oracle.hmc_run(2, 2, beta, 0.3, 4, 30000, seed=21)
    e = -rec[2000:, 0] / 4
    m, err = jackknife_mean(e)
    assert abs(m - ex.e_2x2_bessel(beta)) < 3.5 * err + 1e-6


@pytest.mark.parametrize("Lx,Ly", [(2, 3), (2, 4)])
def test_hmc_samples_exact_small_torus(Lx, Ly):
    beta = 1.0
    N = Lx * Ly
    rec, _ = oracle.hmc_run(Lx, Ly, beta, 0.25, 4, 40000, seed=31 + Ly)
    e = -rec[2000:, 0] / N
    ups = (rec[2000:, 0] - beta * (rec[2000:, 1] ** 2 + rec[2000:, 2] ** 2)) / (2 * N)
    e_ex, u_ex = ex.exact_observables(Lx, Ly, beta)
    me, ee = jackknife_mean(e)
    mu, eu = jackknife_mean(ups)
    assert abs(me - e_ex) < 3.5 * ee + 1e-6
    assert abs(mu - u_ex) < 3.5 * eu + 1e-5


def test_trajectory_rejection_restores_the_state():
    """With a huge step almost every trajectory is rejected: the state is unchanged."""
    Lx = Ly = 6
    th, _ = random_state(Lx, Ly, 4)
    rejected = 0
    for t in range(20):
        out_th, _, info = oracle.hmc_trajectory(th, Lx, Ly, 1.0, 1.5, 6, 9, t)
        if not info["accepted"]:
            rejected += 1
            assert np.array_equal(out_th, th)
        assert info["dH"] == pytest.approx(info["K1"] + info["V1"] - info["K0"] - info["V0"],
                                           abs=1e-9)
    assert rejected >= 15
