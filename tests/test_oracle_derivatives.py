"""Pins of the oracle's beta derivatives against exact tori (CPU only).

``oracle.beta_derivatives`` estimates d<e>/dbeta and d<Upsilon>/dbeta of one
fixed-beta chain from its per-sweep bond sums: the fluctuation formula
d<O>/dbeta = <dO/dbeta> - cov(O, E) of the Boltzmann weight e^{-beta H},
Eq. (1).  For Upsilon_s = (J C - beta J^2 (Ix^2 + Iy^2)) / (2N) the first
term is -J^2 <Ix^2 + Iy^2> / (2N); for e it vanishes.

The exact values here come from elsewhere: a central difference in beta of
the exact <e>(beta) and <Upsilon>(beta) of the 2x4 and 4x2 tori, where
<Upsilon> is the curvature of the transfer-matrix free energy under a
boundary twist (``exact_small``).  On a side of 2 one current vanishes
identically (each pair is bonded in both directions), so the 2x4 torus
checks the y currents and the 4x2 torus the x currents.  A sign error, a
missing factor or a dropped explicit-beta term in the oracle fails here; the
test plants the last two in a copy of the oracle's function to show it.
"""
import numpy as np
import pytest

import oracle
import exact_small as ex
from stats_util import jackknife_func

N_SWEEPS = 400000
THERM = 4000


def _exact_derivatives(Lx, Ly, beta, h=2e-3):
    ep, up = ex.exact_observables(Lx, Ly, beta + h)
    em, um = ex.exact_observables(Lx, Ly, beta - h)
    return (ep - em) / (2 * h), (up - um) / (2 * h)


def _series(Lx, Ly, beta, seed):
    rec, _ = oracle.run(Lx, Ly, beta, N_SWEEPS, seed=seed)
    return rec[THERM:, :3]


def _errors(sums, N, beta, explicit_sign=1.0, J=1.0):
    """Binned-jackknife value and error of both derivatives from the chain.

    explicit_sign multiplies the explicit-beta term of d<Upsilon>/dbeta (1 is
    the formula; -1 and 0 are the planted mistakes)."""
    Cb, Ix, Iy = sums[:, 0], sums[:, 1], sums[:, 2]
    E = -J * Cb
    e = E / N
    jj = Ix * Ix + Iy * Iy
    u = (J * Cb - beta * J * J * jj) / (2.0 * N)
    de = jackknife_func([e, E, e * E], lambda a, b, ab: -(ab - a * b))
    du = jackknife_func([u, E, u * E, jj],
                        lambda a, b, ab, j: -(ab - a * b) - explicit_sign * J * J * j / (2.0 * N))
    return de, du


@pytest.mark.parametrize("Lx,Ly,beta", [(2, 4, 0.5), (2, 4, 1.0), (4, 2, 0.5), (4, 2, 1.0)])
def test_beta_derivatives_match_exact_tori(Lx, Ly, beta):
    N = Lx * Ly
    sums = _series(Lx, Ly, beta, seed=300 + 10 * Lx + int(10 * beta))
    got = oracle.beta_derivatives(sums, N, beta)
    (de, de_err), (du, du_err) = _errors(sums, N, beta)
    # the oracle's estimator is the jackknife's full-sample value
    assert got["de"] == pytest.approx(de, rel=1e-9)
    assert got["dupsilon"] == pytest.approx(du, rel=1e-9)
    ex_de, ex_du = _exact_derivatives(Lx, Ly, beta)
    # the covariance-only reading of d<Upsilon>/dbeta, reported beside the full one
    (cov_only, cov_err) = _errors(sums, N, beta, explicit_sign=0.0)[1]
    print(f"{Lx}x{Ly} beta {beta}: d<e>/dbeta {got['de']:.5f} +- {de_err:.5f} "
          f"(exact {ex_de:.5f}); d<Y>/dbeta {got['dupsilon']:.5f} +- {du_err:.5f} "
          f"(exact {ex_du:.5f}; covariance only {cov_only:.5f} +- {cov_err:.5f})")
    assert abs(got["de"] - ex_de) <= 3.5 * de_err
    assert abs(got["dupsilon"] - ex_du) <= 3.5 * du_err
    # the explicit-beta term is resolved: without it, or with its sign
    # flipped, the estimate misses the exact derivative by many errors
    assert abs(cov_only - ex_du) > 8 * cov_err
    (flip, flip_err) = _errors(sums, N, beta, explicit_sign=-1.0)[1]
    assert abs(flip - ex_du) > 8 * flip_err


def test_planted_mistakes_in_the_oracle_formula_fail():
    """Copies of oracle.beta_derivatives with a flipped or dropped explicit-beta
    term, or the covariance's sign flipped, miss the exact derivative."""
    import inspect
    import textwrap
    src = textwrap.dedent(inspect.getsource(oracle.beta_derivatives))
    good_term = "- J * J * jj.mean() / (2.0 * N)"
    good_cov = '"de": -np.mean('
    assert good_term in src and good_cov in src
    mutants = {
        "explicit term sign": src.replace(good_term, "+ J * J * jj.mean() / (2.0 * N)"),
        "explicit term dropped": src.replace(good_term, "+ 0.0"),
        "explicit term factor 2": src.replace(good_term, "- J * J * jj.mean() / N"),
        "covariance sign": src.replace(good_cov, '"de": np.mean('),
    }
    Lx, Ly, beta = 4, 2, 1.0
    N = Lx * Ly
    sums = _series(Lx, Ly, beta, seed=77)
    (_, de_err), (_, du_err) = _errors(sums, N, beta)
    ex_de, ex_du = _exact_derivatives(Lx, Ly, beta)
    good = oracle.beta_derivatives(sums, N, beta)
    assert abs(good["de"] - ex_de) <= 3.5 * de_err
    assert abs(good["dupsilon"] - ex_du) <= 3.5 * du_err
    for name, code in mutants.items():
        ns = {"np": np}
        exec(code, ns)
        bad = ns["beta_derivatives"](sums, N, beta)
        missed = (abs(bad["de"] - ex_de) > 3.5 * de_err
                  or abs(bad["dupsilon"] - ex_du) > 3.5 * du_err)
        assert missed, name
