"""d<O>/dbeta through autograd: the backward kernel against the oracle's
formula, exact 2x2 derivatives, finite differences and oracle chains (GPU)."""
import numpy as np
import pytest

import oracle
import exact_small as ex
from stats_util import jackknife_func

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0811_2111_gb300 import build as _build  # noqa: E402

_build.build()
from paper_0811_2111_gb300.lattice import Batch  # noqa: E402
from paper_0811_2111_gb300.autograd import chain_averages  # noqa: E402


def test_backward_kernel_equals_oracle_formula_on_the_same_series():
    betas = [0.8, 1.0, 1.3]
    with Batch([16, 16, 16], betas, 5, sweeps_per_round=100) as b:
        b.run(30)
        stats = b.series_stats(500, 2500).cpu().numpy()
        obs = [b.observables(i, 500, 2500) for i in range(3)]
    for i, beta in enumerate(betas):
        sums = np.stack([obs[i]["C"], obs[i]["Ix"], obs[i]["Iy"]], axis=1)
        ref = oracle.beta_derivatives(sums, 256, beta)
        got = dict(e=stats[i, 0], upsilon=stats[i, 1], de=stats[i, 3], dupsilon=stats[i, 4],
                   varE_over_N=stats[i, 6])
        for k, v in ref.items():
            assert got[k] == pytest.approx(v, rel=1e-9, abs=1e-12), k
        assert stats[i, 7] == 2500


@pytest.mark.parametrize("beta", [0.5, 1.0])
def test_derivative_of_2x2_energy_is_exact(beta):
    """d<e>/dbeta on the 2x2 torus against the Bessel-sum partition function."""
    n = 200000
    with Batch([2], [beta], 7, sweeps_per_round=1000) as b:
        b.run(n // 1000 + 10)
        stats = b.series_stats(10000, n).cpu().numpy()[0]
        o = b.observables(0, 10000, n)
    h = 1e-4
    exact = (ex.e_2x2_bessel(beta + h) - ex.e_2x2_bessel(beta - h)) / (2 * h)
    E = -o["C"]
    val, err = jackknife_func([E / 4, E, E * E / 4], lambda a, b, ab: -(ab - a * b), n_bins=50)
    assert stats[3] == pytest.approx(val, rel=1e-6)
    print(f"beta {beta}: gpu {stats[3]:.5f} +- {err:.5f} exact {exact:.5f}")
    assert abs(stats[3] - exact) <= 3.5 * err
    # on a side of 2 the currents vanish: Upsilon_s = -e_s / 2 sweep by sweep
    assert stats[4] == pytest.approx(-stats[3] / 2, rel=1e-9)


def test_autograd_matches_finite_differences():
    """Backward at beta vs (<O>(beta + 0.01) - <O>(beta - 0.01)) / 0.02 for O = e and
    O = Upsilon, 8 chains each; the covariance-only part of d<Upsilon>/dbeta (the
    explicit-beta term -J^2 <Ix^2 + Iy^2> / (2N) left out) is reported beside it."""
    L, chains, therm, meas = 16, 8, 2000, 60000
    grid = [0.99, 1.0, 1.01]
    betas = torch.tensor([b for b in grid for _ in range(chains)], dtype=torch.float64,
                         requires_grad=True)
    e, u = chain_averages(betas, L, 11, therm, meas, sweeps_per_round=1000)
    (g_e,) = torch.autograd.grad(e.sum(), betas, retain_graph=True)
    (g_u,) = torch.autograd.grad(u.sum(), betas)
    with Batch([L] * chains, [grid[1]] * chains, 11, sweeps_per_round=1000,
               lattice_id0=chains) as b:
        b.run((therm + meas) // 1000)
        s = b.series_stats(therm, meas).cpu().numpy()
    for name, val, grad in (("e", e, g_e), ("Y", u, g_u)):
        v = val.detach().cpu().numpy().reshape(3, chains)
        d = grad.cpu().numpy().reshape(3, chains)
        fd = (v[2] - v[0]) / 0.02
        fd_err = np.hypot(v[2].std(ddof=1), v[0].std(ddof=1)) / np.sqrt(chains) / 0.02
        bw, bw_err = d[1].mean(), d[1].std(ddof=1) / np.sqrt(chains)
        extra = ""
        if name == "Y":
            extra = f" (covariance only {s[:, 5].mean():.4f})"
            # the same chains' full and covariance-only parts differ by the
            # explicit-beta term, which is negative
            assert np.all(s[:, 4] < s[:, 5])
        print(f"d<{name}>/dbeta: backward {bw:.4f} +- {bw_err:.4f}, finite difference "
              f"{fd.mean():.4f} +- {fd_err:.4f}{extra}")
        assert abs(bw - fd.mean()) <= 3.5 * np.hypot(bw_err, fd_err), name


def test_autograd_matches_oracle_chains():
    """Backward d<e>/dbeta and d<Upsilon>/dbeta at L=32, beta=1 vs oracle chains."""
    L, beta, therm, meas, chains = 32, 1.0, 2000, 20000, 8
    betas = torch.full((chains,), beta, dtype=torch.float64, requires_grad=True)
    e, u = chain_averages(betas, L, 21, therm, meas, sweeps_per_round=1000)
    (g_e,) = torch.autograd.grad(e.sum(), betas, retain_graph=False)
    betas2 = torch.full((chains,), beta, dtype=torch.float64, requires_grad=True)
    e2, u2 = chain_averages(betas2, L, 21, therm, meas, sweeps_per_round=1000)
    (g_u,) = torch.autograd.grad(u2.sum(), betas2)
    de = g_e.cpu().numpy()
    du = g_u.cpu().numpy()
    ref_de, ref_du = [], []
    for c in range(4):
        rec, _ = oracle.run(L, L, beta, therm + meas // 2, seed=900 + c)
        r = oracle.beta_derivatives(rec[therm:, :3], L * L, beta)
        ref_de.append(r["de"])
        ref_du.append(r["dupsilon"])
    for name, g, o in (("de", de, np.array(ref_de)), ("dY", du, np.array(ref_du))):
        err = np.hypot(g.std(ddof=1) / np.sqrt(g.size), o.std(ddof=1) / np.sqrt(o.size))
        print(f"{name}: gpu {g.mean():.4f} oracle {o.mean():.4f} +- {err:.4f}")
        assert abs(g.mean() - o.mean()) <= 3.5 * err


def test_backward_combines_both_outputs():
    betas = torch.tensor([0.9, 1.1], dtype=torch.float64, requires_grad=True)
    e, u = chain_averages(betas, 8, 3, 200, 2000, sweeps_per_round=100)
    w = torch.tensor([2.0, -1.0], dtype=torch.float64)
    (g,) = torch.autograd.grad((w * e).sum() + (3.0 * u).sum(), betas)
    with Batch([8, 8], [0.9, 1.1], 3, sweeps_per_round=100) as b:
        b.run(22)
        s = b.series_stats(200, 2000).cpu().numpy()
    assert np.allclose(g.cpu().numpy(), w.numpy() * s[:, 3] + 3.0 * s[:, 4], rtol=1e-12)
