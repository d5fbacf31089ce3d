"""Precision variants against the FP64 oracle on the identically seeded L=512
lattice (beta=1.12, seed 7): the error of each sincos path and reduction is
measured and bounded (GPU)."""
import numpy as np
import pytest

import oracle
from gpu_util import ANGLE_TOL, compare_record, lockstep_sweep, nthreads, record_tolerance
from stats_util import jackknife_mean

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0811_2111_gb300 import build as _build  # noqa: E402

_build.build()
from paper_0811_2111_gb300.lattice import Lattice  # noqa: E402
from paper_0811_2111_gb300 import workloads as WL  # noqa: E402

BANDS = {"accurate": 1e-6, "libm": 1e-6, "fast": 2e-5}


@pytest.mark.parametrize("sincos,reduce", [("accurate", "exact"), ("libm", "exact"),
                                           ("fast", "exact"), ("accurate", "compensated"),
                                           ("fast", "compensated")])
def test_precision_variant_errors_at_L512(sincos, reduce):
    w = WL.PRECISION_CHECK
    L, n = w.L, 20
    fast = sincos == "fast"
    stats = dict(out_1e6=0, out_band=0, in_band=0, angle=0.0, rec=np.zeros(5))
    with Lattice(L, w.beta, w.seed, sincos=sincos, reduce=reduce) as lat:
        before, t0 = lat.state()
        for i in range(n):
            lat.sweep(1)
            after, _ = lat.state()
            for band, key in ((1e-6, "out_1e6"), (BANDS[sincos], "out_band")):
                red, blk = lockstep_sweep(before, after, L, w.beta, w.seed, t0 + i, band=band)
                stats[key] += red.out_band_mismatch + blk.out_band_mismatch
            stats["in_band"] += red.in_band + blk.in_band
            stats["angle"] = max(stats["angle"], red.max_angle_err, blk.max_angle_err)
            obs = lat.observables(i, 1)
            diff, _ = compare_record({k: obs[k][0] for k in obs}, after, L)
            stats["rec"] = np.maximum(stats["rec"], diff)
            before = after
    print(f"{sincos}/{reduce}: decisions outside 1e-6 band differing {stats['out_1e6']}, "
          f"outside the {BANDS[sincos]:g} band {stats['out_band']}, max angle error "
          f"{stats['angle']:.2e}, max |record - FP64| (C, Ix, Iy, Mx, My) {stats['rec']}")
    assert stats["out_band"] == 0
    assert stats["angle"] <= ANGLE_TOL
    assert stats["rec"].max() <= record_tolerance(L * L, sincos=sincos, reduce=reduce)


def test_free_running_observables_vs_oracle_L512():
    """Free-running chains on the L=512 precision lattice: GPU (accurate sincos) against
    the FP64 oracle, 12 independent seeds each (the identically seeded pair first).
    A chain's value is its average of e, |m| and Upsilon over sweeps 100..199; the GPU
    and oracle ensemble means must agree within 3 sigma, sigma from the jackknife over
    the independent chains of each side."""
    w = WL.PRECISION_CHECK
    seeds = [w.seed] + [w.seed + 1000 + i for i in range(11)]
    g_means, o_means = [], []
    first_div = None
    for k, seed in enumerate(seeds):
        with Lattice(w.L, w.beta, seed) as lat:
            lat.sweep(w.sweeps)
            g = lat.observables()
        rec, _ = oracle.run(w.L, w.L, w.beta, w.sweeps, seed=seed, nthreads=nthreads())
        e, m, u = oracle.observables(rec[:, :5], w.L * w.L, w.beta)
        if k == 0:
            off = np.abs(g["e"] - e) > 1e-6
            first_div = int(np.argmax(off)) if np.any(off) else w.sweeps
        g_means.append([g["e"][100:].mean(), g["abs_m"][100:].mean(), g["upsilon"][100:].mean()])
        o_means.append([e[100:].mean(), m[100:].mean(), u[100:].mean()])
    g_means, o_means = np.array(g_means), np.array(o_means)
    print(f"free-running L=512: identically seeded per-sweep e equal to 1e-6 for the first "
          f"{first_div} sweeps")
    assert first_div >= 1
    for j, name in enumerate(("e", "|m|", "Upsilon")):
        mg, eg = jackknife_mean(g_means[:, j], n_bins=len(seeds))
        mo, eo = jackknife_mean(o_means[:, j], n_bins=len(seeds))
        err = np.hypot(eg, eo)
        print(f"  <{name}> gpu {mg:.6f} +- {eg:.6f}, oracle {mo:.6f} +- {eo:.6f}")
        assert abs(mg - mo) <= 3.0 * err, name
