"""The work-plan autotuner (GPU): timed candidates, the winner among them,
the on-disk cache, and plans that change nothing but the time.

autotune.tune_lattice and tune_batch time every candidate plan on a throw-away
copy of the workload and cache the fastest per (GPU, library version, shape,
precision).  A plan never changes results, so the tuned plan's sweep must give
the same bits as the library's default plan.
"""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0811_2111_gb300 import build as _build  # noqa: E402

_build.build()
from paper_0811_2111_gb300 import autotune  # noqa: E402
from paper_0811_2111_gb300.lattice import Batch, Lattice  # noqa: E402


def test_lattice_plan_is_the_fastest_candidate_and_is_cached(tmp_path, monkeypatch):
    monkeypatch.setenv("XY_GB300_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    plan = autotune.tune_lattice(512, sweeps=20, repeats=2)
    times = plan["ms_per_sweep"]
    assert set(times) == {f"{a}/{c}" for a, c in autotune.LATTICE_CANDIDATES}
    assert all(t > 0 for t in times.values())
    assert f"{plan['algorithm']}/{plan['ctas_per_sm']}" == min(times, key=times.get)
    with open(tmp_path / "cache.json") as f:
        cache = json.load(f)
    assert any(v == plan for v in cache.values())
    # a second call is served from the cache (the same dict, no re-timing)
    assert autotune.tune_lattice(512, sweeps=20, repeats=2) == plan
    # sides the fused tiles do not take have one plan
    assert autotune.tune_lattice(100, use_cache=False)["algorithm"] == "two_pass"


def test_tuned_lattice_plan_gives_the_default_plans_bits(tmp_path, monkeypatch):
    monkeypatch.setenv("XY_GB300_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    plan = autotune.tune_lattice(1024, sweeps=10, repeats=1)
    out = []
    for kw in ({}, {"algorithm": plan["algorithm"], "ctas_per_sm": plan["ctas_per_sm"]}):
        with Lattice(1024, 1.1, 31, **kw) as lat:
            lat.sweep(6)
            s, _ = lat.state()
            o = lat.observables()
        out.append((s, o))
    assert np.array_equal(out[0][0], out[1][0])
    for k in ("C", "Ix", "Iy", "Mx", "My", "accepted"):
        assert np.array_equal(out[0][1][k], out[1][1][k]), k


def test_batch_plan_is_the_fastest_candidate(tmp_path, monkeypatch):
    monkeypatch.setenv("XY_GB300_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    Ls = [16, 48, 128, 256, 100]
    betas = [0.9, 1.0, 1.05, 1.1, 1.2]
    plan = autotune.tune_batch(Ls, betas, sweeps_per_round=4, rounds=2,
                               group_ctas=(16, 128), ctas_per_sm=(3, 4))
    times = plan["ms_per_round"]
    # banded lattices exist (L = 100), so both band sizes are candidates
    assert len(times) == 2 * 2 * len(autotune.BAND_TARGETS)
    win = min(times, key=times.get)
    assert win == f"{plan['group_ctas']}/{plan['ctas_per_sm']}/{plan['target_band_sites']}"
    states = []
    for kw in ({}, {"group_ctas": plan["group_ctas"], "ctas_per_sm": plan["ctas_per_sm"],
                    "target_band_sites": plan["target_band_sites"]}):
        with Batch(Ls, betas, 9, sweeps_per_round=4, **kw) as b:
            b.run(2)
            states.append([b.state(i) for i in range(len(Ls))])
    for a, c in zip(*states):
        assert np.array_equal(a, c)
