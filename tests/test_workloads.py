"""The seeded workload recipes every test and bench line is measured on (CPU).

They carry no arithmetic of the method, only sizes, seeds and parameters; these
checks pin them to the configurations they stand for: the L = 4096 and
L = 16384 single lattices, the 256-lattice replica-exchange layout (3.18 M
sites in 8 ladders of 32 on a 64-point beta grid), the 41-point
differentiation grid and the unit-length HMC trajectory."""
import math
import os
import sys
from collections import Counter

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_0811_2111_gb300 import workloads as WL  # noqa: E402


def test_single_lattice_workloads():
    assert (WL.LARGE.L, WL.LARGE.beta, WL.LARGE.sweeps) == (4096, 1.12, 1000)
    assert WL.LARGE.updates == 4096 * 4096 * 1000
    assert (WL.HUGE.L, WL.HUGE.sweeps) == (16384, 200)
    assert WL.HUGE.sites * 4 == 1 << 30                  # one FP32 plane pair is 1 GiB
    assert (WL.SMALL.L, WL.SMALL.beta) == (32, 1.0)
    for w in (WL.SMALL, WL.LARGE, WL.HUGE, WL.PRECISION_CHECK):
        assert w.L % 2 == 0 and w.delta == math.pi and w.J == 1.0 and w.start == "hot"


def test_batch_layout():
    Ls, betas, ladders = WL.batch_layout()
    assert len(Ls) == len(betas) == len(ladders) == 256
    assert Counter(Ls) == {L: 32 for L in WL.BATCH_LS}
    assert sum(L * L for L in Ls) == 99392 * 32 == 3180544
    grid = np.array(WL.BATCH_BETA_GRID)
    assert grid.size == 64 and grid[0] == 0.8 and abs(grid[-1] - 1.4) < 1e-12
    # one ladder per side, 32 distinct temperatures each, spanning the grid
    for l in range(8):
        idx = [i for i in range(256) if ladders[i] == l]
        assert len(idx) == 32 and len({Ls[i] for i in idx}) == 1
        b = sorted(betas[i] for i in idx)
        assert len(set(b)) == 32 and b[0] < 0.82 and b[-1] > 1.38
    # every grid point carries exactly four lattices
    assert Counter(betas) == {g: 4 for g in WL.BATCH_BETA_GRID}


def test_differentiation_grid():
    b = np.array(WL.DIFF_BETAS)
    assert b.size == 41 and WL.DIFF_L == 256
    assert np.allclose(np.diff(b), 0.01) and b[0] == 0.9 and b[-1] == 1.3


def test_hmc_trajectories_have_unit_length():
    assert WL.HMC_EPS * WL.HMC_NMD == 1.0 and WL.HMC_L == 4096
    for L in (64, 128, 256, 512, 1024, 2048, 4096):
        eps, n = WL.hmc_step_for(L)
        assert abs(eps * n - 1.0) < 1e-12
        # N^(-1/4) scaling from eps = 0.1 at L = 64, up to rounding n to an integer
        assert abs(eps / (0.1 * math.sqrt(64.0 / L)) - 1.0) < 0.05
    assert WL.hmc_step_for(4096) == (WL.HMC_EPS, WL.HMC_NMD)


def test_random_angles_are_seeded_and_in_range():
    a = WL.random_angles(64, 5)
    assert a.dtype == np.float32 and a.shape == (64, 64)
    assert a.min() >= 0.0 and a.max() < np.float32(2 * np.pi)
    assert np.array_equal(a, WL.random_angles(64, 5))
    assert not np.array_equal(a, WL.random_angles(64, 6))
