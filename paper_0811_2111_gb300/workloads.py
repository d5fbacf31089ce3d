"""Seeded workload definitions shared by tests, the smoke check and bench.py.

Only sizes, seeds and parameter values live here -- none of the method's
arithmetic.  Every run starts from the Philox hot start of its seed (uniform
i.i.d. angles), which is the whole input of the method: the paper measures on
no dataset.
"""
import math
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    L: int
    beta: float
    seed: int
    sweeps: int
    J: float = 1.0
    delta: float = math.pi
    start: str = "hot"

    @property
    def sites(self):
        return self.L * self.L

    @property
    def updates(self):
        return self.sites * self.sweeps


# The single-lattice configurations (plain method small/large, precision run).
SMALL = Workload("xy_L32_beta1.0_seed1_1000sweeps", L=32, beta=1.0, seed=1, sweeps=1000)
LARGE = Workload("xy_L4096_beta1.12_seed7_1000sweeps", L=4096, beta=1.12, seed=7, sweeps=1000)
HUGE = Workload("xy_L16384_beta1.12_seed7_200sweeps", L=16384, beta=1.12, seed=7, sweeps=200)
PRECISION_CHECK = Workload("xy_L512_beta1.12_seed7", L=512, beta=1.12, seed=7, sweeps=200)

# Batched replica-exchange configuration: 8 ladders (one per L) of 32
# lattices on alternate points of a 64-point beta grid in [0.8, 1.4].
BATCH_LS = (16, 24, 32, 48, 64, 96, 128, 256)
BATCH_BETA_GRID = tuple(np.linspace(0.8, 1.4, 64).tolist())
BATCH_SEED = 11

# Differentiation configuration: 41 beta values in [0.9, 1.3] at L = 256.
DIFF_L = 256
DIFF_BETAS = tuple(np.round(np.linspace(0.9, 1.3, 41), 10).tolist())
DIFF_SEED = 13


# Hybrid Monte Carlo configuration (the paper's own algorithm, Sec. 1.2): the
# throughput lattice and beta, unit trajectory length.  The step is scaled
# with N^(-1/4), which keeps the mean energy violation, and so the acceptance,
# roughly constant across sides (an L = 64 chain at eps = 0.1, 10 steps,
# accepts ~0.83; L = 4096 has 4096 times the sites, eps / 8).
HMC_L = 4096
HMC_BETA = 1.12
HMC_SEED = 7
HMC_EPS = 0.0125
HMC_NMD = 80
HMC_METROPOLIS_THERM = 2000    # Metropolis sweeps that thermalise the HMC start
HMC_THERM = 30                 # HMC trajectories discarded before timing


def hmc_step_for(L, trajectory_length=1.0):
    """(eps, n_md) with eps = 0.1 (64 / L)^(1/2) (i.e. N^(-1/4) scaling from L = 64)."""
    eps = 0.1 * math.sqrt(64.0 / L)
    n_md = max(1, int(round(trajectory_length / eps)))
    return trajectory_length / n_md, n_md


def random_angles(L, seed):
    """Uniform angles in [0, 2 pi) as float32 natural-order [L, L] (numpy PCG64)."""
    rng = np.random.default_rng(seed)
    return (rng.random((L, L)) * (2 * np.pi)).astype(np.float32) % np.float32(2 * np.pi)


def batch_layout():
    """The replica-exchange workload: 8 ladders, one per side in BATCH_LS; ladder l
    holds 32 lattices on the beta-grid points b = l mod 2, l mod 2 + 2, ..., so every
    grid point carries exactly 4 lattices and every side spans [0.8, 1.4].
    Returns (Ls, betas, ladders) of the 256 lattices, ladder-major."""
    Ls, betas, ladders = [], [], []
    for l, L in enumerate(BATCH_LS):
        for j in range(32):
            Ls.append(L)
            betas.append(BATCH_BETA_GRID[(l % 2) + 2 * j])
            ladders.append(l)
    return Ls, betas, ladders
