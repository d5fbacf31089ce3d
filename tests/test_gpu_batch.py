"""Batched engine and replica exchange against the single-lattice path and the oracle (GPU).

* A lattice in a batch evolves bit-identically to the same lattice alone
  (same Philox counters, same site update), whatever the work plan.
* Every replica-exchange step equals the oracle's step computed from the
  GPU's own energies (both in FP64 from the same fixed-point sums).
* A ladder of 2x2 tori samples each temperature's exact energy.
"""
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
from paper_0811_2111_gb300.lattice import Batch, Lattice  # noqa: E402
from paper_0811_2111_gb300 import _lib as X  # noqa: E402
from paper_0811_2111_gb300 import workloads as WL  # noqa: E402

# whole-lattice path (2 ... 96), large tiles (128, 256), cluster bands (100, 130)
LS = [2, 6, 16, 24, 48, 96, 128, 256, 100, 130]
BETAS = [0.7, 0.9, 1.0, 1.1, 1.2, 0.95, 1.05, 1.12, 0.85, 1.15]


def run_batch(target=0, sincos="accurate", rounds=2, spr=5, seed=23, lid0=5, algorithm="auto",
              group_ctas=0, ctas_per_sm=0):
    with Batch(LS, BETAS, seed, lattice_id0=lid0, sweeps_per_round=spr,
               target_band_sites=target, sincos=sincos, algorithm=algorithm,
               group_ctas=group_ctas, ctas_per_sm=ctas_per_sm) as b:
        b.run(rounds)
        n_ctas = b.info()[3]
        return [b.state(i) for i in range(len(LS))], [b.observables(i) for i in range(len(LS))], n_ctas


@pytest.mark.parametrize("sincos,algorithm", [("accurate", "fused"), ("fast", "fused"),
                                              ("accurate", "two_pass")])
def test_batch_matches_single_lattices(sincos, algorithm):
    """Odd rounds of 5 sweeps (2 rounds) leave the fused variant's state in its
    second buffer half way and in the first at the end; both are checked."""
    states, obs, _ = run_batch(sincos=sincos, algorithm=algorithm)
    for i, (L, beta) in enumerate(zip(LS, BETAS)):
        with Lattice(L, beta, 23, lattice_id=5 + i, sincos=sincos, algorithm="two_pass") as lat:
            lat.sweep(10)
            s, _ = lat.state()
            o = lat.observables()
        assert np.array_equal(states[i], s), f"L={L}"
        assert np.array_equal(obs[i]["accepted"], o["accepted"]), f"L={L}"
        assert np.all(obs[i]["beta"] == beta)
        # exact sums: the same per-site terms give the same record bits
        for k in ("C", "Ix", "Iy", "Mx", "My"):
            assert np.array_equal(obs[i][k], o[k]), (L, k)


@pytest.mark.parametrize("sincos,reduce", [("accurate", "exact"), ("fast", "compensated"),
                                           ("libm", "exact")])
def test_narrow_tiles_match_single_lattices(sincos, reduce):
    """Sides that are multiples of 32 but neither of 128 nor small enough for
    one CTA run on the narrow tiles (32 rows x 16 plane columns): 5 x 5 (160,
    not a power of two), 6 x 6 (192) and 7 x 7 (224) tiles per lattice, several
    lattices of a side in one launch; next to them whole lattices (32, 64, 96,
    and 96 twice, and 4, one pair per row, a thread per Philox pair; 30 and
    90, L/2 odd, a thread per site); all against the single-lattice two-pass
    kernels."""
    Ls = [160, 192, 224, 160, 32, 64, 96, 96, 30, 90, 4]
    betas = [0.8, 1.0, 1.12, 1.3, 0.9, 1.2, 0.7, 1.05, 0.95, 1.15, 1.0]
    with Batch(Ls, betas, 31, lattice_id0=3, sweeps_per_round=3, sincos=sincos,
               reduce=reduce) as b:
        b.run(3)
        states = [b.state(i) for i in range(len(Ls))]
        obs = [b.observables(i) for i in range(len(Ls))]
        assert b.info()[3] == 0                       # no lattice left for the cluster launch
    for i, (L, beta) in enumerate(zip(Ls, betas)):
        with Lattice(L, beta, 31, lattice_id=3 + i, sincos=sincos, reduce=reduce,
                     algorithm="two_pass") as lat:
            lat.sweep(9)
            s, _ = lat.state()
            o = lat.observables()
        assert np.array_equal(states[i], s), f"L={L}"
        assert np.array_equal(obs[i]["accepted"], o["accepted"]), f"L={L}"
        tol = record_tolerance(L * L, sincos=sincos, reduce=reduce)
        for k in ("C", "Ix", "Iy", "Mx", "My"):
            if reduce == "exact":
                assert np.array_equal(obs[i][k], o[k]), (L, k)
            else:
                assert np.max(np.abs(obs[i][k] - o[k])) <= tol, (L, k)


def test_fused_batch_state_after_odd_sweeps():
    with Batch([16, 256], [1.0, 1.1], 4, sweeps_per_round=3) as b:
        b.run(1)
        odd = [b.state(i) for i in range(2)]
    for i, (L, beta) in enumerate(((16, 1.0), (256, 1.1))):
        with Lattice(L, beta, 4, lattice_id=i, algorithm="two_pass") as lat:
            lat.sweep(3)
            s, _ = lat.state()
        assert np.array_equal(odd[i], s)


def test_batch_is_independent_of_the_work_plan():
    """Band sizes, the two-pass algorithm, the CTAs per grouped tile launch (1 to
    more than all tiles) and the tile kernel's CTAs per SM: the same bits."""
    ref_states, ref_obs, n0 = run_batch(target=8192)
    for target, algorithm, group, ctas in ((256, "auto", 0, 0), (1024, "auto", 0, 0),
                                           (65536, "auto", 0, 0), (2048, "two_pass", 0, 0),
                                           (256, "two_pass", 0, 0), (8192, "auto", 1, 0),
                                           (8192, "auto", 4096, 2), (8192, "auto", 64, 2),
                                           (8192, "auto", 128, 4)):
        states, obs, n = run_batch(target=target, algorithm=algorithm, group_ctas=group,
                                   ctas_per_sm=ctas)
        for i in range(len(LS)):
            assert np.array_equal(states[i], ref_states[i])
            assert np.array_equal(obs[i]["accepted"], ref_obs[i]["accepted"])
            for k in ("C", "Ix", "Iy", "Mx", "My"):
                assert np.array_equal(obs[i][k], ref_obs[i][k]), (target, algorithm, k)
        print(f"target {target} {algorithm} group {group} ctas {ctas}: {n} CTAs (8192: {n0})")


def test_replica_exchange_matches_oracle_step_by_step():
    Ls = [16] * 9
    betas = [0.8, 0.9, 1.0, 1.1, 1.0, 1.1, 1.2, 1.3, 1.05]
    ladders = [0, 0, 0, 0, 3, 3, 3, 3, -1]
    seed, lid0, spr = 31, 100, 3
    # slot layout: ladders in ascending id, positions in ascending initial beta
    ladder_ids = sorted(set(l for l in ladders if l >= 0))
    ladder_start, pos_lattice, pos_beta = [], [], []
    for l in ladder_ids:
        members = sorted([i for i in range(len(Ls)) if ladders[i] == l], key=lambda i: betas[i])
        ladder_start.append(len(pos_lattice))
        pos_lattice += members
        pos_beta += [betas[i] for i in members]
    n_swaps = 0
    with Batch(Ls, betas, seed, ladders=ladders, lattice_id0=lid0, sweeps_per_round=spr) as b:
        slots, _, _ = b.exchange_stats()
        assert list(slots) == pos_lattice
        beta_now = b.betas()
        for r in range(60):
            b.run(1)
            last = (r + 1) * spr - 1
            energy = np.array([-b.J * b.observables(i, last, 1)["C"][0] for i in range(len(Ls))])
            want_pos, want_beta, swapped = oracle.exchange(ladder_start, pos_lattice, pos_beta,
                                                           beta_now, energy, r, seed, lid0)
            slots, acc, att = b.exchange_stats()
            beta_now = b.betas()
            assert list(slots) == list(want_pos), f"round {r}"
            assert np.array_equal(beta_now, want_beta), f"round {r}"
            pos_lattice = list(want_pos)
            n_swaps += int(swapped.sum())
        assert acc.sum() == n_swaps
        assert beta_now[8] == 1.05                        # not on a ladder: never moves
    assert 0 < n_swaps < 60 * 4


def test_replica_exchange_samples_exact_2x2_energies():
    betas = [0.5, 1.0, 2.0]
    with Batch([2, 2, 2], betas, 3, ladders=[0, 0, 0], sweeps_per_round=2) as b:
        b.run(20000)
        obs = [b.observables(i) for i in range(3)]
    e = np.stack([o["e"] for o in obs])
    bl = np.stack([o["beta"] for o in obs])
    assert np.all(np.sort(bl, axis=0) == np.array(betas)[:, None])
    for beta in betas:
        series = e.T[bl.T == beta]
        m, err = jackknife_mean(series[2000:])
        print(f"beta {beta}: gpu {m:.5f} +- {err:.5f} exact {ex.e_2x2_bessel(beta):.5f}")
        assert abs(m - ex.e_2x2_bessel(beta)) <= 3.5 * err + 1e-6


def test_replica_exchange_ladder_energies_match_oracle_chains():
    """One L = 16 ladder of the replica-exchange workload's kind (8 lattices on every
    eighth point of its 64-point beta grid, exchange every 10 sweeps): <e> at each
    beta, collected from whichever lattice holds that beta, against the oracle's
    parallel-tempering chains (independent seed) within 3.5 sigma, binned jackknife."""
    L, spr, rounds, therm = 16, 10, 2000, 200
    betas = [WL.BATCH_BETA_GRID[4 + 8 * i] for i in range(8)]
    with Batch([L] * 8, betas, 41, ladders=[0] * 8, sweeps_per_round=spr) as b:
        b.run(rounds)
        obs = [b.observables(i) for i in range(8)]
    e_g = np.stack([o["e"] for o in obs])
    b_g = np.stack([o["beta"] for o in obs])
    rec = oracle.pt_run(L, L, betas, rounds, spr, seed=4242)
    e_o = -rec[:, :, 0] / (L * L)
    b_o = rec[:, :, 6]
    for beta in betas:
        sg = e_g.T[b_g.T == beta]
        so = e_o.T[b_o.T == beta]
        assert sg.size == so.size == rounds * spr
        mg, eg = jackknife_mean(sg[therm * spr:])
        mo, eo = jackknife_mean(so[therm * spr:])
        print(f"beta {beta:.4f}: gpu {mg:.5f} +- {eg:.5f}, oracle {mo:.5f} +- {eo:.5f}")
        assert abs(mg - mo) <= 3.5 * np.hypot(eg, eo)


def test_replica_exchange_configuration_runs():
    """The batched workload: 256 lattices, 8 ladders of 32 over a 64-point beta grid."""
    Ls, betas, ladders = WL.batch_layout()
    with Batch(Ls, betas, WL.BATCH_SEED, ladders=ladders, sweeps_per_round=10) as b:
        b.run(20)
        n, nrec, nxt, n_ctas = b.info()
        # fused tiles: L = 256 (16 CTAs per lattice, 4 groups of 8), L = 128 (4 CTAs,
        # one group), one launch per sweep each; L = 16 ... 96 whole lattices in one
        # launch per round; then the exchange
        assert b.launches_per_round() == (4 + 1) * 10 + 1 + 1
        bl = b.betas()
        slots, acc, att = b.exchange_stats()
        e0 = b.observables(0)["e"]
    assert n == 256 and nrec == 200 and nxt == 200
    assert sorted(bl) == sorted(betas)                   # temperatures are only permuted
    assert np.isfinite(e0).all() and -2.0 < e0[-1] < 0.0
    rate = acc.sum() / max(att.sum(), 1)
    print(f"{n_ctas} CTAs, exchange acceptance {rate:.3f}")
    assert 0.05 < rate < 0.99


def test_batch_error_paths():
    with pytest.raises(X.XYError):
        Batch([16, 18], [1.0, 1.0], 1, ladders=[0, 0])   # a ladder mixing sides
    with pytest.raises(X.XYError):
        Batch([512], [1.0], 1)                           # beyond the batch side limit
    with pytest.raises(X.XYError):
        Batch([15], [1.0], 1)                            # odd side


def test_batches_alive_together_keep_their_launch_limits():
    """A kernel's shared-memory limit is one value per process: a batch
    created after another, with smaller lattices on the same kernels (whole
    lattices 16 < 96, cluster bands 130 < 200), leaves the first one runnable
    and its lattices as they would be alone."""
    with Batch([96, 200], [1.0, 1.1], 5, sweeps_per_round=2) as a:
        with Batch([16, 130], [1.0, 1.1], 6, sweeps_per_round=2) as b:
            b.run(1)
            a.run(1)
            b.run(1)
            states = [a.state(i) for i in range(2)]
    for i, (L, beta) in enumerate(((96, 1.0), (200, 1.1))):
        with Lattice(L, beta, 5, lattice_id=i, algorithm="two_pass") as lat:
            lat.sweep(2)
            s, _ = lat.state()
        assert np.array_equal(states[i], s), f"L={L}"
