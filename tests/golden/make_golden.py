"""Write the stored expected values used by the GPU tests.  Calls only oracle/.

ensemble_L32_beta1.0.json: per-chain means of e, |m|, Upsilon and the
acceptance rate for 64 independent FP64 oracle chains of the small
configuration (L=32, beta=1, J=1, delta=pi, hot start), 10^4 sweeps each,
first 10^3 discarded; seeds 5000..5063, lattice_id 0.  The GPU long-run test
compares the mean of its own independent chains with this ensemble, using
the ensemble's chain-to-chain spread as the error (single-chain jackknife
errors underestimate it near the BKT region).

Run:  python tests/golden/make_golden.py
"""
import json
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

L, BETA, SWEEPS, DISCARD = 32, 1.0, 10000, 1000
SEEDS = list(range(5000, 5064))


def chain(seed):
    import oracle
    rec, _ = oracle.run(L, L, BETA, SWEEPS, seed=seed)
    e, m, u = oracle.observables(rec[DISCARD:, :5], L * L, BETA)
    return [float(e.mean()), float(m.mean()), float(u.mean()),
            float(rec[DISCARD:, 5].mean() / (L * L))]


def main():
    with mp.get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as pool:
        rows = pool.map(chain, SEEDS)
    out = {
        "what": "per-chain means of the FP64 oracle, small configuration",
        "L": L, "beta": BETA, "J": 1.0, "delta": "pi", "start": "hot",
        "sweeps": SWEEPS, "discard": DISCARD, "seeds": SEEDS, "lattice_id": 0,
        "columns": ["e", "abs_m", "upsilon", "acceptance"],
        "chains": rows,
        "written_by": "tests/golden/make_golden.py (oracle only)",
    }
    with open(os.path.join(HERE, "ensemble_L32_beta1.0.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
