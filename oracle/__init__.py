"""FP64 CPU oracle for the checkerboard Metropolis XY path.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline arm, never by the library.  The arithmetic
lives in ``xy_oracle.c`` (plain C, double precision, its own Philox); this
module only marshals numpy arrays through ctypes.

Site order is natural: s = y * Lx + x.  Colour of a site: (x + y) mod 2.
Every function cites the passage it follows in ``xy_oracle.c``.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_U32 = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_I64 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_U8 = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


def _optional(nd):
    """ndpointer that also accepts None (passed as NULL)."""
    class _Opt(nd):
        @classmethod
        def from_param(cls, obj):
            if obj is None:
                return None
            return super().from_param(obj)
    return _Opt


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_philox4x32_10.argtypes = [_U32, _U32, _U32]
        L.orc_philox_words.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32,
                                       C.c_uint32, C.c_int64, _U32]
        L.orc_measure.argtypes = [C.c_int, C.c_int, _D, _D]
        L.orc_delta_energy.argtypes = [C.c_int, C.c_int, _D, C.c_int64, C.c_double, C.c_double]
        L.orc_delta_energy.restype = C.c_double
        L.orc_start.argtypes = [C.c_int, C.c_int, C.c_uint64, C.c_uint32, C.c_int, _D]
        L.orc_attempt_sites.argtypes = [C.c_int, C.c_int, _D, _I64, C.c_int64, C.c_double,
                                        C.c_double, C.c_double, C.c_uint64, C.c_uint32,
                                        C.c_uint32, C.c_int, _optional(_D), _optional(_D),
                                        _optional(_D), _optional(_U8)]
        L.orc_half_sweep.argtypes = [C.c_int, C.c_int, _D, C.c_int, C.c_double, C.c_double,
                                     C.c_double, C.c_uint64, C.c_uint32, C.c_uint32, C.c_int,
                                     _optional(_D), _optional(_D), _optional(_D),
                                     _optional(_U8)]
        L.orc_half_sweep.restype = C.c_int64
        L.orc_sweep.argtypes = [C.c_int, C.c_int, _D, C.c_double, C.c_double, C.c_double,
                                C.c_uint64, C.c_uint32, C.c_uint32, C.c_int, C.c_int]
        L.orc_sweep.restype = C.c_int64
        L.orc_run.argtypes = [C.c_int, C.c_int, C.c_uint64, C.c_uint32, C.c_double, C.c_double,
                              C.c_double, C.c_int, C.c_int, C.c_uint32, C.c_int64, C.c_int,
                              _optional(_D), _optional(_D)]
        L.orc_run.restype = C.c_int
        L.orc_max_threads.restype = C.c_int
        _I32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
        L.orc_exchange.argtypes = [C.c_int, _I32, C.c_int, _I32, _D, _D, _D, C.c_uint32,
                                   C.c_uint64, C.c_uint32, _optional(_U8)]
        L.orc_pt_run.argtypes = [C.c_int, C.c_int, C.c_int, _D, C.c_double, C.c_double,
                                 C.c_uint64, C.c_uint32, C.c_int, C.c_int, _D]
        L.orc_pt_run.restype = C.c_int
        L.orc_hmc_momenta.argtypes = [C.c_int, C.c_int, C.c_uint64, C.c_uint32, C.c_uint32, _D]
        L.orc_hmc_force.argtypes = [C.c_int, C.c_int, _D, C.c_double, C.c_double, _D]
        L.orc_hmc_hamiltonian.argtypes = [C.c_int, C.c_int, _D, _D, C.c_double, C.c_double, _D]
        L.orc_hmc_leapfrog.argtypes = [C.c_int, C.c_int, _D, _D, C.c_double, C.c_double,
                                       C.c_double, C.c_int]
        L.orc_hmc_leapfrog.restype = C.c_int
        L.orc_hmc_trajectory.argtypes = [C.c_int, C.c_int, _D, C.c_double, C.c_double,
                                         C.c_double, C.c_int, C.c_uint64, C.c_uint32,
                                         C.c_uint32, _D, _optional(_D)]
        L.orc_hmc_trajectory.restype = C.c_int
        L.orc_hmc_run.argtypes = [C.c_int, C.c_int, C.c_uint64, C.c_uint32, C.c_double,
                                  C.c_double, C.c_double, C.c_int, C.c_int, C.c_uint32,
                                  C.c_int64, _optional(_D), _optional(_D)]
        L.orc_hmc_run.restype = C.c_int
        _lib = L
    return _lib


def max_threads() -> int:
    return int(lib().orc_max_threads())


def philox4x32_10(ctr, key):
    """Philox4x32-10 of one counter block (Salmon et al., SC'11)."""
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def philox_words(seed, sweep, lattice_id, domain, first, n):
    """Words for counters (first + i, sweep, lattice_id, domain), shape (n, 4)."""
    out = np.zeros((n, 4), np.uint32)
    lib().orc_philox_words(seed, sweep, lattice_id, domain, first, n, out)
    return out


def measure(theta, Lx, Ly=None):
    """{C, Ix, Iy, Mx, My} of one configuration (Eq. (1) bond sums)."""
    Ly = Lx if Ly is None else Ly
    th = np.ascontiguousarray(theta, np.float64).reshape(-1)
    out = np.zeros(5, np.float64)
    lib().orc_measure(Lx, Ly, th, out)
    return out


def observables(sums, N, beta, J=1.0):
    """e, |m|, Upsilon from bond/spin sums (arrays of shape (..., 5))."""
    sums = np.asarray(sums, np.float64)
    Cb, Ix, Iy, Mx, My = (sums[..., i] for i in range(5))
    e = -J * Cb / N
    m = np.sqrt(Mx * Mx + My * My) / N
    ups = (J * Cb - beta * J * J * (Ix * Ix + Iy * Iy)) / (2.0 * N)
    return e, m, ups


def delta_energy(theta, Lx, Ly, s, theta_new, J=1.0):
    th = np.ascontiguousarray(theta, np.float64).reshape(-1)
    return float(lib().orc_delta_energy(Lx, Ly, th, int(s), float(theta_new), float(J)))


def start(Lx, Ly, seed, lattice_id=0, hot=True):
    th = np.zeros(Lx * Ly, np.float64)
    lib().orc_start(Lx, Ly, seed, lattice_id, 1 if hot else 0, th)
    return th


def attempt_sites(theta, Lx, Ly, sites, beta, seed, sweep, lattice_id=0, J=1.0,
                  delta=np.pi, nthreads=1):
    """Metropolis step of `sweep` at each listed site against `theta` (unchanged).

    Returns (theta_prop, u1, p, accept) per listed site."""
    th = np.ascontiguousarray(theta, np.float64).reshape(-1)
    sites = np.ascontiguousarray(sites, np.int64)
    n = sites.size
    tp, u1, p = (np.zeros(n, np.float64) for _ in range(3))
    acc = np.zeros(n, np.uint8)
    lib().orc_attempt_sites(Lx, Ly, th, sites, n, beta, J, delta, seed, lattice_id, sweep,
                            nthreads, tp, u1, p, acc)
    return tp, u1, p, acc.astype(bool)


def half_sweep(theta, Lx, Ly, colour, beta, seed, sweep, lattice_id=0, J=1.0,
               delta=np.pi, nthreads=1):
    """Apply the colour-`colour` half-sweep to a copy of theta.

    Returns (new_theta, theta_prop, u1, p, accept); per-site arrays are
    indexed by natural site id and only meaningful on sites of that colour."""
    th = np.array(theta, np.float64).reshape(-1)
    N = Lx * Ly
    tp, u1, p = (np.full(N, np.nan) for _ in range(3))
    acc = np.zeros(N, np.uint8)
    r = lib().orc_half_sweep(Lx, Ly, th, colour, beta, J, delta, seed, lattice_id, sweep,
                             nthreads, tp, u1, p, acc)
    if r < 0:
        raise MemoryError("oracle half-sweep failed")
    return th, tp, u1, p, acc.astype(bool)


def sweep(theta, Lx, Ly, beta, seed, sweep_index, lattice_id=0, J=1.0, delta=np.pi,
          order=0, nthreads=1):
    """One sweep in place on a float64 array; returns accepted count."""
    assert theta.dtype == np.float64 and theta.flags.c_contiguous
    r = lib().orc_sweep(Lx, Ly, theta, beta, J, delta, seed, lattice_id, sweep_index, order,
                        nthreads)
    if r < 0:
        raise ValueError("checkerboard order needs even Lx and Ly")
    return int(r)


def run(Lx, Ly, beta, n_sweeps, seed, lattice_id=0, J=1.0, delta=np.pi, start=1, order=0,
        first_sweep=0, theta=None, nthreads=1):
    """Free-running chain; returns (records[n, 6], final_theta).

    records[i] = (C, Ix, Iy, Mx, My, accepted) after sweep first_sweep + i.
    start: 1 hot, 0 cold, -1 from `theta`."""
    N = Lx * Ly
    th = np.zeros(N, np.float64) if theta is None else np.array(theta, np.float64).reshape(-1)
    rec = np.zeros((n_sweeps, 6), np.float64)
    r = lib().orc_run(Lx, Ly, seed, lattice_id, beta, J, delta, start, order, first_sweep,
                      n_sweeps, nthreads, th, rec)
    if r != 0:
        raise ValueError("oracle run failed (odd side with checkerboard order?)")
    return rec, th


def exchange(ladder_start, pos_lattice, pos_beta, beta_of_lattice, energy, round_index, seed,
             lattice_id0=0):
    """One replica-exchange step; returns (pos_lattice, beta_of_lattice, swapped) updated copies."""
    ls = np.ascontiguousarray(ladder_start, np.int32)
    pl = np.array(pos_lattice, np.int32)
    pb = np.ascontiguousarray(pos_beta, np.float64)
    bl = np.array(beta_of_lattice, np.float64)
    en = np.ascontiguousarray(energy, np.float64)
    sw = np.zeros(pl.size, np.uint8)
    lib().orc_exchange(ls.size, ls, pl.size, pl, pb, bl, en, round_index, seed, lattice_id0, sw)
    return pl, bl, sw.astype(bool)


def pt_run(Lx, Ly, betas, rounds, sweeps_per_round, seed, lattice_id0=0, J=1.0, delta=np.pi):
    """Parallel tempering of one ladder; records (n, rounds*sweeps_per_round, 7):
    C, Ix, Iy, Mx, My, accepted, beta of each lattice after each sweep."""
    b = np.ascontiguousarray(betas, np.float64)
    total = rounds * sweeps_per_round
    rec = np.zeros((b.size, total, 7), np.float64)
    r = lib().orc_pt_run(Lx, Ly, b.size, b, J, delta, seed, lattice_id0, sweeps_per_round,
                         rounds, rec)
    if r != 0:
        raise ValueError("oracle parallel-tempering run failed")
    return rec


def beta_derivatives(sums, N, beta, J=1.0):
    """Averages and beta derivatives of one fixed-beta chain from its per-sweep sums.

    sums: (n, >=3) array of C, Ix, Iy per sweep.  From <O> = sum O e^{-beta E}/Z,
    d<O>/dbeta = <dO/dbeta> - cov(O, E) with E = -J C; for e = E/N the first term
    vanishes, for Upsilon = (J C - beta J^2 (Ix^2 + Iy^2))/(2N) it is
    -J^2 <Ix^2 + Iy^2>/(2N).  Returns dict(e, upsilon, de, dupsilon, varE_over_N)."""
    sums = np.asarray(sums, np.float64)
    Cb, Ix, Iy = sums[:, 0], sums[:, 1], sums[:, 2]
    E = -J * Cb
    e = E / N
    jj = Ix * Ix + Iy * Iy
    ups = (J * Cb - beta * J * J * jj) / (2.0 * N)
    dE = E - E.mean()
    return {"e": e.mean(), "upsilon": ups.mean(),
            "de": -np.mean((e - e.mean()) * dE),
            "dupsilon": -np.mean((ups - ups.mean()) * dE) - J * J * jj.mean() / (2.0 * N),
            "varE_over_N": np.mean(dE * dE) / N}


# ---------------------------------------------------------------------------
# Hybrid Monte Carlo (Sec. 1.2): momenta, force, leap-frog, trajectories.
# ---------------------------------------------------------------------------

def _f64(a):
    a = np.array(a, np.float64).reshape(-1)
    return np.ascontiguousarray(a)


def hmc_momenta(Lx, Ly, seed, traj, lattice_id=0):
    """Gaussian momenta of trajectory `traj` (Box-Muller of domain-3 words)."""
    p = np.zeros(Lx * Ly, np.float64)
    lib().orc_hmc_momenta(Lx, Ly, seed, traj, lattice_id, p)
    return p


def hmc_force(theta, Lx, Ly, beta, J=1.0):
    """F_s = -beta J sum_nn sin(theta_s - theta_j)."""
    F = np.zeros(Lx * Ly, np.float64)
    lib().orc_hmc_force(Lx, Ly, _f64(theta), beta, J, F)
    return F


def hmc_hamiltonian(theta, p, Lx, Ly, beta, J=1.0):
    """(K, V): kinetic sum p^2/2 and potential beta H(theta)."""
    out = np.zeros(2, np.float64)
    lib().orc_hmc_hamiltonian(Lx, Ly, _f64(theta), _f64(p), beta, J, out)
    return float(out[0]), float(out[1])


def hmc_leapfrog(theta, p, Lx, Ly, beta, eps, n_steps, J=1.0):
    """n_steps leap-frog steps; returns new (theta, p) copies (angles wrapped into [0, 2pi))."""
    th, pp = _f64(theta), _f64(p)
    if lib().orc_hmc_leapfrog(Lx, Ly, th, pp, beta, J, eps, n_steps) != 0:
        raise MemoryError("oracle leap-frog failed")
    return th, pp


def hmc_trajectory(theta, Lx, Ly, beta, eps, n_steps, seed, traj, lattice_id=0, J=1.0):
    """One trajectory from `theta`; returns (theta_after_test, p_end, dict(dH, accepted,
    K0, V0, K1, V1))."""
    th = _f64(theta)
    out = np.zeros(6, np.float64)
    pend = np.zeros(Lx * Ly, np.float64)
    if lib().orc_hmc_trajectory(Lx, Ly, th, beta, J, eps, n_steps, seed, traj, lattice_id,
                                out, pend) != 0:
        raise MemoryError("oracle trajectory failed")
    return th, pend, {"dH": out[0], "accepted": bool(out[1]), "K0": out[2], "V0": out[3],
                      "K1": out[4], "V1": out[5]}


def hmc_run(Lx, Ly, beta, eps, n_steps, n_traj, seed, lattice_id=0, J=1.0, start=1,
            first_traj=0, theta=None):
    """HMC chain; returns (records[n, 7], final_theta).

    records[i] = (C, Ix, Iy, Mx, My, dH, accepted) after trajectory first_traj + i.
    start: 1 hot, 0 cold, -1 from `theta`."""
    th = np.zeros(Lx * Ly, np.float64) if theta is None else _f64(theta)
    rec = np.zeros((n_traj, 7), np.float64)
    if lib().orc_hmc_run(Lx, Ly, seed, lattice_id, beta, J, eps, n_steps, start, first_traj,
                         n_traj, th, rec) != 0:
        raise ValueError("oracle HMC run failed")
    return rec, th
