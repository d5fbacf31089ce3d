"""Helpers for GPU-vs-oracle parity tests (lock-step comparison).

Lock-step: before every half-sweep the oracle starts from the GPU's own FP32
state promoted to FP64, evaluates every site of that colour in double
precision with the same Philox words, and the GPU's decisions (read off the
state change) are compared site by site.  Where |u1 - exp(-beta dE)| is
inside the band the two precisions may legitimately disagree; those sites
are counted and the GPU's decision is adopted.  Everywhere else the
decisions must be identical, and every angle must equal the oracle's choice
(proposal or old angle) to within the angle tolerance.
"""
import os

import numpy as np

import oracle

TWO_PI = 2 * np.pi
ANGLE_TOL = 1e-5           # rad, circular distance
BAND_ACCURATE = 1e-6       # |u - e^{-beta dE}| band for the accurate path


def circ(a, b):
    d = np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)) % TWO_PI
    return np.minimum(d, TWO_PI - d)


def colour_mask(L):
    y, x = np.divmod(np.arange(L * L), L)
    return [((x + y) & 1) == c for c in (0, 1)]


def nthreads():
    return max(1, min(32, os.cpu_count() or 1))


class HalfResult:
    def __init__(self):
        self.in_band = 0
        self.out_band_mismatch = 0
        self.max_angle_err = 0.0
        self.accepted = 0
        self.sites = 0


def check_half(state64, before32, after32, L, colour, beta, seed, sweep, J, delta, band,
               lattice_id=0):
    """Compare one GPU half-sweep with the oracle's; returns a HalfResult."""
    mask = colour_mask(L)[colour]
    idx = np.flatnonzero(mask)
    tp, u1, p, acc = oracle.attempt_sites(state64, L, L, idx, beta, seed, sweep,
                                          lattice_id=lattice_id, J=J, delta=delta,
                                          nthreads=nthreads())
    b = before32.reshape(-1)[idx]
    a = after32.reshape(-1)[idx]
    gpu_changed = a != b
    unobservable = circ(tp, b) < 2e-6          # proposal rounds back onto the old angle
    in_band = np.abs(u1 - p) < band
    mism = (gpu_changed != acc) & ~unobservable
    res = HalfResult()
    res.in_band = int(np.count_nonzero(mism & in_band))
    res.out_band_mismatch = int(np.count_nonzero(mism & ~in_band))
    dec = np.where(unobservable, acc, gpu_changed)
    expect = np.where(dec, tp, b.astype(np.float64))
    res.max_angle_err = float(circ(a, expect).max()) if idx.size else 0.0
    res.accepted = int(np.count_nonzero(dec))
    res.sites = int(idx.size)
    return res


def lockstep_sweep(before32, after32, L, beta, seed, sweep, J=1.0, delta=np.pi,
                   band=BAND_ACCURATE, lattice_id=0):
    """Both halves of one GPU sweep against the oracle; returns (red, black) results."""
    s0 = before32.reshape(-1).astype(np.float64)
    red = check_half(s0, before32, after32, L, 0, beta, seed, sweep, J, delta, band, lattice_id)
    m_red = colour_mask(L)[0]
    s1 = s0.copy()
    s1[m_red] = after32.reshape(-1)[m_red].astype(np.float64)
    blk = check_half(s1, before32, after32, L, 1, beta, seed, sweep, J, delta, band, lattice_id)
    return red, blk


# Per sincos path: the standard deviation of one black site's term error
# against FP64 on the same state (the rounding of the term to fixed point,
# 2^-19 / sqrt(12) for the four bond cosines, plus the FP32 evaluation from
# FP32 unit vectors), and a bound on the systematic error per bond from the
# unit vectors' mean length bias (measured mean |v|^2 - 1: -1e-9 for the
# polynomial, +1.8e-8 for CUDA's sincosf, a few 1e-8 for __sincosf, whose
# per-value error is up to 7e-7).
RECORD_ERR = {"accurate": (7e-7, 2e-9), "libm": (7e-7, 4e-8), "fast": (1.5e-6, 3e-7)}


def record_tolerance(N, fast=False, sincos=None, reduce="exact"):
    """Absolute tolerance of a record's sums against the oracle on the same state.

    Exact sums (reduce "exact"): the record is the exact sum of the N/2 black
    sites' terms, each rounded to fixed point, so the error is the sum of the
    per-term errors: 6 sigma sqrt(N/2) for the random part and 2N x the bias
    bound for the systematic part (2N bonds).  At L = 4096 (accurate sincos)
    that is 0.08, below the change of C from a single wrong bond, |cos a -
    cos b|, for all but a small fraction of angle pairs.  Compensated FP32
    sums add their own rounding, ~2e-3 per sqrt(1024 sites)."""
    mode = sincos or ("fast" if fast else "accurate")
    sigma, bias = RECORD_ERR[mode]
    tol = 6.0 * sigma * np.sqrt(N / 2.0) + 2.0 * N * bias
    if reduce == "compensated":
        tol += 2e-3 * max(1.0, np.sqrt(N / 1024.0))
    return tol


def compare_record(obs_row, state32, L, J=1.0):
    """Max abs difference of (C, Ix, Iy, Mx, My) between a GPU record and the oracle."""
    ref = oracle.measure(state32.reshape(-1).astype(np.float64), L, L)
    got = np.array([obs_row[k] for k in ("C", "Ix", "Iy", "Mx", "My")])
    return np.abs(got - ref), ref
