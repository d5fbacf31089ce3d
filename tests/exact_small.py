"""Exact thermodynamics of tiny periodic XY lattices (test pins).

Two independent routes, both from the definition Z = int prod_s dtheta_s
exp(-beta H), H = -J sum_bonds cos(theta_i - theta_j - psi_bond) (Eq. (1),
with an optional uniform twist psi on x or y bonds):

* ``z_ring_bessel``: a periodic ring of n spins with coupling K has
  Z = (2 pi)^n sum_k I_k(K)^n (character expansion of exp(K cos)).  The 2x2
  torus is a 4-ring with coupling 2 beta J, because each pair is bonded twice.
* ``log_z_trapezoid``: the periodic trapezoid rule on M points per angle
  (spectrally convergent for these analytic periodic integrands), contracted
  with a row transfer matrix.  Works for 2 x Ly and Lx x 2 tori.

Observables follow from derivatives of ln Z:
  <e> = -(1/N) d ln Z / d beta,
  Upsilon_mu = (1/N) d^2 F / d psi_mu^2 at psi = 0, F = -ln Z / beta,
  Upsilon = (Upsilon_x + Upsilon_y) / 2,
evaluated with central finite differences on the exact ln Z.
<|m|> needs the full grid; ``mean_abs_m_grid`` sums it directly (tiny N only).
"""
import numpy as np
from scipy.special import ive


def bonds(Lx, Ly):
    """List of (i, j, direction) for the 2N bonds s -> s+x, s -> s+y."""
    out = []
    for y in range(Ly):
        for x in range(Lx):
            s = y * Lx + x
            out.append((s, y * Lx + (x + 1) % Lx, 0))
            out.append((s, ((y + 1) % Ly) * Lx + x, 1))
    return out


def z_ring_bessel(n, K, kmax=60):
    """ln Z / (2 pi)^n of an n-spin periodic ring with coupling K."""
    k = np.arange(-kmax, kmax + 1)
    # I_k(K) = ive(k, K) * exp(K); keep the exp(n K) factor in the log
    terms = ive(k, K) ** n
    return n * K + np.log(terms.sum())


def log_z_trapezoid(Lx, Ly, beta, J=1.0, psi=(0.0, 0.0), M=32):
    """ln of the trapezoid-rule partition sum (normalisation dropped).

    Contracted with a row transfer matrix, so one side must be 2; a 2 x Ly
    torus is used as is, an Lx x 2 torus through the x <-> y symmetry
    (Z(Lx, Ly, psi_x, psi_y) = Z(Ly, Lx, psi_y, psi_x))."""
    if Lx != 2:
        if Ly != 2:
            raise ValueError("one side must be 2")
        return log_z_trapezoid(2, Lx, beta, J, (psi[1], psi[0]), M)
    t = 2 * np.pi * np.arange(M) / M
    diff = t[:, None] - t[None, :]
    K = beta * J
    # row of two sites (a, b): bonds a->b and b->a, both twisted by psi_x
    w_row = np.exp(K * (np.cos(diff - psi[0]) + np.cos(-diff - psi[0]) - 2.0))
    # vertical bond from row r to row r+1 (site -> site + y), twisted by psi_y
    w_up = np.exp(K * (np.cos(diff - psi[1]) - 1.0))
    # T[(a,b),(c,d)] = w_row(a,b) w_up(a,c) w_up(b,d)
    T = (w_row[:, :, None, None] * w_up[:, None, :, None] * w_up[None, :, None, :])
    T = T.reshape(M * M, M * M)
    P = np.eye(M * M)
    for _ in range(Ly):
        P = P @ T
    n_bonds = 2 * 2 * Ly
    return float(np.log(np.trace(P)) + K * n_bonds)


def exact_observables(Lx, Ly, beta, J=1.0, M=32, h_beta=1e-4, h_psi=1e-3):
    """(<e>, <Upsilon>) of an Lx x Ly torus from the trapezoid ln Z."""
    N = Lx * Ly
    lz = lambda b, px=0.0, py=0.0: log_z_trapezoid(Lx, Ly, b, J, (px, py), M)
    e = -(lz(beta + h_beta) - lz(beta - h_beta)) / (2 * h_beta) / N
    F = lambda px, py: -lz(beta, px, py) / beta
    f0 = F(0.0, 0.0)
    ups_x = (F(h_psi, 0.0) - 2 * f0 + F(-h_psi, 0.0)) / h_psi ** 2 / N
    ups_y = (F(0.0, h_psi) - 2 * f0 + F(0.0, -h_psi)) / h_psi ** 2 / N
    return e, 0.5 * (ups_x + ups_y)


def mean_abs_m_grid(Lx, Ly, beta, J=1.0, M=16):
    """<|m|> by direct trapezoid summation (global rotation fixed: theta_0 = 0)."""
    N = Lx * Ly
    t = 2 * np.pi * np.arange(M) / M
    bl = bonds(Lx, Ly)
    grids = np.meshgrid(*([t] * (N - 1)), indexing="ij", sparse=False)
    th = [np.zeros_like(grids[0])] + list(grids)
    E = np.zeros_like(grids[0])
    for (i, j, _) in bl:
        E -= J * np.cos(th[i] - th[j])
    w = np.exp(-beta * (E - E.min()))
    mx = sum(np.cos(a) for a in th)
    my = sum(np.sin(a) for a in th)
    am = np.sqrt(mx * mx + my * my) / N
    return float((w * am).sum() / w.sum())


def e_2x2_bessel(beta, J=1.0, h=1e-5):
    """<e> of the 2x2 torus: a 4-ring with coupling 2 beta J."""
    lz = lambda b: z_ring_bessel(4, 2 * b * J)
    return -(lz(beta + h) - lz(beta - h)) / (2 * h) / 4
