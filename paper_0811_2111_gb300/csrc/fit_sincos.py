"""Fit the polynomial coefficients of xyd::sincos_poly (xy_device.cuh).

Weighted Remez exchange for the absolute error of
    sin r ~ r + r^3 (c3 + c5 r^2 + c7 r^4),
    cos r ~ 1 + r^2 (c2 + c4 r^2 + c6 r^4 + c8 r^6)
on |r| <= pi/4 (the range left by the reduction modulo pi/2).  Run it to
reproduce the constants in the kernel header:  python fit_sincos.py
"""
import numpy as np

R2_MAX = (np.pi / 4) ** 2


def remez(h, w, deg, a, b, iters=12, grid_n=100001):
    """Coefficients (lowest first) of the degree-`deg` polynomial P minimising
    max |w(u) (P(u) - h(u))| on [a, b], and that maximum."""
    n = deg + 1
    k = np.arange(n + 1)
    x = (a + b) / 2 + (b - a) / 2 * np.cos(np.pi * k[::-1] / n)
    grid = np.linspace(a, b, grid_n)
    for _ in range(iters):
        A = np.zeros((n + 1, n + 1))
        A[:, :n] = w(x)[:, None] * x[:, None] ** np.arange(n)
        A[:, n] = (-1.0) ** k
        sol = np.linalg.solve(A, w(x) * h(x))
        c = sol[:n]
        err = w(grid) * (np.polyval(c[::-1], grid) - h(grid))
        d = np.diff(err)
        turn = np.nonzero(d[:-1] * d[1:] <= 0)[0] + 1
        ext = np.concatenate([[0], turn, [grid_n - 1]])
        alt = []
        for i in ext:
            if alt and np.sign(err[i]) == np.sign(err[alt[-1]]):
                if abs(err[i]) > abs(err[alt[-1]]):
                    alt[-1] = i
            else:
                alt.append(i)
        while len(alt) > n + 1:
            alt.pop(0 if abs(err[alt[0]]) < abs(err[alt[-1]]) else -1)
        x = grid[alt]
    return c, float(np.max(np.abs(err)))


def _series(u, taylor, exact):
    u = np.asarray(u, np.float64)
    small = u < 1e-6
    safe = np.where(small, 1.0, u)
    return np.where(small, taylor(u), exact(safe))


def sin_target(u):
    return _series(u, lambda v: -1 / 6 + v / 120 - v * v / 5040,
                   lambda v: (np.sin(np.sqrt(v)) - np.sqrt(v)) / v ** 1.5)


def cos_target(u):
    return _series(u, lambda v: -0.5 + v / 24 - v * v / 720,
                   lambda v: (np.cos(np.sqrt(v)) - 1) / v)


def fit():
    cs, es = remez(sin_target, lambda u: np.asarray(u, np.float64) ** 1.5, 2, 0.0, R2_MAX)
    cc, ec = remez(cos_target, lambda u: np.asarray(u, np.float64), 3, 0.0, R2_MAX)
    return cs, es, cc, ec


if __name__ == "__main__":
    cs, es, cc, ec = fit()
    print("sin r^3, r^5, r^7:", ", ".join(f"{float(np.float32(v))!r}f" for v in cs),
          f"(max abs error {es:.3g})")
    print("cos r^2, r^4, r^6, r^8:", ", ".join(f"{float(np.float32(v))!r}f" for v in cc),
          f"(max abs error {ec:.3g})")
