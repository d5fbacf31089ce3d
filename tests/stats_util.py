"""Binned-jackknife statistics for Markov-chain series (test helper).

Chain samples are correlated; the error of a mean is estimated by cutting
the series into `n_bins` contiguous bins and jackknifing over bins.  With
bins much longer than the autocorrelation time this is unbiased.
"""
import numpy as np


def jackknife_mean(x, n_bins=50):
    """(mean, error) of the mean of a 1-d series."""
    x = np.asarray(x, np.float64)
    nb = min(n_bins, x.size)
    m = x.size // nb
    bins = x[: nb * m].reshape(nb, m).mean(axis=1)
    total = bins.sum()
    jk = (total - bins) / (nb - 1)
    mean = jk.mean()
    err = np.sqrt((nb - 1) / nb * np.sum((jk - mean) ** 2))
    return float(bins.mean()), float(err)


def jackknife_func(series, func, n_bins=50):
    """(value, error) of func(means of several series) by binned jackknife.

    `series` is a list of equal-length 1-d arrays; func takes their means."""
    xs = [np.asarray(s, np.float64) for s in series]
    n = xs[0].size
    nb = min(n_bins, n)
    m = n // nb
    binned = [s[: nb * m].reshape(nb, m).mean(axis=1) for s in xs]
    totals = [b.sum() for b in binned]
    jk = np.array([func(*[(t - b[i]) / (nb - 1) for t, b in zip(totals, binned)])
                   for i in range(nb)])
    full = func(*[b.mean() for b in binned])
    err = np.sqrt((nb - 1) / nb * np.sum((jk - jk.mean()) ** 2))
    return float(full), float(err)


def jackknife_cov(x, y, n_bins=50):
    """(cov(x, y), error) of the covariance <xy> - <x><y> over a chain."""
    return jackknife_func([x, y, np.asarray(x) * np.asarray(y)],
                          lambda a, b, ab: ab - a * b, n_bins)
