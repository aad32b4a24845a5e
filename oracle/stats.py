"""Monte Carlo error tools used by the statistical parity tests.

TEST INFRASTRUCTURE ONLY (see the ``oracle`` package docstring).

- ``ess_geyer``: effective sample size from Geyer's (1992) initial positive
  sequence estimator of the integrated autocorrelation time.
- ``mcse``: Monte Carlo standard error of a chain mean, sd * sqrt(1/ESS).
- ``mcse_batch_means``: batch-means MCSE with about sqrt(n) batches.

The paper judges its chains by ESS and autocorrelation (Sec. 3 and Sec. 5.3);
these are the textbook estimators, written out in numpy.
"""
from __future__ import annotations

import numpy as np


def autocov(x):
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    xc = x - x.mean()
    m = 1 << int(np.ceil(np.log2(2 * n)))
    f = np.fft.rfft(xc, m)
    ac = np.fft.irfft(f * np.conj(f), m)[:n] / n
    return ac


def ess_geyer(x) -> float:
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    if n < 4:
        return float(n)
    ac = autocov(x)
    if ac[0] <= 0:
        return float(n)
    rho = ac / ac[0]
    # pair sums Gamma_m = rho_{2m} + rho_{2m+1}; keep the initial positive, monotone run
    s = 0.0
    prev = np.inf
    m = 0
    while 2 * m + 1 < n:
        g = rho[2 * m] + rho[2 * m + 1]
        if g <= 0:
            break
        g = min(g, prev)
        s += g
        prev = g
        m += 1
    tau = 2.0 * s - 1.0
    tau = max(tau, 1.0 / n)
    return float(n / tau)


def mcse(x) -> float:
    x = np.asarray(x, dtype=np.float64)
    return float(x.std(ddof=1) / np.sqrt(ess_geyer(x)))


def mcse_batch_means(x) -> float:
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    b = max(int(np.sqrt(n)), 2)
    k = n // b
    if k < 2:
        return float(x.std(ddof=1) / np.sqrt(n))
    means = x[: k * b].reshape(k, b).mean(axis=1)
    return float(means.std(ddof=1) / np.sqrt(k))
