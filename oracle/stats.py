"""Oracle for the statistics of Monte Carlo series (test infrastructure only).

tau_int: integrated autocorrelation time with the automatic window of Madras
and Sokal (J. Stat. Phys. 50, 109 (1988)): rho(t) = C(t)/C(0) with C the
autocovariance about the sample mean (normalised by n), tau(W) = 1/2 +
sum_{t=1}^{W} rho(t), W the smallest lag with W >= c tau(W).
binder: U = 1 - <m^4> / (3 <m^2>^2).
Written with plain numpy, one lag at a time.
"""
from __future__ import annotations

import math

import numpy as np


def tau_int(x, c: float = 6.0):
    x = np.asarray(x, dtype=np.float64)
    n = len(x)
    d = x - x.mean()
    c0 = float(np.dot(d, d)) / n
    if c0 <= 0.0:
        return 0.5, 0.0, 0
    tau, W = 0.5, 0
    for lag in range(1, n // 2 + 1):
        rho = float(np.dot(d[:-lag], d[lag:])) / (n * c0)
        tau += rho
        W = lag
        if lag >= c * tau:
            break
    return tau, tau * math.sqrt(2.0 * (2 * W + 1) / n), W


def binder(m):
    m = np.asarray(m, dtype=np.float64)
    m2 = np.mean(m ** 2)
    m4 = np.mean(m ** 4)
    return 1.0 - m4 / (3.0 * m2 * m2)


def moments(E, M, N):
    """The six FP64 moment sums of a trace: count, sum|m|, sum m^2, sum m^4,
    sum e, sum e^2 with m = M/N, e = E/N."""
    m = np.asarray(M, dtype=np.float64) / N
    e = np.asarray(E, dtype=np.float64) / N
    return np.array([len(m), np.abs(m).sum(), (m ** 2).sum(), (m ** 4).sum(), e.sum(), (e ** 2).sum()])
