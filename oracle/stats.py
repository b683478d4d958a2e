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


def statistical_inefficiency(x):
    """g = 1 + 2 tau with tau = sum_{t>=1} (1 - t/T) C(t), where C(t) is the
    normalised fluctuation autocorrelation of the series about its own mean,
    C(t) = [sum_{n<T-t} d_n d_{n+t} / (T - t)] / [sum_n d_n^2 / T], and the sum
    stops before the first lag with C(t) <= 0; g is at least 1 (Chodera,
    J. Chem. Theory Comput. 12, 1799 (2016), the method Section 3.1 uses to
    discard non-equilibrated data).  One lag at a time."""
    a = np.asarray(x, dtype=np.float64)
    T = len(a)
    d = a - a.mean()
    var = float(np.dot(d, d)) / T
    if not var > 0.0:
        return 1.0
    tau = 0.0
    for t in range(1, T):
        C = float(np.dot(d[:T - t], d[t:])) / ((T - t) * var)
        if C <= 0.0:
            break
        tau += (1.0 - t / T) * C
    return max(1.0, 1.0 + 2.0 * tau)


def detect_equilibration(x, stride: int = 1):
    """Automatic equilibration detection (same reference): for every candidate
    start t0 = 0, stride, 2 stride, ... (at most T - 2), the effective number
    of samples of x[t0:] is N(t0) = (T - t0) / g(x[t0:]); the result is the
    t0 with the largest N (the smallest such t0 on ties), with its g and N."""
    a = np.asarray(x, dtype=np.float64)
    T = len(a)
    best = (-1.0, 0, 1.0)
    for t0 in range(0, T - 1, max(1, int(stride))):
        g = statistical_inefficiency(a[t0:])
        n_eff = (T - t0) / g
        if n_eff > best[0]:
            best = (n_eff, t0, g)
    return best[1], best[2], best[0]
