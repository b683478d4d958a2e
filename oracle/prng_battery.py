"""Oracle of the random-stream quality battery (test infrastructure only).

The paper checks its generator's bit stream with the tests of NIST SP 800-22
(supplementary, PRNG tests), then floats shaped from it for uniformity in
100 bins, lag-1 independence, and the bits "float >= median" with the same
bit tests.  This module restates those statistics in plain numpy / scipy:

  bits(words)            the stream: every 32-bit word, most significant bit first
  floats(words)          the paper's shaping: the low 23 bits as a fraction,
                         (w & 0x7FFFFF) / 2^23 in [0, 1)
  frequency              S = sum(2b - 1), p = erfc(|S| / sqrt(2n))
  block_frequency(M)     N = n // M blocks, chi2 = 4M sum (ones_j / M - 1/2)^2,
                         p = Q(N/2, chi2/2)
  runs                   pi = ones / n; p = 0 if |pi - 1/2| >= 2/sqrt(n); else
                         V = 1 + #changes, p = erfc(|V - 2n pi(1-pi)| /
                         (2 sqrt(2n) pi (1 - pi)))
  longest_run(M)         longest run of ones per M-bit block in the classes
                         <= 4, 5, 6, 7, 8, >= 9 (M = 128); class
                         probabilities exact from the count of M-bit strings
                         whose longest run is <= k; chi2 over the classes,
                         p = Q(5/2, chi2/2)
  spectral               on the first n bits, n the largest power of two
                         <= min(bits, 2^20); X = DFT of 2b - 1;
                         T = sqrt(ln(20) n); N1 = #{|X_k| < T, k < n/2};
                         d = (N1 - 0.95 n/2) / sqrt(0.95 * 0.05 n / 4),
                         p = erfc(|d| / sqrt(2))
  cusum(reverse)         z = max |partial sum of 2b - 1|; p from the
                         distribution of the maximum of a random walk's
                         excursion (sums of normal CDF differences)
  float_uniformity       100 equal bins, chi2 with 99 degrees of freedom
  float_pairs            non-overlapping pairs in a 10 x 10 grid, chi2 with 99
  median_bits            b_i = f_i >= median(f) (as many ones as zeros by
                         construction, so the frequency test would be void),
                         then the runs and longest-run tests

Q is the regularised upper incomplete gamma function.  Plain loops only where
numpy has no primitive; no blocking or reordering beyond the definitions.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special


def bits(words) -> np.ndarray:
    w = np.ascontiguousarray(words, dtype=np.uint32)
    shifts = np.arange(31, -1, -1, dtype=np.uint32)
    return ((w[:, None] >> shifts) & 1).astype(np.uint8).ravel()


def floats(words) -> np.ndarray:
    w = np.ascontiguousarray(words, dtype=np.uint32)
    return (w & 0x7FFFFF).astype(np.float64) / float(1 << 23)


def frequency(b):
    b = np.asarray(b, dtype=np.int64)
    n = len(b)
    S = int((2 * b - 1).sum())
    return float(special.erfc(abs(S) / math.sqrt(2.0 * n))), float(S)


def block_frequency(b, M: int = 128):
    b = np.asarray(b, dtype=np.int64)
    N = len(b) // M
    ones = b[:N * M].reshape(N, M).sum(axis=1)
    chi2 = 4.0 * M * float(((ones / M - 0.5) ** 2).sum())
    return float(special.gammaincc(N / 2.0, chi2 / 2.0)), chi2


def runs(b):
    b = np.asarray(b, dtype=np.int64)
    n = len(b)
    pi = float(b.sum()) / n
    if abs(pi - 0.5) >= 2.0 / math.sqrt(n):
        return 0.0, float("nan")
    V = 1 + int((b[1:] != b[:-1]).sum())
    num = abs(V - 2.0 * n * pi * (1.0 - pi))
    den = 2.0 * math.sqrt(2.0 * n) * pi * (1.0 - pi)
    return float(special.erfc(num / den)), float(V)


def strings_with_longest_run_at_most(M: int, k: int) -> int:
    """Number of M-bit strings whose longest run of ones is <= k (exact):
    f(m) = 2^m for m <= k, else f(m) = sum_{j=0..k} f(m - 1 - j) (the string
    ends in a zero preceded by a valid string, after j trailing ones)."""
    f = [0] * (M + 1)
    for m in range(M + 1):
        if m <= k:
            f[m] = 1 << m
        else:
            f[m] = sum(f[m - 1 - j] for j in range(k + 1))
    return f[M]


def longest_run_class_probs(M: int = 128, lo: int = 4, hi: int = 9):
    """P(longest run <= lo), P(= lo+1), ..., P(>= hi) for M fair bits."""
    cum = [strings_with_longest_run_at_most(M, k) / 2.0 ** M for k in range(lo, hi)]
    probs = [cum[0]] + [cum[i] - cum[i - 1] for i in range(1, len(cum))] + [1.0 - cum[-1]]
    return np.array(probs)


def longest_run(b, M: int = 128, lo: int = 4, hi: int = 9):
    b = np.asarray(b, dtype=np.int64)
    N = len(b) // M
    blk = b[:N * M].reshape(N, M)
    best = np.zeros(N, dtype=np.int64)
    cur = np.zeros(N, dtype=np.int64)
    for pos in range(M):                        # run length ending at each position, all blocks at once
        cur = (cur + 1) * blk[:, pos]
        best = np.maximum(best, cur)
    counts = np.bincount(np.clip(best, lo, hi) - lo, minlength=hi - lo + 1).astype(np.float64)
    p = longest_run_class_probs(M, lo, hi)
    chi2 = float(((counts - N * p) ** 2 / (N * p)).sum())
    return float(special.gammaincc((hi - lo) / 2.0, chi2 / 2.0)), chi2


SPECTRAL_MAX_BITS = 1 << 20


def spectral(b):
    b = np.asarray(b, dtype=np.float64)
    n = 1
    while 2 * n <= min(len(b), SPECTRAL_MAX_BITS):
        n *= 2
    b = b[:n]
    X = np.fft.fft(2.0 * b - 1.0)
    mod = np.abs(X[: n // 2])
    T = math.sqrt(math.log(1.0 / 0.05) * n)
    N0 = 0.95 * n / 2.0
    N1 = float((mod < T).sum())
    d = (N1 - N0) / math.sqrt(n * 0.95 * 0.05 / 4.0)
    return float(special.erfc(abs(d) / math.sqrt(2.0))), d


def _phi(x):
    return 0.5 * special.erfc(-x / math.sqrt(2.0))


def cusum(b, reverse: bool = False):
    b = np.asarray(b, dtype=np.int64)
    if reverse:
        b = b[::-1]
    n = len(b)
    z = int(np.abs(np.cumsum(2 * b - 1)).max())
    if z == 0:
        return 0.0, 0.0
    sq = math.sqrt(n)
    s1 = 0.0
    for k in range(math.floor((-n / z + 1) / 4), math.floor((n / z - 1) / 4) + 1):
        s1 += _phi((4 * k + 1) * z / sq) - _phi((4 * k - 1) * z / sq)
    s2 = 0.0
    for k in range(math.floor((-n / z - 3) / 4), math.floor((n / z - 1) / 4) + 1):
        s2 += _phi((4 * k + 3) * z / sq) - _phi((4 * k + 1) * z / sq)
    return float(1.0 - s1 + s2), float(z)


def float_uniformity(f, bins: int = 100):
    f = np.asarray(f, dtype=np.float64)
    counts = np.bincount(np.minimum((f * bins).astype(np.int64), bins - 1), minlength=bins)
    e = len(f) / bins
    chi2 = float(((counts - e) ** 2 / e).sum())
    return float(special.gammaincc((bins - 1) / 2.0, chi2 / 2.0)), chi2


def float_pairs(f, bins: int = 10):
    f = np.asarray(f, dtype=np.float64)
    n = len(f) // 2
    x = np.minimum((f[0:2 * n:2] * bins).astype(np.int64), bins - 1)
    y = np.minimum((f[1:2 * n:2] * bins).astype(np.int64), bins - 1)
    counts = np.bincount(x * bins + y, minlength=bins * bins)
    e = n / (bins * bins)
    chi2 = float(((counts - e) ** 2 / e).sum())
    return float(special.gammaincc((bins * bins - 1) / 2.0, chi2 / 2.0)), chi2


def median_bits(f):
    f = np.asarray(f, dtype=np.float64)
    return (f >= np.median(f)).astype(np.uint8)


TESTS = ("frequency", "block_frequency", "runs", "longest_run", "spectral", "cusum_forward",
         "cusum_backward", "float_uniformity", "float_pairs", "median_runs", "median_longest_run")


def battery(words):
    """(p-values, statistics) of the eleven tests on a stream of 32-bit words,
    in the order of TESTS."""
    b = bits(words)
    f = floats(words)
    mb = median_bits(f)
    res = [frequency(b), block_frequency(b), runs(b), longest_run(b), spectral(b), cusum(b, False),
           cusum(b, True), float_uniformity(f), float_pairs(f), runs(mb), longest_run(mb)]
    return np.array([r[0] for r in res]), np.array([r[1] for r in res])
