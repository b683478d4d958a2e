"""Pins of the random-stream battery oracle (oracle/prng_battery.py): bit
order and float shaping by construction, the longest-run class
probabilities against brute-force enumeration, p-values uniform on streams of
numpy's PCG64 generator (a library generator independent of Philox),
near-zero p-values on streams with the defect each test targets, the
cumulative-sums p-value against a Monte Carlo estimate of the tail of the
maximum excursion, and a hand-computed frequency case."""
from __future__ import annotations

import itertools
import math
import zlib

import numpy as np
import pytest
from scipy import stats

from oracle import prng_battery as pb


def test_bit_order_and_float_shaping():
    assert list(pb.bits([0x80000001])) == [1] + [0] * 30 + [1]
    assert list(pb.bits([0x00000002, 0xFFFFFFFF])) == [0] * 30 + [1, 0] + [1] * 32
    f = pb.floats([0x00000000, 0xFF800000, 0x007FFFFF, 0x00400000])
    assert list(f) == [0.0, 0.0, (2**23 - 1) / 2**23, 0.5]     # the top 9 bits are dropped


@pytest.mark.parametrize("M", [1, 2, 5, 8, 13])
def test_longest_run_counts_brute_force(M):
    longest = []
    for s in itertools.product((0, 1), repeat=M):
        best = cur = 0
        for v in s:
            cur = cur + 1 if v else 0
            best = max(best, cur)
        longest.append(best)
    longest = np.array(longest)
    for k in range(M + 1):
        assert pb.strings_with_longest_run_at_most(M, k) == int((longest <= k).sum())


def test_longest_run_class_probs():
    p = pb.longest_run_class_probs(128)
    assert abs(p.sum() - 1.0) < 1e-15 and np.all(p > 0)
    # M = 8 against the brute-force class frequencies (classes <= 1, 2, 3, >= 4)
    q = pb.longest_run_class_probs(8, 1, 4)
    longest = [max((len(r) for r in "".join(map(str, s)).split("0")), default=0)
               for s in itertools.product((0, 1), repeat=8)]
    brute = np.bincount(np.clip(longest, 1, 4) - 1, minlength=4) / 256.0
    assert np.allclose(q, brute, atol=1e-15)


def test_frequency_hand_case():
    # 1110: S = 2, |S| / sqrt(n) = 1, p = P(|N(0,1)| > 1) = erfc(1 / sqrt 2)
    p, S = pb.frequency([1, 1, 1, 0])
    assert S == 2.0 and abs(p - 2 * (1 - stats.norm.cdf(1.0))) < 1e-12


def test_pvalues_uniform_on_a_library_generator():
    rng = np.random.default_rng(20240426)
    P = np.array([pb.battery(rng.integers(0, 2**32, size=4096, dtype=np.uint64).astype(np.uint32))[0]
                  for _ in range(120)])
    for j, name in enumerate(pb.TESTS):
        ks = stats.kstest(P[:, j], "uniform").pvalue
        assert ks > 1e-3, (name, ks)


def test_defects_are_caught():
    n = 4096
    rng = np.random.default_rng(5)
    good = rng.integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)
    biased = (rng.random((n, 32)) < 0.55).astype(np.uint64)
    biased = (biased << np.arange(31, -1, -1, dtype=np.uint64)).sum(axis=1).astype(np.uint32)
    alternating = np.full(n, 0x55555555, dtype=np.uint32)
    periodic = np.tile(good[:16], n // 16)
    half = (good & np.uint32(0xFFBFFFFF))                   # floats never in [0.5, 1)
    pairs = np.repeat(good[: n // 2], 2)                    # f(2i+1) = f(2i)
    p, _ = pb.battery(biased)
    assert p[pb.TESTS.index("frequency")] < 1e-6 and p[pb.TESTS.index("cusum_forward")] < 1e-6
    p, _ = pb.battery(alternating)
    assert p[pb.TESTS.index("runs")] < 1e-6 and p[pb.TESTS.index("frequency")] == 1.0
    assert p[pb.TESTS.index("longest_run")] < 1e-6
    p, _ = pb.battery(periodic)
    assert p[pb.TESTS.index("spectral")] < 1e-6
    p, _ = pb.battery(half)
    assert p[pb.TESTS.index("float_uniformity")] < 1e-6
    p, _ = pb.battery(pairs)
    assert p[pb.TESTS.index("float_pairs")] < 1e-6


def test_cusum_pvalue_matches_monte_carlo_tail():
    # p(z) approximates P(max_k |S_k| >= z) for n fair +-1 steps
    rng = np.random.default_rng(8)
    n, reps = 4000, 20000
    steps = rng.integers(0, 2, size=(reps, n), dtype=np.int8) * 2 - 1
    zmax = np.abs(np.cumsum(steps, axis=1, dtype=np.int32)).max(axis=1)
    for z in (60, 100, 150):
        b = np.zeros(n, dtype=np.int64)
        b[:z] = 1                                               # a walk whose excursion is exactly z
        b[z:] = np.tile([0, 1], (n - z) // 2 + 1)[: n - z]
        p, zz = pb.cusum(b)
        assert zz == z
        emp = float((zmax >= z).mean())
        se = math.sqrt(emp * (1 - emp) / reps)
        assert abs(p - emp) < 4 * se + 0.01, (z, p, emp)


# --------------------------------------------------------------------------
# The library's host battery (C ABI) against the oracle.
# --------------------------------------------------------------------------
def _philox_words(seed, s, t, phase, n_words):
    import oracle
    key = [seed & 0xFFFFFFFF, seed >> 32]
    out = np.empty(n_words, dtype=np.uint32)
    for q in range(n_words // 4):
        out[4 * q:4 * q + 4] = oracle.philox4x32_10([q, t, s, phase], key)
    return out


def test_library_battery_matches_oracle():
    from paper_2404_16990_gb300 import ising
    rng = np.random.default_rng(77)
    streams = [rng.integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32) for n in (4096, 5000, 40_000)]
    streams.append(_philox_words(2, 0, 0, 0, 1 << 14))
    streams.append(np.full(4096, 0x55555555, dtype=np.uint32))          # a failing stream: runs pre-test passes
    biased = (rng.random((4096, 32)) < 0.6).astype(np.uint64)
    streams.append((biased << np.arange(31, -1, -1, dtype=np.uint64)).sum(axis=1).astype(np.uint32))
    for w in streams:
        p_ref, s_ref = pb.battery(w)
        p_lib, s_lib = ising.ising_prng_battery(w)
        for j, name in enumerate(pb.TESTS):
            if np.isnan(s_ref[j]):
                assert np.isnan(s_lib[j]) and p_lib[j] == p_ref[j] == 0.0, name
                continue
            assert abs(s_lib[j] - s_ref[j]) <= 1e-9 * max(1.0, abs(s_ref[j])), (name, len(w), s_lib[j], s_ref[j])
            assert abs(p_lib[j] - p_ref[j]) <= 1e-9 + 1e-7 * p_ref[j], (name, len(w), p_lib[j], p_ref[j])
    with pytest.raises(ising.IsingError):
        ising.ising_prng_battery(np.zeros(4095, dtype=np.uint32))


def test_statistics_by_hand():
    # the statistic each test returns, counted by hand on short strings
    for s, V in (("1100", 2), ("1010", 4), ("0110100111", 6), ("0000011111", 2)):
        b = [int(ch) for ch in s]
        assert pb.runs(b)[1] == V, s                      # number of maximal blocks of equal bits
    # block frequency, M = 4 on 11110000 0110: blocks 1111, 0000, 0110 have
    # 4, 0, 2 ones: 4M sum (ones/M - 1/2)^2 = 16 (1/4 + 1/4 + 0) = 8
    assert pb.block_frequency([1, 1, 1, 1, 0, 0, 0, 0, 0, 1, 1, 0], M=4)[1] == 8.0
    # longest run of ones per 8-bit block, classes <= 1, 2, 3, >= 4 (lo = 1, hi = 4):
    # 01101110 -> 3, 00000000 -> 0, 11111011 -> 5, 10101010 -> 1 ; counts 2, 0, 1, 1
    blocks = "01101110" "00000000" "11111011" "10101010"
    p8 = pb.longest_run_class_probs(8, 1, 4)
    e = 4 * p8
    want = float((((np.array([2, 0, 1, 1]) - e) ** 2) / e).sum())
    assert abs(pb.longest_run([int(ch) for ch in blocks], M=8, lo=1, hi=4)[1] - want) < 1e-12
    # float uniformity with 4 bins on 0.1, 0.3, 0.35, 0.9: counts 1, 2, 0, 1 against 1 each
    assert pb.float_uniformity([0.1, 0.3, 0.35, 0.9], bins=4)[1] == 2.0
    # float pairs with 2 bins: (0.1, 0.2), (0.6, 0.7), (0.1, 0.9), (0.2, 0.3): cells 00 x2, 11, 01
    assert pb.float_pairs([0.1, 0.2, 0.6, 0.7, 0.1, 0.9, 0.2, 0.3], bins=2)[1] == 2.0


@pytest.mark.parametrize("name,words", [("block_frequency", 512), ("longest_run", 512),
                                        ("float_uniformity", 1000), ("float_pairs", 2000)])
def test_chi2_pvalues_uniform_at_scale(name, words):
    # under fair input every p-value is uniform; thousands of short streams
    # resolve the degrees of freedom and normalisation of each chi^2 test
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    fn = getattr(pb, name)
    P = []
    for _ in range(4000):
        w = rng.integers(0, 2**32, size=words, dtype=np.uint64).astype(np.uint32)
        P.append(fn(pb.floats(w) if name.startswith("float") else pb.bits(w))[0])
    assert stats.kstest(P, "uniform").pvalue > 1e-3, name
