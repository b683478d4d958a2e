"""Pins for the CPU oracle: each test checks the oracle against something the
paper or the mathematics fixes (published known-answer vectors, closed forms,
exact enumeration, Kaufman's and Onsager's solutions, hand-derived worked
cases), never against a retyped copy of itself."""
from __future__ import annotations

import math
import os

import mpmath as mp
import numpy as np
import pytest
from scipy import stats

import exact
import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
NT = max(1, min(8, os.cpu_count() or 1))


# --------------------------------------------------------------------------
# Philox4x32-10 (replaces the paper's hardware generator, supplementary PRNG
# section): the published known-answer vectors.
# --------------------------------------------------------------------------
def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            v = [int(x, 16) for x in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answers(ctr, key, expect):
    assert list(oracle.philox4x32_10(ctr, key)) == expect


def test_site_random_keying():
    # counter (p >> 2, t, s, phase), key (lo32, hi32 of seed), lane p & 3
    seed = 0x0123456789ABCDEF
    for p, t, s, ph in [(0, 0, 0, 0), (5, 7, 3, 1), (1 << 20 | 3, 999, 11, 2)]:
        block = oracle.philox4x32_10([p >> 2, t, s, ph], [seed & 0xFFFFFFFF, seed >> 32])
        assert oracle.site_random(seed, p, t, s, ph) == block[p & 3]


def test_random_stream_uniformity_and_lag1():
    # The paper's own generator checks: 100-bin uniformity and lag-1
    # independence of floats in [0,1) (supplementary, ranged float tests).
    n = 100_000
    u = np.array([oracle.site_random(7, p, 3, 1, 0) for p in range(n)], dtype=np.float64) / 2.0**32
    counts, _ = np.histogram(u, bins=100, range=(0.0, 1.0))
    chi2 = ((counts - n / 100) ** 2 / (n / 100)).sum()
    assert stats.chi2.sf(chi2, 99) > 1e-3
    r = np.corrcoef(u[:-1], u[1:])[0, 1]
    assert abs(r) < 4.0 / math.sqrt(n)
    # bit balance of the top bit (the initial-state draw uses it)
    top = (u >= 0.5).mean()
    assert abs(top - 0.5) < 4 * 0.5 / math.sqrt(n)


# --------------------------------------------------------------------------
# Acceptance thresholds: floor(2^32 exp(-dE/T)) clamped, against the exact
# value computed with 60-digit arithmetic.
# --------------------------------------------------------------------------
def test_thresholds_exact():
    rng = np.random.default_rng(3)
    temps = list(rng.uniform(0.2, 50.0, size=400)) + [0.5, 1.0, 1.5, exact.T_C, 2.269185, 3.0]
    with mp.workdps(60):
        for T in temps:
            thr = oracle.thresholds(T)
            for k, dE in enumerate((4, 8)):
                v = mp.exp(-mp.mpf(dE) / mp.mpf(T)) * mp.mpf(2) ** 32
                if abs(v - mp.nint(v)) < mp.mpf(10) ** -5:
                    continue  # within rounding of an integer: either floor is fine
                assert int(thr[k]) == min(int(mp.floor(v)), 2**32 - 1), (T, dE)


def test_thresholds_limits_and_errors():
    assert list(oracle.thresholds(0.1)) == [0, 0]          # T -> 0: only dE <= 0 accepted
    assert list(oracle.thresholds(1e12)) == [2**32 - 1, 2**32 - 1]  # T -> inf: clamped
    thr = oracle.thresholds(2.269185)
    assert thr[1] < thr[0]
    for bad in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(ValueError):
            oracle.thresholds(bad)


# --------------------------------------------------------------------------
# Energy and magnetization: closed forms for ordered states.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("L", [2, 4, 6, 16])
def test_energy_closed_forms(L):
    cold = np.ones((L, L), np.int8)
    assert oracle.energy(cold) == -2 * L * L
    assert oracle.magnetization(cold) == L * L
    y, x = np.indices((L, L))
    neel = np.where((x + y) % 2 == 0, 1, -1).astype(np.int8)
    assert oracle.energy(neel) == 2 * L * L
    assert oracle.magnetization(neel) == 0
    one = cold.copy()
    one[L // 2, L - 1] = -1
    if L > 2:
        assert oracle.energy(one) == -2 * L * L + 8
    assert oracle.magnetization(one) == L * L - 2
    stripe = cold.copy()
    stripe[:, 0] = -1                         # two vertical domain walls of length L
    if L > 2:
        assert oracle.energy(stripe) == -2 * L * L + 4 * L


def test_energy_matches_enumeration_definition():
    # E of every 3x... state of a 4x4 torus equals the bond sum of the
    # brute-force enumeration.
    E, M = exact.enumerate_EM(4)
    rng = np.random.default_rng(0)
    for idx in rng.integers(0, 1 << 16, size=200):
        bits = (int(idx) >> np.arange(16)) & 1
        s = (1 - 2 * bits).reshape(4, 4).astype(np.int8)
        assert oracle.energy(s) == E[idx]
        assert oracle.magnetization(s) == M[idx]


# --------------------------------------------------------------------------
# Initial state.
# --------------------------------------------------------------------------
def test_init_cold_and_random():
    assert (oracle.init(64, 1, 0, cold=True) == 1).all()
    s = oracle.init(256, 1, 0)
    frac = (s == 1).mean()
    assert abs(frac - 0.5) < 4 * 0.5 / 256
    assert not np.array_equal(s, oracle.init(256, 2, 0))
    assert not np.array_equal(s, oracle.init(256, 1, 1))
    assert np.array_equal(s, oracle.init(256, 1, 0, n_threads=NT))
    # the draw is the top bit of the site's phase-2 word
    for (y, x) in [(0, 0), (3, 17), (255, 255)]:
        r = oracle.site_random(1, y * 256 + x, 0, 0, 2)
        assert s[y, x] == (-1 if r >> 31 else 1)


# --------------------------------------------------------------------------
# Deterministic limits.
# --------------------------------------------------------------------------
def _golden_t0_cases():
    cases, lines = [], []
    with open(os.path.join(GOLDEN, "zero_temperature_sweeps.txt")) as f:
        lines = [ln.rstrip("\n") for ln in f if ln.strip() and not ln.startswith("#")]
    i = 0
    while i < len(lines):
        _, name, L = lines[i].split()
        L = int(L)
        grid = lambda rows: np.array([[1 if ch == "+" else -1 for ch in r] for r in rows], np.int8)
        cases.append((name, grid(lines[i + 1:i + 1 + L]), grid(lines[i + 1 + L:i + 1 + 2 * L])))
        i += 1 + 2 * L
    return cases


@pytest.mark.parametrize("name,start,after", _golden_t0_cases())
def test_zero_temperature_worked_cases(name, start, after):
    s = np.ascontiguousarray(start.copy())
    E, M = oracle.sweeps(s, 0.1, seed=5, s=0, t0=0, n=1)
    assert np.array_equal(s, after), name
    assert E[0] == oracle.energy(after) and M[0] == after.sum()


def test_zero_temperature_cold_start_frozen():
    s = oracle.init(32, 9, 0, cold=True)
    E, M = oracle.sweeps(s, 0.15, seed=9, s=0, t0=0, n=50)
    assert (E == -2 * 32 * 32).all() and (M == 32 * 32).all()


def test_zero_temperature_energy_never_rises():
    s = oracle.init(32, 11, 0)
    e0 = oracle.energy(s)
    prev = e0
    for t in range(40):
        for c in (0, 1):
            oracle.half_sweep(s, c, 0.1, 11, 0, t)
            e = oracle.energy(s)
            assert e <= prev
            prev = e
    assert prev < e0


def test_infinite_temperature_negates_every_spin():
    # thr = 2^32 - 1: every move is accepted unless r == 2^32-1.  The black
    # half-sweep negates all black spins, the white one all white spins.
    s0 = oracle.init(32, 4, 0)
    s = s0.copy()
    E, M = oracle.sweeps(s, 1e12, seed=4, s=0, t0=0, n=1)
    assert np.array_equal(s, -s0)
    assert E[0] == oracle.energy(s0) and M[0] == -s0.sum()


# --------------------------------------------------------------------------
# Exact-solution pins (the closed forms themselves are cross-checked first).
# --------------------------------------------------------------------------
def test_kaufman_matches_bruteforce_and_transfer_matrix():
    E, _ = exact.enumerate_EM(4)
    for K in (0.15, 0.3, 1 / exact.T_C, 0.6, 1.1):
        with mp.workdps(50):
            lnz_brute = mp.log(mp.fsum([mp.e ** (-mp.mpf(K) * int(e)) for e in E]))
        assert abs(float(lnz_brute - exact.kaufman_lnZ(4, 4, K))) < 1e-12
        for L in (6, 8):
            assert abs(exact.transfer_matrix_lnZ(L, K) - float(exact.kaufman_lnZ(L, L, K))) < 1e-9


def test_onsager_matches_large_kaufman():
    for T in (1.5, 2.0, 3.0, 5.0):
        u_kaufman = exact.kaufman_mean_energy(256, T) / 256**2
        assert abs(u_kaufman - exact.onsager_u(T)) < 1e-6
    assert abs(exact.onsager_u(exact.T_C) + math.sqrt(2.0)) < 1e-12
    assert abs(exact.onsager_u(exact.T_C * (1 + 1e-7)) + math.sqrt(2.0)) < 1e-5


def _chain_stats(L, T, n_chains, burn, n_meas, seed):
    sig = [oracle.init(L, seed, s) for s in range(n_chains)]
    oracle.sweeps_batch(sig, [T] * n_chains, [seed] * n_chains, list(range(n_chains)), 0, burn, NT)
    E, M = oracle.sweeps_batch(sig, [T] * n_chains, [seed] * n_chains, list(range(n_chains)),
                               burn, n_meas, NT)
    return E.astype(np.float64), M.astype(np.float64)


def _mean_and_se(per_chain):
    m = per_chain.mean()
    se = per_chain.std(ddof=1) / math.sqrt(len(per_chain))
    return m, se


@pytest.mark.parametrize("T", [1.5, exact.T_C, 3.0])
def test_4x4_joint_distribution_matches_enumeration(T):
    """Sampled (E, |M|) histogram of 4x4 chains against exact enumeration."""
    E_all, M_all = exact.enumerate_EM(4)
    w = exact.boltzmann_weights(E_all, T)
    keys = E_all * 1000 + np.abs(M_all)
    uniq, inv = np.unique(keys, return_inverse=True)
    p = np.bincount(inv, weights=w)
    E, M = _chain_stats(4, T, n_chains=256, burn=200, n_meas=800, seed=20240426)
    thin = 20
    ks = (E[:, ::thin] * 1000 + np.abs(M[:, ::thin])).astype(np.int64).ravel()
    obs = np.array([(ks == u).sum() for u in uniq], dtype=np.float64)
    n = obs.sum()
    exp_ = p * n
    # merge sparse bins
    order = np.argsort(exp_)
    o2, e2, acc_o, acc_e = [], [], 0.0, 0.0
    for i in order:
        acc_o += obs[i]; acc_e += exp_[i]
        if acc_e >= 10:
            o2.append(acc_o); e2.append(acc_e); acc_o = acc_e = 0.0
    if acc_e > 0:
        o2[-1] += acc_o; e2[-1] += acc_e
    o2, e2 = np.array(o2), np.array(e2)
    chi2 = ((o2 - e2) ** 2 / e2).sum()
    assert len(o2) >= 3
    assert stats.chi2.sf(chi2, len(o2) - 1) > 1e-3, (T, chi2, len(o2))


@pytest.mark.parametrize("T", [2.0, exact.T_C, 3.0])
def test_finite_lattice_energy_matches_kaufman(T):
    L = 16
    E, _ = _chain_stats(L, T, n_chains=64, burn=500, n_meas=2000, seed=77)
    m, se = _mean_and_se(E.mean(axis=1))
    ref = exact.kaufman_mean_energy(L, T)
    assert abs(m - ref) < 3 * se + 1e-9, (T, m, ref, se)


@pytest.mark.parametrize("T", [1.5, 3.0])
def test_energy_per_spin_matches_onsager(T):
    L = 64
    E, M = _chain_stats(L, T, n_chains=16, burn=300, n_meas=700, seed=123)
    m, se = _mean_and_se(E.mean(axis=1) / L**2)
    assert abs(m - exact.onsager_u(T)) < 3 * se, (T, m, exact.onsager_u(T), se)


def test_spontaneous_magnetization_matches_onsager():
    L, T = 64, 1.5
    _, M = _chain_stats(L, T, n_chains=16, burn=300, n_meas=700, seed=321)
    m, se = _mean_and_se(np.abs(M).mean(axis=1) / L**2)
    assert abs(m - exact.onsager_m(T)) < 3 * se, (m, exact.onsager_m(T), se)


def test_high_temperature_susceptibility_series():
    # T -> inf: <M^2>/N -> 1; at T = 20 the square-lattice high-temperature
    # series chi = 1 + 4v + 12v^2 + 36v^3 + 100v^4 + 276v^5 + 740v^6 + 1972v^7,
    # v = tanh(1/T), holds to ~1e-7.
    L, T = 32, 20.0
    _, M = _chain_stats(L, T, n_chains=32, burn=50, n_meas=1000, seed=99)
    m, se = _mean_and_se((M**2).mean(axis=1) / L**2)
    v = math.tanh(1.0 / T)
    chi = sum(c * v**k for k, c in enumerate([1, 4, 12, 36, 100, 276, 740, 1972]))
    assert abs(m - chi) < 3 * se, (m, chi, se)
    e, se_e = _mean_and_se(_chain_stats(L, T, 32, 50, 400, 98)[0].mean(axis=1) / L**2)
    assert abs(e - exact.onsager_u(T)) < 3 * se_e


# --------------------------------------------------------------------------
# The light-cone window helper gives the full-lattice values.
# --------------------------------------------------------------------------
def test_window_light_cone_matches_full_lattice():
    L, T, seed, n = 64, exact.T_C, 17, 5
    full = oracle.init(L, seed, 2)
    oracle.sweeps(full, T, seed, 2, 0, n)
    rng = np.random.default_rng(1)
    for y, x in list(rng.integers(0, L, size=(12, 2))) + [(0, 0), (L - 1, L - 1), (0, L - 1)]:
        assert oracle.window_state(L, seed, 2, False, T, int(y), int(x), 0, n) == full[y, x]
