"""Pins for the Swendsen-Wang oracle (oracle/cluster_oracle.c): each test
checks it against what the mathematics fixes -- the bond probability
1 - exp(-2/T) in 60-digit arithmetic, the bond statistics, cluster partitions
against scipy's connected components, exact enumeration of the 4x4 torus,
Kaufman's finite-lattice energy, Onsager's magnetization, the T -> 0 and
T -> inf limits, and the collapse of the autocorrelation time at T_c that
is the point of a cluster algorithm (Section 1 names it as the cure for
critical slowing down)."""
from __future__ import annotations

import math
import os

import mpmath as mp
import numpy as np
import pytest
from scipy import sparse, stats
from scipy.sparse import csgraph

import exact
import oracle
from oracle import stats as ostats

NT = max(1, min(8, os.cpu_count() or 1))


# --------------------------------------------------------------------------
# Bond threshold: floor(2^32 (1 - exp(-2/T))) clamped, 60-digit arithmetic.
# --------------------------------------------------------------------------
def test_sw_threshold_exact():
    rng = np.random.default_rng(11)
    temps = list(rng.uniform(0.05, 80.0, size=400)) + [0.5, 1.0, 1.5, exact.T_C, 2.269185, 3.0, 1e3]
    with mp.workdps(60):
        for T in temps:
            v = (1 - mp.exp(-mp.mpf(2) / mp.mpf(T))) * mp.mpf(2) ** 32
            if abs(v - mp.nint(v)) < mp.mpf(10) ** -5:
                continue  # within rounding of an integer: either floor is fine
            assert oracle.sw_threshold(T) == min(int(mp.floor(v)), 2**32 - 1), T


def test_sw_threshold_limits_and_errors():
    assert oracle.sw_threshold(0.01) == 2**32 - 1          # T -> 0: every equal pair bonded
    assert oracle.sw_threshold(1e9) == 8                   # 2^32 * 2e-9 = 8.59
    for bad in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(ValueError):
            oracle.sw_threshold(bad)


# --------------------------------------------------------------------------
# Bonds: only between equal spins, at rate p among them, fresh every step.
# --------------------------------------------------------------------------
def _pairs_equal(sigma):
    right = sigma == np.roll(sigma, -1, axis=1)
    down = sigma == np.roll(sigma, -1, axis=0)
    return right, down


@pytest.mark.parametrize("T", [1.5, exact.T_C, 3.0])
def test_bonds_between_equal_spins_at_rate_p(T):
    L, seed = 64, 4242
    sigma = oracle.init(L, seed)
    right_eq, down_eq = _pairs_equal(sigma)
    p = 1.0 - math.exp(-2.0 / T)
    n_on = n_eq = 0
    prev = None
    for t in range(20):
        b = oracle.sw_bonds(sigma, T, seed, 3, t)
        r, d = (b & 1) != 0, (b & 2) != 0
        assert not np.any(r & ~right_eq) and not np.any(d & ~down_eq)
        assert not np.any(b & ~np.uint8(3))
        n_on += int(r.sum() + d.sum())
        n_eq += int(right_eq.sum() + down_eq.sum())
        if prev is not None:
            assert not np.array_equal(prev, b)
        prev = b
    sd = math.sqrt(n_eq * p * (1 - p))
    assert abs(n_on - n_eq * p) < 4 * sd, (n_on, n_eq * p, sd)


def test_bonds_right_and_down_draws_are_distinct_lanes():
    # every equal pair bonded at T -> 0; at T = T_c the right and down bonds
    # of one site are not copies of each other
    sigma = np.ones((32, 32), np.int8)
    assert np.all(oracle.sw_bonds(sigma, 0.01, 5, 0, 0) == 3)
    b = oracle.sw_bonds(sigma, exact.T_C, 5, 0, 0)
    assert np.mean(((b & 1) != 0) != ((b & 2) != 0)) > 0.3


# --------------------------------------------------------------------------
# Cluster labels: the connected components of the bond graph on the torus
# (scipy.sparse.csgraph), named by their smallest site index.
# --------------------------------------------------------------------------
def _reference_labels(bonds):
    L = bonds.shape[0]
    N = L * L
    idx = np.arange(N).reshape(L, L)
    r = (bonds & 1) != 0
    d = (bonds & 2) != 0
    rows = np.concatenate([idx[r], idx[d]])
    cols = np.concatenate([np.roll(idx, -1, axis=1)[r], np.roll(idx, -1, axis=0)[d]])
    g = sparse.coo_matrix((np.ones(len(rows)), (rows, cols)), shape=(N, N))
    n, comp = csgraph.connected_components(g, directed=False)
    smallest = np.full(n, N, dtype=np.int64)
    np.minimum.at(smallest, comp, np.arange(N))
    return smallest[comp].reshape(L, L).astype(np.uint32), n


@pytest.mark.parametrize("L,density", [(2, 0.5), (3, 0.4), (4, 0.3), (8, 0.5), (16, 0.45), (33, 0.5),
                                       (64, 0.55), (64, 0.2), (128, 0.5)])
def test_labels_match_connected_components(L, density):
    rng = np.random.default_rng(L * 1000 + int(density * 100))
    for _ in range(3):
        bonds = ((rng.random((L, L)) < density).astype(np.uint8)
                 | ((rng.random((L, L)) < density).astype(np.uint8) << 1))
        lab, n = oracle.sw_labels(bonds)
        ref, n_ref = _reference_labels(bonds)
        assert n == n_ref
        assert np.array_equal(lab, ref)


def test_labels_extremes():
    L = 16
    lab, n = oracle.sw_labels(np.zeros((L, L), np.uint8))
    assert n == L * L and np.array_equal(lab.ravel(), np.arange(L * L))
    lab, n = oracle.sw_labels(np.full((L, L), 3, np.uint8))
    assert n == 1 and np.all(lab == 0)
    # a single wrapped row: the right bonds of row 5 only
    b = np.zeros((L, L), np.uint8)
    b[5, :] = 1
    lab, n = oracle.sw_labels(b)
    assert n == L * L - L + 1 and np.all(lab[5] == 5 * L)


# --------------------------------------------------------------------------
# The chain: stationary distribution, energies, magnetization, limits.
# --------------------------------------------------------------------------
def _sw_chains(L, T, n_chains, burn, n_meas, seed):
    sig = [oracle.init(L, seed, s) for s in range(n_chains)]
    sims = list(range(n_chains))
    oracle.sw_sweeps_batch(sig, [T] * n_chains, [seed] * n_chains, sims, 0, burn, NT)
    E, M = oracle.sw_sweeps_batch(sig, [T] * n_chains, [seed] * n_chains, sims, burn, n_meas, NT)
    return E.astype(np.float64), M.astype(np.float64)


def _mean_and_se(per_chain):
    return per_chain.mean(), per_chain.std(ddof=1) / math.sqrt(len(per_chain))


@pytest.mark.parametrize("T", [1.5, exact.T_C, 3.0])
def test_sw_4x4_joint_distribution_matches_enumeration(T):
    E_all, M_all = exact.enumerate_EM(4)
    w = exact.boltzmann_weights(E_all, T)
    keys = E_all * 1000 + np.abs(M_all)
    uniq, inv = np.unique(keys, return_inverse=True)
    p = np.bincount(inv, weights=w)
    E, M = _sw_chains(4, T, n_chains=256, burn=20, n_meas=400, seed=20240426)
    thin = 4
    ks = (E[:, ::thin] * 1000 + np.abs(M[:, ::thin])).astype(np.int64).ravel()
    obs = np.array([(ks == u).sum() for u in uniq], dtype=np.float64)
    assert obs.sum() == ks.size            # no state outside the enumeration
    exp_ = p * obs.sum()
    order = np.argsort(exp_)
    o2, e2, acc_o, acc_e = [], [], 0.0, 0.0
    for i in order:
        acc_o += obs[i]
        acc_e += exp_[i]
        if acc_e >= 10:
            o2.append(acc_o)
            e2.append(acc_e)
            acc_o = acc_e = 0.0
    if acc_e > 0:
        o2[-1] += acc_o
        e2[-1] += acc_e
    o2, e2 = np.array(o2), np.array(e2)
    chi2 = ((o2 - e2) ** 2 / e2).sum()
    assert len(o2) >= 3
    assert stats.chi2.sf(chi2, len(o2) - 1) > 1e-3, (T, chi2, len(o2))


@pytest.mark.parametrize("T", [2.0, exact.T_C, 3.0])
def test_sw_energy_matches_kaufman(T):
    L = 16
    E, _ = _sw_chains(L, T, n_chains=64, burn=50, n_meas=600, seed=78)
    m, se = _mean_and_se(E.mean(axis=1))
    ref = exact.kaufman_mean_energy(L, T)
    assert abs(m - ref) < 3 * se + 1e-9, (T, m, ref, se)


def test_sw_magnetization_matches_onsager():
    L, T = 64, 1.5
    _, M = _sw_chains(L, T, n_chains=16, burn=50, n_meas=300, seed=322)
    m, se = _mean_and_se(np.abs(M).mean(axis=1) / L**2)
    assert abs(m - exact.onsager_m(T)) < 3 * se, (m, exact.onsager_m(T), se)


def test_sw_zero_temperature_one_cluster():
    # T -> 0: every bond between equal spins is active, so a cold lattice is one
    # cluster; each step flips all of it or nothing.
    L = 16
    sigma = np.ones((L, L), np.int8)
    E, M = oracle.sw_sweeps(sigma, 0.01, 9, 0, 0, 64)
    assert np.all(E == -2 * L * L)
    assert set(np.unique(M)) == {-L * L, L * L}


def test_sw_infinite_temperature_independent_coins():
    # T -> inf: almost no bonds, every site its own cluster flipped with
    # probability 1/2, so one step from any state gives i.i.d. +-1 spins:
    # <M> = 0, <M^2> = N, <E> = 0, <E^2> = 2N.
    L, T = 32, 1e9
    N = L * L
    sigma = np.ones((L, L), np.int8)
    _, n = oracle.sw_labels(oracle.sw_bonds(sigma, T, 1, 0, 0))
    assert n == N
    E, M = oracle.sw_sweeps(sigma, T, 1, 0, 0, 4000)
    E, M = E.astype(np.float64), M.astype(np.float64)
    assert abs(M.mean()) < 4 * math.sqrt(N / len(M))
    assert abs((M**2).mean() / N - 1.0) < 4 * math.sqrt(2.0 / len(M))
    assert abs(E.mean()) < 4 * math.sqrt(2 * N / len(E))
    assert abs((E**2).mean() / (2 * N) - 1.0) < 4 * math.sqrt(2.0 / len(E))


def test_sw_beats_metropolis_autocorrelation_at_tc():
    # the reason for the cluster move: at T_c, tau_int(|M|) per step is O(1)
    # for Swendsen-Wang but grows like L^2.17 for single-site Metropolis
    L, T, n = 32, exact.T_C, 6000
    s1 = oracle.init(L, 5)
    oracle.sw_sweeps(s1, T, 5, 0, 0, 200)
    _, M_sw = oracle.sw_sweeps(s1, T, 5, 0, 200, n)
    s2 = oracle.init(L, 5)
    oracle.sweeps(s2, T, 5, 0, 0, 2000)
    _, M_mp = oracle.sweeps(s2, T, 5, 0, 2000, n)
    tau_sw = ostats.tau_int(np.abs(M_sw))[0]
    tau_mp = ostats.tau_int(np.abs(M_mp))[0]
    assert tau_sw < 10.0, tau_sw
    assert tau_mp > 5 * tau_sw, (tau_mp, tau_sw)


@pytest.mark.parametrize("L,T", [(8, 2.0), (16, exact.T_C), (32, 3.0)])
def test_sw_step_flips_each_cluster_by_its_root_coin(L, T):
    # one step = this step's bonds -> clusters named by their smallest site r0
    # -> every site flips iff the top bit of the phase-8 draw of r0 (lane r0 & 3
    # of Philox block (r0 >> 2, t, s, 8)) is 1
    seed, s = 0x5151, 3
    key = [seed & 0xFFFFFFFF, seed >> 32]
    sigma = oracle.init(L, seed, s)
    for t in range(3):
        before = sigma.copy()
        lab, _ = oracle.sw_labels(oracle.sw_bonds(before, T, seed, s, t))
        oracle.sw_sweeps(sigma, T, seed, s, t, 1)
        coin = {int(r): int(oracle.philox4x32_10([int(r) >> 2, t, s, 8], key)[int(r) & 3]) >> 31
                for r in np.unique(lab)}
        want = np.where(np.vectorize(coin.get)(lab) == 1, -before, before)
        assert np.array_equal(sigma, want), (L, T, t)
