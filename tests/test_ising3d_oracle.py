"""Pins of the three-dimensional oracle (oracle/ising3d_oracle.c): thresholds
in 60-digit arithmetic, energy closed forms, the T -> 0 and T -> inf limits,
exact enumeration of the 2 x 2 x 2 torus (every neighbour pair joined by two
bonds), and the simple-cubic high-temperature series of the energy and the
susceptibility (coefficients from counting closed polygons and self-avoiding
walks on the lattice: 3 squares per site; 6, 30, 150, 726 walks of 1..4 steps)."""
from __future__ import annotations

import itertools
import math
import os

import mpmath as mp
import numpy as np
import pytest
from scipy import stats

import oracle

NT = max(1, min(8, os.cpu_count() or 1))


def test_thresholds3d_exact():
    rng = np.random.default_rng(31)
    temps = list(rng.uniform(0.3, 60.0, size=300)) + [1.0, 4.5, 4.511528]
    with mp.workdps(60):
        for T in temps:
            thr = oracle.thresholds3d(T)
            for k, dE in enumerate((4, 8, 12)):
                v = mp.exp(-mp.mpf(dE) / mp.mpf(T)) * mp.mpf(2) ** 32
                if abs(v - mp.nint(v)) < mp.mpf(10) ** -5:
                    continue
                assert int(thr[k]) == min(int(mp.floor(v)), 2**32 - 1), (T, dE)
    assert list(oracle.thresholds3d(0.1)) == [0, 0, 0]
    with pytest.raises(ValueError):
        oracle.thresholds3d(0.0)


@pytest.mark.parametrize("L", [2, 4, 6])
def test_energy3d_closed_forms(L):
    N = L ** 3
    cold = np.ones((L, L, L), np.int8)
    assert oracle.energy3d(cold) == -3 * N and oracle.magnetization3d(cold) == N
    z, y, x = np.indices((L, L, L))
    neel = np.where((x + y + z) % 2 == 0, 1, -1).astype(np.int8)
    assert oracle.energy3d(neel) == 3 * N and oracle.magnetization3d(neel) == 0
    one = cold.copy()
    one[1, 0, L - 1] = -1                         # six bonds broken (at L = 2: three neighbours, two bonds each)
    assert oracle.energy3d(one) == -3 * N + 12 and oracle.magnetization3d(one) == N - 2


def test_init3d_cold_and_random():
    assert np.all(oracle.init3d(4, 1, cold=True) == 1)
    r = oracle.init3d(16, 5)
    assert set(np.unique(r)) == {-1, 1}
    assert abs(int(r.sum())) < 4 * math.sqrt(r.size)


def test_infinite_temperature_negates_every_spin3d():
    s0 = oracle.init3d(8, 9)
    s = s0.copy()
    oracle.sweeps3d(s, 1e12, 9, 0, 0, 1)           # thresholds clamp to 2^32 - 1
    assert np.array_equal(s, -s0)


def test_zero_temperature3d():
    cold = np.ones((6, 6, 6), np.int8)
    E, M = oracle.sweeps3d(cold, 0.05, 1, 0, 0, 5)
    assert np.all(E == -3 * 216) and np.all(M == 216)
    s = oracle.init3d(8, 2)
    last = oracle.energy3d(s)
    for t in range(6):
        E, _ = oracle.sweeps3d(s, 0.05, 2, 0, t, 1)
        assert E[0] <= last
        last = E[0]


def test_zero_temperature_neel_worked_case():
    # From the Neel state (+1 on (x+y+z) even) at T -> 0: in the black
    # half-sweep every black site sees six -1 neighbours (dE = -12) and
    # flips, so after it every spin is -1; the white half-sweep then finds
    # every site aligned (dE = +12 > 0, no draw can pass thr = 0).  One sweep
    # ends in all -1.  Updating a colour that mixes neighbours (e.g. (x+y)
    # parity) does not.
    L = 4
    z, y, x = np.indices((L, L, L))
    s = np.where((x + y + z) % 2 == 0, 1, -1).astype(np.int8)
    E, M = oracle.sweeps3d(s, 0.05, 1, 0, 0, 1)
    assert np.all(s == -1) and E[0] == -3 * L**3 and M[0] == -(L**3)


def _brute_energy(sigma):
    return -int(sum((sigma * np.roll(sigma, -1, axis=a)).sum() for a in range(3)))


def _chains3d(L, T, n_chains, burn, n_meas, seed):
    sig = [oracle.init3d(L, seed, s) for s in range(n_chains)]
    sims = list(range(n_chains))
    oracle.sweeps3d_batch(sig, [T] * n_chains, [seed] * n_chains, sims, 0, burn, NT)
    E, M = oracle.sweeps3d_batch(sig, [T] * n_chains, [seed] * n_chains, sims, burn, n_meas, NT)
    return E.astype(np.float64), M.astype(np.float64)


@pytest.mark.parametrize("T", [2.0, 4.5, 8.0])
def test_2x2x2_joint_distribution_matches_enumeration(T):
    states = np.array(list(itertools.product((1, -1), repeat=8)), dtype=np.int8).reshape(-1, 2, 2, 2)
    E_all = np.array([_brute_energy(s) for s in states])
    M_all = states.reshape(len(states), -1).sum(axis=1)
    assert np.array_equal(E_all, [oracle.energy3d(s) for s in states])
    w = np.exp(-(E_all - E_all.min()) / T)
    keys = E_all * 100 + np.abs(M_all)
    uniq, inv = np.unique(keys, return_inverse=True)
    p = np.bincount(inv, weights=w) / w.sum()
    E, M = _chains3d(2, T, n_chains=256, burn=50, n_meas=600, seed=4242)
    ks = (E[:, ::5] * 100 + np.abs(M[:, ::5])).astype(np.int64).ravel()
    obs = np.array([(ks == u).sum() for u in uniq], dtype=np.float64)
    assert obs.sum() == ks.size
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


def test_high_temperature_series3d():
    # ln Z / N = ln 2 + 3 ln cosh b + 3 t^4 + O(t^6), t = tanh b, so
    # u = -3 t - 12 t^3 (1 - t^2) + O(t^5); chi = <M^2>/N = 1 + 6v + 30v^2 +
    # 150v^3 + 726v^4 + O(v^5), v = t
    L, T = 12, 20.0
    t = math.tanh(1.0 / T)
    E, M = _chains3d(L, T, n_chains=32, burn=30, n_meas=600, seed=77)
    N = L ** 3
    e = E.mean(axis=1) / N
    u = -3 * t - 12 * t**3 * (1 - t * t)
    assert abs(e.mean() - u) < 3 * e.std(ddof=1) / math.sqrt(len(e)) + 1e-4, (e.mean(), u)
    chi = (M ** 2).mean(axis=1) / N
    series = 1 + 6 * t + 30 * t**2 + 150 * t**3 + 726 * t**4
    assert abs(chi.mean() - series) < 3 * chi.std(ddof=1) / math.sqrt(len(chi)) + 4000 * t**5, (chi.mean(), series)
