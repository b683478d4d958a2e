"""Pins for the Wolff oracle (oracle/wolff_oracle.c): each test checks it
against what the definitions and the mathematics fix -- the seed site from
its draw, the flipped set against the connected component of the seed built
independently (bonds drawn here in Python from the phase-10 definition,
components by scipy), the change of E and M, exact enumeration of the 4x4
torus, Kaufman's finite-lattice energy, and the T -> 0 and T -> inf limits
(the whole same-spin domain, a single site)."""
from __future__ import annotations

import math
import os

import numpy as np
import pytest
from scipy import sparse, stats
from scipy.sparse import csgraph

import exact
import oracle

NT = max(1, min(8, os.cpu_count() or 1))


def _bond_draw(seed, s, t, p, lane):
    key = [seed & 0xFFFFFFFF, seed >> 32]
    return int(oracle.philox4x32_10([p >> 1, t, s, 10], key)[lane])


def _component_flip(sigma, T, seed, s, t):
    """The expected lattice after Wolff step t, built without the oracle's
    growth: every bond between equal spins is active iff its phase-10 draw is
    below the bond threshold; the cluster is the connected component of the
    seed; it flips."""
    L = sigma.shape[0]
    N = L * L
    thr = oracle.sw_threshold(T)
    rows, cols = [], []
    for y in range(L):
        for x in range(L):
            p = y * L + x
            for lane, q in ((2 * (p & 1), y * L + (x + 1) % L), (2 * (p & 1) + 1, ((y + 1) % L) * L + x)):
                if sigma.flat[p] == sigma.flat[q] and _bond_draw(seed, s, t, p, lane) < thr:
                    rows.append(p)
                    cols.append(q)
    g = sparse.coo_matrix((np.ones(len(rows)), (rows, cols)), shape=(N, N))
    _, lab = csgraph.connected_components(g, directed=False)
    r = int(oracle.philox4x32_10([0, t, s, 9], [seed & 0xFFFFFFFF, seed >> 32])[0])
    p0 = (r * N) >> 32
    assert p0 == oracle.wolff_seed(L, seed, s, t)
    out = sigma.copy().ravel()
    members = lab == lab[p0]
    out[members] = -out[members]
    return out.reshape(L, L), int(members.sum())


@pytest.mark.parametrize("L,T,seed", [(4, 2.0, 3), (8, 1.5, 11), (16, 2.269185, 5), (16, 3.5, 9), (32, 2.4, 21)])
def test_wolff_step_is_the_seed_component(L, T, seed):
    sigma = oracle.init(L, seed, 1)
    for t in range(6):
        want, size = _component_flip(sigma, T, seed, 1, t)
        E, M, C = oracle.wolff_sweeps(sigma, T, seed, 1, t, 1)
        assert np.array_equal(sigma, want), (L, T, t)
        assert C[0] == size
        assert E[0] == oracle.energy(sigma) and M[0] == oracle.magnetization(sigma)


def test_wolff_seed_covers_the_lattice():
    # floor(r N / 2^32) of 2^32-uniform r: every site, about equally often
    L, n = 8, 20000
    counts = np.bincount([oracle.wolff_seed(L, 7, 0, t) for t in range(n)], minlength=L * L)
    assert counts.min() > 0
    chi2 = ((counts - n / L**2) ** 2 / (n / L**2)).sum()
    assert stats.chi2.sf(chi2, L * L - 1) > 1e-3


def _wolff_chains(L, T, n_chains, burn, n_meas, seed):
    sig = [oracle.init(L, seed, s) for s in range(n_chains)]
    sims = list(range(n_chains))
    oracle.wolff_sweeps_batch(sig, [T] * n_chains, [seed] * n_chains, sims, 0, burn, NT)
    E, M = oracle.wolff_sweeps_batch(sig, [T] * n_chains, [seed] * n_chains, sims, burn, n_meas, NT)
    return E.astype(np.float64), M.astype(np.float64)


@pytest.mark.parametrize("T", [1.5, exact.T_C, 3.0])
def test_wolff_4x4_joint_distribution_matches_enumeration(T):
    E_all, M_all = exact.enumerate_EM(4)
    w = exact.boltzmann_weights(E_all, T)
    keys = E_all * 1000 + np.abs(M_all)
    uniq, inv = np.unique(keys, return_inverse=True)
    p = np.bincount(inv, weights=w)
    E, M = _wolff_chains(4, T, n_chains=256, burn=40, n_meas=800, seed=20240427)
    thin = 8
    ks = (E[:, ::thin] * 1000 + np.abs(M[:, ::thin])).astype(np.int64).ravel()
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


@pytest.mark.parametrize("T", [2.0, exact.T_C, 3.0])
def test_wolff_energy_matches_kaufman(T):
    L = 16
    E, _ = _wolff_chains(L, T, n_chains=64, burn=200, n_meas=3000, seed=79)
    per_chain = E.mean(axis=1)
    m, se = per_chain.mean(), per_chain.std(ddof=1) / math.sqrt(len(per_chain))
    ref = exact.kaufman_mean_energy(L, T)
    assert abs(m - ref) < 3 * se + 1e-9, (T, m, ref, se)


def test_wolff_zero_temperature_flips_the_domain():
    # T -> 0: every bond between equal spins is active, so from a cold lattice
    # the cluster is the whole lattice and every step flips it
    L = 16
    sigma = np.ones((L, L), np.int8)
    E, M, C = oracle.wolff_sweeps(sigma, 0.01, 9, 0, 0, 10)
    assert np.all(C == L * L) and np.all(E == -2 * L * L)
    assert list(M) == [(-1) ** (i + 1) * L * L for i in range(10)]


def test_wolff_infinite_temperature_flips_one_site():
    # T -> inf: no active bond, the cluster is the seed alone
    L, T = 16, 1e9
    sigma = oracle.init(L, 4, 0)
    before = sigma.copy()
    E, M, C = oracle.wolff_sweeps(sigma, T, 4, 0, 0, 1)
    assert C[0] == 1
    diff = np.argwhere(sigma != before)
    assert len(diff) == 1
    y, x = diff[0]
    assert y * L + x == oracle.wolff_seed(L, 4, 0, 0)
