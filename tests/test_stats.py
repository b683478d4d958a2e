"""Statistics: the oracle's tau_int and Binder cumulant pinned to closed forms
(AR(1) process, i.i.d. noise, Gaussian and two-peak magnetization
distributions), and the library's host implementation (C ABI) against it."""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import stats as ostats
from paper_2404_16990_gb300 import ising


def ar1(rho, n, seed):
    rng = np.random.default_rng(seed)
    eps = rng.standard_normal(n)
    x = np.empty(n)
    x[0] = eps[0] / math.sqrt(1 - rho * rho)
    for i in range(1, n):
        x[i] = rho * x[i - 1] + eps[i]
    return x


@pytest.mark.parametrize("rho", [0.0, 0.5, 0.9])
def test_tau_int_ar1_closed_form(rho):
    # tau_int of AR(1) = (1 + rho) / (2 (1 - rho))
    x = ar1(rho, 400_000, seed=int(rho * 10) + 1)
    tau, err, W = ostats.tau_int(x)
    exact = (1 + rho) / (2 * (1 - rho))
    bias = rho ** (W + 1) / (1 - rho) if rho > 0 else 0.0   # truncated tail
    assert abs(tau - exact) < 4 * err + bias + 1e-3, (tau, exact, err, W)


def test_tau_int_constant_and_alternating():
    assert ostats.tau_int(np.ones(100))[0] == 0.5
    # perfectly anticorrelated series: rho(1) = -1 (1 - 1/n), the window stops at lag 1
    x = np.tile([1.0, -1.0], 500)
    tau, _, W = ostats.tau_int(x)
    assert W == 1 and abs(tau - (0.5 - (1 - 1 / 1000))) < 1e-12


def test_binder_limits():
    rng = np.random.default_rng(0)
    g = rng.standard_normal(2_000_000)          # Gaussian m (disordered phase): U -> 0
    assert abs(ostats.binder(g)) < 5e-3
    two = np.where(rng.random(1000) < 0.5, 0.7, -0.7)   # ordered phase: U -> 2/3
    assert abs(ostats.binder(two) - 2.0 / 3.0) < 1e-12


def test_library_tau_int_matches_oracle():
    for rho, seed, n in [(0.0, 3, 50_000), (0.6, 4, 50_000), (0.95, 5, 50_000), (0.9, 6, 3000), (0.99, 7, 200_000)]:
        x = ar1(rho, n, seed)
        lib = ising.ising_tau_int(x, 6.0)
        ref = ostats.tau_int(x, 6.0)
        assert lib[2] == ref[2]
        assert abs(lib[0] - ref[0]) < 1e-9 * max(1.0, ref[0])
        assert abs(lib[1] - ref[1]) < 1e-9 * max(1.0, ref[1])
    with pytest.raises(ising.IsingError):
        ising.ising_tau_int([1.0], 6.0)
    with pytest.raises(ising.IsingError):
        ising.ising_tau_int([1.0, 2.0], 0.0)


def test_library_binder_matches_oracle():
    rng = np.random.default_rng(7)
    rows = []
    ms = []
    for k in range(5):
        M = rng.integers(-4096, 4097, size=300)
        E = rng.integers(-8192, 8192, size=300)
        rows.append(ostats.moments(E, M, 4096))
        ms.append(M / 4096)
    rows.append(np.zeros(6))
    U = ising.ising_binder(np.array(rows))
    for k in range(5):
        assert abs(U[k] - ostats.binder(ms[k])) < 1e-12
    assert math.isnan(U[5])
