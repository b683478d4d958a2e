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
    # the window stops at the first lag with W >= c tau(W); the step from
    # tau(W-1) to tau(W) is rho(W), so 0 <= W - c tau < 1 - c rho(W), and
    # rho(W) is tiny at these windows
    assert 0.0 <= W - 6.0 * tau < 1.5, (W, tau)


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


# --------------------------------------------------------------------------
# Statistical inefficiency and automatic equilibration detection (the method
# Section 3.1 cites for discarding non-equilibrated data).
# --------------------------------------------------------------------------
def test_statistical_inefficiency_worked_case():
    # x = 1, 2, 3, 4: mean 2.5, deviations -1.5, -0.5, 0.5, 1.5, variance 1.25;
    # C(1) = (0.75 - 0.25 + 0.75) / (3 * 1.25) = 1/3, C(2) = (-0.75 - 0.75) /
    # (2 * 1.25) < 0 stops the sum; g = 1 + 2 (1 - 1/4) (1/3) = 1.5
    assert abs(ostats.statistical_inefficiency([1.0, 2.0, 3.0, 4.0]) - 1.5) < 1e-15
    # anticorrelated: C(1) < 0 at once, g = 1; constant: g = 1
    assert ostats.statistical_inefficiency([1.0, -1.0] * 50) == 1.0
    assert ostats.statistical_inefficiency(np.full(10, 3.0)) == 1.0


@pytest.mark.parametrize("rho", [0.0, 0.5, 0.9])
def test_statistical_inefficiency_ar1_closed_form(rho):
    # g = 1 + 2 tau = (1 + rho) / (1 - rho) for AR(1)
    x = ar1(rho, 200_000, seed=40 + int(rho * 10))
    g = ostats.statistical_inefficiency(x)
    exact = (1 + rho) / (1 - rho)
    assert abs(g - exact) < 0.06 * exact, (g, exact)


def test_statistical_inefficiency_affine_invariant():
    x = ar1(0.7, 5000, seed=9)
    g = ostats.statistical_inefficiency(x)
    assert abs(ostats.statistical_inefficiency(-3.0 * x + 17.0) - g) < 1e-9 * g


def test_equilibration_stationary_series_starts_early():
    x = ar1(0.5, 20_000, seed=11)
    t0, g, n_eff = ostats.detect_equilibration(x, stride=100)
    assert t0 <= 0.1 * len(x)
    assert abs(g - 3.0) < 0.3 and abs(n_eff - (len(x) - t0) / g) < 1e-9


def test_equilibration_detects_an_offset_block():
    rng = np.random.default_rng(12)
    x = rng.standard_normal(10_000)
    x[:1000] += 3.0                                   # non-equilibrated start
    t0, g, _ = ostats.detect_equilibration(x, stride=10)
    assert 990 <= t0 <= 1100, t0
    assert g < 1.3


def test_equilibration_detects_a_relaxation():
    # exponential relaxation of amplitude 10 on top of AR(1) noise of unit
    # stationary variance: the transient falls below the noise after
    # ln(10) * 300 ~ 700 steps; the detected start lies between 2 and 10 decay times
    n, tau0 = 30_000, 300.0
    noise = ar1(0.8, n, seed=13) * math.sqrt(1 - 0.64)
    x = 10.0 * np.exp(-np.arange(n) / tau0) + noise
    t0, _, _ = ostats.detect_equilibration(x, stride=50)
    assert 2 * tau0 <= t0 <= 10 * tau0, t0


def test_library_equilibration_matches_oracle():
    rng = np.random.default_rng(21)
    cases = []
    for n, rho, amp, tau0 in [(800, 0.3, 4.0, 50.0), (3000, 0.9, 10.0, 200.0), (6000, 0.7, 5.0, 400.0),
                              (20_000, 0.95, 8.0, 1500.0), (2000, 0.0, 0.0, 1.0)]:
        noise = ar1(rho, n, seed=int(rng.integers(1 << 30))) * math.sqrt(1 - rho * rho)
        cases.append(amp * np.exp(-np.arange(n) / tau0) + noise)
    step = rng.standard_normal(5000)
    step[:700] -= 2.5
    cases.append(step)
    for x in cases:
        for stride in (1 if len(x) <= 800 else 0, 37):
            s = stride or max(1, len(x) // 256)
            t_ref, g_ref, n_ref = ostats.detect_equilibration(x, s)
            t_lib, g_lib, n_lib = ising.ising_equilibration(x, stride)
            assert t_lib == t_ref, (len(x), stride, t_lib, t_ref)
            assert abs(g_lib - g_ref) < 1e-9 * g_ref and abs(n_lib - n_ref) < 1e-9 * n_ref
        assert abs(ising.ising_stat_inefficiency(x) - ostats.statistical_inefficiency(x)) < \
            1e-9 * ostats.statistical_inefficiency(x)
    assert ising.ising_stat_inefficiency([1.0, 2.0, 3.0, 4.0]) == 1.5
    with pytest.raises(ising.IsingError):
        ising.ising_equilibration([1.0], 0)
    with pytest.raises(ising.IsingError):
        ising.ising_equilibration([1.0, 2.0, 3.0], -1)
