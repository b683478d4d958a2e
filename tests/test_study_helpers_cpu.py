"""Host-side helpers of the measurement studies, on the CPU: the Binder
crossing by linear interpolation, the studies' own Kolmogorov-Smirnov test
against scipy's, and the Binder cumulant against the statistics oracle."""
from __future__ import annotations

import numpy as np
import pytest
from scipy import stats

from oracle import stats as ostats
from paper_2404_16990_gb300 import binder_study, prng_study


def test_binder_crossing_of_two_lines():
    # U_a = 1 - T, U_b = 0.5 (T - 0.2): they cross at T = 1.1 / 1.5
    Ts = np.linspace(0.0, 2.0, 11)
    assert binder_study._crossing(Ts, 1.0 - Ts, 0.5 * (Ts - 0.2)) == pytest.approx(1.1 / 1.5)
    # a crossing exactly on a grid point, and no crossing at all
    assert binder_study._crossing([1.0, 2.0, 3.0], [0.0, 1.0, 2.0], [1.0, 1.0, 1.0]) == 2.0
    assert binder_study._crossing([1.0, 2.0, 3.0], [2.0, 3.0, 4.0], [1.0, 1.0, 1.0]) is None


def test_binder_of_matches_the_oracle():
    rng = np.random.default_rng(3)
    for m in (rng.standard_normal(5000), np.where(rng.random(300) < 0.5, 0.6, -0.6), rng.random(1000) - 0.3):
        assert binder_study._binder_of(m) == pytest.approx(ostats.binder(m), rel=1e-12, abs=1e-12)
    assert np.isnan(binder_study._binder_of(np.zeros(10)))


@pytest.mark.parametrize("n", [20, 200, 5000])
def test_ks_uniform_matches_scipy(n):
    rng = np.random.default_rng(n)
    for p in (rng.random(n), rng.random(n) ** 1.3):
        d, q = prng_study._ks_uniform(p)
        ref = stats.kstest(p, "uniform")
        assert d == pytest.approx(ref.statistic, rel=1e-12)
        # the asymptotic (Stephens-corrected) p-value against scipy's exact one
        assert abs(q - ref.pvalue) < 0.02 + 0.1 * ref.pvalue
