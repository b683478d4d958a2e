"""Plant plausible mistakes in a copy of the statistics oracle's source
(oracle/stats.py, on the CPU) and check that at least one pin of
test_stats.py catches each: the autocovariance normalisation, tau's
starting value, the Madras-Sokal window constant, the Binder factor and
power, the statistical inefficiency's (1 - t/T) weight and lag
normalisation, and the equilibration criterion."""
from __future__ import annotations

import inspect
import types

import pytest

from oracle import stats as ostats
import test_stats as pins

MUTATIONS = {
    "autocov_normalised_by_n_minus_lag": ("rho = float(np.dot(d[:-lag], d[lag:])) / (n * c0)",
                                          "rho = float(np.dot(d[:-lag], d[lag:])) / ((n - lag) * c0)"),
    "tau_starts_at_one": ("tau, W = 0.5, 0", "tau, W = 1.0, 0"),
    "window_constant_dropped": ("if lag >= c * tau:", "if lag >= tau:"),
    "binder_factor": ("return 1.0 - m4 / (3.0 * m2 * m2)", "return 1.0 - m4 / (2.0 * m2 * m2)"),
    "binder_power": ("return 1.0 - m4 / (3.0 * m2 * m2)", "return 1.0 - m4 / (3.0 * m2)"),
    "inefficiency_weight_dropped": ("tau += (1.0 - t / T) * C", "tau += C"),
    "inefficiency_lag_normalisation": ("C = float(np.dot(d[:T - t], d[t:])) / ((T - t) * var)",
                                       "C = float(np.dot(d[:T - t], d[t:])) / (T * var)"),
    "inefficiency_factor_two": ("return max(1.0, 1.0 + 2.0 * tau)", "return max(1.0, 1.0 + tau)"),
    "equilibration_uses_g_times_n": ("n_eff = (T - t0) / g", "n_eff = (T - t0) * g"),
}

CHECKS = [
    ("tau_const_alternating", lambda: pins.test_tau_int_constant_and_alternating()),
    ("binder_limits", lambda: pins.test_binder_limits()),
    ("inefficiency_worked", lambda: pins.test_statistical_inefficiency_worked_case()),
    ("equilibration_offset", lambda: pins.test_equilibration_detects_an_offset_block()),
    ("tau_ar1_0.9", lambda: pins.test_tau_int_ar1_closed_form(0.9)),
    ("inefficiency_ar1_0.5", lambda: pins.test_statistical_inefficiency_ar1_closed_form(0.5)),
]


def _module_from(src: str):
    mod = types.ModuleType("stats_variant")
    mod.__file__ = ostats.__file__
    exec(compile(src, "stats_variant", "exec"), mod.__dict__)
    return mod


def _catches(mod, monkeypatch, stop_early=True):
    monkeypatch.setattr(pins, "ostats", mod)
    caught = []
    for name, fn in CHECKS:
        try:
            fn()
        except Exception as e:
            caught.append((name, type(e).__name__))
            if stop_early:
                break
    return caught


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, monkeypatch):
    old, new = MUTATIONS[name]
    src = inspect.getsource(ostats)
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    assert _catches(_module_from(src.replace(old, new)), monkeypatch), f"no pin caught {name}"


def test_unmodified_source_passes_same_checks(monkeypatch):
    assert _catches(_module_from(inspect.getsource(ostats)), monkeypatch, stop_early=False) == []
