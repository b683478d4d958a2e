"""Plant plausible mistakes in a copy of the random-stream battery oracle's
source (oracle/prng_battery.py, on the CPU) and check that at least one pin
of test_prng_battery.py catches each: bit order, float shaping, the
normalisation or degrees of freedom of each test's statistic, the run count,
the longest-run recurrence, the spectral threshold, the cumulative-sums
series."""
from __future__ import annotations

import inspect
import types

import pytest

from oracle import prng_battery as pb
import test_prng_battery as pins

MUTATIONS = {
    "bits_lsb_first": ("shifts = np.arange(31, -1, -1, dtype=np.uint32)", "shifts = np.arange(0, 32, dtype=np.uint32)"),
    "floats_24_bits": ("return (w & 0x7FFFFF).astype(np.float64) / float(1 << 23)",
                       "return (w & 0xFFFFFF).astype(np.float64) / float(1 << 24)"),
    "frequency_normalisation": ("special.erfc(abs(S) / math.sqrt(2.0 * n))", "special.erfc(abs(S) / math.sqrt(n))"),
    "block_frequency_factor": ("chi2 = 4.0 * M * float(", "chi2 = 2.0 * M * float("),
    "runs_denominator": ("den = 2.0 * math.sqrt(2.0 * n) * pi * (1.0 - pi)", "den = math.sqrt(2.0 * n) * pi * (1.0 - pi)"),
    "runs_count_off_by_one": ("V = 1 + int((b[1:] != b[:-1]).sum())", "V = int((b[1:] != b[:-1]).sum())"),
    "longest_run_recurrence": ("f[m] = sum(f[m - 1 - j] for j in range(k + 1))", "f[m] = sum(f[m - 1 - j] for j in range(k))"),
    "longest_run_dof": ("special.gammaincc((hi - lo) / 2.0, chi2 / 2.0)", "special.gammaincc((hi - lo + 1) / 2.0, chi2 / 2.0)"),
    "spectral_threshold": ("T = math.sqrt(math.log(1.0 / 0.05) * n)", "T = math.sqrt(math.log(1.0 / 0.01) * n)"),
    "spectral_expected_count": ("N0 = 0.95 * n / 2.0", "N0 = 0.95 * n"),
    "cusum_second_series_sign": ("return float(1.0 - s1 + s2), float(z)", "return float(1.0 - s1 - s2), float(z)"),
    "float_uniformity_dof": ("special.gammaincc((bins - 1) / 2.0, chi2 / 2.0)", "special.gammaincc(bins / 2.0, chi2 / 2.0)"),
    "float_pairs_expected": ("e = n / (bins * bins)", "e = 2 * n / (bins * bins)"),
}

CHECKS = [
    ("bit_order", lambda: pins.test_bit_order_and_float_shaping()),
    ("frequency_hand", lambda: pins.test_frequency_hand_case()),
    ("longest_run_brute_13", lambda: pins.test_longest_run_counts_brute_force(13)),
    ("longest_run_classes", lambda: pins.test_longest_run_class_probs()),
    ("cusum_monte_carlo", lambda: pins.test_cusum_pvalue_matches_monte_carlo_tail()),
    ("statistics_by_hand", lambda: pins.test_statistics_by_hand()),
    ("defects", lambda: pins.test_defects_are_caught()),
    ("uniform_pvalues", lambda: pins.test_pvalues_uniform_on_a_library_generator()),
    ("chi2_scale_block", lambda: pins.test_chi2_pvalues_uniform_at_scale("block_frequency", 512)),
    ("chi2_scale_float", lambda: pins.test_chi2_pvalues_uniform_at_scale("float_uniformity", 1000)),
    ("chi2_scale_pairs", lambda: pins.test_chi2_pvalues_uniform_at_scale("float_pairs", 2000)),
    ("chi2_scale_longest", lambda: pins.test_chi2_pvalues_uniform_at_scale("longest_run", 512)),
]


def _module_from(src: str):
    mod = types.ModuleType("prng_battery_variant")
    mod.__file__ = pb.__file__
    exec(compile(src, "prng_battery_variant", "exec"), mod.__dict__)
    return mod


def _catches(mod, monkeypatch, stop_early=True):
    monkeypatch.setattr(pins, "pb", mod)
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
    src = inspect.getsource(pb)
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    assert _catches(_module_from(src.replace(old, new)), monkeypatch), f"no pin caught {name}"


def test_unmodified_source_passes_same_checks(monkeypatch):
    assert _catches(_module_from(inspect.getsource(pb)), monkeypatch, stop_early=False) == []
