"""Plant plausible mistakes in a copy of the oracle source (on the CPU) and
check that at least one pin catches each: a dropped neighbour, swapped
thresholds, the colour order reversed, zero-energy moves rejected, a wrong
Philox multiplier, an energy sign error."""
from __future__ import annotations

import numpy as np
import pytest

import exact
import oracle
import test_oracle_pins as pins

MUTATIONS = {
    "dropped_neighbour": ("+ sigma[(size_t)y * L + wrap(x - 1, L)] + sigma[(size_t)y * L + wrap(x + 1, L)];",
                          "+ sigma[(size_t)y * L + wrap(x - 1, L)];"),
    "swapped_thresholds": ("flip = r < thr[dE == 8 ? 1 : 0];", "flip = r < thr[dE == 8 ? 0 : 1];"),
    "colour_order": ("oracle_half_sweep(L, sigma, 0, thr, seed, s, t, n_threads);\n"
                     "        oracle_half_sweep(L, sigma, 1, thr, seed, s, t, n_threads);",
                     "oracle_half_sweep(L, sigma, 1, thr, seed, s, t, n_threads);\n"
                     "        oracle_half_sweep(L, sigma, 0, thr, seed, s, t, n_threads);"),
    "zero_moves_rejected": ("    if (dE <= 0) {\n        flip = 1;\n    } else {\n        uint32_t p",
                            "    if (dE < 0) {\n        flip = 1;\n    } else if (dE == 0) {\n"
                            "        flip = 0;\n    } else {\n        uint32_t p"),
    "philox_multiplier": ("#define ORC_PHILOX_MUL_A 0xD2511F53u", "#define ORC_PHILOX_MUL_A 0xD2511F55u"),
    "energy_sign": ("e -= (int64_t)(s * (r + d));", "e += (int64_t)(s * (r + d));"),
}


def _caught(variant_so) -> list:
    caught = []
    with oracle.use_library(variant_so):
        checks = [
            ("kat", lambda: [pins.test_philox_known_answers(c, k, e) for c, k, e in pins._kat_rows()]),
            ("t0_golden", lambda: [pins.test_zero_temperature_worked_cases(*c) for c in pins._golden_t0_cases()]),
            ("closed_forms", lambda: pins.test_energy_closed_forms(4)),
            ("chi2_4x4", lambda: pins.test_4x4_joint_distribution_matches_enumeration(exact.T_C)),
        ]
        for name, fn in checks:
            try:
                fn()
            except AssertionError:
                caught.append(name)
    return caught


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTATIONS[name]
    src = oracle.source_text()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    so = oracle.compile_variant(src.replace(old, new), str(tmp_path), "oracle_" + name)
    caught = _caught(so)
    assert caught, f"no pin caught the planted mistake {name}"


def test_unmodified_source_passes_same_checks(tmp_path):
    so = oracle.compile_variant(oracle.source_text(), str(tmp_path), "oracle_clean")
    assert _caught(so) == []
