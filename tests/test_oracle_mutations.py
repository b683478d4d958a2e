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


# --------------------------------------------------------------------------
# The same for the Swendsen-Wang oracle (cluster_oracle.c).
# --------------------------------------------------------------------------
import test_cluster_oracle as swpins  # noqa: E402

SW_MUTATIONS = {
    "sw_bond_probability": ("double p = -expm1(-2.0 / T);", "double p = -expm1(-1.0 / T);"),
    "sw_down_bond_dropped": ("if (me == down && r_down < thr) b |= 2u;", ""),
    "sw_bond_unequal_spins": ("if (me == right && r_right < thr) b |= 1u;",
                              "if (me != right && r_right < thr) b |= 1u;"),
    "sw_coin_per_site": ("oracle_site_random(seed, root, t, s, ORC_SW_PHASE_COIN)",
                         "oracle_site_random(seed, (uint32_t)p, t, s, ORC_SW_PHASE_COIN)"),
    "sw_left_neighbour_missed": ("if (bonds[left] & 1u) nb[k++] = left;", ""),
    "sw_same_lane_both_bonds": ("uint32_t r_down = out[2u * (p & 1u) + 1u];",
                                "uint32_t r_down = out[2u * (p & 1u)];"),
}


def _caught_sw(variant_so) -> list:
    caught = []
    with oracle.use_library(variant_so):
        checks = [
            ("threshold", swpins.test_sw_threshold_exact),
            ("bonds", lambda: swpins.test_bonds_between_equal_spins_at_rate_p(exact.T_C)),
            ("lanes", swpins.test_bonds_right_and_down_draws_are_distinct_lanes),
            ("labels", lambda: swpins.test_labels_match_connected_components(16, 0.45)),
            ("chi2_4x4", lambda: swpins.test_sw_4x4_joint_distribution_matches_enumeration(exact.T_C)),
        ]
        for name, fn in checks:
            try:
                fn()
            except AssertionError:
                caught.append(name)
    return caught


@pytest.mark.parametrize("name", sorted(SW_MUTATIONS))
def test_sw_pins_catch_planted_mistake(name, tmp_path):
    old, new = SW_MUTATIONS[name]
    src = oracle.source_text("cluster_oracle.c")
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    so = oracle.compile_variant(src.replace(old, new), str(tmp_path), "sw_" + name, which="cluster_oracle.c")
    assert _caught_sw(so), f"no pin caught the planted mistake {name}"


def test_sw_unmodified_source_passes_same_checks(tmp_path):
    so = oracle.compile_variant(oracle.source_text("cluster_oracle.c"), str(tmp_path), "sw_clean",
                                which="cluster_oracle.c")
    assert _caught_sw(so) == []


# --------------------------------------------------------------------------
# The same for the three-dimensional oracle (ising3d_oracle.c).
# --------------------------------------------------------------------------
import test_ising3d_oracle as pins3d  # noqa: E402

MUTATIONS_3D = {
    "3d_dropped_neighbour": ("sigma[at3(L, x, y, z - 1)] + sigma[at3(L, x, y, z + 1)];",
                             "sigma[at3(L, x, y, z + 1)];"),
    "3d_threshold_index": ("< thr[dE / 4 - 1];", "< thr[dE / 4 - 1 > 0 ? dE / 4 - 2 : 0];"),
    "3d_colour_rule": ("if (((x + y + z) & 1) != c) continue;", "if (((x + y) & 1) != c) continue;"),
    "3d_energy_missing_axis": ("sigma[at3(L, x + 1, y, z)] + sigma[at3(L, x, y + 1, z)] + sigma[at3(L, x, y, z + 1)];",
                               "sigma[at3(L, x + 1, y, z)] + sigma[at3(L, x, y + 1, z)];"),
}


def _caught_3d(variant_so) -> list:
    caught = []
    with oracle.use_library(variant_so):
        checks = [
            ("closed_forms", lambda: pins3d.test_energy3d_closed_forms(4)),
            ("chi2_2x2x2", lambda: pins3d.test_2x2x2_joint_distribution_matches_enumeration(4.5)),
            ("chi2_2x2x2_cold", lambda: pins3d.test_2x2x2_joint_distribution_matches_enumeration(2.0)),
            ("series", pins3d.test_high_temperature_series3d),
            ("t0", pins3d.test_zero_temperature3d),
            ("t0_neel", pins3d.test_zero_temperature_neel_worked_case),
        ]
        for name, fn in checks:
            try:
                fn()
            except AssertionError:
                caught.append(name)
    return caught


@pytest.mark.parametrize("name", sorted(MUTATIONS_3D))
def test_3d_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTATIONS_3D[name]
    src = oracle.source_text("ising3d_oracle.c")
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    so = oracle.compile_variant(src.replace(old, new), str(tmp_path), "o3d_" + name, which="ising3d_oracle.c")
    assert _caught_3d(so), f"no pin caught the planted mistake {name}"


def test_3d_unmodified_source_passes_same_checks(tmp_path):
    so = oracle.compile_variant(oracle.source_text("ising3d_oracle.c"), str(tmp_path), "o3d_clean",
                                which="ising3d_oracle.c")
    assert _caught_3d(so) == []

# --------------------------------------------------------------------------
# The same for the Wolff oracle (wolff_oracle.c).
# --------------------------------------------------------------------------
import test_wolff_oracle as wpins  # noqa: E402

WOLFF_MUTATIONS = {
    "wolff_unequal_spins": ("if (in[j] || sigma[j] != s0) continue;", "if (in[j]) continue;"),
    "wolff_bonds_ignored": ("if (!wolff_bond_active(seed, s, t, thr, owner[k], dir[k])) continue;", ""),
    "wolff_own_draw_for_left_and_up": ("const uint32_t owner[4] = { p, left, p, up };",
                                       "const uint32_t owner[4] = { p, p, p, p };"),
    "wolff_same_lane_both_bonds": ("2u * (p & 1u) + (uint32_t)dir", "2u * (p & 1u)"),
    "wolff_seed_mapping": ("return (uint32_t)((r * (uint64_t)L * (uint64_t)L) >> 32);",
                           "return (uint32_t)(r % ((uint64_t)L * (uint64_t)L));"),
}


def _caught_wolff(variant_so) -> list:
    caught = []
    with oracle.use_library(variant_so):
        checks = [
            ("component", lambda: wpins.test_wolff_step_is_the_seed_component(8, 1.5, 11)),
            ("chi2_4x4", lambda: wpins.test_wolff_4x4_joint_distribution_matches_enumeration(exact.T_C)),
            ("kaufman", lambda: wpins.test_wolff_energy_matches_kaufman(exact.T_C)),
            ("t0", wpins.test_wolff_zero_temperature_flips_the_domain),
            ("t_inf", wpins.test_wolff_infinite_temperature_flips_one_site),
        ]
        for name, fn in checks:
            try:
                fn()
            except AssertionError:
                caught.append(name)
    return caught


@pytest.mark.parametrize("name", sorted(WOLFF_MUTATIONS))
def test_wolff_pins_catch_planted_mistake(name, tmp_path):
    old, new = WOLFF_MUTATIONS[name]
    src = oracle.source_text("wolff_oracle.c")
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    so = oracle.compile_variant(src.replace(old, new), str(tmp_path), "wolff_" + name, which="wolff_oracle.c")
    assert _caught_wolff(so), f"no pin caught the planted mistake {name}"


def test_wolff_unmodified_source_passes_same_checks(tmp_path):
    so = oracle.compile_variant(oracle.source_text("wolff_oracle.c"), str(tmp_path), "wolff_clean",
                                which="wolff_oracle.c")
    assert _caught_wolff(so) == []
