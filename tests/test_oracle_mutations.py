"""Plant plausible mistakes in a copy of the oracle source (on the CPU) and
check that at least one pin catches each: a dropped or wrong neighbour,
swapped, ceiled or mis-scaled thresholds, the colour order or colour rule,
zero-energy moves rejected, the sign of dE, Philox's multiplier, key
schedule, rounds and word order, the output lane, the energy's sign or a
dropped bond, the sense of the initial-state bit."""
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
    "energy_down_bond_dropped": ("e -= (int64_t)(s * (r + d));", "e -= (int64_t)(s * r);"),
    "philox_key_bumped_before_first_round": ("        if (round > 0) {\n            k0 += ORC_PHILOX_WEYL_A;",
                                             "        if (round >= 0) {\n            k0 += ORC_PHILOX_WEYL_A;"),
    "philox_low_words_swapped": ("uint32_t n1 = (uint32_t)prod_b;", "uint32_t n1 = (uint32_t)prod_a;"),
    "philox_seven_rounds": ("for (int round = 0; round < 10; ++round)", "for (int round = 0; round < 7; ++round)"),
    "output_lane_from_wrong_bits": ("return out[p & 3u];", "return out[(p >> 1) & 3u];"),
    "threshold_ceil": ("(uint32_t)floor(v);", "(uint32_t)ceil(v);"),
    "threshold_energy_scale": ("double dE = 4.0 * (double)(k + 1);", "double dE = 2.0 * (double)(k + 1);"),
    "up_neighbour_is_the_site": ("int h = sigma[(size_t)wrap(y - 1, L) * L + x]", "int h = sigma[(size_t)wrap(y, L) * L + x]"),
    "column_colouring": ("if (((x + y) & 1) == c) update_site", "if ((x & 1) == c) update_site"),
    "dE_sign": ("int dE = 2 * sigma[i] * h;", "int dE = -2 * sigma[i] * h;"),
    "initial_bit_sense": ("                v = (oracle_site_random(seed, p, 0u, s, 2u) >> 31) ? (int8_t)-1 : (int8_t)1;\n"
                          "            }\n            sigma[(size_t)y * L + x] = v;",
                          "                v = (oracle_site_random(seed, p, 0u, s, 2u) >> 31) ? (int8_t)1 : (int8_t)-1;\n"
                          "            }\n            sigma[(size_t)y * L + x] = v;"),
}


def _caught(variant_so) -> list:
    caught = []
    with oracle.use_library(variant_so):
        checks = [
            ("kat", lambda: [pins.test_philox_known_answers(c, k, e) for c, k, e in pins._kat_rows()]),
            ("keying", lambda: pins.test_site_random_keying()),
            ("thresholds", lambda: (pins.test_thresholds_exact(), pins.test_thresholds_limits_and_errors())),
            ("init", lambda: pins.test_init_cold_and_random()),
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
    "sw_threshold_ceil": ("*thr = (v >= 4294967296.0) ? 0xFFFFFFFFu : (uint32_t)floor(v);",
                          "*thr = (v >= 4294967296.0) ? 0xFFFFFFFFu : (uint32_t)ceil(v);"),
    "sw_right_neighbour_not_wrapped": ("int8_t right = sigma[(size_t)y * L + (x + 1) % L];",
                                       "int8_t right = sigma[(size_t)y * L + (x + 1 < L ? x + 1 : x)];"),
    "sw_up_neighbour_missed": ("if (bonds[up] & 2u) nb[k++] = up;", ""),
    "sw_label_is_the_discoverer": ("label[nb[i]] = (uint32_t)start;", "label[nb[i]] = u;"),
    "sw_every_cluster_flipped": ("if (coin) sigma[p] = (int8_t)(-sigma[p]);", "sigma[p] = (int8_t)(-sigma[p]); (void)coin;"),
    "sw_coin_from_the_bond_phase": ("#define ORC_SW_PHASE_COIN 8u", "#define ORC_SW_PHASE_COIN 7u"),
    "sw_coin_low_bit": ("uint32_t coin = oracle_site_random(seed, root, t, s, ORC_SW_PHASE_COIN) >> 31;",
                        "uint32_t coin = oracle_site_random(seed, root, t, s, ORC_SW_PHASE_COIN) & 1u;"),
}


def _caught_sw(variant_so) -> list:
    caught = []
    with oracle.use_library(variant_so):
        checks = [
            ("threshold", swpins.test_sw_threshold_exact),
            ("root_coin", lambda: swpins.test_sw_step_flips_each_cluster_by_its_root_coin(16, exact.T_C)),
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
    "3d_threshold_ceil": ("thr[k] = (v >= 4294967296.0) ? 0xFFFFFFFFu : (uint32_t)floor(v);",
                          "thr[k] = (v >= 4294967296.0) ? 0xFFFFFFFFu : (uint32_t)ceil(v);"),
    "3d_threshold_scale": ("double v = ldexp(exp(-4.0 * (double)(k + 1) / T), 32);",
                           "double v = ldexp(exp(-2.0 * (double)(k + 1) / T), 32);"),
    "3d_dE_sign": ("int dE = 2 * sigma[i] * h;", "int dE = -2 * sigma[i] * h;"),
    "3d_white_first": ("        half_sweep3(L, sigma, 0, thr, seed, s, t);\n        half_sweep3(L, sigma, 1, thr, seed, s, t);",
                       "        half_sweep3(L, sigma, 1, thr, seed, s, t);\n        half_sweep3(L, sigma, 0, thr, seed, s, t);"),
    "3d_y_neighbour_twice": ("sigma[at3(L, x, y - 1, z)] +\n                        sigma[at3(L, x, y + 1, z)]",
                             "sigma[at3(L, x, y + 1, z)] +\n                        sigma[at3(L, x, y + 1, z)]"),
}


def _caught_3d(variant_so) -> list:
    caught = []
    with oracle.use_library(variant_so):
        checks = [
            ("thresholds", pins3d.test_thresholds3d_exact),
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
    "wolff_only_the_seed_flipped": ("for (size_t i = 0; i < tail; ++i) sigma[queue[i]] = (int8_t)(-s0);",
                                    "sigma[queue[0]] = (int8_t)(-s0);"),
    "wolff_seed_from_another_lane": ("uint64_t r = wolff_draw(seed, 0u, t, s, ORC_WOLFF_PHASE_SEED, 0u);",
                                     "uint64_t r = wolff_draw(seed, 0u, t, s, ORC_WOLFF_PHASE_SEED, 1u);"),
    "wolff_bond_directions_swapped": ("const int dir[4] = { 0, 0, 1, 1 };", "const int dir[4] = { 1, 1, 0, 0 };"),
    "wolff_down_neighbour_misplaced": ("const uint32_t down = (uint32_t)((y + 1) % L) * L + (uint32_t)x;",
                                       "const uint32_t down = (uint32_t)((y + 1) % L) * L + (uint32_t)((x + 1) % L);"),
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
