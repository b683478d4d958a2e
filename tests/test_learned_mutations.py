"""Plant plausible mistakes in a copy of the learned-proposal oracle's source
(oracle/learned.py, on the CPU) and check that at least one pin of
test_learned_oracle.py catches each: the sampler's comparison or sigmoid, the
sign in log q, the Metropolis-Hastings ratio, the local energy, the two
autoregressive masks, the backward pass, Adam's bias correction, the patch
offsets, the round's acceptance test, the 53-bit uniform and the bf16 / e4m3
rounding."""
from __future__ import annotations

import inspect
import types

import pytest

from oracle import learned as ol
import test_learned_oracle as pins

MUTATIONS = {
    "sampler_comparison_reversed": ("np.where(np.asarray(R[:, i], np.float64) < thr[:, i], 1.0, -1.0)",
                                    "np.where(np.asarray(R[:, i], np.float64) >= thr[:, i], 1.0, -1.0)"),
    "threshold_of_minus_z": ("(np.float32(1.0) + np.exp(-z32))", "(np.float32(1.0) + np.exp(z32))"),
    "log_q_sign": ("log_sigmoid(np.asarray(win, np.float64) * z)", "log_sigmoid(-np.asarray(win, np.float64) * z)"),
    "mh_proposal_terms_swapped": ("return -float(dE) / T + lq_old - lq_new", "return -float(dE) / T + lq_new - lq_old"),
    "mh_energy_sign": ("return -float(dE) / T + lq_old - lq_new", "return float(dE) / T + lq_old - lq_new"),
    "local_energy_vertical_dropped": ("    e -= (w[..., 0:S - 1, 1:S - 1] * w[..., 1:S, 1:S - 1]).sum(axis=(-1, -2))", "    pass"),
    "local_energy_last_row_dropped": ("w[..., 1:S - 1, 0:S - 1] * w[..., 1:S - 1, 1:S]", "w[..., 1:S - 2, 0:S - 1] * w[..., 1:S - 2, 1:S]"),
    "mask_a_sees_the_site": ("MASK_A = [(-1, -1), (-1, 0), (-1, 1), (0, -1)]", "MASK_A = [(-1, -1), (-1, 0), (-1, 1), (0, 0)]"),
    "mask_b_looks_ahead": ("MASK_B = [(-1, -1), (-1, 0), (-1, 1), (0, -1), (0, 0)]",
                           "MASK_B = [(-1, -1), (-1, 0), (-1, 1), (0, -1), (0, 1)]"),
    "relu_gate_dropped_in_backward": ("dA2 = dH2 * (H2 > 0)", "dA2 = dH2"),
    "backward_tap_not_adjoint": ('dH1 += shift_back(dA2 @ W["W2"][t].T, dy, dx)', 'dH1 += shift(dA2 @ W["W2"][t].T, dy, dx)'),
    "weight_not_transposed_in_backward": ('dH2 += shift_back(dA3 @ W["W3"][t].T, dy, dx)',
                                          'dH2 += shift_back(dA3 @ W["W3"][t], dy, dx)'),
    "adam_without_bias_correction": ("mhat = m / (1 - b1 ** step)", "mhat = m"),
    "adam_beta2_wrong": ("def adam_step(flat, m, v, g, step, lr, b1=0.9, b2=0.999, eps=1e-8):",
                         "def adam_step(flat, m, v, g, step, lr, b1=0.9, b2=0.99, eps=1e-8):"),
    "adam_beta1_wrong": ("def adam_step(flat, m, v, g, step, lr, b1=0.9, b2=0.999, eps=1e-8):",
                         "def adam_step(flat, m, v, g, step, lr, b1=0.8, b2=0.999, eps=1e-8):"),
    "adam_eps_inside_root": ("flat = (flat - lr * mhat / (np.sqrt(vhat) + eps)).astype(np.float32)",
                             "flat = (flat - lr * mhat / np.sqrt(vhat + eps)).astype(np.float32)"),
    "adam_second_moment_unsquared": ("v = (b2 * v + (1 - b2) * g * g).astype(np.float32)",
                                     "v = (b2 * v + (1 - b2) * np.abs(g)).astype(np.float32)"),
    "patch_offsets": ("OFFSETS = [(0, 0), (8, 8), (0, 8), (8, 0)]", "OFFSETS = [(0, 0), (8, 8), (0, 8), (0, 8)]"),
    "round_dm_sign": ("dMt += int(new[j][1:P + 1, 1:P + 1].astype(np.int64).sum() - wins[j]",
                      "dMt -= int(new[j][1:P + 1, 1:P + 1].astype(np.int64).sum() - wins[j]"),
    "u53_high_word_scale": ("(int(r0) >> 5) * 67108864", "(int(r0) >> 5) * 134217728"),
    "round_acceptance_reversed": ("ok = math.log(u) < log_alpha", "ok = math.log(u) > log_alpha"),
    "round_uniform_ignored": ("ok = math.log(u) < log_alpha", "ok = 0.0 < log_alpha"),
    "bf16_truncates": ("((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000)", "(u & 0xFFFF0000)"),
    "e4m3_three_exponent_bits": ("e = np.maximum(e, -6.0)", "e = np.maximum(e, -2.0)"),
}

# cheap pins first; a mutation counts as caught at the first pin that fails
CHECKS = [
    ("ar_mask", lambda: pins.test_autoregressive_mask()),
    ("q_normalised", lambda: pins.test_q_is_normalised()),
    ("local_energy", lambda: pins.test_local_energy_matches_full_hamiltonian()),
    ("patch_tiling", lambda: pins.test_patch_origins_tile_the_lattice_and_rings_avoid_interiors()),
    ("adam", lambda: pins.test_adam_first_step_is_signed_lr()),
    ("adam_closed_forms", lambda: pins.test_adam_closed_forms_fix_betas_and_epsilon()),
    ("gradient_fd", lambda: pins.test_gradient_matches_finite_differences()),
    ("sampler_path_4", lambda: pins.test_sampler_path_probability_is_q(4, 2.0)),
    ("sampler_path_10", lambda: pins.test_sampler_path_probability_is_q(10, 0.7)),
    ("round_bookkeeping", lambda: pins.test_learned_round_runs_and_keeps_energy_bookkeeping()),
    ("round_limits", lambda: pins.test_learned_round_limits_with_a_uniform_proposal()),
    ("u53", lambda: pins.test_u53_is_the_rounded_half_code_and_uniform()),
    ("e4m3", lambda: pins.test_e4m3_rounding_matches_torch()),
    ("bf16", lambda: pins.test_bf16_rounding_matches_torch()),
    ("fp8_mask", lambda: pins.test_fp8_forward_is_close_to_bf16_and_keeps_the_mask()),
    ("detailed_balance", lambda: pins.test_detailed_balance_exact_on_4x4_torus()),
    ("sampler_chi2", lambda: pins.test_sampler_distribution_matches_q()),
]


def _module_from(src: str):
    mod = types.ModuleType("learned_variant")
    mod.__file__ = ol.__file__
    exec(compile(src, "learned_variant", "exec"), mod.__dict__)
    return mod


def _first_catch(mod, monkeypatch, stop_early=True):
    monkeypatch.setattr(pins, "ol", mod)
    caught = []
    for name, fn in CHECKS:
        try:
            fn()
        except pytest.skip.Exception:
            continue
        except Exception as e:              # AssertionError, or a crash the mistake causes
            caught.append((name, type(e).__name__))
            if stop_early:
                break
    return caught


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, monkeypatch):
    old, new = MUTATIONS[name]
    src = inspect.getsource(ol)
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    caught = _first_catch(_module_from(src.replace(old, new)), monkeypatch)
    assert caught, f"no pin caught the planted mistake {name}"


def test_unmodified_source_passes_same_checks(monkeypatch):
    assert _first_catch(_module_from(inspect.getsource(ol)), monkeypatch, stop_early=False) == []
