"""Pins for the learned-proposal oracle: finite-difference gradients, the
autoregressive mask property, normalisation of q, the local energy against
the full Hamiltonian, exact detailed balance of the MH patch move on a 4x4
torus (all 2^16 states), bf16 rounding against torch, and one Adam step."""
from __future__ import annotations

import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import learned as ol


def rand_windows(B, S, seed):
    rng = np.random.default_rng(seed)
    return np.where(rng.random((B, S, S)) < 0.5, -1, 1).astype(np.int8)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(10000) * 10 ** rng.uniform(-5, 5, 10000),
                        [1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 0.0, 65504.0]]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(ol.bf16(x), ref)


def test_gradient_matches_finite_differences():
    win = rand_windows(6, 10, 1)
    flat = ol.init_params(3, gain=1.5)
    g = ol.grad(win, flat, exact=True)
    rng = np.random.default_rng(2)
    idx = list(rng.integers(0, ol.N_PARAMS, size=40)) + [0, 16 * 16 - 1, ol.N_PARAMS - 1]
    h = 1e-6
    for i in idx:
        e = np.zeros(ol.N_PARAMS)
        e[i] = h
        fd = (ol.loss(win, flat + e, exact=True) - ol.loss(win, flat - e, exact=True)) / (2 * h)
        assert abs(fd - g[i]) < 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])
    d = rng.standard_normal(ol.N_PARAMS)
    fd = (ol.loss(win, flat + 1e-6 * d, exact=True) - ol.loss(win, flat - 1e-6 * d, exact=True)) / 2e-6
    assert abs(fd - g @ d) < 1e-5 * max(1.0, abs(fd))


def test_autoregressive_mask():
    # z at interior position p depends only on ring values and earlier interior values
    win = rand_windows(4, 10, 5)
    flat = ol.init_params(7, gain=2.0)
    z0, _ = ol.forward(win, flat, exact=True)
    for (r, c) in [(1, 1), (3, 5), (8, 8), (5, 1)]:
        w2 = win.copy()
        w2[:, r, c] *= -1
        z1, _ = ol.forward(w2, flat, exact=True)
        order = np.arange(100).reshape(10, 10)
        before = order <= order[r, c]
        assert np.array_equal(z0[:, before], z1[:, before])
        assert not np.allclose(z0[:, ~before], z1[:, ~before])


def test_q_is_normalised():
    # S = 4 (2x2 interior): sum over the 16 interiors of q(x | ring) = 1
    flat = ol.init_params(11, gain=2.0)
    ring = rand_windows(5, 4, 9)
    for b in range(5):
        total = 0.0
        for bits in itertools.product([-1, 1], repeat=4):
            w = ring[b:b + 1].copy()
            w[0, 1:3, 1:3] = np.array(bits).reshape(2, 2)
            z, _ = ol.forward(w, flat)
            total += math.exp(ol.log_q(w, z)[0])
        assert abs(total - 1.0) < 1e-12


def test_local_energy_matches_full_hamiltonian():
    rng = np.random.default_rng(4)
    L = 32
    for trial in range(20):
        s = np.where(rng.random((L, L)) < 0.5, -1, 1).astype(np.int8)
        x0, y0 = int(rng.integers(0, L)), int(rng.integers(0, L))
        w_old = ol.extract(s, x0, y0)
        new = s.copy()
        ys, xs = (y0 + np.arange(8)) % L, (x0 + np.arange(8)) % L
        new[np.ix_(ys, xs)] = np.where(rng.random((8, 8)) < 0.5, -1, 1)
        w_new = ol.extract(new, x0, y0)
        assert ol.local_energy(w_new) - ol.local_energy(w_old) == oracle.energy(new) - oracle.energy(s)


def test_patch_origins_tile_the_lattice_and_rings_avoid_interiors():
    L = 64
    cover = np.zeros((L, L), int)
    for r in range(4):
        inter = np.zeros((L, L), int)
        ring = np.zeros((L, L), int)
        for (x0, y0) in ol.patch_origins(L, r):
            ys, xs = (y0 + np.arange(8)) % L, (x0 + np.arange(8)) % L
            inter[np.ix_(ys, xs)] += 1
            ys2, xs2 = (y0 - 1 + np.arange(10)) % L, (x0 - 1 + np.arange(10)) % L
            ring[np.ix_(ys2, xs2)] += 1
        ring -= inter
        assert inter.max() == 1
        assert (ring[inter > 0] == 0).all()          # no ring site is another patch's interior
        cover += inter
    assert (cover == 1).all()                          # four rounds cover every site once


def test_detailed_balance_exact_on_4x4_torus():
    """One patch move (2x2 interior, its ring = the rest of a 4x4 torus):
    pi(s) P(s -> s') = pi(s') P(s' -> s) for every pair, all 2^16 states."""
    T = 2.3
    flat = ol.init_params(21, gain=2.5)
    rings = np.array(list(itertools.product([-1, 1], repeat=12)), dtype=np.int8)   # 4096 rings
    inter = np.array(list(itertools.product([-1, 1], repeat=4)), dtype=np.int8)    # 16 interiors
    ring_pos = [(r, c) for r in range(4) for c in range(4) if not (1 <= r <= 2 and 1 <= c <= 2)]
    W = np.zeros((4096, 16, 4, 4), np.int8)
    for k, (r, c) in enumerate(ring_pos):
        W[:, :, r, c] = rings[:, k][:, None]
    W[:, :, 1:3, 1:3] = inter.reshape(16, 2, 2)[None]
    flatW = W.reshape(-1, 4, 4)
    z, _ = ol.forward(flatW, flat)
    lq = ol.log_q(flatW, z).reshape(4096, 16)
    E = ol.local_energy(flatW).reshape(4096, 16)
    # full energy = local + ring-ring bonds (same for all interiors of a ring): pi ~ exp(-E_local/T) per ring
    for b in range(0, 4096, 37):
        for i in range(16):
            for j in range(16):
                if i == j:
                    continue
                la_ij = ol.log_acceptance(int(E[b, j] - E[b, i]), lq[b, i], lq[b, j], T)
                la_ji = ol.log_acceptance(int(E[b, i] - E[b, j]), lq[b, j], lq[b, i], T)
                flow_ij = -E[b, i] / T + lq[b, j] + min(0.0, la_ij)
                flow_ji = -E[b, j] / T + lq[b, i] + min(0.0, la_ji)
                assert abs(flow_ij - flow_ji) < 1e-9


def test_adam_first_step_is_signed_lr():
    g = np.array([0.5, -2.0, 1e-3, 0.0], np.float32)
    p, m, v = ol.adam_step(np.zeros(4, np.float32), np.zeros(4, np.float32), np.zeros(4, np.float32), g, 1, 0.01)
    assert np.allclose(p[:3], -0.01 * np.sign(g[:3]), rtol=1e-4) and p[3] == 0.0


def test_adam_closed_forms_fix_betas_and_epsilon():
    """Adam's later steps and its epsilon, against values worked out by hand
    from the definition (Kingma & Ba 2015, bias-corrected moments; beta1 =
    0.9, beta2 = 0.999, eps = 1e-8 outside the square root):
    * gradient 1 then 0: after step 2, m = 0.09 and v = 0.000999, so the
      second update is lr (0.09/0.19) / sqrt(0.000999/0.001999) = lr (9/19) /
      sqrt(999/1999) = 0.670058... lr (a beta2 of 0.99 would give 0.6716 lr,
      a beta1 of 0.8 0.6287 lr);
    * gradient 1, 0, 0: the third update is lr (0.081/0.271) /
      sqrt(0.000998001/0.002997001) = 0.517957... lr;
    * a first gradient of 1e-8: the update is lr 1e-8 / (1e-8 + 1e-8) =
      lr / 2 (epsilon inside the root would give about lr 1e-4)."""
    lr = 0.01
    z = np.zeros(3, np.float32)
    g1 = np.array([1.0, -1.0, 1e-8], np.float32)
    p1, m, v = ol.adam_step(z, z, z, g1, 1, lr)
    assert np.allclose(p1[:2], [-lr, lr], rtol=1e-6)
    assert abs(p1[2] + lr / 2) < 1e-6 * lr
    g0 = np.zeros(3, np.float32)
    p2, m, v = ol.adam_step(p1, m, v, g0, 2, lr)
    second = (9.0 / 19.0) / math.sqrt(999.0 / 1999.0)
    assert abs((p1[0] - p2[0]) / lr - second) < 1e-5 and abs((p2[1] - p1[1]) / lr - second) < 1e-5
    assert abs(second - 0.670058) < 1e-6
    p3, m, v = ol.adam_step(p2, m, v, g0, 3, lr)
    third = (0.081 / 0.271) / math.sqrt(0.000998001 / 0.002997001)
    assert abs((p2[0] - p3[0]) / lr - third) < 1e-5
    assert abs(third - 0.517957) < 1e-6


def test_learned_round_runs_and_keeps_energy_bookkeeping():
    L, T, seed = 32, 2.3, 3
    s = oracle.init(L, seed, 0)
    e0, m0 = oracle.energy(s), oracle.magnetization(s)
    flat = ol.init_params(1, gain=0.5)
    acc, dE, dM, recs = ol.learned_round(s, flat, T, seed, 0, 0)
    assert len(recs) == (L // 16) ** 2
    assert oracle.energy(s) - e0 == dE and oracle.magnetization(s) - m0 == dM
    assert acc == sum(r["accept"] for r in recs)


def test_e4m3_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("torch without float8_e4m3fn")
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.standard_normal(20000) * 10 ** rng.uniform(-4, 2.4, 20000),
                        [0.0, 448.0, -448.0, 2 ** -9, 3 * 2 ** -10, 1.0625, 1.1875, 240.0, 0.015625]])
    x = x[np.abs(x) <= 448].astype(np.float32)
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(ol.e4m3(x.astype(np.float64)), ref)
    assert ol.e4m3(np.array([1000.0, -1e6]))[0] == 448.0          # saturating


def test_fp8_forward_is_close_to_bf16_and_keeps_the_mask():
    win = rand_windows(8, 10, 3)
    flat = ol.init_params(5, gain=1.0)
    z8, _ = ol.forward(win, flat, prec="fp8")
    z16, _ = ol.forward(win, flat)
    inner = ol.interior_mask(10)
    assert np.median(np.abs(z8 - z16)[:, inner]) < 0.1
    w2 = win.copy()
    w2[:, 4, 4] *= -1
    z8b, _ = ol.forward(w2, flat, prec="fp8")
    order = np.arange(100).reshape(10, 10)
    before = order <= order[4, 4]
    assert np.array_equal(z8[:, before], z8b[:, before])


def _forced_draws(target, P):
    """u32 draws that make a sampler obeying x_p = +1 iff R_p < thr_p
    produce `target`'s interior (0 is below every positive threshold,
    2^32 - 1 below none)."""
    x = np.asarray(target, np.int64)[:, 1:P + 1, 1:P + 1].reshape(len(target), P * P)
    return np.where(x > 0, 0.0, 4294967295.0)


@pytest.mark.parametrize("S,gain", [(4, 2.0), (10, 0.7)])
def test_sampler_path_probability_is_q(S, gain):
    # the probability with which the sampler produces x, the product of its
    # per-site thresholds / 2^32 along x's path, equals q(x | ring) up to the
    # 2^-32 quantization and the float32 sigmoid
    P = S - 2
    flat = ol.init_params(31, gain=gain)
    target = rand_windows(64, S, 17)
    got, lq, thr = ol.sample(target, flat, _forced_draws(target, P))
    assert np.array_equal(got, target)
    x = target[:, 1:P + 1, 1:P + 1].reshape(64, P * P)
    p_plus = thr / 4294967296.0
    log_path = np.where(x > 0, np.log(p_plus), np.log1p(-p_plus)).sum(axis=1)
    z, _ = ol.forward(target, flat)
    assert np.allclose(lq, ol.log_q(target, z), atol=0, rtol=0)
    assert np.max(np.abs(log_path - lq)) < 2e-5 * P * P


def test_sampler_distribution_matches_q():
    # independent uniform u32 draws: chi^2 of the 16 interiors of a 2x2 patch
    # against q(. | ring), two rings sampled in one batch
    from scipy import stats
    flat = ol.init_params(41, gain=2.0)
    rng = np.random.default_rng(43)
    n, rings = 6000, rand_windows(2, 4, 47)
    R = rng.integers(0, 2**32, size=(2 * n, 4)).astype(np.float64)
    got, _, _ = ol.sample(np.repeat(rings, n, axis=0), flat, R)
    codes = ((got[:, 1:3, 1:3].reshape(2 * n, 4) > 0) * (1 << np.arange(4))).sum(axis=1)
    all16 = np.where((np.arange(16)[:, None] >> np.arange(4)) & 1, 1, -1).reshape(16, 2, 2)
    for b in range(2):
        counts = np.bincount(codes[b * n:(b + 1) * n], minlength=16)
        w = np.repeat(rings[b][None], 16, axis=0)
        w[:, 1:3, 1:3] = all16
        z, _ = ol.forward(w, flat)
        expct = np.exp(ol.log_q(w, z)) * n
        o, e, acc_o, acc_e = [], [], 0.0, 0.0         # rarest first, pooled to >= 10 expected
        for i in np.argsort(expct):
            acc_o += counts[i]
            acc_e += expct[i]
            if acc_e >= 10:
                o.append(acc_o)
                e.append(acc_e)
                acc_o = acc_e = 0.0
        o[-1] += acc_o
        e[-1] += acc_e
        o, e = np.array(o), np.array(e)
        chi2 = ((o - e) ** 2 / e).sum()
        assert len(o) >= 4 and stats.chi2.sf(chi2, len(o) - 1) > 1e-4, (b, chi2, len(o))


def test_u53_is_the_rounded_half_code_and_uniform():
    # u53 = (k + 1/2) / 2^53, k = (r0 >> 5) 2^26 + (r1 >> 6), correctly rounded
    # to float64 (exact rational arithmetic here); so u is in (0, 1] and only
    # the top code reaches 1.0
    from fractions import Fraction
    from scipy import stats
    rng = np.random.default_rng(5)
    words = [(0, 0), (0, 63), (0, 64), (31, 2**32 - 1), (32, 0), (2**31, 0), (2**32 - 1, 2**32 - 65),
             (2**32 - 1, 2**32 - 1)] + [tuple(int(v) for v in w) for w in rng.integers(0, 2**32, size=(2000, 2))]
    for r0, r1 in words:
        k = (r0 >> 5) * 2**26 + (r1 >> 6)
        assert ol.u53(r0, r1) == float(Fraction(2 * k + 1, 2**54)), (r0, r1)
    assert ol.u53(0, 0) == 2.0**-54 and ol.u53(0, 64) - ol.u53(0, 0) == 2.0**-53
    assert ol.u53(2**32 - 1, 2**32 - 65) < 1.0 == ol.u53(2**32 - 1, 2**32 - 1)
    u = [ol.u53(int(a), int(b)) for a, b in rng.integers(0, 2**32, size=(20000, 2))]
    assert stats.kstest(u, "uniform").pvalue > 1e-3


def test_learned_round_limits_with_a_uniform_proposal():
    # all-zero parameters: z = 0, q uniform, so log alpha = -dE / T.  As
    # T -> inf every proposal is accepted; as T -> 0 exactly those that do not
    # raise the energy (Metropolis-Hastings in both limits)
    L, seed = 32, 9
    flat = np.zeros(ol.N_PARAMS)
    for T, rnd in ((1e9, 0), (1e9, 1), (0.05, 2), (0.05, 3)):
        s = oracle.init(L, seed, 0)
        acc, _, _, recs = ol.learned_round(s, flat, T, seed, 0, rnd)
        assert all(abs(r["lq_old"] - r["lq_new"]) < 1e-12 for r in recs)
        for r in recs:
            assert r["accept"] == (r["dE"] <= 0 if T < 1 else True), (T, r["dE"], r["log_alpha"])
        assert acc == sum(r["accept"] for r in recs)
        if T > 1:
            assert acc == len(recs)
        else:
            assert any(r["dE"] > 0 for r in recs) and any(r["dE"] < 0 for r in recs)


def test_training_windows_follow_their_draws():
    # snapshots that differ everywhere tell which one a window came from; the
    # ring and interior of each window are the periodic neighbourhood of its origin
    L, n_snap, seed = 32, 5, 0x1234_5678_9ABC
    rng = np.random.default_rng(2)
    pool = np.where(rng.random((n_snap, L, L)) < 0.5, -1, 1).astype(np.int8)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for step in (0, 7):
        wins = ol.train_windows(pool, seed, step, 64)
        for b in range(64):
            r = oracle.philox4x32_10([b, step, 0, 6], key)
            snap, x0, y0 = int(r[0]) % n_snap, int(r[1]) % L, int(r[2]) % L
            ys, xs = (y0 - 1 + np.arange(10)) % L, (x0 - 1 + np.arange(10)) % L
            assert np.array_equal(wins[b], pool[snap][np.ix_(ys, xs)])
    # over many draws every snapshot and origin row is used about equally often
    from scipy import stats
    snaps = [int(oracle.philox4x32_10([b, 3, 0, 6], key)[0]) % n_snap for b in range(5000)]
    counts = np.bincount(snaps, minlength=n_snap)
    assert stats.chisquare(counts).pvalue > 1e-3
