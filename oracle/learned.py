"""Oracle for the learned patch proposal (test infrastructure only).

The paper has no learned component; it motivates one by the critical slowing
down of local updates near T_c (Section 1).  The definitions written out here,
in plain numpy, are the project's:

Window.  A P x P interior patch of the lattice plus its one-site ring: an
S x S window, S = P + 2, positions p = (r, c) in raster order; interior =
1 <= r, c <= P, ring = the rest.

Net (masked-convolution autoregressive model, PixelCNN style, 16 channels):
  features F[p] (16): x_int at the 4 taps strictly before p in raster order
    (dy, dx) in {(-1,-1), (-1,0), (-1,1), (0,-1)} ("mask A"), then x_ring at
    the 9 taps (dy, dx) in {-1,0,1}^2, then 3 zeros; x_int = spin at interior
    positions, 0 elsewhere; x_ring = spin at ring positions, 0 elsewhere;
    positions outside the window read 0.
  layer 1: A1[p] = b1 + F[p] @ W1            (W1: 16 x 16)
  layers 2, 3: A[p] = b + sum_t H[p + tap_t] @ W[t]   over the 5 "mask B"
    taps (dy, dx) in {(-1,-1), (-1,0), (-1,1), (0,-1), (0,0)} (W: 5 x 16 x 16)
  H_l = bf16(relu(A_l)) for l = 1, 2, 3
  layer 4: z[p] = b4 + sum_t H3[p + tap_t] @ W4[t]  (W4: 5 x 16), the logit of
    P(x_p = +1 | x_<p, ring) at interior p.
  Each z[p] depends only on ring values and interior values strictly before p.
  Weights enter as bf16 (rounded from fp32 masters); `exact=True` skips every
  bf16 rounding (pure float64, for finite differences).

log q(x | ring) = sum over interior p of log sigmoid(x_p z_p).
Move (Metropolis-Hastings with an independence proposal given the ring):
  x' ~ q(. | ring) position by position (x'_p = +1 iff u_p < sigmoid(z_p)),
  log alpha = -beta dE + log q(x | ring) - log q(x' | ring), accept iff
  log u < log alpha, dE = E(x') - E(x) over the bonds touching the interior.
"""
from __future__ import annotations

import math

import numpy as np

C = 16
MASK_A = [(-1, -1), (-1, 0), (-1, 1), (0, -1)]
MASK_B = [(-1, -1), (-1, 0), (-1, 1), (0, -1), (0, 0)]
RING9 = [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
N_FEAT = 16
SIZES = {"W1": (N_FEAT, C), "b1": (C,), "W2": (5, C, C), "b2": (C,), "W3": (5, C, C), "b3": (C,),
         "W4": (5, C), "b4": (1,)}
ORDER = ["W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4"]
N_PARAMS = sum(int(np.prod(SIZES[k])) for k in ORDER)   # 2945


# ---------------------------------------------------------------------------
def bf16(a):
    """Round to bfloat16 (via float32, round to nearest even), back to float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def e4m3(a):
    """Round to float8 E4M3 (1-4-3, bias 7, largest finite 448; round to
    nearest even, saturating), back to float64."""
    a = np.asarray(a, dtype=np.float64)
    sgn = np.sign(a)
    x = np.minimum(np.abs(a), 448.0)
    e = np.floor(np.log2(np.maximum(x, 2.0 ** -10)))
    e = np.maximum(e, -6.0)                       # subnormals: step 2^-9
    step = 2.0 ** (e - 3.0)
    q = np.minimum(np.round(x / step) * step, 448.0)   # np.round: half to even
    return sgn * q


LAYER_W = {"W1": 0, "W2": 1, "W3": 2, "W4": 3}


def fp8_scales(flat):
    """Per-layer power-of-two weight scales: 2^floor(log2(448 / max|W|))."""
    P = unpack(flat)
    out = []
    for k in ("W1", "W2", "W3", "W4"):
        mx = float(np.max(np.abs(np.asarray(P[k], np.float32).astype(np.float64))))
        e = math.floor(math.log2(448.0 / mx)) if mx > 0 else 0
        out.append(2.0 ** min(max(e, -60), 60))
    return out


def unpack(flat):
    flat = np.asarray(flat, dtype=np.float64)
    assert flat.size == N_PARAMS
    out, o = {}, 0
    for k in ORDER:
        n = int(np.prod(SIZES[k]))
        out[k] = flat[o:o + n].reshape(SIZES[k])
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[k], dtype=np.float64).ravel() for k in ORDER])


def init_params(seed: int, gain: float = 1.0) -> np.ndarray:
    """Seeded fp32 initial weights (inputs of the method, not its arithmetic)."""
    rng = np.random.default_rng(seed)
    d = {k: np.zeros(SIZES[k]) for k in ORDER}
    d["W1"][:13] = rng.standard_normal((13, C)) * gain / math.sqrt(13)
    d["W2"] = rng.standard_normal((5, C, C)) * gain / math.sqrt(5 * C)
    d["W3"] = rng.standard_normal((5, C, C)) * gain / math.sqrt(5 * C)
    d["W4"] = rng.standard_normal((5, C)) * gain / math.sqrt(5 * C)
    d["b1"] = rng.standard_normal(C) * 0.05
    d["b2"] = rng.standard_normal(C) * 0.05
    d["b3"] = rng.standard_normal(C) * 0.05
    return pack(d).astype(np.float32).astype(np.float64)


def interior_mask(S):
    m = np.zeros((S, S), bool)
    m[1:S - 1, 1:S - 1] = True
    return m


def shift(a, dy, dx):
    """out[..., r, c, ...] = a[..., r+dy, c+dx, ...] (zero outside); a: [B, S, S, ...]."""
    B, S = a.shape[0], a.shape[1]
    out = np.zeros_like(a)
    r0, r1 = max(0, -dy), min(S, S - dy)
    c0, c1 = max(0, -dx), min(S, S - dx)
    out[:, r0:r1, c0:c1] = a[:, r0 + dy:r1 + dy, c0 + dx:c1 + dx]
    return out


def shift_back(a, dy, dx):
    """Adjoint of shift: out[r+dy, c+dx] += a[r, c]."""
    return shift(a, -dy, -dx)


def features(win):
    """win: [B, S, S] of +-1 -> F [B, S, S, 16]."""
    win = np.asarray(win, dtype=np.float64)
    B, S, _ = win.shape
    inner = interior_mask(S)
    x_int = np.where(inner, win, 0.0)
    x_ring = np.where(~inner, win, 0.0)
    F = np.zeros((B, S, S, N_FEAT))
    for k, (dy, dx) in enumerate(MASK_A):
        F[..., k] = shift(x_int, dy, dx)
    for k, (dy, dx) in enumerate(RING9):
        F[..., 4 + k] = shift(x_ring, dy, dx)
    return F


def forward(win, flat, exact=False, prec="bf16"):
    """Teacher-forced pass.  Returns (z [B, S, S], cache).  prec = "bf16"
    (weights and hidden activations rounded to bf16) or "fp8" (weights as
    e4m3(W s_l) / s_l, hidden activations as e4m3)."""
    P = unpack(flat)
    if prec == "fp8" and not exact:
        sc = fp8_scales(flat)
        q = e4m3
        W = {k: (e4m3(np.asarray(v, np.float32).astype(np.float64) * sc[LAYER_W[k]]) / sc[LAYER_W[k]]
                 if k.startswith("W") else v) for k, v in P.items()}
    else:
        q = (lambda a: a) if exact else bf16
        W = {k: q(v) if k.startswith("W") else v for k, v in P.items()}
    F = features(win)
    A1 = F @ W["W1"] + P["b1"]
    H1 = q(np.maximum(A1, 0.0))
    A2 = sum(shift(H1, dy, dx) @ W["W2"][t] for t, (dy, dx) in enumerate(MASK_B)) + P["b2"]
    H2 = q(np.maximum(A2, 0.0))
    A3 = sum(shift(H2, dy, dx) @ W["W3"][t] for t, (dy, dx) in enumerate(MASK_B)) + P["b3"]
    H3 = q(np.maximum(A3, 0.0))
    z = sum(shift(H3, dy, dx) @ W["W4"][t] for t, (dy, dx) in enumerate(MASK_B)) + P["b4"][0]
    if not exact:
        z = z.astype(np.float32).astype(np.float64)
    return z, {"F": F, "H1": H1, "H2": H2, "H3": H3, "W": W}


def log_sigmoid(t):
    t = np.asarray(t, dtype=np.float64)
    return -(np.maximum(-t, 0.0) + np.log1p(np.exp(-np.abs(t))))


def log_q(win, z):
    S = win.shape[1]
    inner = interior_mask(S)
    return (log_sigmoid(np.asarray(win, np.float64) * z) * inner).sum(axis=(1, 2))


def loss(win, flat, exact=False):
    z, _ = forward(win, flat, exact)
    return -log_q(win, z).mean()


def grad(win, flat, exact=False):
    """d loss / d params (mean negative log-likelihood over the batch), float64,
    through the bf16-rounded weights (gradient applied to the fp32 masters)."""
    win = np.asarray(win, dtype=np.float64)
    B, S, _ = win.shape
    z, cache = forward(win, flat, exact)
    W = cache["W"]
    inner = interior_mask(S)
    # d(-log sigmoid(x z))/dz = sigmoid(z) - (x+1)/2
    dz = np.where(inner, 1.0 / (1.0 + np.exp(-z)) - (win + 1.0) / 2.0, 0.0) / B
    g = {k: np.zeros(SIZES[k]) for k in ORDER}
    g["b4"][0] = dz.sum()
    H3 = cache["H3"]
    dH3 = np.zeros_like(H3)
    for t, (dy, dx) in enumerate(MASK_B):
        g["W4"][t] = np.einsum("brc,brci->i", dz, shift(H3, dy, dx))
        dH3 += shift_back(dz[..., None] * W["W4"][t][None, None, None, :], dy, dx)
    dA3 = dH3 * (H3 > 0)
    g["b3"] = dA3.sum(axis=(0, 1, 2))
    H2 = cache["H2"]
    dH2 = np.zeros_like(H2)
    for t, (dy, dx) in enumerate(MASK_B):
        g["W3"][t] = np.einsum("brci,brco->io", shift(H2, dy, dx), dA3)
        dH2 += shift_back(dA3 @ W["W3"][t].T, dy, dx)
    dA2 = dH2 * (H2 > 0)
    g["b2"] = dA2.sum(axis=(0, 1, 2))
    H1 = cache["H1"]
    dH1 = np.zeros_like(H1)
    for t, (dy, dx) in enumerate(MASK_B):
        g["W2"][t] = np.einsum("brci,brco->io", shift(H1, dy, dx), dA2)
        dH1 += shift_back(dA2 @ W["W2"][t].T, dy, dx)
    dA1 = dH1 * (H1 > 0)
    g["b1"] = dA1.sum(axis=(0, 1, 2))
    g["W1"] = np.einsum("brck,brco->ko", cache["F"], dA1)
    return pack(g)


def adam_step(flat, m, v, g, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) of fp32 masters; step counts from 1."""
    flat = np.asarray(flat, dtype=np.float32)
    g = np.asarray(g, dtype=np.float32)
    m = (b1 * m + (1 - b1) * g).astype(np.float32)
    v = (b2 * v + (1 - b2) * g * g).astype(np.float32)
    mhat = m / (1 - b1 ** step)
    vhat = v / (1 - b2 ** step)
    flat = (flat - lr * mhat / (np.sqrt(vhat) + eps)).astype(np.float32)
    return flat, m, v


# ---------------------------------------------------------------------------
# Patches on a periodic lattice
# ---------------------------------------------------------------------------
OFFSETS = [(0, 0), (8, 8), (0, 8), (8, 0)]   # (ox, oy) of round index % 4


def patch_origins(L, round_index, P=8):
    """Top-left interior sites (x0, y0) of the gapped patch checkerboard: one
    patch every 2P sites in each direction, offset (ox, oy) cycling with the
    round index; patch index j = b * (L / 2P) + a."""
    ox, oy = OFFSETS[round_index % 4] if P == 8 else [(0, 0), (P, P), (0, P), (P, 0)][round_index % 4]
    n = L // (2 * P)
    return [((2 * P * a + ox) % L, (2 * P * b + oy) % L) for b in range(n) for a in range(n)]


def extract(sigma, x0, y0, P=8):
    L = sigma.shape[0]
    S = P + 2
    ys = (y0 - 1 + np.arange(S)) % L
    xs = (x0 - 1 + np.arange(S)) % L
    return sigma[np.ix_(ys, xs)].astype(np.int8)


def local_energy(win):
    """Energy of the bonds with at least one interior end (window coordinates)."""
    w = np.asarray(win, dtype=np.int64)
    S = w.shape[-1]
    e = 0
    e -= (w[..., 1:S - 1, 0:S - 1] * w[..., 1:S - 1, 1:S]).sum(axis=(-1, -2))   # horizontal, rows 1..P
    e -= (w[..., 0:S - 1, 1:S - 1] * w[..., 1:S, 1:S - 1]).sum(axis=(-1, -2))   # vertical, cols 1..P
    return e


def log_acceptance(dE, lq_old, lq_new, T):
    """log of the Metropolis-Hastings ratio pi(x') q(x|b) / (pi(x) q(x'|b))."""
    return -float(dE) / T + lq_old - lq_new


def u32_to_unit(r):
    """(r + 0.5) / 2^32 in float64."""
    return (np.asarray(r, dtype=np.float64) + 0.5) / 4294967296.0


def u53(r0, r1):
    """53-bit uniform from two u32 words: ((r0 >> 5) * 2^26 + (r1 >> 6) + 0.5) / 2^53
    in float64 arithmetic, i.e. (k + 1/2) / 2^53 rounded to nearest-even for
    the code k.  It lies in (0, 1]: for k >= 2^52 the half rounds, and the top
    code (probability 2^-53) gives exactly 1.0."""
    return (float((int(r0) >> 5) * 67108864 + (int(r1) >> 6)) + 0.5) / 9007199254740992.0


def sample_threshold(z):
    """floor(2^32 sigmoid(z)) with the sigmoid evaluated in float32 (the
    precision the sampling decision is defined in); 2^32 - 1 if it rounds to 1."""
    z32 = np.asarray(z, dtype=np.float32)
    with np.errstate(over="ignore"):
        s32 = np.float32(1.0) / (np.float32(1.0) + np.exp(-z32))
    t = np.floor(s32.astype(np.float64) * 4294967296.0)
    return np.where(s32 >= np.float32(1.0), 4294967295.0, t)


def sample(win_ring, flat, R, prec="bf16"):
    """Autoregressive sample of the interior given the ring.  win_ring:
    [B, S, S] (interior values ignored), R [B, P*P] raw u32 draws in raster
    order.  x'_p = +1 iff R_p < floor(2^32 sigmoid(z_p)).  Returns (windows,
    log q(x'), per-site thresholds)."""
    w = np.array(win_ring, dtype=np.float64)
    B, S, _ = w.shape
    P = S - 2
    w[:, 1:S - 1, 1:S - 1] = 0.0
    thr = np.zeros((B, P * P))
    for i in range(P * P):
        r, c = 1 + i // P, 1 + i % P
        z, _ = forward(w, flat, prec=prec)
        thr[:, i] = sample_threshold(z[:, r, c])
        w[:, r, c] = np.where(np.asarray(R[:, i], np.float64) < thr[:, i], 1.0, -1.0)
    z, _ = forward(w, flat, prec=prec)
    return w.astype(np.int8), log_q(w, z), thr


def sampling_draws(seed, s, j, round_index, P=8):
    """The raw u32 draws of patch j: lane i % 4 of Philox counter
    (16 j + i/4, round, s, 4), i.e. rank p = 64 j + i."""
    import oracle
    return np.array([oracle.site_random(seed, 64 * j + i, round_index, s, 4) for i in range(P * P)], np.float64)


def train_windows(pool, seed, step, batch, P=8):
    """The windows of training step `step`: window b comes from snapshot
    r0 % n_snap with top-left interior site (x0, y0) = (r1 % L, r2 % L), where
    (r0, r1, r2, r3) = Philox4x32-10 of counter (b, step, 0, 6) keyed by the
    seed (lo32, hi32).  pool: [n_snap, L, L] spins."""
    import oracle
    pool = np.asarray(pool)
    n_snap, L = pool.shape[0], pool.shape[1]
    key = [seed & 0xFFFFFFFF, seed >> 32]
    out = []
    for b in range(batch):
        r = oracle.philox4x32_10([b, step, 0, 6], key)
        out.append(extract(pool[int(r[0]) % n_snap], int(r[1]) % L, int(r[2]) % L, P))
    return np.stack(out)


def learned_round(sigma, flat, T, seed, s, round_index, P=8, prec="bf16"):
    """One MH patch round on lattice sigma (in place).  Uniforms: Philox
    phase 4 (sampling: counter (16 j + i/4, round, s, 4), lane i % 4) and phase
    5 (acceptance: counter (j, round, s, 5), lanes 0, 1).  Returns
    (accepted count, dE total, dM total, per-patch records)."""
    import oracle
    L = sigma.shape[0]
    origins = patch_origins(L, round_index, P)
    wins = np.stack([extract(sigma, x0, y0, P) for (x0, y0) in origins])
    z, _ = forward(wins, flat, prec=prec)
    lq_old = log_q(wins, z)
    R = np.stack([sampling_draws(seed, s, j, round_index, P) for j in range(len(origins))])
    new, lq_new, thr = sample(wins, flat, R, prec=prec)
    dE = local_energy(new) - local_energy(wins)
    acc = 0
    dEt = dMt = 0
    recs = []
    for j, (x0, y0) in enumerate(origins):
        log_alpha = log_acceptance(int(dE[j]), float(lq_old[j]), float(lq_new[j]), T)
        r0 = oracle.site_random(seed, 4 * j + 0, round_index, s, 5)
        r1 = oracle.site_random(seed, 4 * j + 1, round_index, s, 5)
        u = u53(r0, r1)
        ok = math.log(u) < log_alpha
        recs.append({"j": j, "log_alpha": log_alpha, "u": u, "accept": ok, "new": new[j], "old": wins[j],
                     "draws": R[j], "thr": thr[j],
                     "lq_old": float(lq_old[j]), "lq_new": float(lq_new[j]), "dE": int(dE[j])})
        if ok:
            acc += 1
            dEt += int(dE[j])
            dMt += int(new[j][1:P + 1, 1:P + 1].astype(np.int64).sum() - wins[j][1:P + 1, 1:P + 1].astype(np.int64).sum())
            ys = (y0 + np.arange(P)) % L
            xs = (x0 + np.arange(P)) % L
            sigma[np.ix_(ys, xs)] = new[j][1:P + 1, 1:P + 1]
    return acc, dEt, dMt, recs
