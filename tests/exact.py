"""Exact results for the 2D Ising model used to pin the oracle.

Nothing here shares code with the oracle or the CUDA path: these are the
closed forms and brute-force definitions the physics fixes.

* ``enumerate_EM``   -- brute force over all 2^(L*L) states of a small torus.
* ``transfer_matrix_lnZ`` -- row-to-row transfer matrix, Z = Tr T^L.
* ``kaufman_lnZ``    -- Kaufman's (1949) exact partition function of the finite
  m x n torus, the sum of four products over the gamma_l of the transfer
  matrix spectrum.
* ``onsager_u`` / ``onsager_m`` -- Onsager's infinite-lattice energy per spin
  (complete elliptic integral form) and Yang's spontaneous magnetization
  |M| = [1 - sinh^-4(2J/T)]^(1/8) below T_c (Section 3.1, code validation).
"""
from __future__ import annotations

import math

import mpmath as mp
import numpy as np

T_C = 2.0 / math.log(1.0 + math.sqrt(2.0))  # 2.269185...


def enumerate_EM(L: int):
    """All states of the L x L periodic lattice: returns (E, M) int arrays."""
    N = L * L
    idx = np.arange(1 << N, dtype=np.int64)
    bits = ((idx[:, None] >> np.arange(N, dtype=np.int64)) & 1).astype(np.int8)
    s = (1 - 2 * bits).reshape(-1, L, L).astype(np.int16)
    E = -(s * np.roll(s, -1, axis=2)).sum(axis=(1, 2)) - (s * np.roll(s, -1, axis=1)).sum(axis=(1, 2))
    M = s.sum(axis=(1, 2))
    return E.astype(np.int64), M.astype(np.int64)


def boltzmann_weights(E: np.ndarray, T: float) -> np.ndarray:
    w = np.exp(-(E - E.min()) / T)
    return w / w.sum()


def transfer_matrix_lnZ(L: int, K: float) -> float:
    """ln Z of the L x L torus from the 2^L x 2^L row transfer matrix."""
    n = 1 << L
    rows = 1 - 2 * ((np.arange(n)[:, None] >> np.arange(L)) & 1)
    horiz = (rows * np.roll(rows, -1, axis=1)).sum(axis=1)          # bonds within a row
    vert = rows @ rows.T                                               # bonds between rows
    Tm = np.exp(K * (vert + 0.5 * horiz[:, None] + 0.5 * horiz[None, :]))
    ev = np.linalg.eigvalsh(Tm)
    lmax = ev.max()
    return float(L * math.log(lmax) + math.log(np.sum((ev / lmax) ** L)))


def kaufman_lnZ(m: int, n: int, K, dps: int = 50):
    """ln Z for m rows x n columns, periodic, coupling K = J/T (mpmath)."""
    with mp.workdps(dps):
        K = mp.mpf(K)

        def gamma(l):
            if l == 0:
                return 2 * K + mp.log(mp.tanh(K))
            return mp.acosh(mp.cosh(2 * K) * mp.coth(2 * K) - mp.cos(mp.pi * l / n))

        g_odd = [gamma(2 * r + 1) for r in range(n)]
        g_even = [gamma(2 * r) for r in range(n)]
        z1 = mp.fprod([2 * mp.cosh(m * g / 2) for g in g_odd])
        z2 = mp.fprod([2 * mp.sinh(m * g / 2) for g in g_odd])
        z3 = mp.fprod([2 * mp.cosh(m * g / 2) for g in g_even])
        z4 = mp.fprod([2 * mp.sinh(m * g / 2) for g in g_even])
        pref = mp.mpf(m * n) / 2 * mp.log(2 * mp.sinh(2 * K)) - mp.log(2)
        return pref + mp.log(z1 + z2 + z3 + z4)


def kaufman_mean_energy(L: int, T: float) -> float:
    """<E> = -d ln Z / d beta (J = 1) on the L x L torus, by a high-precision
    central difference of Kaufman's ln Z."""
    with mp.workdps(60):
        K = 1 / mp.mpf(T)
        h = mp.mpf(10) ** -20
        d = (kaufman_lnZ(L, L, K + h, dps=60) - kaufman_lnZ(L, L, K - h, dps=60)) / (2 * h)
        return float(-d)


def kaufman_energy_variance(L: int, T: float) -> float:
    """Var(E) = d^2 ln Z / d beta^2 on the L x L torus."""
    with mp.workdps(80):
        K = 1 / mp.mpf(T)
        h = mp.mpf(10) ** -15
        f0 = kaufman_lnZ(L, L, K, dps=80)
        fp = kaufman_lnZ(L, L, K + h, dps=80)
        fm = kaufman_lnZ(L, L, K - h, dps=80)
        return float((fp - 2 * f0 + fm) / (h * h))


def onsager_u(T: float) -> float:
    """Energy per spin of the infinite lattice (J = 1)."""
    from scipy.special import ellipk
    b = 1.0 / T
    k = 2.0 * math.sinh(2 * b) / math.cosh(2 * b) ** 2
    c = 2.0 * math.tanh(2 * b) ** 2 - 1.0
    if abs(c) < 1e-15:   # at T_c the product c * K1 -> 0 (K1 diverges only logarithmically)
        return -(1.0 / math.tanh(2 * b))
    K1 = ellipk(k * k)  # scipy takes the parameter m = k^2
    return -(1.0 / math.tanh(2 * b)) * (1.0 + (2.0 / math.pi) * (2.0 * math.tanh(2 * b) ** 2 - 1.0) * K1)


def onsager_m(T: float) -> float:
    """Spontaneous magnetization per spin; 0 at and above T_c."""
    if T >= T_C:
        return 0.0
    return (1.0 - math.sinh(2.0 / T) ** -4) ** 0.125
