"""Seeded synthetic workloads (lattice sizes, temperatures, seeds, starts).

This module holds no arithmetic of the method: it only fixes the inputs that
both the CUDA path and the CPU oracle are run on.  The paper's own workloads
are synthetic lattices (Section 3.1: random starts at L = 1024..4096 over a
temperature scan; Table 1: many simulations of one size at once), so every
input here is generated, never read from a dataset.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np

T_CRITICAL = 2.269185  # critical temperature as printed in Section 3.1 (J = 1)

MASK64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """SplitMix64 output for state x (Steele, Lea, Flood, OOPSLA 2014): the
    per-lattice seed derivation of the batched workload."""
    z = (x + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


@dataclass
class Workload:
    """A set of independent lattices advanced together."""
    name: str
    Ls: List[int]
    temps: List[float]
    seeds: List[int]
    cold: bool
    n_sweeps: int
    notes: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def n_sims(self) -> int:
        return len(self.Ls)

    @property
    def spins(self) -> int:
        return int(sum(L * L for L in self.Ls))

    @property
    def flips(self) -> int:
        """Flip attempts of the whole workload: one per spin per sweep."""
        return self.spins * self.n_sweeps


def single_l64() -> Workload:
    """One 64 x 64 lattice at T = 2.269185, random start from seed 1, 1000
    sweeps, E and M recorded every sweep."""
    return Workload("single_L64_T2.269185_random_1000sweeps", [64], [T_CRITICAL], [1],
                    cold=False, n_sweeps=1000)


def single_l16384(T: float = T_CRITICAL, cold: bool = False, n_sweeps: int = 1000) -> Workload:
    """One 16384 x 16384 lattice (268M spins), cold start or random start
    from seed 2."""
    start = "cold" if cold else "random"
    return Workload(f"single_L16384_T{T:g}_{start}_{n_sweeps}sweeps", [16384], [T], [2],
                    cold=cold, n_sweeps=n_sweeps)


def l16384_runs(n_sweeps: int = 1000) -> List[Workload]:
    """The six 16384^2 runs: T in {1.5, 2.269185, 3.0} x {cold, random}."""
    return [single_l16384(T, cold, n_sweeps) for T in (1.5, T_CRITICAL, 3.0) for cold in (True, False)]


def batch754(n_sweeps: int = 10000, master_seed: int = 20240426) -> Workload:
    """754 independent lattices: L = 2^(7+U{0..3}) in {128, 256, 512, 1024}
    (log-uniform), T ~ U[1.8, 2.8], random starts, per-lattice seed
    splitmix64(master + i).  754 is the paper's largest count of parallel
    simulations (Section 3.2)."""
    rng = np.random.default_rng(master_seed)
    exps = rng.integers(0, 4, size=754)
    temps = rng.uniform(1.8, 2.8, size=754)
    Ls = [int(2 ** (7 + e)) for e in exps]
    seeds = [splitmix64(master_seed + i) for i in range(754)]
    return Workload("batch754_L128-1024_T1.8-2.8_random", Ls, [float(t) for t in temps], seeds,
                    cold=False, n_sweeps=n_sweeps)


def binder_scan(n_sweeps: int = 50000, t_lo: float = 2.20, t_hi: float = 2.34) -> Workload:
    """L in {1024, 2048, 4096} x 16 temperatures in [t_lo, t_hi] (default
    [2.20, 2.34]) x 3 replicas (144 lattices)."""
    Ls, temps, seeds = [], [], []
    i = 0
    for L in (1024, 2048, 4096):
        for T in np.linspace(t_lo, t_hi, 16):
            for r in range(3):
                Ls.append(L)
                temps.append(float(T))
                seeds.append(splitmix64(0x5EED0000 + i))
                i += 1
    return Workload("binder_L1024-4096_16T_3rep", Ls, temps, seeds, cold=False, n_sweeps=n_sweeps)


def learned_l256(T: float) -> Workload:
    """64 replicas of a 256 x 256 lattice at one temperature."""
    return Workload(f"learned_L256_T{T:g}_64rep", [256] * 64, [T] * 64,
                    [splitmix64(0x1EA2 + k) for k in range(64)], cold=False, n_sweeps=0)


def random_batch(n: int, Ls=(64, 128, 192, 256), tmin=1.5, tmax=3.5, seed=0) -> Workload:
    """A small mixed batch for tests (sizes drawn from Ls)."""
    rng = np.random.default_rng(seed)
    L = [int(rng.choice(Ls)) for _ in range(n)]
    T = [float(x) for x in rng.uniform(tmin, tmax, size=n)]
    S = [splitmix64(seed * 1000003 + i) for i in range(n)]
    return Workload(f"random_batch_{n}", L, T, S, cold=False, n_sweeps=0)
