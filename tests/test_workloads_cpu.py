"""The seeded input generators (paper_2404_16990_gb300/workloads.py) on the
CPU: the shapes and ranges of each workload, and that the 754-lattice batch,
whose draws depend on numpy's generator, stays the batch the measurements
were taken on."""
from __future__ import annotations

import numpy as np

from paper_2404_16990_gb300 import workloads as wl


def test_splitmix64_is_a_64_bit_bijection_sample():
    xs = [wl.splitmix64(i) for i in range(20000)]
    assert len(set(xs)) == len(xs) and all(0 <= x < 2**64 for x in xs)
    bits = np.array([[(x >> b) & 1 for b in range(64)] for x in xs[:4000]])
    assert np.all(np.abs(bits.mean(axis=0) - 0.5) < 0.05)          # every output bit balanced


def test_batch754_shape_and_recorded_size():
    w = wl.batch754()
    assert w.n_sims == 754 and set(w.Ls) <= {128, 256, 512, 1024} and len(set(w.Ls)) == 4
    assert all(1.8 <= t <= 2.8 for t in w.temps)
    assert w.seeds == [wl.splitmix64(20240426 + i) for i in range(754)]
    # the batch every batch754 figure was measured on (sum of L^2)
    assert w.spins == 263_176_192
    assert w.flips == 263_176_192 * 10000


def test_fixed_workloads():
    assert wl.single_l64().Ls == [64] and wl.single_l64().temps == [wl.T_CRITICAL]
    runs = wl.l16384_runs()
    assert len(runs) == 6 and {r.temps[0] for r in runs} == {1.5, wl.T_CRITICAL, 3.0}
    assert sorted(r.cold for r in runs) == [False] * 3 + [True] * 3
    b = wl.binder_scan()
    assert b.n_sims == 144 and b.spins == 48 * (1024**2 + 2048**2 + 4096**2)
    assert len(set(b.seeds)) == 144
    l = wl.learned_l256(2.3)
    assert l.Ls == [256] * 64 and len(set(l.seeds)) == 64
    r = wl.random_batch(10, seed=3)
    assert r.n_sims == 10 and r == wl.random_batch(10, seed=3)
