"""Randomised plan invariance: random uneven batches (sides 64..512, random
temperatures, cold or random starts) run under random plans -- automatic,
resident with random unit sizes and block sizes, streaming and persistent
streaming with random words per thread, rows per thread and block sizes,
with and without graph replay -- must give the oracle's lattices and E/M
traces bit for bit.  No choice of plan may change a result bit."""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
from paper_2404_16990_gb300 import ising, workloads

pytestmark = pytest.mark.gpu
NT = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def _random_plan(rng, Ls):
    kind = rng.choice(["auto", "resident", "stream", "persist"])
    if kind == "auto":
        return ising.ISING_PLAN_AUTO, {}
    if kind == "resident":
        if max(Ls) > 1024:
            kind = "stream"
        else:
            return ising.ISING_PLAN_RESIDENT, {"sweeps_per_unit": int(rng.choice([1, 3, 8, 64])),
                                               "threads": int(rng.choice([0, 128, 256, 512]))}
    V = int(rng.choice([1, 2, 4]))
    while V > 1 and any((L // 64) % V for L in Ls):
        V //= 2
    plan = ising.ISING_PLAN_STREAM if kind == "stream" else ising.ISING_PLAN_PERSIST
    return plan, {"words_per_thread": V, "rows_per_item": int(rng.choice([1, 2, 3, 4, 8])),
                  "threads": int(rng.choice([64, 128, 256]))}


@pytest.mark.parametrize("case", range(12))
def test_random_batch_random_plan(case):
    import torch
    rng = np.random.default_rng(1000 + case)
    n = int(rng.integers(1, 7))
    Ls = [int(x) for x in rng.choice([64, 128, 192, 256, 320, 448, 512], size=n)]
    temps = [float(x) for x in rng.uniform(0.8, 4.0, size=n)]
    seeds = [workloads.splitmix64(7000 + 97 * case + i) for i in range(n)]
    cold = bool(rng.integers(0, 2))
    sweeps = int(rng.integers(1, 9))
    plan, kw = _random_plan(rng, Ls)
    graph = bool(rng.integers(0, 2))
    stream = torch.cuda.Stream() if graph else None
    sim = ising.IsingSim(Ls=Ls, temps=temps, seeds=seeds, cold=cold, trace_cap=sweeps, stream=stream)
    sim.set_plan(plan, **kw)
    if graph:
        sim.set_graph(True)
    sim.sweep(sweeps)
    Eg, Mg = sim.trace(sweeps)
    refs = [np.ones((L, L), np.int8) if cold else oracle.init(L, sd, i) for i, (L, sd) in enumerate(zip(Ls, seeds))]
    Eo, Mo = oracle.sweeps_batch(refs, temps, seeds, list(range(n)), 0, sweeps, NT)
    info = (case, Ls, plan, kw, graph, cold, sweeps)
    assert np.array_equal(Eg, Eo) and np.array_equal(Mg, Mo), info
    for i in range(n):
        assert np.array_equal(sim.spins(i), refs[i]), (info, i)
    sim.close()
