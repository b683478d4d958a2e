"""GPU parity of the cluster-resident plan (ISING_PLAN_CLUSTER: one
thread-block cluster per lattice, strips of rows in shared memory, the rows
next to a strip read from the neighbouring CTAs' shared memory) against the
CPU oracle, bit for bit: every cluster size from 1 to 8, sides that are not
powers of two, uneven batches, cold and random starts, several calls, graph
replay, and the 64-lattice 256^2 workload of the learned-proposal study."""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
from paper_2404_16990_gb300 import ising, workloads

pytestmark = pytest.mark.gpu

NT = max(1, min(16, os.cpu_count() or 1))
TC = workloads.T_CRITICAL


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def _check(Ls, temps, seeds, rows, n, cold=False, graph=False, calls=(5,)):
    import torch
    stream = torch.cuda.Stream()
    sim = ising.IsingSim(Ls=Ls, temps=temps, seeds=seeds, cold=cold, trace_cap=n, stream=stream)
    sim.set_plan(ising.ISING_PLAN_CLUSTER, rows_per_item=rows)
    assert ising.ising_get_plan(sim.h)["plan"] == ising.ISING_PLAN_CLUSTER
    sim.set_graph(graph)
    done = 0
    for k in list(calls) + [n - sum(calls)]:
        if k > 0:
            sim.sweep(k)
            done += k
    assert sim.sweeps_done == n
    refs = [oracle.init(L, s, i, cold=cold) for i, (L, s) in enumerate(zip(Ls, seeds))]
    Eo, Mo = oracle.sweeps_batch(refs, temps, seeds, list(range(len(refs))), 0, n, NT)
    Eg, Mg = sim.trace(n)
    assert np.array_equal(Eg, Eo) and np.array_equal(Mg, Mo)
    for i in range(len(refs)):
        assert np.array_equal(sim.spins(i), refs[i]), (i, Ls[i])
    return sim


@pytest.mark.parametrize("L,rows,T,cold", [
    (64, 64, TC, False),          # C = 1: the strip's neighbours are itself
    (128, 64, 1.5, True),         # C = 2: both neighbours are the other CTA
    (256, 64, TC, False),         # C = 4
    (512, 64, 3.0, False),        # C = 8
    (1024, 32, 2.0, True),        # C = 8 (capped), 128 rows each
    (1024, 128, TC, False),       # C = 8
    (256, 128, 2.6, False),       # C = 2
])
def test_cluster_sizes_bit_exact(L, rows, T, cold):
    _check([L], [T], [300 + L + rows], rows, 12, cold=cold, calls=(5,))


def test_uneven_batch_with_sides_not_powers_of_two():
    """Sides 192 (C = 2, 96 rows), 320 (C = 4, 80 rows), 576 (C = 8, 72 rows)
    beside powers of two, in one handle: one launch per side."""
    wl = workloads.random_batch(14, Ls=(64, 192, 256, 320, 576, 1024), seed=17)
    _check(wl.Ls, wl.temps, wl.seeds, 64, 9, calls=(3, 4))


def test_graph_replay_and_cold_start():
    wl = workloads.random_batch(6, Ls=(128, 256, 512), seed=5)
    _check(wl.Ls, wl.temps, wl.seeds, 64, 12, cold=True, graph=True, calls=(4, 4))


def test_learned_study_workload_100_sweeps():
    """64 replicas of 256^2 (the learned-proposal study's plain chain), one
    seed, simulation indices 0 .. 63."""
    L, n = 256, 100
    temps = [TC] * 64
    import torch
    stream = torch.cuda.Stream()
    sim = ising.IsingSim(L, temps, 2024, trace_cap=n, stream=stream)
    sim.set_plan(ising.ISING_PLAN_CLUSTER)
    sim.set_graph(True)
    sim.sweep(50)
    sim.sweep(50)
    refs = [oracle.init(L, 2024, i) for i in range(64)]
    Eo, Mo = oracle.sweeps_batch(refs, temps, [2024] * 64, list(range(64)), 0, n, NT)
    Eg, Mg = sim.trace(n)
    assert np.array_equal(Eg, Eo) and np.array_equal(Mg, Mo)
    for i in (0, 17, 63):
        assert np.array_equal(sim.spins(i), refs[i])


def test_cluster_plan_rejects_large_lattices():
    sim = ising.IsingSim(Ls=[256, 2048], temps=[2.0, 2.0], seeds=[1, 2])
    with pytest.raises(ising.IsingError) as e:
        sim.set_plan(ising.ISING_PLAN_CLUSTER)
    assert e.value.code == ising.ISING_EINVAL
    sim.sweep(2)                                    # the previous plan is kept and still runs
    assert sim.sweeps_done == 2
