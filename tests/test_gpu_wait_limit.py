"""The bounded device waits run out cleanly: with a wait limit of one
microsecond (ising_set_wait_limit_ns), a wait that cannot be satisfied in
that time sets the handle's error word, the kernel returns without finishing
its sweeps, the next synchronising call reports ISING_ETIMEOUT, and the
device stays usable -- a fresh handle then sweeps bit for bit like the
oracle.  Nothing here faults or spins without bound: each wait checks the
GPU's global timer against the limit and gives up.

The waits are made to run out by uneven work, not by a broken kernel:
* the persistent streaming kernel's grid barrier: blocks whose tiles are
  small 128^2 lattices reach the barrier long (tens of microseconds) before
  the blocks sweeping a 1024^2 lattice's tiles;
* the resident kernel's chunk wait: with one sweep per work unit, blocks of
  small 64^2 groups finish a chunk long before the 1024^2 group and take the
  next tickets, among them the 1024^2 group's next chunk, which must wait
  for the previous one."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2404_16990_gb300 import ising

pytestmark = pytest.mark.gpu

LIMIT_NS = 1000


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def _fresh_handle_matches_oracle(Ls, temps, seeds, plan, **kw):
    sim = ising.IsingSim(Ls=Ls, temps=temps, seeds=seeds, trace_cap=4)
    sim.set_plan(plan, **kw)
    sim.sweep(4)
    refs = [oracle.init(L, s, i) for i, (L, s) in enumerate(zip(Ls, seeds))]
    Eo, Mo = oracle.sweeps_batch(refs, temps, seeds, list(range(len(refs))), 0, 4, 8)
    Eg, Mg = sim.trace(4)
    assert np.array_equal(Eg, Eo) and np.array_equal(Mg, Mo)
    for i in range(len(refs)):
        assert np.array_equal(sim.spins(i), refs[i])


def test_persistent_grid_barrier_wait_runs_out():
    Ls = [1024, 1024, 128, 128, 128, 128]
    temps = [2.3] * 6
    seeds = [31 + i for i in range(6)]
    sim = ising.IsingSim(Ls=Ls, temps=temps, seeds=seeds)
    sim.set_plan(ising.ISING_PLAN_PERSIST, words_per_thread=2, rows_per_item=8)
    ising.ising_set_wait_limit_ns(sim.h, LIMIT_NS)
    sim.sweep(20)                                   # enqueues only
    with pytest.raises(ising.IsingError) as e:
        sim.observables()
    assert e.value.code == ising.ISING_ETIMEOUT
    with pytest.raises(ising.IsingError) as e:      # the handle stays failed
        sim.spins(0)
    assert e.value.code == ising.ISING_ETIMEOUT
    _fresh_handle_matches_oracle(Ls, temps, seeds, ising.ISING_PLAN_PERSIST, words_per_thread=2, rows_per_item=8)


def test_resident_chunk_wait_runs_out():
    Ls = [1024] + [64] * 8
    temps = [2.5] * 9
    seeds = [77 + i for i in range(9)]
    sim = ising.IsingSim(Ls=Ls, temps=temps, seeds=seeds)
    sim.set_plan(ising.ISING_PLAN_RESIDENT, sweeps_per_unit=1)
    ising.ising_set_wait_limit_ns(sim.h, LIMIT_NS)
    sim.sweep(50)
    with pytest.raises(ising.IsingError) as e:
        sim.observables()
    assert e.value.code == ising.ISING_ETIMEOUT
    _fresh_handle_matches_oracle(Ls, temps, seeds, ising.ISING_PLAN_RESIDENT, sweeps_per_unit=1)


def test_default_limit_restored_by_zero():
    """Setting the limit back to 0 (the 10 s default) on a handle whose waits
    never ran out leaves its sweeps exact."""
    Ls, temps, seeds = [1024, 128, 128], [2.2, 2.4, 2.6], [5, 6, 7]
    sim = ising.IsingSim(Ls=Ls, temps=temps, seeds=seeds, trace_cap=4)
    sim.set_plan(ising.ISING_PLAN_PERSIST, words_per_thread=2, rows_per_item=8)
    ising.ising_set_wait_limit_ns(sim.h, 5_000_000_000)
    ising.ising_set_wait_limit_ns(sim.h, 0)
    sim.sweep(4)
    refs = [oracle.init(L, s, i) for i, (L, s) in enumerate(zip(Ls, seeds))]
    Eo, Mo = oracle.sweeps_batch(refs, temps, seeds, [0, 1, 2], 0, 4, 8)
    Eg, Mg = sim.trace(4)
    assert np.array_equal(Eg, Eo) and np.array_equal(Mg, Mo)
