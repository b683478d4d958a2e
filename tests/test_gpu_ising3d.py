"""GPU parity of the three-dimensional sweep (ising3d_* C ABI) against the
CPU oracle, bit for bit: initial states, spins and E/M traces after sweeps of
single lattices and uneven batches, graph replay, a 256^3 lattice, and the
API's argument checks."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2404_16990_gb300 import ising

pytestmark = pytest.mark.gpu
TC3 = 4.5115


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def _start(L, seed, s, cold):
    return np.ones((L, L, L), np.int8) if cold else oracle.init3d(L, seed, s)


def test_initial_states_and_observables():
    Ls, temps, seeds = [64, 128], [TC3, 3.0], [5, 6]
    sim = ising.IsingSim3D(Ls, temps, seeds)
    E, M = sim.observables()
    for i, (L, sd) in enumerate(zip(Ls, seeds)):
        ref = oracle.init3d(L, sd, i)
        assert np.array_equal(sim.spins(i), ref)
        assert E[i] == oracle.energy3d(ref) and M[i] == oracle.magnetization3d(ref)
    sim.close()


@pytest.mark.parametrize("cold", [False, True])
def test_sweeps_bit_exact_uneven_batch(cold):
    Ls, temps, seeds = [64, 128, 64, 192], [TC3, 3.0, 6.0, 0.5], [11, 12, 13, 14]
    n = 12
    sim = ising.IsingSim3D(Ls, temps, seeds, cold=cold, trace_cap=n)
    sim.sweep(n)
    Eg, Mg = sim.trace(n)
    for i, (L, T, sd) in enumerate(zip(Ls, temps, seeds)):
        ref = _start(L, sd, i, cold)
        Eo, Mo = oracle.sweeps3d(ref, T, sd, i, 0, n)
        assert np.array_equal(sim.spins(i), ref), (i, L, T)
        assert np.array_equal(Eg[i], Eo) and np.array_equal(Mg[i], Mo), (i, L, T)
    assert sim.sweeps_done == n
    sim.close()


def test_graph_replay_matches_direct_launches():
    import torch
    s = torch.cuda.Stream()
    a = ising.IsingSim3D([64, 128], [TC3, 4.0], [3, 4], trace_cap=20, stream=s)
    b = ising.IsingSim3D([64, 128], [TC3, 4.0], [3, 4], trace_cap=20, stream=s)
    b.set_graph(True)
    for _ in range(4):
        a.sweep(5)
        b.sweep(5)
    for i in range(2):
        assert np.array_equal(a.spins(i), b.spins(i))
    Ea, Ma = a.trace(20)
    Eb, Mb = b.trace(20)
    assert np.array_equal(Ea, Eb) and np.array_equal(Ma, Mb)
    a.close()
    b.close()


def test_256_cubed_bit_exact():
    L, T, sd, n = 256, TC3, 21, 3
    sim = ising.IsingSim3D([L], [T], [sd], trace_cap=n)
    sim.sweep(n)
    ref = oracle.init3d(L, sd, 0)
    Eo, Mo = oracle.sweeps3d(ref, T, sd, 0, 0, n)
    Eg, Mg = sim.trace(n)
    assert np.array_equal(Eg[0], Eo) and np.array_equal(Mg[0], Mo)
    assert np.array_equal(sim.spins(0), ref)
    sim.close()


def test_arguments_rejected():
    for Ls, temps in [([96], [4.0]), ([2048], [4.0]), ([64], [0.0]), ([64], [float("nan")])]:
        with pytest.raises(ising.IsingError):
            ising.IsingSim3D(Ls, temps, [1])
