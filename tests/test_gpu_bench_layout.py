"""GPU parity of the two throughput workloads in the launch layout the
benchmark times, against the CPU oracle bit for bit.

* The 16384^2 configuration: two handles of three lattices (T = 1.5, 2.269185,
  3.0; one handle cold, one random from seed 2), the streaming plan forced to
  4 words x 4 rows per thread in blocks of 128 threads (the plan the
  autotuner picks for the benchmark on GB300) or 256 (the library's default),
  CUDA-graph replay of a 1000-sweep call with E/M recorded every sweep.  Run
  in full at 2048^2 (all six lattices, 1000 sweeps, lattices and traces;
  128 threads) and 4096^2 (all six on the GPU; the two cold lattices at
  T = 1.5 and 3.0 in full against the oracle; 256 threads), and at the
  benchmark's own 16384^2 on light-cone samples after 50 sweeps (both).
* The 754-lattice batch (L in {128 .. 1024}, T in [1.8, 2.8], random
  starts): 100 sweeps of every lattice under the cooperative persistent plan
  the autotuner picks for it on GB300 (2 words x 8 rows per thread, 128
  threads) and under whatever the autotuner picks in the test, and 10,000
  sweeps of the whole batch with a 32-lattice sample (16 of side 128, 16 of
  side 256) compared in full, traces included.

The oracle runs on every host thread (rows of one colour split across
threads, or lattices across threads); these are the slowest GPU tests."""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
from paper_2404_16990_gb300 import ising, workloads

pytestmark = pytest.mark.gpu

NT = max(1, min(16, os.cpu_count() or 1))
TC = workloads.T_CRITICAL
T_RUNS = (1.5, TC, 3.0)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def site_from_words(words_t, L: int, y: int, x: int) -> int:
    wn = L // 64
    c = (x + y) & 1
    j = x >> 1
    w = int(words_t[(c * L + y) * wn + j // 32].item()) & 0xFFFFFFFF
    return -1 if (w >> (j % 32)) & 1 else 1


def bench_handles(L: int, n: int, seed: int = 2, threads: int = 128):
    """The benchmark's two handles on one non-default stream, streaming plan
    4 x 4 with `threads` per block, graph replay on, n sweeps each."""
    import torch
    stream = torch.cuda.Stream()
    sims = []
    for cold in (True, False):
        s = ising.IsingSim(Ls=[L] * 3, temps=list(T_RUNS), seeds=[seed] * 3, cold=cold, trace_cap=n,
                           stream=stream)
        s.set_plan(ising.ISING_PLAN_STREAM, words_per_thread=4, rows_per_item=4, threads=threads)
        s.set_graph(True)
        sims.append(s)
    for s in sims:
        plan = ising.ising_get_plan(s.h)
        assert (plan["plan"], plan["words_per_thread"], plan["rows_per_item"], plan["threads"]) == \
            (ising.ISING_PLAN_STREAM, 4, 4, threads)
    for s in sims:          # two calls: the graph of n/2 sweeps is captured, then replayed
        s.sweep(n // 2)
        s.sweep(n - n // 2)
    return sims


def test_bench_layout_2048_1000_sweeps_bit_exact():
    L, n, seed = 2048, 1000, 2
    sims = bench_handles(L, n, seed, threads=128)
    for h, cold in enumerate((True, False)):
        sim = sims[h]
        assert sim.sweeps_done == n
        Eg, Mg = sim.trace(n)
        for i, T in enumerate(T_RUNS):
            ref = oracle.init(L, seed, i, cold=cold, n_threads=NT)
            Eo, Mo = oracle.sweeps(ref, T, seed, i, 0, n, n_threads=NT)
            assert np.array_equal(Eg[i], Eo) and np.array_equal(Mg[i], Mo), (cold, T)
            assert np.array_equal(sim.spins(i), ref), (cold, T)


def test_bench_layout_4096_1000_sweeps_cold_lattices_bit_exact():
    """Config 2's cold starts at T = 1.5 and 3.0, 1000 sweeps, in the
    benchmark's layout (all six lattices swept on the GPU)."""
    L, n, seed = 4096, 1000, 2
    sims = bench_handles(L, n, seed, threads=256)
    cold = sims[0]
    Eg, Mg = cold.trace(n)
    for i in (0, 2):
        ref = oracle.init(L, seed, i, cold=True, n_threads=NT)
        Eo, Mo = oracle.sweeps(ref, T_RUNS[i], seed, i, 0, n, n_threads=NT)
        assert np.array_equal(Eg[i], Eo) and np.array_equal(Mg[i], Mo), T_RUNS[i]
        assert np.array_equal(cold.spins(i), ref), T_RUNS[i]
    # the random handle and the critical cold lattice: E and M against their own lattices
    for sim in sims:
        E, M = sim.observables()
        for i in range(3):
            s = sim.spins(i)
            assert oracle.energy(s) == E[i] and int(s.sum(dtype=np.int64)) == M[i]


@pytest.mark.parametrize("threads", [128, 256])
def test_bench_layout_16384_light_cone_after_50_sweeps(threads):
    """The benchmark's own lattices: every one of the six sampled at 10
    sites (corners and edges included) after 50 graph-replayed sweeps."""
    L, n, seed = 16384, 50, 2
    sims = bench_handles(L, n, seed, threads=threads)
    rng = np.random.default_rng(50)
    for h, cold in enumerate((True, False)):
        for i, T in enumerate(T_RUNS):
            words = sims[h].words(i)
            pts = [(int(y), int(x)) for y, x in rng.integers(0, L, size=(7, 2))] + [(0, 0), (L - 1, L - 1), (1, L - 2)]
            for y, x in pts:
                want = oracle.window_state(L, seed, i, cold, T, y, x, 0, n)
                assert site_from_words(words, L, y, x) == want, (cold, T, y, x)


# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def batch754_after_100():
    """The oracle's 754 lattices and traces after 100 sweeps (lattices spread
    over the host threads)."""
    wl = workloads.batch754()
    refs = [oracle.init(L, s, i) for i, (L, s) in enumerate(zip(wl.Ls, wl.seeds))]
    E, M = oracle.sweeps_batch(refs, wl.temps, wl.seeds, list(range(len(refs))), 0, 100, NT)
    return wl, refs, E, M


def _check_754(sim, wl, refs, Eo, Mo, n):
    Eg, Mg = sim.trace(n)
    assert np.array_equal(Eg, Eo) and np.array_equal(Mg, Mo)
    for i in range(len(refs)):
        assert np.array_equal(sim.spins(i), refs[i]), (i, wl.Ls[i])


def test_batch754_tuned_persistent_plan_100_sweeps(batch754_after_100):
    import torch
    wl, refs, Eo, Mo = batch754_after_100
    stream = torch.cuda.Stream()
    sim = ising.IsingSim(Ls=wl.Ls, temps=wl.temps, seeds=wl.seeds, trace_cap=100, stream=stream)
    sim.set_plan(ising.ISING_PLAN_PERSIST, words_per_thread=2, rows_per_item=8, threads=128)
    sim.set_graph(True)
    sim.sweep(40)
    sim.sweep(60)
    plan = ising.ising_get_plan(sim.h)
    assert (plan["plan"], plan["words_per_thread"], plan["rows_per_item"], plan["threads"]) == \
        (ising.ISING_PLAN_PERSIST, 2, 8, 128)
    _check_754(sim, wl, refs, Eo, Mo, 100)


def test_batch754_autotuned_plan_100_sweeps(batch754_after_100, tmp_path, monkeypatch):
    import torch
    monkeypatch.setenv("ISING_TUNE_CACHE", str(tmp_path / "tune.txt"))
    wl, refs, Eo, Mo = batch754_after_100
    stream = torch.cuda.Stream()
    sim = ising.IsingSim(Ls=wl.Ls, temps=wl.temps, seeds=wl.seeds, trace_cap=100, stream=stream)
    sim.set_graph(True)
    sim.sweep(10)
    assert sim.autotune(probe_sweeps=5, force=True) > 0
    sim.sweep(90)
    _check_754(sim, wl, refs, Eo, Mo, 100)


def test_batch754_10000_sweeps_sample_bit_exact():
    import torch
    wl = workloads.batch754()
    n = 10000
    stream = torch.cuda.Stream()
    sim = ising.IsingSim(Ls=wl.Ls, temps=wl.temps, seeds=wl.seeds, trace_cap=n, stream=stream)
    sim.set_plan(ising.ISING_PLAN_PERSIST, words_per_thread=2, rows_per_item=8, threads=128)
    sim.set_graph(True)
    sim.sweep(n)
    rng = np.random.default_rng(754)
    pick = []
    for L in (128, 256):
        idx = [i for i, Li in enumerate(wl.Ls) if Li == L]
        pick += sorted(rng.choice(idx, 16, replace=False).tolist())
    refs = [oracle.init(wl.Ls[i], wl.seeds[i], i) for i in pick]
    Eo, Mo = oracle.sweeps_batch(refs, [wl.temps[i] for i in pick], [wl.seeds[i] for i in pick], pick, 0, n, NT)
    Eg, Mg = sim.trace(n)
    for k, i in enumerate(pick):
        assert np.array_equal(Eg[i], Eo[k]) and np.array_equal(Mg[i], Mo[k]), (i, wl.Ls[i])
        assert np.array_equal(sim.spins(i), refs[k]), (i, wl.Ls[i])
    # every other lattice: E and M consistent with its own final spins
    E, M = sim.observables()
    for i in rng.choice(len(wl.Ls), 24, replace=False):
        s = sim.spins(int(i))
        assert oracle.energy(s) == E[i] and int(s.sum(dtype=np.int64)) == M[i]
