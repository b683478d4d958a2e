"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, bit
for bit -- initial states, lattices after sweeps, E/M traces, thresholds --
for single lattices (resident and streaming kernels), uneven batches,
ragged tilings, the full 16384^2 workload the benchmark times (full lattice
for the first sweeps, light-cone samples later, properties after 1000
sweeps), the 65536^2 maximum, and the API's edge cases."""
from __future__ import annotations

import os

import numpy as np
import pytest

import exact
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


def unpack_words(words: np.ndarray, L: int) -> np.ndarray:
    """Documented layout: word[(c*L + y)*(L/64) + k], bit b -> x = 2(32k+b) + ((y+c)&1),
    bit 1 = spin -1."""
    wn = L // 64
    w = words.view(np.uint32).reshape(2, L, wn)
    bits = ((w[..., None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(2, L, wn * 32)
    out = np.empty((L, L), np.int8)
    for c in (0, 1):
        for par in (0, 1):
            ys = np.arange(par, L, 2)
            x0 = (par + c) & 1
            out[ys, x0::2] = np.where(bits[c, ys, :] == 1, -1, 1)
    return out


def site_from_words(words_t, L: int, y: int, x: int) -> int:
    wn = L // 64
    c = (x + y) & 1
    j = x >> 1
    w = int(words_t[(c * L + y) * wn + j // 32].item()) & 0xFFFFFFFF
    return -1 if (w >> (j % 32)) & 1 else 1


# ---------------------------------------------------------------------------
def test_single_l64_config_bit_exact():
    """64x64, T = 2.269185, random start seed 1, 1000 sweeps, E/M each sweep."""
    wl = workloads.single_l64()
    sim = ising.IsingSim(64, wl.temps, wl.seeds[0], trace_cap=wl.n_sweeps)
    ref = oracle.init(64, wl.seeds[0], 0)
    assert np.array_equal(sim.spins(0), ref)
    E0, M0 = sim.observables()
    assert E0[0] == oracle.energy(ref) and M0[0] == oracle.magnetization(ref)
    assert np.array_equal(sim.thresholds()[0], oracle.thresholds(wl.temps[0]))
    sim.sweep(wl.n_sweeps)
    Eo, Mo = oracle.sweeps(ref, wl.temps[0], wl.seeds[0], 0, 0, wl.n_sweeps)
    Eg, Mg = sim.trace(wl.n_sweeps)
    assert np.array_equal(Eg[0], Eo) and np.array_equal(Mg[0], Mo)
    assert np.array_equal(sim.spins(0), ref)
    assert sim.sweeps_done == wl.n_sweeps


@pytest.mark.parametrize("L,V,R,T,cold", [
    (128, 2, 3, TC, False),
    (384, 2, 5, 1.5, False),
    (448, 1, 7, 3.0, True),       # 7 words per row: odd, V = 1
    (1024, 4, 4, TC, False),
    (1280, 4, 6, 1.5, True),
    (2048, 2, 4, 3.0, False),
])
def test_streaming_kernel_bit_exact(L, V, R, T, cold):
    n = 12
    sim = ising.IsingSim(L, [T], 77 + L, cold=cold, trace_cap=n)
    sim.set_plan(ising.ISING_PLAN_STREAM, words_per_thread=V, rows_per_item=R)
    ref = oracle.init(L, 77 + L, 0, cold=cold, n_threads=NT)
    assert np.array_equal(sim.spins(0), ref)
    sim.sweep(5)
    sim.sweep(n - 5)
    Eo, Mo = oracle.sweeps(ref, T, 77 + L, 0, 0, n, n_threads=NT)
    Eg, Mg = sim.trace(n)
    assert np.array_equal(Eg[0], Eo) and np.array_equal(Mg[0], Mo)
    assert np.array_equal(sim.spins(0), ref)


@pytest.mark.parametrize("Ls", [(2048,), (4096,), (1024, 2048, 4096)])
def test_default_streaming_tiling_bit_exact(Ls):
    """The streaming plan with the default tiling, which depends on the
    blocks each candidate gives (on a 152-SM GB300: 1 x 2 for 2048^2, 2 x 2
    for 4096^2): bit-exact, and the tiling in use is one of the candidates."""
    n = 3
    temps = [TC, 1.5, 3.0][:len(Ls)]
    seeds = [91 + i for i in range(len(Ls))]
    sim = ising.IsingSim(Ls=list(Ls), temps=temps, seeds=seeds, trace_cap=n)
    sim.set_plan(ising.ISING_PLAN_STREAM)
    plan = ising.ising_get_plan(sim.h)
    assert (plan["words_per_thread"], plan["rows_per_item"]) in {(4, 4), (2, 2), (1, 2), (1, 1)}
    refs = [oracle.init(L, s_, i, n_threads=NT) for i, (L, s_) in enumerate(zip(Ls, seeds))]
    sim.sweep(n)
    Eo, Mo = oracle.sweeps_batch(refs, temps, seeds, list(range(len(refs))), 0, n, NT)
    Eg, Mg = sim.trace(n)
    assert np.array_equal(Eg, Eo) and np.array_equal(Mg, Mo)
    for i in range(len(refs)):
        assert np.array_equal(sim.spins(i), refs[i]), i


@pytest.mark.parametrize("L,k,threads", [(64, 1, 64), (192, 3, 96), (256, 8, 0), (512, 5, 512), (1024, 2, 512)])
def test_resident_kernel_bit_exact(L, k, threads):
    n = 11
    T = [1.8, TC, 2.9][L % 3]
    sim = ising.IsingSim(L, [T], 5 + L, trace_cap=n)
    sim.set_plan(ising.ISING_PLAN_RESIDENT, sweeps_per_unit=k, threads=threads)
    ref = oracle.init(L, 5 + L, 0)
    sim.sweep(n)
    Eo, Mo = oracle.sweeps(ref, T, 5 + L, 0, 0, n, n_threads=NT)
    Eg, Mg = sim.trace(n)
    assert np.array_equal(Eg[0], Eo) and np.array_equal(Mg[0], Mo)
    assert np.array_equal(sim.spins(0), ref)


def _batch_check(wl, n, plan=None, **kw):
    sim = ising.IsingSim(Ls=wl.Ls, temps=wl.temps, seeds=wl.seeds, trace_cap=n)
    if plan is not None:
        sim.set_plan(plan, **kw)
    refs = [oracle.init(L, s, i) for i, (L, s) in enumerate(zip(wl.Ls, wl.seeds))]
    for i in range(len(refs)):
        assert np.array_equal(sim.spins(i), refs[i])
    sim.sweep(n)
    Eo, Mo = oracle.sweeps_batch(refs, wl.temps, wl.seeds, list(range(len(refs))), 0, n, NT)
    Eg, Mg = sim.trace(n)
    assert np.array_equal(Eg, Eo) and np.array_equal(Mg, Mo)
    for i in range(len(refs)):
        assert np.array_equal(sim.spins(i), refs[i]), i
    assert np.array_equal(sim.thresholds(), np.stack([oracle.thresholds(T) for T in wl.temps]))


@pytest.mark.parametrize("plan,kw", [
    (None, {}),
    (ising.ISING_PLAN_RESIDENT, {"sweeps_per_unit": 3, "threads": 256}),
    (ising.ISING_PLAN_STREAM, {"words_per_thread": 1, "rows_per_item": 3}),
])
def test_uneven_batch_bit_exact(plan, kw):
    wl = workloads.random_batch(40, Ls=(64, 128, 192, 256, 320), seed=11)
    _batch_check(wl, 17, plan, **kw)


def test_mixed_resident_and_streamed_batch():
    wl = workloads.random_batch(9, Ls=(64, 128, 2048), seed=3)
    assert 2048 in wl.Ls and min(wl.Ls) < 1024
    _batch_check(wl, 9, ising.ISING_PLAN_MIXED)
    _batch_check(wl, 5)         # the default plan streams every lattice


def test_batch754_sample_and_prefix():
    """The 754-lattice workload: every lattice for the first sweeps."""
    wl = workloads.batch754()
    _batch_check(wl, 3)


# ---------------------------------------------------------------------------
def test_l16384_bench_configuration():
    """The benchmark's 16384^2 workload in its launch configuration: initial
    state and first two sweeps compared in full, later sweeps on light-cone
    samples, and E/M against the lattice itself."""
    L, T, seed = 16384, TC, 2
    sim = ising.IsingSim(L, [T], seed, trace_cap=16)
    ref = oracle.init(L, seed, 0, n_threads=NT)
    assert np.array_equal(sim.spins(0), ref)
    sim.sweep(2)
    Eo, Mo = oracle.sweeps(ref, T, seed, 0, 0, 2, n_threads=NT)
    Eg, Mg = sim.trace(2)
    assert np.array_equal(Eg[0], Eo) and np.array_equal(Mg[0], Mo)
    assert np.array_equal(sim.spins(0), ref)
    del ref
    sim.sweep(8)
    words = sim.words(0)
    rng = np.random.default_rng(5)
    pts = [(int(y), int(x)) for y, x in rng.integers(0, L, size=(24, 2))] + [(0, 0), (L - 1, 5), (7, L - 1)]
    for y, x in pts:
        assert site_from_words(words, L, y, x) == oracle.window_state(L, seed, 0, False, T, y, x, 0, 10), (y, x)


def _energy_np(s: np.ndarray) -> int:
    s16 = s.astype(np.int16)
    return int(-(s16 * np.roll(s16, -1, 1)).sum(dtype=np.int64) - (s16 * np.roll(s16, -1, 0)).sum(dtype=np.int64))


@pytest.mark.parametrize("T,cold", [(1.5, True), (3.0, False)])
def test_l16384_1000_sweeps_properties(T, cold):
    L, n = 16384, 1000
    sim = ising.IsingSim(L, [T], 2, cold=cold, trace_cap=n)
    sim.sweep(n)
    E, M = sim.observables()
    Et, Mt = sim.trace(n)
    assert Et[0, -1] == E[0] and Mt[0, -1] == M[0]
    s = sim.spins(0)
    assert int(s.sum(dtype=np.int64)) == M[0]
    assert _energy_np(s) == E[0]
    N = L * L
    e = Et[0, -100:].mean() / N
    assert abs(e - exact.onsager_u(T)) < 2e-3
    if T < TC:
        assert abs(abs(Mt[0, -100:]).mean() / N - exact.onsager_m(T)) < 2e-3


def test_max_size_lattice_light_cone():
    L, T, seed = ising.ISING_MAX_L, 2.5, 9
    sim = ising.IsingSim(L, [T], seed)
    sim.sweep(3)
    words = sim.words(0)
    rng = np.random.default_rng(2)
    pts = [(int(y), int(x)) for y, x in rng.integers(0, L, size=(12, 2))] + [(0, 0), (L - 1, L - 1)]
    for y, x in pts:
        assert site_from_words(words, L, y, x) == oracle.window_state(L, seed, 0, False, T, y, x, 0, 3), (y, x)


# ---------------------------------------------------------------------------
def test_trace_ring_wraps():
    sim = ising.IsingSim(128, [2.0], 4, trace_cap=7)
    ref = oracle.init(128, 4, 0)
    sim.sweep(20)
    Eo, Mo = oracle.sweeps(ref, 2.0, 4, 0, 0, 20)
    Eg, Mg = sim.trace(100)
    assert Eg.shape == (1, 7)
    assert np.array_equal(Eg[0], Eo[-7:]) and np.array_equal(Mg[0], Mo[-7:])
    Eg, _ = sim.trace(3)
    assert np.array_equal(Eg[0], Eo[-3:])


def test_save_load_resume_bit_exact():
    wl = workloads.random_batch(6, Ls=(64, 128, 2048), seed=8)
    a = ising.IsingSim(Ls=wl.Ls, temps=wl.temps, seeds=wl.seeds)
    a.sweep(60)
    b = ising.IsingSim(Ls=wl.Ls, temps=wl.temps, seeds=wl.seeds)
    b.sweep(25)
    state = ising.ising_save(b.h)
    c = ising.IsingSim(Ls=wl.Ls, temps=wl.temps, seeds=wl.seeds, cold=True)
    ising.ising_load(c.h, state)
    assert c.sweeps_done == 25
    c.sweep(35)
    for i in range(len(wl.Ls)):
        assert np.array_equal(a.spins(i), c.spins(i))
    assert all(np.array_equal(x, y) for x, y in zip(a.observables(), c.observables()))
    d = ising.IsingSim(128, [2.0], 1)
    with pytest.raises(ising.IsingError):
        ising.ising_load(d.h, state)


def test_graph_replay_identical():
    import torch
    wl = workloads.random_batch(5, Ls=(64, 256, 2048), seed=21)
    s = torch.cuda.Stream()
    a = ising.IsingSim(Ls=wl.Ls, temps=wl.temps, seeds=wl.seeds, trace_cap=30, stream=s)
    b = ising.IsingSim(Ls=wl.Ls, temps=wl.temps, seeds=wl.seeds, trace_cap=30, stream=s)
    b.set_graph(True)
    for _ in range(3):
        a.sweep(10)
        b.sweep(10)
    for i in range(len(wl.Ls)):
        assert np.array_equal(a.spins(i), b.spins(i))
    assert all(np.array_equal(x, y) for x, y in zip(a.trace(30), b.trace(30)))


def test_set_get_spins_and_observables():
    rng = np.random.default_rng(0)
    sim = ising.IsingSim(192, [2.2], 3)
    s = np.where(rng.random((192, 192)) < 0.3, -1, 1).astype(np.int8)
    sim.set_spins(0, s)
    assert np.array_equal(sim.spins(0), s)
    E, M = sim.observables()
    assert E[0] == oracle.energy(s) and M[0] == s.sum()
    bad = s.copy()
    bad[3, 3] = 0
    with pytest.raises(ising.IsingError):
        sim.set_spins(0, bad)


def test_moments_match_trace():
    wl = workloads.random_batch(4, Ls=(64, 128, 2048), seed=5)
    sim = ising.IsingSim(Ls=wl.Ls, temps=wl.temps, seeds=wl.seeds, trace_cap=200)
    sim.sweep(10)
    ising.ising_set_measure(sim.h, True)
    sim.sweep(200)
    mom = ising.ising_moments(sim.h)
    E, M = sim.trace(200)
    for i, L in enumerate(wl.Ls):
        m = M[i] / L**2
        e = E[i] / L**2
        ref = [200, np.abs(m).sum(), (m**2).sum(), (m**4).sum(), e.sum(), (e**2).sum()]
        assert np.allclose(mom[i], ref, rtol=1e-12, atol=1e-12)
    ising.ising_reset_moments(sim.h)
    assert (ising.ising_moments(sim.h) == 0).all()


def test_zero_sweeps_and_empty_handle():
    sim = ising.IsingSim(64, [2.0], 1)
    before = sim.spins(0)
    sim.sweep(0)
    assert np.array_equal(before, sim.spins(0)) and sim.sweeps_done == 0
    empty = ising.IsingSim(64, [], 1)
    assert empty.n == 0
    empty.sweep(5)
    E, M = empty.observables()
    assert E.size == 0 and M.size == 0
    with pytest.raises(ising.IsingError):
        sim.sweep(-1)


def test_temperature_limits_on_gpu():
    cold = ising.IsingSim(128, [0.1], 1, cold=True, trace_cap=20)
    cold.sweep(20)
    E, M = cold.trace(20)
    assert (E == -2 * 128 * 128).all() and (M == 128 * 128).all()
    hot = ising.IsingSim(128, [1e12], 2)
    s0 = hot.spins(0)
    hot.sweep(1)
    assert np.array_equal(hot.spins(0), -s0)


def test_autotune_keeps_state_and_bits(tmp_path, monkeypatch):
    monkeypatch.setenv("ISING_TUNE_CACHE", str(tmp_path / "tune.txt"))
    wl = workloads.random_batch(12, Ls=(64, 128, 256, 1152), seed=31)
    sim = ising.IsingSim(Ls=wl.Ls, temps=wl.temps, seeds=wl.seeds, trace_cap=6)
    sim.sweep(3)
    before = [sim.spins(i) for i in range(sim.n)]
    E0, M0 = sim.observables()
    assert sim.autotune(probe_sweeps=3, force=True) > 0
    assert sim.sweeps_done == 3
    for i in range(sim.n):
        assert np.array_equal(sim.spins(i), before[i])
    assert all(np.array_equal(a, b) for a, b in zip((E0, M0), sim.observables()))
    sim.sweep(6)
    refs = [oracle.init(L, s, i) for i, (L, s) in enumerate(zip(wl.Ls, wl.seeds))]
    Eo, Mo = oracle.sweeps_batch(refs, wl.temps, wl.seeds, list(range(len(refs))), 0, 9, NT)
    Eg, Mg = sim.trace(6)
    assert np.array_equal(Eg, Eo[:, 3:]) and np.array_equal(Mg, Mo[:, 3:])
    for i in range(len(refs)):
        assert np.array_equal(sim.spins(i), refs[i])
    plan = ising.ising_get_plan(sim.h)
    sim2 = ising.IsingSim(Ls=wl.Ls, temps=wl.temps, seeds=wl.seeds)
    assert sim2.autotune(probe_sweeps=3, force=False) == 0.0      # taken from the cache
    assert ising.ising_get_plan(sim2.h)["plan"] == plan["plan"]


@pytest.mark.parametrize("Ls,V,R", [((2048,), 2, 4), ((64, 128, 192, 256, 1024), 1, 3), ((256,) * 12, 4, 2)])
def test_persistent_streaming_kernel_bit_exact(Ls, V, R):
    """All sweeps of a call in one cooperative launch (grid barrier between
    half-sweeps), plain and through a CUDA graph."""
    import torch
    wl = workloads.random_batch(len(Ls), Ls=Ls, seed=len(Ls) + V)
    n = 9
    s = torch.cuda.Stream()
    sims = []
    for graph in (False, True):
        sim = ising.IsingSim(Ls=wl.Ls, temps=wl.temps, seeds=wl.seeds, trace_cap=n, stream=s)
        sim.set_plan(ising.ISING_PLAN_PERSIST, words_per_thread=V, rows_per_item=R)
        sim.set_graph(graph)
        sim.sweep(4)
        sim.sweep(n - 4)
        sims.append(sim)
        assert ising.ising_kernel_launches(sim.h) == 2   # one launch per call
    refs = [oracle.init(L, sd, i) for i, (L, sd) in enumerate(zip(wl.Ls, wl.seeds))]
    Eo, Mo = oracle.sweeps_batch(refs, wl.temps, wl.seeds, list(range(len(refs))), 0, n, NT)
    for sim in sims:
        Eg, Mg = sim.trace(n)
        assert np.array_equal(Eg, Eo) and np.array_equal(Mg, Mo)
        for i in range(len(refs)):
            assert np.array_equal(sim.spins(i), refs[i])
        assert sim.sweeps_done == n
