"""GPU parity of the Swendsen-Wang cluster step (through the C ABI) against
the CPU oracle: bond thresholds, cluster labels (the unique partition with
minimum-index roots), whole steps bit for bit on uneven batches, steps mixed
with Metropolis sweeps, graph replay, lattices whose clusters span many tiles
(up to 4096^2 in full), sampled sites of 16384^2 and 32768^2 lattices, the
T -> 0 / T -> inf limits, and the API's errors; and the same for the Wolff
single-cluster step (uneven batches, cold and random starts, steps mixed with
sweeps and Swendsen-Wang steps, a 2048^2 lattice at T_c, the limits)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import stats as ostats
from paper_2404_16990_gb300 import ising, workloads

pytestmark = pytest.mark.gpu

TC = workloads.T_CRITICAL


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def _oracle_start(L, seed, s, cold):
    return np.ones((L, L), np.int8) if cold else oracle.init(L, seed, s)


def test_sw_thresholds_match_oracle():
    temps = [0.01, 0.5, 1.5, TC, 3.0, 7.5, 1e3, 1e9]
    sim = ising.IsingSim(64, temps, 3)
    assert list(sim.sw_thresholds()) == [oracle.sw_threshold(T) for T in temps]
    sim.close()


@pytest.mark.parametrize("L,T,pre", [(64, TC, 0), (128, 1.5, 0), (320, 3.0, 2), (1024, TC, 5), (1024, 0.8, 1),
                                     (2048, 2.4, 0)])
def test_sw_labels_match_oracle(L, T, pre):
    seed = 1000 + L
    sim = ising.IsingSim(L, [T, T], seed)
    sim.sweep(pre)
    for s in (0, 1):
        sigma = sim.spins(s)
        bonds = oracle.sw_bonds(sigma, T, seed, s, pre)
        ref, _ = oracle.sw_labels(bonds)
        got = sim.sw_labels(s)
        assert np.array_equal(got, ref), (L, T, s)
    assert sim.sweeps_done == pre          # labels alone take no step
    sim.close()


def test_sw_steps_bit_exact_uneven_batch():
    Ls = [64, 128, 64, 256, 192, 64, 320]
    temps = [TC, 1.5, 0.5, 3.0, TC, 1e3, 2.1]
    seeds = [11, 12, 13, 14, 15, 16, 17]
    n = 12
    for cold in (False, True):
        sim = ising.IsingSim(Ls=Ls, temps=temps, seeds=seeds, cold=cold, trace_cap=n)
        sim.sw_sweep(n)
        Eg, Mg = sim.trace(n)
        for i, (L, T, sd) in enumerate(zip(Ls, temps, seeds)):
            ref = _oracle_start(L, sd, i, cold)
            Eo, Mo = oracle.sw_sweeps(ref, T, sd, i, 0, n)
            assert np.array_equal(sim.spins(i), ref), (i, L, T, cold)
            assert np.array_equal(Eg[i], Eo) and np.array_equal(Mg[i], Mo), (i, L, T, cold)
        assert sim.sweeps_done == n
        sim.close()


def test_sw_mixed_with_metropolis_sweeps():
    L, T, seed = 256, TC, 77
    sim = ising.IsingSim(L, [T], seed, trace_cap=16)
    ref = oracle.init(L, seed, 0)
    t = 0
    for kind, k in (("mp", 2), ("sw", 3), ("mp", 1), ("sw", 2), ("sw", 1), ("mp", 3)):
        if kind == "mp":
            sim.sweep(k)
            Eo, Mo = oracle.sweeps(ref, T, seed, 0, t, k)
        else:
            sim.sw_sweep(k)
            Eo, Mo = oracle.sw_sweeps(ref, T, seed, 0, t, k)
        t += k
        Eg, Mg = sim.trace(k)
        assert np.array_equal(Eg[0], Eo) and np.array_equal(Mg[0], Mo), (kind, t)
        assert np.array_equal(sim.spins(0), ref), (kind, t)
    sim.close()


def test_sw_graph_replay_matches_direct_launches():
    import torch
    Ls, temps, seeds = [128, 256, 64], [TC, 2.0, 2.6], [5, 6, 7]
    s = torch.cuda.Stream()
    a = ising.IsingSim(Ls=Ls, temps=temps, seeds=seeds, trace_cap=20, stream=s)
    b = ising.IsingSim(Ls=Ls, temps=temps, seeds=seeds, trace_cap=20, stream=s)
    b.set_graph(True)
    for _ in range(4):
        a.sw_sweep(5)
        b.sw_sweep(5)
    torch.cuda.synchronize()
    for i in range(3):
        assert np.array_equal(a.spins(i), b.spins(i))
    Ea, Ma = a.trace(20)
    Eb, Mb = b.trace(20)
    assert np.array_equal(Ea, Eb) and np.array_equal(Ma, Mb)
    a.close()
    b.close()


@pytest.mark.parametrize("L,T,n", [(2048, TC, 3), (4096, TC, 2), (4096, 2.0, 1)])
def test_sw_large_lattices_bit_exact(L, T, n):
    """Clusters at and below T_c percolate across hundreds of tiles."""
    seed = 31 + L
    sim = ising.IsingSim(L, [T], seed, trace_cap=n)
    ref = oracle.init(L, seed, 0, n_threads=8)
    sim.sw_sweep(n)
    Eo, Mo = oracle.sw_sweeps(ref, T, seed, 0, 0, n)
    Eg, Mg = sim.trace(n)
    assert np.array_equal(Eg[0], Eo) and np.array_equal(Mg[0], Mo)
    assert np.array_equal(sim.spins(0), ref)
    sim.close()


def _coin(seed, p, t, s):
    return oracle.site_random(seed, p, t, s, 8) >> 31


@pytest.mark.parametrize("L", [16384, 32768])
def test_sw_maximum_sizes_limits(L):
    """T -> inf (bond threshold 0: no bonds): every site flips by its own
    coin, checked on sampled sites; T -> 0 from a cold start: one cluster,
    all spins equal."""
    import torch
    seed = 4 + L
    assert oracle.sw_threshold(1e12) == 0
    sim = ising.IsingSim(L, [1e12, 0.01], seed, cold=True, trace_cap=3)
    sim.sw_sweep(2)
    Eg, Mg = sim.trace(2)
    N = L * L
    assert np.all(Eg[1] == -2 * N) and np.all(np.abs(Mg[1]) == N)
    words = sim.words(0).cpu().numpy().view(np.uint32)
    wn = L // 64
    rng = np.random.default_rng(L)
    for _ in range(400):
        y, x = int(rng.integers(L)), int(rng.integers(L))
        p = y * L + x
        expect = -1 if (_coin(seed, p, 0, 0) ^ _coin(seed, p, 1, 0)) else 1
        c, j = (x + y) & 1, x >> 1
        bit = (int(words[(c * L + y) * wn + j // 32]) >> (j % 32)) & 1
        assert (-1 if bit else 1) == expect, (y, x)
    # E, M of the T -> inf lattice from its own words (the trace entry)
    table = np.array([bin(v).count("1") for v in range(256)], dtype=np.uint8)
    spins_pop = int(np.take(table, words.view(np.uint8)).sum(dtype=np.int64))
    assert Mg[0][1] == N - 2 * spins_pop
    del words
    sim.close()
    torch.cuda.empty_cache()


def test_sw_autocorrelation_collapses_at_tc():
    """Physics through the GPU path: tau_int(|M|) per step at T_c is O(1)."""
    L, n = 128, 4000
    sim = ising.IsingSim(L, [TC] * 4, 9, trace_cap=n)
    sim.sw_sweep(200)
    sim.sw_sweep(n)
    _, M = sim.trace(n)
    taus = [ostats.tau_int(np.abs(M[i]).astype(np.float64))[0] for i in range(4)]
    assert max(taus) < 15.0, taus
    sim.close()


def test_sw_errors():
    import torch
    sim = ising.IsingSim(128, [TC], 1)
    need = ising.ising_sw_scratch_bytes(sim.h)
    assert need >= 128 * 128 * 4
    small = torch.empty(need - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(ising.IsingError) as e:
        ising.ising_sw_sweep(sim.h, 1, small.data_ptr(), small.numel())
    assert e.value.code == ising.ISING_ENOMEM
    big = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(ising.IsingError) as e:
        ising.ising_sw_sweep(sim.h, 1, big.data_ptr() + 16, need)
    assert e.value.code == ising.ISING_EINVAL
    with pytest.raises(ising.IsingError) as e:
        ising.ising_sw_sweep(sim.h, -1, big.data_ptr(), need)
    assert e.value.code == ising.ISING_EINVAL
    with pytest.raises(ising.IsingError) as e:
        ising.ising_sw_labels(sim.h, 3, big.data_ptr(), need)
    assert e.value.code == ising.ISING_EINVAL
    ising.ising_sw_sweep(sim.h, 0, big.data_ptr(), need)       # no-op
    assert sim.sweeps_done == 0
    sim.close()
    huge = ising.IsingSim(65536, [TC], 1, cold=True)
    with pytest.raises(ising.IsingError) as e:
        ising.ising_sw_scratch_bytes(huge.h)
    assert e.value.code == ising.ISING_EINVAL
    huge.close()


# --------------------------------------------------------------------------
# Wolff single-cluster step
# --------------------------------------------------------------------------
WOLFF_METHODS = [ising.ISING_WOLFF_GROWTH, ising.ISING_WOLFF_LABELS]


@pytest.mark.parametrize("method", WOLFF_METHODS)
def test_wolff_steps_bit_exact_uneven_batch(method):
    Ls = [64, 128, 64, 256, 192, 64, 320]
    temps = [TC, 1.5, 0.5, 3.0, TC, 1e3, 2.1]
    seeds = [21, 22, 23, 24, 25, 26, 27]
    n = 25
    for cold in (False, True):
        sim = ising.IsingSim(Ls=Ls, temps=temps, seeds=seeds, cold=cold, trace_cap=n)
        ising.ising_wolff_set_method(sim.h, method)
        sim.wolff_sweep(n)
        Eg, Mg = sim.trace(n)
        for i, (L, T, sd) in enumerate(zip(Ls, temps, seeds)):
            ref = _oracle_start(L, sd, i, cold)
            Eo, Mo, _ = oracle.wolff_sweeps(ref, T, sd, i, 0, n)
            assert np.array_equal(sim.spins(i), ref), (i, L, T, cold)
            assert np.array_equal(Eg[i], Eo) and np.array_equal(Mg[i], Mo), (i, L, T, cold)
        assert sim.sweeps_done == n
        sim.close()


@pytest.mark.parametrize("method", WOLFF_METHODS + [ising.ISING_WOLFF_AUTO])
def test_wolff_mixed_with_sweeps_and_sw_steps(method):
    L, T, seed = 256, TC, 78
    sim = ising.IsingSim(L, [T], seed, trace_cap=16)
    ising.ising_wolff_set_method(sim.h, method)
    ref = oracle.init(L, seed, 0)
    t = 0
    for kind, k in (("mp", 2), ("wolff", 4), ("sw", 2), ("wolff", 3), ("mp", 1), ("wolff", 1)):
        if kind == "mp":
            sim.sweep(k)
            Eo, Mo = oracle.sweeps(ref, T, seed, 0, t, k)
        elif kind == "sw":
            sim.sw_sweep(k)
            Eo, Mo = oracle.sw_sweeps(ref, T, seed, 0, t, k)
        else:
            sim.wolff_sweep(k)
            Eo, Mo, _ = oracle.wolff_sweeps(ref, T, seed, 0, t, k)
        t += k
        Eg, Mg = sim.trace(k)
        assert np.array_equal(Eg[0], Eo) and np.array_equal(Mg[0], Mo), (kind, t)
        assert np.array_equal(sim.spins(0), ref), (kind, t)
    sim.close()


@pytest.mark.parametrize("method", WOLFF_METHODS)
def test_wolff_2048_at_tc_bit_exact(method):
    L, T, seed, n = 2048, TC, 5, 6
    sim = ising.IsingSim(L, [T], seed, trace_cap=n)
    ising.ising_wolff_set_method(sim.h, method)
    sim.sweep(20)
    ref = sim.spins(0)
    sim.wolff_sweep(n)
    Eo, Mo, C = oracle.wolff_sweeps(ref, T, seed, 0, 20, n)
    Eg, Mg = sim.trace(n)
    assert np.array_equal(sim.spins(0), ref)
    assert np.array_equal(Eg[0], Eo) and np.array_equal(Mg[0], Mo)
    assert C.max() > 1


@pytest.mark.parametrize("method", WOLFF_METHODS)
def test_wolff_limits(method):
    # T -> 0 from a cold start: the whole lattice every step; T -> inf: one site
    L = 128
    sim = ising.IsingSim(L, [0.01, 1e9], 3, cold=True, trace_cap=4)
    ising.ising_wolff_set_method(sim.h, method)
    sim.wolff_sweep(4)
    E, M = sim.trace(4)
    assert list(M[0]) == [-(L * L), L * L, -(L * L), L * L]
    assert np.all(E[0] == -2 * L * L)
    dM = np.diff(np.concatenate([[L * L], M[1]]))
    assert set(np.abs(dM).tolist()) == {2}              # one site per step
    assert np.count_nonzero(sim.spins(1) == -1) <= 4
    sim.close()


def test_wolff_labelling_at_4096_tc_and_graph_replay():
    """One large lattice at T_c, where a cluster spans much of it: labelling
    (all SMs) and growth (one block) give the same steps; graph replay of
    the labelling path gives the same as direct launches."""
    import torch
    L, T, seed, n = 4096, TC, 12, 3
    s = torch.cuda.Stream()
    a = ising.IsingSim(L, [T], seed, trace_cap=n, stream=s)
    b = ising.IsingSim(L, [T], seed, trace_cap=n, stream=s)
    ising.ising_wolff_set_method(a.h, ising.ISING_WOLFF_LABELS)
    ising.ising_wolff_set_method(b.h, ising.ISING_WOLFF_GROWTH)
    a.set_graph(True)
    a.wolff_sweep(1)
    a.wolff_sweep(2)
    b.wolff_sweep(3)
    torch.cuda.synchronize()
    assert np.array_equal(a.spins(0), b.spins(0))
    Ea, Ma = a.trace(n)
    Eb, Mb = b.trace(n)
    assert np.array_equal(Ea, Eb) and np.array_equal(Ma, Mb)
    assert np.abs(np.diff(Ma[0])).max() > 2                              # clusters of more than one site
    a.close()
    b.close()


def test_wolff_scratch_errors():
    sim = ising.IsingSim(64, [TC], 1)
    with pytest.raises(ising.IsingError) as e:
        ising.ising_wolff_set_method(sim.h, 3)
    assert e.value.code == ising.ISING_EINVAL
    with pytest.raises(ising.IsingError):
        ising.ising_wolff_sweep(sim.h, 1, 0, 0)          # no scratch
    with pytest.raises(ising.IsingError):
        sim.wolff_sweep(-1)
    sim.close()

