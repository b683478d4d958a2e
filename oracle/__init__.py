"""CPU oracle for the checkerboard Metropolis Ising sweep.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline arm of ``bench.py`` may import this package.  The product package
(``paper_2404_16990_gb300``) never imports it, and this package never imports
the product package.  The two share no code; only the seeded workload
definitions in ``paper_2404_16990_gb300.workloads`` (which hold none of the
method's arithmetic) serve both sides.

The arithmetic lives in ``ising_oracle.c`` (plain C, one byte per spin, the
definitions of Section 1 and Algorithm 5 written out site by site) and
``cluster_oracle.c`` (the Swendsen-Wang cluster step named in Section 1) and
``ising3d_oracle.c`` (the same sweep on the simple cubic lattice) and
``wolff_oracle.c`` (the Wolff single-cluster step);
this module compiles them with gcc and wraps them with ctypes and numpy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ising_oracle.c")
_SOURCES = ("ising_oracle.c", "cluster_oracle.c", "ising3d_oracle.c", "wolff_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle sources into oracle/liboracle.so (gcc, OpenMP)."""
    srcs = [os.path.join(_HERE, f) for f in _SOURCES]
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(f) for f in srcs)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
           "-Wall", "-Wextra", "-o", tmp, *srcs, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        i8p = ctypes.POINTER(ctypes.c_int8)
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
        lib.oracle_philox4x32_10.restype = None
        lib.oracle_site_random.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                           ctypes.c_uint32, ctypes.c_uint32]
        lib.oracle_site_random.restype = ctypes.c_uint32
        lib.oracle_thresholds.argtypes = [ctypes.c_double, u32p]
        lib.oracle_thresholds.restype = ctypes.c_int
        lib.oracle_init_parallel.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32,
                                             ctypes.c_int, i8p, ctypes.c_int]
        lib.oracle_init_parallel.restype = ctypes.c_int
        lib.oracle_energy.argtypes = [ctypes.c_int, i8p]
        lib.oracle_energy.restype = ctypes.c_int64
        lib.oracle_magnetization.argtypes = [ctypes.c_int, i8p]
        lib.oracle_magnetization.restype = ctypes.c_int64
        lib.oracle_half_sweep.argtypes = [ctypes.c_int, i8p, ctypes.c_int, u32p, ctypes.c_uint64,
                                          ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int]
        lib.oracle_half_sweep.restype = None
        lib.oracle_sweeps.argtypes = [ctypes.c_int, i8p, u32p, ctypes.c_uint64, ctypes.c_uint32,
                                      ctypes.c_uint32, ctypes.c_int64, i64p, i64p, ctypes.c_int]
        lib.oracle_sweeps.restype = None
        lib.oracle_sweeps_batch.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(i8p), u32p,
                                            ctypes.POINTER(ctypes.c_uint64), u32p,
                                            ctypes.c_uint32, ctypes.c_int64, i64p, i64p,
                                            ctypes.c_int]
        lib.oracle_sweeps_batch.restype = None
        lib.oracle_window_init.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32,
                                           ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_int, i8p]
        lib.oracle_window_init.restype = ctypes.c_int
        lib.oracle_window_sweeps.argtypes = [ctypes.c_int, i8p, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_int, u32p, ctypes.c_uint64,
                                             ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int64]
        lib.oracle_window_sweeps.restype = None
        lib.oracle_max_threads.argtypes = []
        lib.oracle_max_threads.restype = ctypes.c_int
        u8p = ctypes.POINTER(ctypes.c_uint8)
        lib.oracle_sw_threshold.argtypes = [ctypes.c_double, u32p]
        lib.oracle_sw_threshold.restype = ctypes.c_int
        lib.oracle_sw_bonds.argtypes = [ctypes.c_int, i8p, ctypes.c_uint64, ctypes.c_uint32,
                                        ctypes.c_uint32, ctypes.c_uint32, u8p]
        lib.oracle_sw_bonds.restype = None
        lib.oracle_sw_labels.argtypes = [ctypes.c_int, u8p, u32p]
        lib.oracle_sw_labels.restype = ctypes.c_int64
        lib.oracle_sw_step.argtypes = [ctypes.c_int, i8p, ctypes.c_uint32, ctypes.c_uint64,
                                       ctypes.c_uint32, ctypes.c_uint32, u8p, u32p]
        lib.oracle_sw_step.restype = ctypes.c_int
        lib.oracle_sw_sweeps.argtypes = [ctypes.c_int, i8p, ctypes.c_uint32, ctypes.c_uint64,
                                         ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int64, i64p, i64p]
        lib.oracle_sw_sweeps.restype = ctypes.c_int
        lib.oracle_sw_sweeps_batch.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                               ctypes.POINTER(i8p), u32p,
                                               ctypes.POINTER(ctypes.c_uint64), u32p,
                                               ctypes.c_uint32, ctypes.c_int64, i64p, i64p,
                                               ctypes.c_int]
        lib.oracle_sw_sweeps_batch.restype = ctypes.c_int
        lib.oracle_wolff_seed.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32]
        lib.oracle_wolff_seed.restype = ctypes.c_uint32
        lib.oracle_wolff_step.argtypes = [ctypes.c_int, i8p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32,
                                          ctypes.c_uint32]
        lib.oracle_wolff_step.restype = ctypes.c_int64
        lib.oracle_wolff_steps.argtypes = [ctypes.c_int, i8p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32,
                                           ctypes.c_uint32, ctypes.c_int64, i64p, i64p, i64p]
        lib.oracle_wolff_steps.restype = ctypes.c_int
        lib.oracle_wolff_steps_batch.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                                 ctypes.POINTER(i8p), u32p, ctypes.POINTER(ctypes.c_uint64),
                                                 u32p, ctypes.c_uint32, ctypes.c_int64, i64p, i64p, ctypes.c_int]
        lib.oracle_wolff_steps_batch.restype = ctypes.c_int
        lib.oracle3d_thresholds.argtypes = [ctypes.c_double, u32p]
        lib.oracle3d_thresholds.restype = ctypes.c_int
        lib.oracle3d_init.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, i8p]
        lib.oracle3d_init.restype = ctypes.c_int
        lib.oracle3d_energy.argtypes = [ctypes.c_int, i8p]
        lib.oracle3d_energy.restype = ctypes.c_int64
        lib.oracle3d_magnetization.argtypes = [ctypes.c_int, i8p]
        lib.oracle3d_magnetization.restype = ctypes.c_int64
        lib.oracle3d_sweeps.argtypes = [ctypes.c_int, i8p, u32p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.c_int64, i64p, i64p]
        lib.oracle3d_sweeps.restype = None
        lib.oracle3d_sweeps_batch.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(i8p), u32p,
                                              ctypes.POINTER(ctypes.c_uint64), u32p, ctypes.c_uint32,
                                              ctypes.c_int64, i64p, i64p, ctypes.c_int]
        lib.oracle3d_sweeps_batch.restype = None
        _lib = lib
        return lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def philox4x32_10(counter, key) -> np.ndarray:
    """One Philox4x32-10 block: counter = 4 u32 words, key = 2 u32 words."""
    c = np.ascontiguousarray(counter, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().oracle_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                                 _ptr(out, ctypes.c_uint32))
    return out


def site_random(seed: int, p: int, t: int, s: int, phase: int) -> int:
    return int(_load().oracle_site_random(seed, p, t, s, phase))


def thresholds(T: float) -> np.ndarray:
    """u32 thresholds [dE=4, dE=8] at temperature T."""
    thr = np.zeros(2, dtype=np.uint32)
    rc = _load().oracle_thresholds(float(T), _ptr(thr, ctypes.c_uint32))
    if rc != 0:
        raise ValueError(f"invalid temperature {T!r}")
    return thr


def init(L: int, seed: int, s: int = 0, cold: bool = False, n_threads: int = 1) -> np.ndarray:
    """Initial L x L lattice of int8 spins (+1/-1)."""
    sigma = np.empty((L, L), dtype=np.int8)
    rc = _load().oracle_init_parallel(L, seed, s, 1 if cold else 0, _ptr(sigma, ctypes.c_int8),
                                      max(1, n_threads))
    if rc != 0:
        raise ValueError(f"invalid L {L}")
    return sigma


def energy(sigma: np.ndarray) -> int:
    sigma = np.ascontiguousarray(sigma, dtype=np.int8)
    return int(_load().oracle_energy(sigma.shape[0], _ptr(sigma, ctypes.c_int8)))


def magnetization(sigma: np.ndarray) -> int:
    sigma = np.ascontiguousarray(sigma, dtype=np.int8)
    return int(_load().oracle_magnetization(sigma.shape[0], _ptr(sigma, ctypes.c_int8)))


def half_sweep(sigma: np.ndarray, colour: int, T: float, seed: int, s: int, t: int,
               n_threads: int = 1) -> None:
    """In place: one half-sweep of colour 0 (black, (x+y) even) or 1 (white)."""
    assert sigma.dtype == np.int8 and sigma.flags.c_contiguous
    thr = thresholds(T)
    _load().oracle_half_sweep(sigma.shape[0], _ptr(sigma, ctypes.c_int8), colour,
                              _ptr(thr, ctypes.c_uint32), seed, s, t, max(1, n_threads))


def sweeps(sigma: np.ndarray, T: float, seed: int, s: int, t0: int, n: int,
           n_threads: int = 1):
    """In place: n sweeps from sweep index t0.  Returns (E trace, M trace)."""
    assert sigma.dtype == np.int8 and sigma.flags.c_contiguous
    thr = thresholds(T)
    E = np.zeros(max(n, 0), dtype=np.int64)
    M = np.zeros(max(n, 0), dtype=np.int64)
    _load().oracle_sweeps(sigma.shape[0], _ptr(sigma, ctypes.c_int8), _ptr(thr, ctypes.c_uint32),
                          seed, s, t0, n, _ptr(E, ctypes.c_int64), _ptr(M, ctypes.c_int64),
                          max(1, n_threads))
    return E, M


def sweeps_batch(sigmas, temps, seeds, sims, t0: int, n: int, n_threads: int = 1):
    """In place over a list of int8 lattices.  Returns traces [n_lat, n]."""
    n_lat = len(sigmas)
    Ls = np.array([s.shape[0] for s in sigmas], dtype=np.int32)
    thr = np.concatenate([thresholds(T) for T in temps]).astype(np.uint32) if n_lat else \
        np.zeros(0, dtype=np.uint32)
    seeds_a = np.array([int(x) for x in seeds], dtype=np.uint64)
    sims_a = np.array([int(x) for x in sims], dtype=np.uint32)
    ptrs = (ctypes.POINTER(ctypes.c_int8) * max(n_lat, 1))()
    for j, s in enumerate(sigmas):
        assert s.dtype == np.int8 and s.flags.c_contiguous
        ptrs[j] = _ptr(s, ctypes.c_int8)
    E = np.zeros((n_lat, max(n, 0)), dtype=np.int64)
    M = np.zeros((n_lat, max(n, 0)), dtype=np.int64)
    _load().oracle_sweeps_batch(n_lat, _ptr(Ls, ctypes.c_int), ptrs, _ptr(thr, ctypes.c_uint32),
                                _ptr(seeds_a, ctypes.c_uint64), _ptr(sims_a, ctypes.c_uint32),
                                t0, n, _ptr(E, ctypes.c_int64), _ptr(M, ctypes.c_int64),
                                max(1, n_threads))
    return E, M


def window_state(L: int, seed: int, s: int, cold: bool, T: float, y: int, x: int,
                 t0: int, n: int) -> int:
    """Exact value of site (x, y) after sweeps t0..t0+n-1 from the initial state
    (t0 must be 0 for the initial state to apply), computed on a light-cone
    window of radius 2n+1 around the site."""
    r = 2 * n + 1
    h = w = 2 * r + 1
    win = np.empty((h, w), dtype=np.int8)
    lib = _load()
    lib.oracle_window_init(L, seed, s, 1 if cold else 0, y - r, x - r, h, w,
                           _ptr(win, ctypes.c_int8))
    thr = thresholds(T)
    lib.oracle_window_sweeps(L, _ptr(win, ctypes.c_int8), y - r, x - r, h, w,
                             _ptr(thr, ctypes.c_uint32), seed, s, t0, n)
    return int(win[r, r])


# --- Swendsen-Wang cluster step (cluster_oracle.c) ---------------------------

def sw_threshold(T: float) -> int:
    """u32 bond threshold floor(2^32 (1 - exp(-2/T))), clamped to 2^32 - 1."""
    thr = np.zeros(1, dtype=np.uint32)
    if _load().oracle_sw_threshold(float(T), _ptr(thr, ctypes.c_uint32)) != 0:
        raise ValueError(f"invalid temperature {T!r}")
    return int(thr[0])


def sw_bonds(sigma: np.ndarray, T: float, seed: int, s: int, t: int) -> np.ndarray:
    """Active bonds of step t: uint8 [L, L], bit 0 = right bond, bit 1 = down."""
    sigma = np.ascontiguousarray(sigma, dtype=np.int8)
    L = sigma.shape[0]
    bonds = np.zeros((L, L), dtype=np.uint8)
    _load().oracle_sw_bonds(L, _ptr(sigma, ctypes.c_int8), seed, t, s, sw_threshold(T),
                            _ptr(bonds, ctypes.c_uint8))
    return bonds


def sw_labels(bonds: np.ndarray):
    """(labels uint32 [L, L] = smallest site index of each site's cluster,
    number of clusters)."""
    bonds = np.ascontiguousarray(bonds, dtype=np.uint8)
    L = bonds.shape[0]
    lab = np.zeros((L, L), dtype=np.uint32)
    n = int(_load().oracle_sw_labels(L, _ptr(bonds, ctypes.c_uint8), _ptr(lab, ctypes.c_uint32)))
    if n < 0:
        raise MemoryError("oracle_sw_labels: allocation failed")
    return lab, n


def sw_sweeps(sigma: np.ndarray, T: float, seed: int, s: int, t0: int, n: int):
    """In place: n Swendsen-Wang steps with indices t0..t0+n-1.  Returns the
    (E, M) traces."""
    assert sigma.dtype == np.int8 and sigma.flags.c_contiguous
    E = np.zeros(max(n, 0), dtype=np.int64)
    M = np.zeros(max(n, 0), dtype=np.int64)
    rc = _load().oracle_sw_sweeps(sigma.shape[0], _ptr(sigma, ctypes.c_int8), sw_threshold(T), seed, s,
                                  t0, n, _ptr(E, ctypes.c_int64), _ptr(M, ctypes.c_int64))
    if rc != 0:
        raise MemoryError("oracle_sw_sweeps: allocation failed")
    return E, M


def sw_sweeps_batch(sigmas, temps, seeds, sims, t0: int, n: int, n_threads: int = 1):
    """In place over a list of int8 lattices.  Returns traces [n_lat, n]."""
    n_lat = len(sigmas)
    Ls = np.array([x.shape[0] for x in sigmas], dtype=np.int32)
    thr = np.array([sw_threshold(T) for T in temps], dtype=np.uint32)
    seeds_a = np.array([int(x) for x in seeds], dtype=np.uint64)
    sims_a = np.array([int(x) for x in sims], dtype=np.uint32)
    ptrs = (ctypes.POINTER(ctypes.c_int8) * max(n_lat, 1))()
    for j, x in enumerate(sigmas):
        assert x.dtype == np.int8 and x.flags.c_contiguous
        ptrs[j] = _ptr(x, ctypes.c_int8)
    E = np.zeros((n_lat, max(n, 0)), dtype=np.int64)
    M = np.zeros((n_lat, max(n, 0)), dtype=np.int64)
    failed = _load().oracle_sw_sweeps_batch(n_lat, _ptr(Ls, ctypes.c_int), ptrs, _ptr(thr, ctypes.c_uint32),
                                            _ptr(seeds_a, ctypes.c_uint64), _ptr(sims_a, ctypes.c_uint32),
                                            t0, n, _ptr(E, ctypes.c_int64), _ptr(M, ctypes.c_int64),
                                            max(1, n_threads))
    if failed:
        raise MemoryError("oracle_sw_sweeps_batch: allocation failed")
    return E, M


# --- three-dimensional sweep (ising3d_oracle.c) ------------------------------

def thresholds3d(T: float) -> np.ndarray:
    """u32 thresholds [dE = 4, 8, 12] at temperature T."""
    thr = np.zeros(3, dtype=np.uint32)
    if _load().oracle3d_thresholds(float(T), _ptr(thr, ctypes.c_uint32)) != 0:
        raise ValueError(f"invalid temperature {T!r}")
    return thr


def init3d(L: int, seed: int, s: int = 0, cold: bool = False) -> np.ndarray:
    sigma = np.empty((L, L, L), dtype=np.int8)          # [z, y, x]
    if _load().oracle3d_init(L, seed, s, 1 if cold else 0, _ptr(sigma, ctypes.c_int8)) != 0:
        raise ValueError(f"invalid L {L}")
    return sigma


def energy3d(sigma: np.ndarray) -> int:
    sigma = np.ascontiguousarray(sigma, dtype=np.int8)
    return int(_load().oracle3d_energy(sigma.shape[0], _ptr(sigma, ctypes.c_int8)))


def magnetization3d(sigma: np.ndarray) -> int:
    sigma = np.ascontiguousarray(sigma, dtype=np.int8)
    return int(_load().oracle3d_magnetization(sigma.shape[0], _ptr(sigma, ctypes.c_int8)))


def wolff_seed(L: int, seed: int, s: int, t: int) -> int:
    """The seed site p = y*L + x of Wolff step t."""
    return int(_load().oracle_wolff_seed(L, seed, s, t))


def wolff_sweeps(sigma: np.ndarray, T: float, seed: int, s: int, t0: int, n: int):
    """In place: n Wolff steps with indices t0..t0+n-1.  Returns the (E, M)
    traces and the cluster sizes."""
    assert sigma.dtype == np.int8 and sigma.flags.c_contiguous
    E = np.zeros(max(n, 0), dtype=np.int64)
    M = np.zeros(max(n, 0), dtype=np.int64)
    C = np.zeros(max(n, 0), dtype=np.int64)
    rc = _load().oracle_wolff_steps(sigma.shape[0], _ptr(sigma, ctypes.c_int8), sw_threshold(T), seed, s, t0, n,
                                    _ptr(E, ctypes.c_int64), _ptr(M, ctypes.c_int64), _ptr(C, ctypes.c_int64))
    if rc != 0:
        raise MemoryError("oracle_wolff_steps: allocation failed")
    return E, M, C


def wolff_sweeps_batch(sigmas, temps, seeds, sims, t0: int, n: int, n_threads: int = 1):
    """In place over a list of int8 lattices.  Returns traces [n_lat, n]."""
    n_lat = len(sigmas)
    Ls = np.array([x.shape[0] for x in sigmas], dtype=np.int32)
    thr = np.array([sw_threshold(T) for T in temps], dtype=np.uint32)
    seeds_a = np.array([int(x) for x in seeds], dtype=np.uint64)
    sims_a = np.array([int(x) for x in sims], dtype=np.uint32)
    ptrs = (ctypes.POINTER(ctypes.c_int8) * max(n_lat, 1))()
    for j, x in enumerate(sigmas):
        assert x.dtype == np.int8 and x.flags.c_contiguous
        ptrs[j] = _ptr(x, ctypes.c_int8)
    E = np.zeros((n_lat, max(n, 0)), dtype=np.int64)
    M = np.zeros((n_lat, max(n, 0)), dtype=np.int64)
    rc = _load().oracle_wolff_steps_batch(n_lat, _ptr(Ls, ctypes.c_int), ptrs, _ptr(thr, ctypes.c_uint32),
                                          _ptr(seeds_a, ctypes.c_uint64), _ptr(sims_a, ctypes.c_uint32), t0, n,
                                          _ptr(E, ctypes.c_int64), _ptr(M, ctypes.c_int64), n_threads)
    if rc != 0:
        raise MemoryError("oracle_wolff_steps_batch: allocation failed")
    return E, M


def sweeps3d(sigma: np.ndarray, T: float, seed: int, s: int, t0: int, n: int):
    """In place: n sweeps of an L^3 lattice [z, y, x] from sweep index t0."""
    assert sigma.dtype == np.int8 and sigma.flags.c_contiguous
    E = np.zeros(max(n, 0), dtype=np.int64)
    M = np.zeros(max(n, 0), dtype=np.int64)
    thr = thresholds3d(T)
    _load().oracle3d_sweeps(sigma.shape[0], _ptr(sigma, ctypes.c_int8), _ptr(thr, ctypes.c_uint32), seed, s, t0, n,
                            _ptr(E, ctypes.c_int64), _ptr(M, ctypes.c_int64))
    return E, M


def sweeps3d_batch(sigmas, temps, seeds, sims, t0: int, n: int, n_threads: int = 1):
    n_lat = len(sigmas)
    Ls = np.array([x.shape[0] for x in sigmas], dtype=np.int32)
    thr = np.concatenate([thresholds3d(T) for T in temps]).astype(np.uint32) if n_lat else np.zeros(0, np.uint32)
    seeds_a = np.array([int(x) for x in seeds], dtype=np.uint64)
    sims_a = np.array([int(x) for x in sims], dtype=np.uint32)
    ptrs = (ctypes.POINTER(ctypes.c_int8) * max(n_lat, 1))()
    for j, x in enumerate(sigmas):
        assert x.dtype == np.int8 and x.flags.c_contiguous
        ptrs[j] = _ptr(x, ctypes.c_int8)
    E = np.zeros((n_lat, max(n, 0)), dtype=np.int64)
    M = np.zeros((n_lat, max(n, 0)), dtype=np.int64)
    _load().oracle3d_sweeps_batch(n_lat, _ptr(Ls, ctypes.c_int), ptrs, _ptr(thr, ctypes.c_uint32),
                                  _ptr(seeds_a, ctypes.c_uint64), _ptr(sims_a, ctypes.c_uint32), t0, n,
                                  _ptr(E, ctypes.c_int64), _ptr(M, ctypes.c_int64), max(1, n_threads))
    return E, M


class use_library:
    """Context manager: route every wrapper above through another build of the
    oracle source (used by the tests that plant mistakes in a copy of
    ising_oracle.c and check that the pins catch them)."""

    def __init__(self, so_path: str):
        self.so_path = so_path
        self._saved = None

    def __enter__(self):
        global _lib
        _load()
        with _lock:
            self._saved = _lib
            _lib = None
        saved_path = globals()["_LIB_PATH"]
        globals()["_LIB_PATH"] = self.so_path
        try:
            _load_no_build()
        finally:
            globals()["_LIB_PATH"] = saved_path
        return self

    def __exit__(self, *exc):
        global _lib
        with _lock:
            _lib = self._saved
        return False


def _load_no_build():
    global _lib
    saved_build = globals()["build"]
    globals()["build"] = lambda force=False: _LIB_PATH
    try:
        _load()
    finally:
        globals()["build"] = saved_build


def compile_variant(src_text: str, out_dir: str, name: str, which: str = "ising_oracle.c") -> str:
    """Compile the oracle with a (modified) copy of source file `which` and
    the other sources unchanged into out_dir/name.so."""
    assert which in _SOURCES
    srcs = []
    for f in _SOURCES:
        path = os.path.join(out_dir, f"{name}_{f}")
        with open(path, "w") as fh:
            fh.write(src_text if f == which else source_text(f))
        srcs.append(path)
    so = os.path.join(out_dir, name + ".so")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                           "-o", so, *srcs, "-lm"])
    return so


def source_text(which: str = "ising_oracle.c") -> str:
    assert which in _SOURCES
    with open(os.path.join(_HERE, which)) as f:
        return f.read()
