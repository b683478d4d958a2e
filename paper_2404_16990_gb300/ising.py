"""ctypes binding of libising (include/ising.h): the same names, argument
marshalling only.  Every step of the simulation runs in the CUDA library; this
module converts numpy/torch arguments to pointers and error codes to
exceptions.  There is no CPU fallback: if libising.so cannot be built or
loaded, every call raises.

``IsingSim`` is a small convenience owner: it allocates the device workspace
as a torch uint8 tensor on the current CUDA device and keeps it alive with the
handle.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import numpy as np

from . import build as _build

ISING_OK = 0
ISING_EINVAL = -1
ISING_ENOMEM = -2
ISING_ECUDA = -3
ISING_ETIMEOUT = -4
ISING_ESTATE = -5
ISING_INIT_RANDOM = 0
ISING_INIT_COLD = 1
ISING_PLAN_AUTO = 0
ISING_PLAN_RESIDENT = 1
ISING_PLAN_STREAM = 2
ISING_PLAN_PERSIST = 3
ISING_PLAN_MIXED = 4
ISING_PLAN_CLUSTER = 5
ISING_CLUSTER_MAX_L = 1024
ISING_MIN_L = 64
ISING_MAX_L = 65536

_lock = threading.Lock()
_lib = None


class IsingError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"ising error {code}: {msg}")
        self.code = code


def library_path() -> str:
    return _build.LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build()  # no-op when up to date; raises if nvcc fails
        lib = ctypes.CDLL(path)
        vp, i64, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_size_t
        i64p = ctypes.POINTER(ctypes.c_int64)
        sig = {
            "ising_last_error": ([], ctypes.c_char_p),
            "ising_version": ([], ctypes.c_char_p),
            "ising_workspace_bytes": ([ctypes.c_int, ctypes.c_int, i64, ctypes.POINTER(sz)], ctypes.c_int),
            "ising_batch_workspace_bytes": ([ctypes.c_int, ctypes.POINTER(ctypes.c_int), i64,
                                             ctypes.POINTER(sz)], ctypes.c_int),
            "ising_create": ([ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                              ctypes.c_uint64, ctypes.c_int, i64, vp, sz, vp], ctypes.c_int),
            "ising_create_batch": ([ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64),
                                    ctypes.c_int, i64, vp, sz, vp], ctypes.c_int),
            "ising_sweep": ([vp, i64], ctypes.c_int),
            "ising_sweeps_done": ([vp], i64),
            "ising_kernel_launches": ([vp], i64),
            "ising_observables": ([vp, i64p, i64p], ctypes.c_int),
            "ising_trace": ([vp, i64p, i64p, i64, i64p], ctypes.c_int),
            "ising_get_spins": ([vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int8)], ctypes.c_int),
            "ising_set_spins": ([vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int8)], ctypes.c_int),
            "ising_get_thresholds": ([vp, ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int),
            "ising_lattice_words": ([vp, ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(sz)], ctypes.c_int),
            "ising_lattice_size": ([vp, ctypes.c_int], ctypes.c_int),
            "ising_num_sims": ([vp], ctypes.c_int),
            "ising_set_measure": ([vp, ctypes.c_int], ctypes.c_int),
            "ising_set_wait_limit_ns": ([vp, ctypes.c_uint64], ctypes.c_int),
            "ising_reset_moments": ([vp], ctypes.c_int),
            "ising_moments": ([vp, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
            "ising_state_bytes": ([vp, ctypes.POINTER(sz)], ctypes.c_int),
            "ising_save": ([vp, vp, sz], ctypes.c_int),
            "ising_load": ([vp, vp, sz], ctypes.c_int),
            "ising_set_plan": ([vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int],
                               ctypes.c_int),
            "ising_set_graph": ([vp, ctypes.c_int], ctypes.c_int),
            "ising_autotune": ([vp, i64, ctypes.c_int, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
            "ising_get_plan": ([vp] + [ctypes.POINTER(ctypes.c_int)] * 5, ctypes.c_int),
            "ising_destroy": ([vp], None),
            "ising_sweep_noalloc": ([vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_uint64), i64, i64, vp, vp], ctypes.c_int),
            "ising_net_workspace_bytes": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(sz)], ctypes.c_int),
            "ising_net_create": ([ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, sz, vp],
                                 ctypes.c_int),
            "ising_net_destroy": ([vp], None),
            "ising_net_set_params": ([vp, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
            "ising_net_get_params": ([vp, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
            "ising_net_score": ([vp, ctypes.POINTER(ctypes.c_int8), ctypes.c_int, ctypes.POINTER(ctypes.c_float),
                                 ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
            "ising_net_sample": ([vp, ctypes.POINTER(ctypes.c_int8), ctypes.c_int, ctypes.POINTER(ctypes.c_uint32),
                                  ctypes.c_uint32, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
            "ising_net_grad": ([vp, ctypes.POINTER(ctypes.c_int8), ctypes.c_int, ctypes.POINTER(ctypes.c_float),
                                ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
            "ising_net_train": ([vp, vp, ctypes.c_int, ctypes.c_int, i64, ctypes.c_int, ctypes.c_float,
                                 ctypes.c_uint64, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
            "ising_learned_round": ([vp, vp, i64, i64p], ctypes.c_int),
            "ising_net_train_windows": ([vp, vp, ctypes.c_int, ctypes.c_int, i64, ctypes.c_int, ctypes.c_uint64,
                                         ctypes.POINTER(ctypes.c_int8)], ctypes.c_int),
            "ising_net_apply_grad": ([vp, ctypes.POINTER(ctypes.c_float), ctypes.c_float], ctypes.c_int),
            "ising_snapshot": ([vp, vp, sz], ctypes.c_int),
            "ising_net_accepted": ([vp, i64p, ctypes.c_int, ctypes.c_int], ctypes.c_int),
            "ising_net_set_precision": ([vp, ctypes.c_int], ctypes.c_int),
            "ising_binder": ([ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.POINTER(ctypes.c_double)],
                             ctypes.c_int),
            "ising_tau_int": ([ctypes.POINTER(ctypes.c_double), i64, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double), i64p], ctypes.c_int),
            "ising_stat_inefficiency": ([ctypes.POINTER(ctypes.c_double), i64, ctypes.POINTER(ctypes.c_double)],
                                        ctypes.c_int),
            "ising_equilibration": ([ctypes.POINTER(ctypes.c_double), i64, i64, i64p, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
            "ising_random_stream": ([ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64,
                                     ctypes.c_uint32, ctypes.c_uint32, vp, vp], ctypes.c_int),
            "ising_prng_battery": ([ctypes.POINTER(ctypes.c_uint32), i64, ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
            "ising3d_workspace_bytes": ([ctypes.c_int, ctypes.POINTER(ctypes.c_int), i64, ctypes.POINTER(sz)], ctypes.c_int),
            "ising3d_create": ([ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64), ctypes.c_int, i64,
                                vp, sz, vp], ctypes.c_int),
            "ising3d_sweep": ([vp, i64], ctypes.c_int),
            "ising3d_set_graph": ([vp, ctypes.c_int], ctypes.c_int),
            "ising3d_sweeps_done": ([vp], i64),
            "ising3d_kernel_launches": ([vp], i64),
            "ising3d_observables": ([vp, i64p, i64p], ctypes.c_int),
            "ising3d_trace": ([vp, i64p, i64p, i64, i64p], ctypes.c_int),
            "ising3d_get_spins": ([vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int8)], ctypes.c_int),
            "ising3d_destroy": ([vp], None),
            "ising_sw_scratch_bytes": ([vp, ctypes.POINTER(sz)], ctypes.c_int),
            "ising_sw_get_thresholds": ([vp, ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int),
            "ising_sw_sweep": ([vp, i64, vp, sz], ctypes.c_int),
            "ising_wolff_set_method": ([vp, ctypes.c_int], ctypes.c_int),
            "ising_wolff_sweep": ([vp, i64, vp, sz], ctypes.c_int),
            "ising_sw_labels": ([vp, ctypes.c_int, vp, sz, ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def ising_last_error() -> str:
    return _load().ising_last_error().decode()


def ising_version() -> str:
    return _load().ising_version().decode()


def _check(rc: int):
    if rc != ISING_OK:
        raise IsingError(rc, ising_last_error())


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def ising_workspace_bytes(L: int, n_sims: int, trace_cap: int = 0) -> int:
    out = ctypes.c_size_t(0)
    _check(_load().ising_workspace_bytes(L, n_sims, trace_cap, ctypes.byref(out)))
    return out.value


def ising_batch_workspace_bytes(Ls: Sequence[int], trace_cap: int = 0) -> int:
    La = np.ascontiguousarray(Ls, dtype=np.int32)
    out = ctypes.c_size_t(0)
    _check(_load().ising_batch_workspace_bytes(len(La), _ptr(La, ctypes.c_int), trace_cap, ctypes.byref(out)))
    return out.value


def ising_create(L: int, n_sims: int, temps: Sequence[float], seed: int, init: int, trace_cap: int,
                 dev_workspace: int, ws_bytes: int, cuda_stream: int = 0) -> ctypes.c_void_p:
    T = np.ascontiguousarray(temps, dtype=np.float64)
    h = ctypes.c_void_p()
    _check(_load().ising_create(ctypes.byref(h), L, n_sims, _ptr(T, ctypes.c_double), seed, init, trace_cap,
                                dev_workspace, ws_bytes, cuda_stream))
    return h


def ising_create_batch(Ls: Sequence[int], temps: Sequence[float], seeds: Sequence[int], init: int,
                       trace_cap: int, dev_workspace: int, ws_bytes: int,
                       cuda_stream: int = 0) -> ctypes.c_void_p:
    La = np.ascontiguousarray(Ls, dtype=np.int32)
    T = np.ascontiguousarray(temps, dtype=np.float64)
    S = np.ascontiguousarray([int(s) for s in seeds], dtype=np.uint64)
    h = ctypes.c_void_p()
    _check(_load().ising_create_batch(ctypes.byref(h), len(La), _ptr(La, ctypes.c_int), _ptr(T, ctypes.c_double),
                                      _ptr(S, ctypes.c_uint64), init, trace_cap, dev_workspace, ws_bytes,
                                      cuda_stream))
    return h


def ising_sweep(h, n: int) -> None:
    _check(_load().ising_sweep(h, n))


def ising_sweeps_done(h) -> int:
    return int(_load().ising_sweeps_done(h))


def ising_kernel_launches(h) -> int:
    return int(_load().ising_kernel_launches(h))


def ising_load_from(h, host_ptr: int, nbytes: int) -> None:
    """ising_load from a raw host address (e.g. a pinned torch tensor)."""
    _check(_load().ising_load(h, host_ptr, nbytes))


def ising_save_to(h, host_ptr: int, nbytes: int) -> None:
    _check(_load().ising_save(h, host_ptr, nbytes))


def ising_num_sims(h) -> int:
    return int(_load().ising_num_sims(h))


def ising_lattice_size(h, sim: int) -> int:
    return int(_load().ising_lattice_size(h, sim))


def ising_observables(h):
    n = ising_num_sims(h)
    E = np.zeros(n, dtype=np.int64)
    M = np.zeros(n, dtype=np.int64)
    _check(_load().ising_observables(h, _ptr(E, ctypes.c_int64), _ptr(M, ctypes.c_int64)))
    return E, M


def ising_trace(h, max_sweeps: int):
    n = ising_num_sims(h)
    cap = max(0, int(max_sweeps))
    E = np.zeros(max(1, n * cap), dtype=np.int64)
    M = np.zeros(max(1, n * cap), dtype=np.int64)
    k = ctypes.c_int64(0)
    _check(_load().ising_trace(h, _ptr(E, ctypes.c_int64), _ptr(M, ctypes.c_int64), cap, ctypes.byref(k)))
    k = k.value
    return E[: n * k].reshape(n, k), M[: n * k].reshape(n, k)


def ising_get_spins(h, sim: int) -> np.ndarray:
    L = ising_lattice_size(h, sim)
    if L <= 0:
        raise IsingError(ISING_EINVAL, f"sim {sim} out of range")
    out = np.empty((L, L), dtype=np.int8)
    _check(_load().ising_get_spins(h, sim, _ptr(out, ctypes.c_int8)))
    return out


def ising_set_spins(h, sim: int, spins: np.ndarray) -> None:
    a = np.ascontiguousarray(spins, dtype=np.int8)
    L = ising_lattice_size(h, sim)
    if a.shape != (L, L):
        raise IsingError(ISING_EINVAL, f"spins must have shape ({L}, {L})")
    _check(_load().ising_set_spins(h, sim, _ptr(a, ctypes.c_int8)))


def ising_lattice_words(h, sim: int):
    """(device address, number of 32-bit words) of lattice sim's packed spins."""
    p = ctypes.c_void_p()
    n = ctypes.c_size_t(0)
    _check(_load().ising_lattice_words(h, sim, ctypes.byref(p), ctypes.byref(n)))
    return int(p.value or 0), n.value


def ising_get_thresholds(h) -> np.ndarray:
    n = ising_num_sims(h)
    out = np.zeros(max(1, 2 * n), dtype=np.uint32)
    _check(_load().ising_get_thresholds(h, _ptr(out, ctypes.c_uint32)))
    return out[: 2 * n].reshape(n, 2)


def ising_set_measure(h, on: bool) -> None:
    _check(_load().ising_set_measure(h, 1 if on else 0))


ISING_MAX_WAIT_LIMIT_NS = 600_000_000_000


def ising_set_wait_limit_ns(h, ns: int) -> None:
    _check(_load().ising_set_wait_limit_ns(h, int(ns)))


def ising_reset_moments(h) -> None:
    _check(_load().ising_reset_moments(h))


def ising_moments(h) -> np.ndarray:
    n = ising_num_sims(h)
    out = np.zeros(max(1, 6 * n), dtype=np.float64)
    _check(_load().ising_moments(h, _ptr(out, ctypes.c_double)))
    return out[: 6 * n].reshape(n, 6)


def ising_state_bytes(h) -> int:
    out = ctypes.c_size_t(0)
    _check(_load().ising_state_bytes(h, ctypes.byref(out)))
    return out.value


def ising_save(h) -> bytes:
    n = ising_state_bytes(h)
    buf = ctypes.create_string_buffer(n)
    _check(_load().ising_save(h, ctypes.cast(buf, ctypes.c_void_p), n))
    return buf.raw


def ising_load(h, state: bytes) -> None:
    buf = ctypes.create_string_buffer(state, len(state))
    _check(_load().ising_load(h, ctypes.cast(buf, ctypes.c_void_p), len(state)))


def ising_set_plan(h, plan: int, words_per_thread: int = 0, rows_per_item: int = 0, sweeps_per_unit: int = 0,
                   threads: int = 0) -> None:
    _check(_load().ising_set_plan(h, plan, words_per_thread, rows_per_item, sweeps_per_unit, threads))


def ising_autotune(h, probe_sweeps: int = 10, force: bool = False) -> float:
    best = ctypes.c_double(0)
    _check(_load().ising_autotune(h, probe_sweeps, 1 if force else 0, ctypes.byref(best)))
    return best.value


def ising_get_plan(h) -> dict:
    v = [ctypes.c_int(0) for _ in range(5)]
    _check(_load().ising_get_plan(h, *[ctypes.byref(x) for x in v]))
    return dict(zip(["plan", "words_per_thread", "rows_per_item", "sweeps_per_unit", "threads"], [x.value for x in v]))


def ising_set_graph(h, on: bool) -> None:
    _check(_load().ising_set_graph(h, 1 if on else 0))


def ising_destroy(h) -> None:
    if h:
        _load().ising_destroy(h)


ISING_NOALLOC_MAX_LATTICES = 64


def ising_sweep_noalloc(dev_words: int, Ls: Sequence[int], temps: Sequence[float], seeds: Sequence[int],
                        t0: int, n: int, dev_EM: int, cuda_stream: int = 0) -> None:
    """Allocation-free sweep of packed lattices held by the caller (device
    addresses dev_words and dev_EM); see ising_sweep_noalloc in ising.h."""
    La = np.ascontiguousarray(Ls, dtype=np.int32)
    T = np.ascontiguousarray(temps, dtype=np.float64)
    S = np.ascontiguousarray([int(s) for s in seeds], dtype=np.uint64)
    if not (len(La) == len(T) == len(S)):
        raise ValueError(f"Ls, temps and seeds must have the same length ({len(La)}, {len(T)}, {len(S)})")
    _check(_load().ising_sweep_noalloc(dev_words, len(La), _ptr(La, ctypes.c_int), _ptr(T, ctypes.c_double),
                                       _ptr(S, ctypes.c_uint64), t0, n, dev_EM, cuda_stream))


def ising_binder(moments: np.ndarray) -> np.ndarray:
    m = np.ascontiguousarray(moments, dtype=np.float64).reshape(-1, 6)
    U = np.zeros(max(1, len(m)), dtype=np.float64)
    _check(_load().ising_binder(_ptr(m, ctypes.c_double), len(m), _ptr(U, ctypes.c_double)))
    return U[: len(m)]


def ising_tau_int(x, c: float = 6.0):
    """(tau_int, error, window) of a 1-D series (Madras-Sokal automatic window)."""
    a = np.ascontiguousarray(x, dtype=np.float64)
    tau, err, w = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_int64(0)
    _check(_load().ising_tau_int(_ptr(a, ctypes.c_double), len(a), c, ctypes.byref(tau), ctypes.byref(err),
                                 ctypes.byref(w)))
    return tau.value, err.value, w.value


def ising_stat_inefficiency(x) -> float:
    a = np.ascontiguousarray(x, dtype=np.float64)
    g = ctypes.c_double()
    _check(_load().ising_stat_inefficiency(_ptr(a, ctypes.c_double), len(a), ctypes.byref(g)))
    return g.value


def ising_equilibration(x, stride: int = 0):
    """(t0, g, n_eff): equilibrated start, its statistical inefficiency and
    effective sample count."""
    a = np.ascontiguousarray(x, dtype=np.float64)
    t0 = ctypes.c_int64()
    g = ctypes.c_double()
    n = ctypes.c_double()
    _check(_load().ising_equilibration(_ptr(a, ctypes.c_double), len(a), stride, ctypes.byref(t0),
                                       ctypes.byref(g), ctypes.byref(n)))
    return t0.value, g.value, n.value


ISING_NET_PARAMS = 2945
ISING_NET_BF16 = 0
ISING_NET_FP8 = 1


class IsingNet:
    """Owner of a learned-proposal network handle and its torch-allocated
    device workspace (ising_net_* in ising.h)."""

    def __init__(self, max_windows: int, max_lattices: int = 1, stream=None, device=None,
                 max_batch: Optional[int] = None):
        import torch
        if device is None:
            device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        lib = _load()
        if max_batch is None:
            max_batch = min(max_windows, 4096)
        nb = ctypes.c_size_t(0)
        _check(lib.ising_net_workspace_bytes(max_windows, max_batch, max_lattices, ctypes.byref(nb)))
        self.workspace = torch.empty(nb.value, dtype=torch.uint8, device=device)
        self.h = ctypes.c_void_p()
        _check(lib.ising_net_create(ctypes.byref(self.h), max_windows, max_batch, max_lattices,
                                    self.workspace.data_ptr(), nb.value, self.stream.cuda_stream))

    def set_params(self, params) -> None:
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == ISING_NET_PARAMS
        _check(_load().ising_net_set_params(self.h, _ptr(p, ctypes.c_float)))

    def set_precision(self, precision: int) -> None:
        _check(_load().ising_net_set_precision(self.h, precision))

    def get_params(self) -> np.ndarray:
        p = np.zeros(ISING_NET_PARAMS, dtype=np.float32)
        _check(_load().ising_net_get_params(self.h, _ptr(p, ctypes.c_float)))
        return p

    def score(self, windows, with_z: bool = False):
        w = np.ascontiguousarray(windows, dtype=np.int8).reshape(-1, 100)
        lq = np.zeros(len(w), dtype=np.float32)
        z = np.zeros((len(w), 100), dtype=np.float32) if with_z else None
        _check(_load().ising_net_score(self.h, _ptr(w, ctypes.c_int8), len(w), _ptr(lq, ctypes.c_float),
                                       _ptr(z, ctypes.c_float) if with_z else None))
        return (lq, z) if with_z else lq

    def sample(self, windows, keys, round_index: int):
        w = np.array(windows, dtype=np.int8).reshape(-1, 100)
        k = np.ascontiguousarray(keys, dtype=np.uint32).reshape(-1, 4)
        lq = np.zeros(len(w), dtype=np.float32)
        _check(_load().ising_net_sample(self.h, _ptr(w, ctypes.c_int8), len(w), _ptr(k, ctypes.c_uint32),
                                        round_index, _ptr(lq, ctypes.c_float)))
        return w, lq

    def grad(self, windows):
        w = np.ascontiguousarray(windows, dtype=np.int8).reshape(-1, 100)
        g = np.zeros(ISING_NET_PARAMS, dtype=np.float32)
        loss = ctypes.c_float(0)
        _check(_load().ising_net_grad(self.h, _ptr(w, ctypes.c_int8), len(w), _ptr(g, ctypes.c_float),
                                      ctypes.byref(loss)))
        return g, loss.value

    def train(self, dev_pool_words: int, n_snap: int, L: int, steps: int, batch: int, lr: float, seed: int):
        losses = np.zeros(max(1, steps), dtype=np.float32)
        _check(_load().ising_net_train(self.h, dev_pool_words, n_snap, L, steps, batch, lr, seed,
                                       _ptr(losses, ctypes.c_float)))
        return losses[:steps]

    def train_windows(self, dev_pool_words: int, n_snap: int, L: int, step: int, batch: int, seed: int):
        out = np.zeros((batch, 10, 10), dtype=np.int8)
        _check(_load().ising_net_train_windows(self.h, dev_pool_words, n_snap, L, step, batch, seed,
                                               _ptr(out, ctypes.c_int8)))
        return out

    def apply_grad(self, grad, lr: float) -> None:
        g = np.ascontiguousarray(grad, dtype=np.float32)
        assert g.size == ISING_NET_PARAMS
        _check(_load().ising_net_apply_grad(self.h, _ptr(g, ctypes.c_float), lr))

    def accepted(self, n: int, reset: bool = True) -> np.ndarray:
        acc = np.zeros(max(1, n), dtype=np.int64)
        _check(_load().ising_net_accepted(self.h, _ptr(acc, ctypes.c_int64), n, 1 if reset else 0))
        return acc[:n]

    def close(self):
        if getattr(self, "h", None):
            _load().ising_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ising_snapshot(h, dev_dst: int, nbytes: int) -> None:
    _check(_load().ising_snapshot(h, dev_dst, nbytes))


def ising_learned_round(h, net: "IsingNet", round_index: int, sync: bool = True):
    """One learned round; returns the accepted patches per lattice when sync,
    else enqueues only (counts accumulate; see IsingNet.accepted)."""
    n = ising_num_sims(h)
    if not sync:
        _check(_load().ising_learned_round(h, net.h, round_index, None))
        return None
    acc = np.zeros(max(1, n), dtype=np.int64)
    _check(_load().ising_learned_round(h, net.h, round_index, _ptr(acc, ctypes.c_int64)))
    return acc[:n]


ISING_PRNG_TESTS = 11
PRNG_TEST_NAMES = ("frequency", "block_frequency", "runs", "longest_run", "spectral", "cusum_forward",
                   "cusum_backward", "float_uniformity", "float_pairs", "median_runs", "median_longest_run")


def ising_random_stream(seed: int, s: int, phase: int, p0: int, n_p: int, t0: int, n_t: int, dev_out: int,
                        cuda_stream: int = 0) -> None:
    _check(_load().ising_random_stream(seed, s, phase, p0, n_p, t0, n_t, dev_out, cuda_stream))


def ising_prng_battery(words):
    """(p-values, statistics) of the eleven battery tests on host words."""
    w = np.ascontiguousarray(words, dtype=np.uint32)
    p = np.zeros(ISING_PRNG_TESTS)
    st = np.zeros(ISING_PRNG_TESTS)
    _check(_load().ising_prng_battery(_ptr(w, ctypes.c_uint32), len(w), _ptr(p, ctypes.c_double),
                                      _ptr(st, ctypes.c_double)))
    return p, st


def ising_sw_scratch_bytes(h) -> int:
    n = ctypes.c_size_t()
    _check(_load().ising_sw_scratch_bytes(h, ctypes.byref(n)))
    return n.value


def ising_sw_get_thresholds(h) -> np.ndarray:
    thr = np.zeros(max(1, ising_num_sims(h)), dtype=np.uint32)
    _check(_load().ising_sw_get_thresholds(h, _ptr(thr, ctypes.c_uint32)))
    return thr[:ising_num_sims(h)]


def ising_sw_sweep(h, n: int, dev_scratch: int, nbytes: int) -> None:
    _check(_load().ising_sw_sweep(h, n, dev_scratch, nbytes))


ISING_WOLFF_AUTO, ISING_WOLFF_GROWTH, ISING_WOLFF_LABELS = 0, 1, 2


def ising_wolff_set_method(h, method: int) -> None:
    _check(_load().ising_wolff_set_method(h, method))


def ising_wolff_sweep(h, n: int, dev_scratch: int, nbytes: int) -> None:
    _check(_load().ising_wolff_sweep(h, n, dev_scratch, nbytes))


def ising_sw_labels(h, sim: int, dev_scratch: int, nbytes: int) -> np.ndarray:
    L = ising_lattice_size(h, sim)
    lab = np.zeros((max(L, 1), max(L, 1)), dtype=np.uint32)
    _check(_load().ising_sw_labels(h, sim, dev_scratch, nbytes, _ptr(lab, ctypes.c_uint32)))
    return lab


class IsingSim:
    """Owner of one handle and its torch-allocated device workspace.

    IsingSim(L=64, temps=[2.269185], seed=1) -> one or more L x L lattices with
    one seed; IsingSim(Ls=[...], temps=[...], seeds=[...]) -> a batch of uneven
    lattices.  `stream` is a torch.cuda.Stream (default: the current stream)."""

    def __init__(self, L: Optional[int] = None, temps: Sequence[float] = (), seed: int = 0, *,
                 Ls: Optional[Sequence[int]] = None, seeds: Optional[Sequence[int]] = None,
                 cold: bool = False, trace_cap: int = 0, stream=None, device=None):
        import torch
        self._torch = torch
        if device is None:
            device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        init = ISING_INIT_COLD if cold else ISING_INIT_RANDOM
        temps = list(temps)
        with torch.cuda.device(device):
            if Ls is None:
                nbytes = ising_workspace_bytes(L, len(temps), trace_cap)
            else:
                nbytes = ising_batch_workspace_bytes(Ls, trace_cap)
            self.workspace = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)
            ptr = self.workspace.data_ptr()
            s = self.stream.cuda_stream
            if Ls is None:
                self.h = ising_create(L, len(temps), temps, seed, init, trace_cap, ptr, nbytes, s)
            else:
                self.h = ising_create_batch(Ls, temps, seeds, init, trace_cap, ptr, nbytes, s)
        self.n = ising_num_sims(self.h)

    def sweep(self, n: int) -> None:
        ising_sweep(self.h, n)

    def observables(self):
        return ising_observables(self.h)

    def trace(self, max_sweeps: int):
        return ising_trace(self.h, max_sweeps)

    def spins(self, sim: int = 0) -> np.ndarray:
        return ising_get_spins(self.h, sim)

    def set_spins(self, sim: int, spins: np.ndarray) -> None:
        ising_set_spins(self.h, sim, spins)

    def words(self, sim: int = 0):
        """Packed spins of lattice sim as a torch int32 view of the workspace."""
        ptr, n = ising_lattice_words(self.h, sim)
        off = ptr - self.workspace.data_ptr()
        return self.workspace[off: off + 4 * n].view(self._torch.int32)

    def thresholds(self) -> np.ndarray:
        return ising_get_thresholds(self.h)

    def set_plan(self, plan: int, **kw) -> None:
        ising_set_plan(self.h, plan, **kw)

    def learned_round(self, net: "IsingNet", round_index: int, sync: bool = True):
        return ising_learned_round(self.h, net, round_index, sync)

    def _sw_scratch(self):
        if getattr(self, "sw_scratch", None) is None:
            nbytes = ising_sw_scratch_bytes(self.h)
            self.sw_scratch = self._torch.empty(max(nbytes, 256), dtype=self._torch.uint8,
                                                device=self.workspace.device)
        return self.sw_scratch.data_ptr(), self.sw_scratch.numel()

    def sw_sweep(self, n: int) -> None:
        """n Swendsen-Wang steps (scratch allocated once, on first use)."""
        ptr, nbytes = self._sw_scratch()
        ising_sw_sweep(self.h, n, ptr, nbytes)

    def sw_labels(self, sim: int = 0) -> np.ndarray:
        ptr, nbytes = self._sw_scratch()
        return ising_sw_labels(self.h, sim, ptr, nbytes)

    def wolff_sweep(self, n: int) -> None:
        """n Wolff single-cluster steps of every lattice (the cluster step's
        scratch, allocated once, on first use)."""
        ptr, nbytes = self._sw_scratch()
        ising_wolff_sweep(self.h, n, ptr, nbytes)

    def sw_thresholds(self) -> np.ndarray:
        return ising_sw_get_thresholds(self.h)

    def autotune(self, probe_sweeps: int = 10, force: bool = False) -> float:
        return ising_autotune(self.h, probe_sweeps, force)

    def set_graph(self, on: bool) -> None:
        ising_set_graph(self.h, on)

    @property
    def sweeps_done(self) -> int:
        return ising_sweeps_done(self.h)

    def close(self) -> None:
        if getattr(self, "h", None):
            ising_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class IsingSim3D:
    """Owner of one three-dimensional handle (lattices of side Ls[i], L^3
    spins each) and its torch-allocated device workspace."""

    def __init__(self, Ls: Sequence[int], temps: Sequence[float], seeds: Sequence[int], *, cold: bool = False,
                 trace_cap: int = 0, stream=None, device=None):
        import torch
        self._torch = torch
        if device is None:
            device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        lib = _load()
        self.Ls = [int(L) for L in Ls]
        n = len(self.Ls)
        Ls_a = np.array(self.Ls, dtype=np.int32)
        T_a = np.array(list(temps), dtype=np.float64)
        S_a = np.array([int(x) for x in seeds], dtype=np.uint64)
        nbytes = ctypes.c_size_t()
        _check(lib.ising3d_workspace_bytes(n, _ptr(Ls_a, ctypes.c_int), trace_cap, ctypes.byref(nbytes)))
        with torch.cuda.device(device):
            self.workspace = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device=device)
        h = ctypes.c_void_p()
        _check(lib.ising3d_create(ctypes.byref(h), n, _ptr(Ls_a, ctypes.c_int), _ptr(T_a, ctypes.c_double),
                                  _ptr(S_a, ctypes.c_uint64), ISING_INIT_COLD if cold else ISING_INIT_RANDOM,
                                  trace_cap, self.workspace.data_ptr(), nbytes.value, self.stream.cuda_stream))
        self.h = h.value
        self.n = n

    def sweep(self, n: int) -> None:
        _check(_load().ising3d_sweep(self.h, n))

    def set_graph(self, on: bool) -> None:
        _check(_load().ising3d_set_graph(self.h, 1 if on else 0))

    @property
    def sweeps_done(self) -> int:
        return int(_load().ising3d_sweeps_done(self.h))

    def observables(self):
        E = np.zeros(self.n, dtype=np.int64)
        M = np.zeros(self.n, dtype=np.int64)
        _check(_load().ising3d_observables(self.h, _ptr(E, ctypes.c_int64), _ptr(M, ctypes.c_int64)))
        return E, M

    def trace(self, max_sweeps: int):
        E = np.zeros((self.n, max(1, max_sweeps)), dtype=np.int64)
        M = np.zeros_like(E)
        k = ctypes.c_int64()
        _check(_load().ising3d_trace(self.h, _ptr(E, ctypes.c_int64), _ptr(M, ctypes.c_int64), max_sweeps,
                                     ctypes.byref(k)))
        return E.reshape(-1)[: self.n * k.value].reshape(self.n, k.value), \
            M.reshape(-1)[: self.n * k.value].reshape(self.n, k.value)

    def spins(self, sim: int = 0) -> np.ndarray:
        L = self.Ls[sim]
        out = np.zeros((L, L, L), dtype=np.int8)
        _check(_load().ising3d_get_spins(self.h, sim, _ptr(out, ctypes.c_int8)))
        return out

    def close(self) -> None:
        if getattr(self, "h", None):
            _load().ising3d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
