"""Entry points that take device addresses or sizes reject invalid arguments
with ISING_EINVAL before any device work, so these run without a GPU: the
fake device addresses below are never dereferenced."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from paper_2404_16990_gb300 import ising

FAKE = 1 << 20          # a 16-byte aligned address that is never dereferenced


def _einval(fn, *args):
    with pytest.raises(ising.IsingError) as e:
        fn(*args)
    assert e.value.code == ising.ISING_EINVAL
    assert ising.ising_last_error()


def test_random_stream_arguments():
    rs = ising.ising_random_stream
    _einval(rs, 1, 0, 0, 0, 16, 0, 1, 0)                       # dev_out NULL
    _einval(rs, 1, 0, 0, 0, 16, 0, 1, FAKE + 4)                # not 16-byte aligned
    _einval(rs, 1, 0, 0, (1 << 34) - 8, 16, 0, 1, FAKE)       # sites beyond 2^34
    _einval(rs, 1, 0, 0, 2**64 - 8, 16, 0, 1, FAKE)           # p0 + n_p wraps
    _einval(rs, 1, 0, 0, 0, 16, 2**32 - 2, 4, FAKE)           # sweeps beyond 2^32


def test_noalloc_arguments():
    sw = ising.ising_sweep_noalloc
    _einval(sw, FAKE, [], [], [], 0, 1, FAKE)                                    # no lattice
    _einval(sw, FAKE, [64] * (ising.ISING_NOALLOC_MAX_LATTICES + 1), [2.0] * (ising.ISING_NOALLOC_MAX_LATTICES + 1),
            [1] * (ising.ISING_NOALLOC_MAX_LATTICES + 1), 0, 1, FAKE)          # too many
    _einval(sw, 0, [64], [2.0], [1], 0, 1, FAKE)                                 # NULL words
    _einval(sw, FAKE, [64], [2.0], [1], 0, 1, 0)                                 # NULL E/M
    _einval(sw, FAKE + 8, [64], [2.0], [1], 0, 1, FAKE)                          # words misaligned
    for L in (32, 96, 65600):
        _einval(sw, FAKE, [L], [2.0], [1], 0, 1, FAKE)                           # L not a multiple of 64 in range
    for T in (0.0, -1.0, float("nan"), float("inf")):
        _einval(sw, FAKE, [64], [T], [1], 0, 1, FAKE)
    _einval(sw, FAKE, [64], [2.0], [1], -1, 1, FAKE)                             # t0 < 0
    _einval(sw, FAKE, [64], [2.0], [1], 0, -1, FAKE)                             # n < 0
    _einval(sw, FAKE, [64], [2.0], [1], 2**32 - 4, 8, FAKE)                      # counter past 2^32
    sw(FAKE, [64, 128], [2.0, 3.0], [1, 2], 5, 0, FAKE)                          # n = 0: nothing to do, OK
    # the binding checks that the three host arrays agree in length before the
    # library reads n_lat entries from each
    for Ls, temps, seeds in (([64, 128], [2.0], [1, 2]), ([64, 128], [2.0, 3.0], [1]), ([64], [2.0, 3.0], [1, 2])):
        with pytest.raises(ValueError):
            sw(FAKE, Ls, temps, seeds, 0, 1, FAKE)


def test_wait_limit_arguments():
    _einval(ising.ising_set_wait_limit_ns, None, 1000)                           # NULL handle
    _einval(ising.ising_set_wait_limit_ns, None, ising.ISING_MAX_WAIT_LIMIT_NS + 1)
    assert "at most" in ising.ising_last_error()


def test_net_workspace_bytes():
    lib = ising._load()
    nb = ctypes.c_size_t(0)
    for bad in ((0, 1, 1), (1, 0, 1), (1, 1, 0), (-5, 1, 1)):
        assert lib.ising_net_workspace_bytes(*bad, ctypes.byref(nb)) == ising.ISING_EINVAL
    assert lib.ising_net_workspace_bytes(1, 1, 1, None) == ising.ISING_EINVAL
    sizes = []
    for w in (1, 64, 4096, 65536):
        assert lib.ising_net_workspace_bytes(w, min(w, 512), 1, ctypes.byref(nb)) == ising.ISING_OK
        sizes.append(nb.value)
    assert all(a < b for a, b in zip(sizes, sizes[1:]))
    assert all(s % 256 == 0 for s in sizes)


def test_statistics_arguments():
    _einval(ising.ising_stat_inefficiency, [1.0])
    _einval(ising.ising_equilibration, [1.0])
    _einval(ising.ising_equilibration, [1.0, 2.0, 3.0], -1)
    _einval(ising.ising_tau_int, [1.0, 2.0], -1.0)
    assert ising.ising_equilibration(np.arange(10.0), 0)[0] >= 0      # stride 0: the default
