"""The Philox stream the kernels draw, read back through ising_random_stream,
against the oracle's Philox4x32-10 bit for bit (aligned and unaligned site
ranges, several sweeps, every phase), and the battery on it."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import prng_battery as pb
from paper_2404_16990_gb300 import ising

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def _device_stream(seed, s, phase, p0, n_p, t0, n_t):
    import torch
    out = torch.empty(n_p * n_t, dtype=torch.int32, device="cuda")
    ising.ising_random_stream(seed, s, phase, p0, n_p, t0, n_t, out.data_ptr(),
                              torch.cuda.current_stream().cuda_stream)
    return out.cpu().numpy().view(np.uint32).reshape(n_t, n_p)


def _oracle_stream(seed, s, phase, p0, n_p, t0, n_t):
    key = [seed & 0xFFFFFFFF, seed >> 32]
    out = np.empty((n_t, n_p), dtype=np.uint32)
    for ti in range(n_t):
        cache = {}
        for j in range(n_p):
            p = p0 + j
            q = p >> 2
            if q not in cache:
                cache[q] = oracle.philox4x32_10([q & 0xFFFFFFFF, t0 + ti, s, phase], key)
            out[ti, j] = cache[q][p & 3]
    return out


@pytest.mark.parametrize("seed,s,phase,p0,n_p,t0,n_t", [
    (2, 0, 0, 0, 4096, 0, 3),
    (0x0123456789ABCDEF, 5, 1, 3, 1001, 17, 2),        # unaligned start and length
    (7, 1, 2, (1 << 33) + 1, 257, 0, 1),               # beyond 2^32 sites (q > 2^30)
    (11, 2, 7, 12345, 1, 0, 2000),                     # one site over many sweeps
    (13, 0, 8, 65530, 20, 4294967000, 296),            # up to the last sweep index
])
def test_stream_matches_oracle(seed, s, phase, p0, n_p, t0, n_t):
    assert np.array_equal(_device_stream(seed, s, phase, p0, n_p, t0, n_t),
                          _oracle_stream(seed, s, phase, p0, n_p, t0, n_t))


def test_stream_arguments_rejected():
    import torch
    out = torch.empty(64, dtype=torch.int32, device="cuda")
    for args in [(1, 0, 0, (1 << 34) - 10, 20, 0, 1), (1, 0, 0, 0, 4, (1 << 32) - 1, 2)]:
        with pytest.raises(ising.IsingError):
            ising.ising_random_stream(*args, out.data_ptr())
    with pytest.raises(ising.IsingError):
        ising.ising_random_stream(1, 0, 0, 0, 4, 0, 1, out.data_ptr() + 4)


def test_battery_of_the_sweep_stream():
    """The black half-sweep's draws of a 1024^2 lattice in sweep 0 and one
    site's draws over 65536 sweeps: library battery equals the oracle's, and
    no test rejects at the 1e-4 level."""
    for words in (_device_stream(2, 0, 0, 0, 1 << 19, 0, 1).ravel(),
                  _device_stream(2, 0, 1, 4321, 1, 0, 1 << 16).ravel()):
        p_lib, s_lib = ising.ising_prng_battery(words)
        p_ref, s_ref = pb.battery(words)
        assert np.allclose(s_lib, s_ref, rtol=1e-9, atol=1e-9)
        assert np.allclose(p_lib, p_ref, rtol=1e-7, atol=1e-9)
        assert p_lib.min() > 1e-4, dict(zip(pb.TESTS, p_lib))
