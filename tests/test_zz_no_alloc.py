"""ising_sweep_noalloc -- the entry point for callers that cannot allocate
device memory (for example code inside an application that owns all device
memory through its own pool, or a latency-critical path where cudaMalloc may
block) -- against the workspace-based entry points, bit for bit, on two calls
in a row.  This file is collected last so that a run stopping at the first
failure has already run every other test."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2404_16990_gb300 import ising

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def test_noalloc_matches_workspace_path_on_two_calls():
    import torch
    Ls = [64, 192, 2048]
    temps = [1.8, 2.269185, 3.1]
    seeds = [11, 12, 13]
    ref = ising.IsingSim(Ls=Ls, temps=temps, seeds=seeds)      # workspace-based path
    # the caller's own buffers: the same initial lattices, packed, one after another
    words = torch.cat([ref.words(i).clone() for i in range(len(Ls))])
    em = torch.zeros(2 * len(Ls), dtype=torch.int64, device="cuda")
    t0 = 0
    for n in (7, 5):                                            # two calls in a row
        ref.sweep(n)
        ising.ising_sweep_noalloc(words.data_ptr(), Ls, temps, seeds, t0, n, em.data_ptr(), 0)
        torch.cuda.synchronize()
        t0 += n
        E, M = ref.observables()
        got = em.cpu().numpy()
        assert np.array_equal(got[0::2], E) and np.array_equal(got[1::2], M)
        expect = torch.cat([ref.words(i) for i in range(len(Ls))])
        assert torch.equal(words, expect)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    n = ising.ISING_NOALLOC_MAX_LATTICES + 1
    words = torch.zeros(n * 64 * 64 // 32, dtype=torch.int32, device="cuda")
    em = torch.zeros(2 * n, dtype=torch.int64, device="cuda")
    with pytest.raises(ising.IsingError) as e:
        ising.ising_sweep_noalloc(words.data_ptr(), [64] * n, [2.0] * n, [1] * n, 0, 1, em.data_ptr(), 0)
    assert e.value.code == ising.ISING_EINVAL
    assert "ISING_NOALLOC_MAX_LATTICES" in ising.ising_last_error()
