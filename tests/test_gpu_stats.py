"""Statistics on traces the GPU produced: automatic equilibration detection
and the statistical inefficiency of the library against the oracle on E and
|M| traces of lattices relaxing from random starts."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import stats as ostats
from paper_2404_16990_gb300 import ising

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def test_equilibration_of_gpu_traces_matches_oracle():
    n = 3000
    sim = ising.IsingSim(128, [1.8, 2.269185, 3.0], 5, trace_cap=n)
    sim.sweep(n)
    E, M = sim.trace(n)
    for i in range(3):
        for x in (E[i].astype(np.float64), np.abs(M[i]).astype(np.float64)):
            t_lib, g_lib, n_lib = ising.ising_equilibration(x, 10)
            t_ref, g_ref, n_ref = ostats.detect_equilibration(x, 10)
            assert t_lib == t_ref and abs(g_lib - g_ref) < 1e-9 * g_ref and abs(n_lib - n_ref) < 1e-9 * n_ref
    # the energy of a random start relaxes: the detected start is past the transient
    t_e, _, _ = ising.ising_equilibration(E[0].astype(np.float64), 10)
    assert t_e > 0
    sim.close()
