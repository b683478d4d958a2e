"""What the trained net gains, on the GPU, end to end: 32 replicas of 128^2
at T = 2.35 (above T_c, where the learned move was measured to shorten
tau_int most), a net trained on the GPU on snapshots of the plain sampler,
then two chains from one equilibrated state -- plain sweeps, and a learned
patch round followed by one sweep per unit.

* The learned chain samples the same distribution: its <|m|> and <e> agree
  with the plain chain's within 3 sigma (sigma from the spread over
  replicas), and its <e> agrees with the exact finite-lattice value (Kaufman)
  within 3 sigma.
* Training is what makes the proposal useful: the trained net's patches are
  accepted far more often than the untrained initial net's.
* Per unit, the learned chain decorrelates |M| no slower than plain sweeps
  (tau_int within two combined standard errors or below).

The Metropolis-Hastings correction keeps the learned chain exact whatever the
net; these checks are about the net, the training and the bookkeeping."""
from __future__ import annotations

import math

import pytest

import exact
from paper_2404_16990_gb300 import learned_study

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


@pytest.fixture(scope="module")
def study():
    return learned_study.run_temperature(T=2.35, L=128, replicas=32, burn=1000, n_snap=4000, snap_every=10,
                                         train_steps=400, batch=256, lr=3e-3, units=6000, sw_burn=200, seed=77,
                                         verbose=False)


def test_learned_chain_samples_the_same_distribution(study):
    assert study["agree_abs_m_sigma"] < 3.0, study["agree_abs_m_sigma"]
    assert study["agree_e_sigma"] < 3.0, study["agree_e_sigma"]
    e_exact = exact.kaufman_mean_energy(128, 2.35) / 128**2
    for chain in ("plain", "learned"):
        c = study[chain]
        assert abs(c["mean_e"] - e_exact) < 3.0 * c["mean_e_err"], (chain, c["mean_e"], e_exact, c["mean_e_err"])


def test_training_raises_acceptance(study):
    assert study["loss_last"] < study["loss_first"]
    assert study["acceptance"] > study["acceptance_untrained"] + 0.1, (study["acceptance"],
                                                                      study["acceptance_untrained"])


def test_learned_unit_decorrelates_no_slower(study):
    p, q = study["plain"], study["learned"]
    sigma = math.hypot(p["tau_int_absM_err"], q["tau_int_absM_err"])
    assert q["tau_int_absM"] <= p["tau_int_absM"] + 2.0 * sigma, (q["tau_int_absM"], p["tau_int_absM"], sigma)
