"""Quality of the Philox4x32-10 streams the kernels draw, in the manner of the
paper's generator checks (supplementary, PRNG tests): the streams are
generated on the GPU exactly as the sweeps, the initial state, the cluster
bonds and coins consume them (ising_random_stream), then split into
sub-streams of `words` 32-bit words; each sub-stream gets the battery
(ising_prng_battery: NIST SP 800-22 bit tests, float uniformity, float pairs,
median bits).  Reported per stream and test: the proportion of sub-streams
passing at alpha = 0.01 and a Kolmogorov-Smirnov p-value of the sub-stream
p-values against uniform (NIST's two second-level checks), plus the stream
kernel's device time.

Streams: spatial = all sites of one phase in sweep 0 (black half-sweep,
white half-sweep, initial state, cluster bonds, cluster coins); temporal =
one site's draws over consecutive sweeps.  --calibrate adds the same protocol
on numpy's PCG64 generator (host), the scale against which to read the
Philox numbers: with 100 sub-streams a good generator still shows a few
(test, stream) pairs below NIST's proportion threshold.
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import ising


def _ks_uniform(p):
    """Kolmogorov-Smirnov statistic and asymptotic p-value of p against U(0,1)."""
    x = np.sort(np.asarray(p, dtype=np.float64))
    n = len(x)
    i = np.arange(1, n + 1)
    d = max(float((i / n - x).max()), float((x - (i - 1) / n).max()))
    lam = (math.sqrt(n) + 0.12 + 0.11 / math.sqrt(n)) * d
    q = 2.0 * sum((-1) ** (k - 1) * math.exp(-2.0 * k * k * lam * lam) for k in range(1, 101))
    return d, min(1.0, max(0.0, q))


STREAMS = {
    "black_half_sweep": dict(seed=2, s=0, phase=0, spatial=True),
    "white_half_sweep": dict(seed=2, s=0, phase=1, spatial=True),
    "initial_state": dict(seed=2, s=0, phase=2, spatial=True),
    "cluster_bonds": dict(seed=2, s=0, phase=7, spatial=True),
    "cluster_coins": dict(seed=2, s=0, phase=8, spatial=True),
    "one_site_over_sweeps": dict(seed=2, s=0, phase=0, spatial=False),
}


def run(sub_streams: int = 100, words: int = 1 << 16, calibrate: int = 0, verbose: bool = True) -> dict:
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    s = torch.cuda.Stream(dev)
    n = sub_streams * words
    out = torch.empty(n, dtype=torch.int32, device=dev)
    res = {"sub_streams": sub_streams, "words_per_sub_stream": words, "tests": list(ising.PRNG_TEST_NAMES),
           "streams": {}}
    for name, cfg in STREAMS.items():
        p0, n_p, t0, n_t = (0, n, 0, 1) if cfg["spatial"] else (4321, 1, 0, n)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ising.ising_random_stream(cfg["seed"], cfg["s"], cfg["phase"], p0, n_p, t0, n_t, out.data_ptr(), s.cuda_stream)
        e0.record(s)
        ising.ising_random_stream(cfg["seed"], cfg["s"], cfg["phase"], p0, n_p, t0, n_t, out.data_ptr(), s.cuda_stream)
        e1.record(s)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        w = out.cpu().numpy().view(np.uint32)
        P = np.array([ising.ising_prng_battery(w[k * words:(k + 1) * words])[0] for k in range(sub_streams)])
        rows = {}
        for j, tname in enumerate(ising.PRNG_TEST_NAMES):
            d, q = _ks_uniform(P[:, j])
            rows[tname] = {"pass_proportion": float((P[:, j] >= 0.01).mean()), "ks_uniform_p": q,
                           "min_p": float(P[:, j].min())}
        res["streams"][name] = {"stream_kernel_ms": ms, "draws_per_ns": n / (ms * 1e6), "tests": rows}
        if verbose:
            worst = min(rows.items(), key=lambda kv: kv[1]["ks_uniform_p"])
            print(json.dumps({"stream": name, "draws_per_ns": n / (ms * 1e6),
                              "min_pass_proportion": min(r["pass_proportion"] for r in rows.values()),
                              "min_ks_p": worst[1]["ks_uniform_p"], "min_ks_test": worst[0]}), flush=True)
    if calibrate:
        rows = {}
        for k in range(calibrate):
            w = np.random.default_rng(1000 + k).integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)
            P = np.array([ising.ising_prng_battery(w[j * words:(j + 1) * words])[0] for j in range(sub_streams)])
            for j, tname in enumerate(ising.PRNG_TEST_NAMES):
                rows.setdefault(tname, []).append(float((P[:, j] >= 0.01).mean()))
        res["pcg64_calibration"] = {t: {"pass_proportions": v, "min": min(v)} for t, v in rows.items()}
        if verbose:
            print(json.dumps({"pcg64_min_pass_proportion": {t: min(v) for t, v in rows.items()}}), flush=True)
    # NIST's acceptable proportion at alpha = 0.01: 0.99 - 3 sqrt(0.99 * 0.01 / m)
    res["proportion_threshold"] = 0.99 - 3.0 * math.sqrt(0.99 * 0.01 / sub_streams)
    if verbose:
        print(json.dumps(res), flush=True)
    return res


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--sub-streams", type=int, default=100)
    ap.add_argument("--words", type=int, default=1 << 16)
    ap.add_argument("--calibrate", type=int, default=0, help="also this many PCG64 streams (host)")
    args = ap.parse_args()
    run(args.sub_streams, args.words, args.calibrate)


if __name__ == "__main__":
    main()
