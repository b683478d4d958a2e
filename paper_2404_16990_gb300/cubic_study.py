"""Three-dimensional sweep: flip rate of the ising3d_* kernels on single
L^3 lattices and a batch near the simple-cubic critical temperature
(T ~ 4.5115), graphs on, CUDA events, L2 flushed between timed calls when
the lattice fits in it; plus the energy per site and |m| after the timed
sweeps, for a sanity check against the known critical values (e ~ -0.99).

Everything runs through the C ABI (libising); this module only orchestrates.
"""
from __future__ import annotations

import argparse
import json

from . import ising

TC3 = 4.5115


def time_case(Ls, temps, seeds, sweeps: int = 100, reps: int = 3) -> dict:
    import torch
    s = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    with torch.cuda.stream(s):
        sim = ising.IsingSim3D(Ls, temps, seeds, stream=s)
        sim.set_graph(True)
        sim.sweep(sweeps)
        torch.cuda.synchronize()
        best = float("inf")
        for r in range(reps):
            flush.fill_(r)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            sim.sweep(sweeps)
            e1.record(s)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        E, M = sim.observables()
    sites = sum(L ** 3 for L in Ls)
    out = {"Ls": list(Ls), "sweeps": sweeps, "ms_per_sweep": best / sweeps,
           "flip_per_ns": sites * sweeps / (best * 1e6),
           "e_per_site": [float(E[i]) / Ls[i] ** 3 for i in range(len(Ls))],
           "abs_m": [abs(float(M[i])) / Ls[i] ** 3 for i in range(len(Ls))]}
    print(json.dumps(out), flush=True)
    sim.close()
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--sweeps", type=int, default=100)
    args = ap.parse_args()
    res = [time_case([256], [TC3], [1], args.sweeps), time_case([512], [TC3], [1], args.sweeps),
           time_case([1024], [TC3], [1], max(10, args.sweeps // 4)),
           time_case([256] * 8, [TC3] * 8, list(range(1, 9)), args.sweeps)]
    print(json.dumps({"cubic_timing": res}))


if __name__ == "__main__":
    main()
