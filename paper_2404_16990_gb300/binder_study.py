"""Binder-cumulant temperature scan: L in {1024, 2048, 4096} x 16 temperatures
in [2.20, 2.34] x 3 replicas (144 lattices, 1.06e9 spins) advanced together,
FP64 moments of m = M/N and e = E/N accumulated on the GPU every sweep, the
Binder cumulant U = 1 - <m^4>/(3<m^2>^2) per (L, T), and tau_int of |M| and E
from the per-sweep traces.  Optionally, the learned patch proposal's cost and
acceptance on the same lattices in BF16 and in FP8 (E4M3) inference, with a net
trained at L = 256 near T_c.

Everything runs through the C ABI (libising); this module only orchestrates.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import ising, workloads


def run(burn: int = 5000, sweeps: int = 50000, learned_rounds: int = 10, seed: int = 77,
        verbose: bool = True) -> dict:
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(dev)
    wl = workloads.binder_scan(n_sweeps=sweeps)
    res = {"lattices": wl.n_sims, "spins": wl.spins, "burn": burn, "sweeps": sweeps}
    with torch.cuda.stream(stream):
        sim = ising.IsingSim(Ls=wl.Ls, temps=wl.temps, seeds=wl.seeds, trace_cap=sweeps, stream=stream)
        sim.set_graph(True)
        res["autotune_probe_flip_per_ns"] = sim.autotune(probe_sweeps=10)
        res["plan"] = ising.ising_get_plan(sim.h)
        sim.sweep(burn)
        ising.ising_set_measure(sim.h, True)
        ising.ising_reset_moments(sim.h)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        done = 0
        while done < sweeps:                       # one graph of 1000 sweeps replayed
            k = min(1000, sweeps - done)
            sim.sweep(k)
            done += k
        e1.record(stream)
        torch.cuda.synchronize(dev)
        secs = e0.elapsed_time(e1) / 1e3
        res["seconds"] = secs
        res["flip_per_ns"] = wl.spins * sweeps / (secs * 1e9)
        mom = ising.ising_moments(sim.h)
        U = ising.ising_binder(mom)
        E, M = sim.trace(sweeps)
    rows = []
    for i, (L, T) in enumerate(zip(wl.Ls, wl.temps)):
        tm = ising.ising_tau_int(np.abs(M[i]).astype(np.float64))[0]
        te = ising.ising_tau_int(E[i].astype(np.float64))[0]
        rows.append({"L": L, "T": T, "U": float(U[i]), "abs_m": float(mom[i, 1] / mom[i, 0]),
                     "e": float(mom[i, 4] / mom[i, 0]), "tau_absM": tm, "tau_E": te})
    table = {}
    for r in rows:
        key = (r["L"], round(r["T"], 6))
        table.setdefault(key, []).append(r)
    summary = []
    for (L, T), rs in sorted(table.items()):
        Us = np.array([r["U"] for r in rs])
        summary.append({"L": L, "T": T, "U": float(Us.mean()), "U_err": float(Us.std(ddof=1) / math.sqrt(len(Us))),
                        "abs_m": float(np.mean([r["abs_m"] for r in rs])),
                        "e": float(np.mean([r["e"] for r in rs])),
                        "tau_absM": float(np.mean([r["tau_absM"] for r in rs])),
                        "tau_E": float(np.mean([r["tau_E"] for r in rs]))})
    res["summary"] = summary
    # learned proposal on the same lattices: BF16 vs FP8 inference
    if learned_rounds > 0:
        from .learned_study import default_params
        with torch.cuda.stream(stream):
            tr = ising.IsingSim(256, [workloads.T_CRITICAL] * 64, seed, stream=stream)
            tr.set_graph(True)
            tr.autotune(probe_sweeps=10)
            tr.sweep(2000)
            per = 256 * 256 // 8
            sets = 150
            pool = torch.empty(sets * 64 * per, dtype=torch.uint8, device=dev)
            for k in range(sets):
                tr.sweep(10)
                ising.ising_snapshot(tr.h, pool.data_ptr() + k * 64 * per, 64 * per)
            nwin = sum((L // 16) ** 2 for L in wl.Ls)
            net = ising.IsingNet(max_windows=max(nwin, 512), max_lattices=wl.n_sims, stream=stream, max_batch=512)
            net.set_params(default_params(seed))
            losses = net.train(pool.data_ptr(), sets * 64, 256, 1500, 512, 3e-3, seed)
            res["learned"] = {"patches_per_round": nwin, "train_loss_last": float(losses[-50:].mean())}
            state = ising.ising_save(sim.h)
            for name, prec in (("bf16", ising.ISING_NET_BF16), ("fp8", ising.ISING_NET_FP8)):
                ising.ising_load(sim.h, state)
                net.set_precision(prec)
                sim.learned_round(net, 0, sync=True)
                ising.ising_load(sim.h, state)
                net.accepted(wl.n_sims, reset=True)
                a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                for r in range(learned_rounds):
                    sim.learned_round(net, r, sync=False)
                a1.record(stream)
                torch.cuda.synchronize(dev)
                acc = net.accepted(wl.n_sims)
                ms = a0.elapsed_time(a1) / learned_rounds
                res["learned"][name] = {"round_ms": ms, "acceptance": float(acc.sum() / (nwin * learned_rounds)),
                                        "sweep_equivalents_per_round": ms / (1e3 * secs / sweeps),
                                        "patches_per_s": nwin / (ms / 1e3)}
            ising.ising_load(sim.h, state)
            tr.close()
            net.close()
    if verbose:
        print(json.dumps(res), flush=True)
    sim.close()
    return res


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--burn", type=int, default=5000)
    ap.add_argument("--sweeps", type=int, default=50000)
    ap.add_argument("--learned-rounds", type=int, default=10)
    args = ap.parse_args()
    run(burn=args.burn, sweeps=args.sweeps, learned_rounds=args.learned_rounds)


if __name__ == "__main__":
    main()
