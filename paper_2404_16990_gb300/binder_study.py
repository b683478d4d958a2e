"""Binder-cumulant temperature scan: L in {1024, 2048, 4096} x 16 temperatures
in [2.20, 2.34] x 3 replicas (144 lattices, 1.06e9 spins) advanced together,
FP64 moments of m = M/N and e = E/N accumulated on the GPU every unit, the
Binder cumulant U = 1 - <m^4>/(3<m^2>^2) per (L, T), tau_int of |M| and E
from the per-unit traces, and -- as in the paper's validation (Section 3.1) --
the non-equilibrated start of each trace found and discarded automatically
(statistical inefficiency, Chodera 2016) before U is taken again from the
rest; the crossings of U(T) between lattice sizes estimate T_c.  A unit is a
checkerboard sweep (--mode plain, the paper's method) or a Swendsen-Wang step
(--mode cluster).  Optionally, the learned patch proposal's cost and
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


def _binder_of(m):
    m = np.asarray(m, dtype=np.float64)
    m2 = float(np.mean(m * m))
    return 1.0 - float(np.mean(m ** 4)) / (3.0 * m2 * m2) if m2 > 0 else float("nan")


def _crossing(Ts, Ua, Ub):
    """Temperature where two U(T) curves cross (linear interpolation between
    neighbouring temperatures; the first sign change), or None."""
    d = np.asarray(Ua) - np.asarray(Ub)
    for i in range(len(Ts) - 1):
        if d[i] == 0.0:
            return float(Ts[i])
        if d[i] * d[i + 1] < 0.0:
            return float(Ts[i] + (Ts[i + 1] - Ts[i]) * d[i] / (d[i] - d[i + 1]))
    return None


def run(burn: int = 5000, sweeps: int = 50000, learned_rounds: int = 10, seed: int = 77,
        mode: str = "plain", sw_burn: int = 200, t_range=(2.20, 2.34), verbose: bool = True) -> dict:
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(dev)
    wl = workloads.binder_scan(n_sweeps=sweeps, t_lo=t_range[0], t_hi=t_range[1])
    res = {"lattices": wl.n_sims, "spins": wl.spins, "mode": mode, "burn": burn, "sw_burn": sw_burn,
           "units": sweeps}
    with torch.cuda.stream(stream):
        sim = ising.IsingSim(Ls=wl.Ls, temps=wl.temps, seeds=wl.seeds, trace_cap=sweeps, stream=stream)
        sim.set_graph(True)
        res["autotune_probe_flip_per_ns"] = sim.autotune(probe_sweeps=10)
        res["plan"] = ising.ising_get_plan(sim.h)
        if sw_burn > 0:
            sim.sw_sweep(sw_burn)
        sim.sweep(burn)
        ising.ising_set_measure(sim.h, True)
        ising.ising_reset_moments(sim.h)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        done = 0
        chunk = 1000 if mode == "plain" else 100
        while done < sweeps:                       # one graph per chunk, replayed
            k = min(chunk, sweeps - done)
            if mode == "plain":
                sim.sweep(k)
            else:
                sim.sw_sweep(k)
            done += k
        e1.record(stream)
        torch.cuda.synchronize(dev)
        secs = e0.elapsed_time(e1) / 1e3
        res["seconds"] = secs
        res["site_updates_per_ns"] = wl.spins * sweeps / (secs * 1e9)
        mom = ising.ising_moments(sim.h)
        U = ising.ising_binder(mom)
        E, M = sim.trace(sweeps)
    rows = []
    for i, (L, T) in enumerate(zip(wl.Ls, wl.temps)):
        absm = np.abs(M[i]).astype(np.float64)
        t0, g, n_eff = ising.ising_equilibration(absm, 0)
        tm = ising.ising_tau_int(absm[t0:])[0] if len(absm) - t0 >= 2 else float("nan")
        te = ising.ising_tau_int(E[i][t0:].astype(np.float64))[0] if len(absm) - t0 >= 2 else float("nan")
        m_eq = M[i][t0:].astype(np.float64) / (L * L)
        rows.append({"L": L, "T": T, "U_all": float(U[i]), "U": _binder_of(m_eq), "t0": int(t0),
                     "n_eff": float(n_eff), "abs_m": float(np.abs(m_eq).mean()),
                     "e": float(E[i][t0:].mean() / (L * L)), "tau_absM": tm, "tau_E": te})
    table = {}
    for r in rows:
        key = (r["L"], round(r["T"], 6))
        table.setdefault(key, []).append(r)
    summary = []
    for (L, T), rs in sorted(table.items()):
        Us = np.array([r["U"] for r in rs])
        summary.append({"L": L, "T": T, "U": float(Us.mean()), "U_err": float(Us.std(ddof=1) / math.sqrt(len(Us))),
                        "U_all": float(np.mean([r["U_all"] for r in rs])),
                        "t0": float(np.mean([r["t0"] for r in rs])),
                        "n_eff": float(np.mean([r["n_eff"] for r in rs])),
                        "abs_m": float(np.mean([r["abs_m"] for r in rs])),
                        "e": float(np.mean([r["e"] for r in rs])),
                        "tau_absM": float(np.mean([r["tau_absM"] for r in rs])),
                        "tau_E": float(np.mean([r["tau_E"] for r in rs]))})
    res["summary"] = summary
    by_L = {}
    for r in summary:
        by_L.setdefault(r["L"], []).append(r)
    Ls = sorted(by_L)
    crossings = {}
    for a in range(len(Ls)):
        for b in range(a + 1, len(Ls)):
            ra, rb = by_L[Ls[a]], by_L[Ls[b]]
            crossings[f"{Ls[a]}/{Ls[b]}"] = _crossing([r["T"] for r in ra], [r["U"] for r in ra],
                                                      [r["U"] for r in rb])
    res["U_crossings"] = crossings
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
                                        "unit_equivalents_per_round": ms / (1e3 * secs / sweeps),
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
    ap.add_argument("--mode", choices=["plain", "cluster"], default="plain",
                    help="measurement unit: checkerboard sweep or Swendsen-Wang step")
    ap.add_argument("--sw-burn", type=int, default=200, help="cluster steps before the plain burn-in")
    ap.add_argument("--t-range", type=float, nargs=2, default=[2.20, 2.34], metavar=("T_LO", "T_HI"))
    args = ap.parse_args()
    run(burn=args.burn, sweeps=args.sweeps, learned_rounds=args.learned_rounds, mode=args.mode,
        sw_burn=args.sw_burn, t_range=tuple(args.t_range))


if __name__ == "__main__":
    main()
