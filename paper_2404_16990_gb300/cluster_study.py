"""Swendsen-Wang and Wolff cluster steps against plain checkerboard
Metropolis sweeps: integrated autocorrelation times and effective independent
samples per second of |M| and E, on the workload of the learned-proposal
study (64 replicas of 256^2 at T in {2.20, T_c, 2.35}), plus step throughput
on larger lattices.

Study (per temperature): the chains start from the same state, reached from
a random start by `sw_burn` cluster steps and `burn` plain sweeps; the plain
chain runs `units` sweeps, the Swendsen-Wang chain `sw_units` steps, the
Wolff chain `wolff_units` steps (its mean cluster size is |dM| / 2 per step);
E and M after every unit; tau_int of |M| and E from the
Madras-Sokal window per replica (averaged); effective samples per second =
replicas * units / (2 tau_int) / seconds, the seconds being each chain's own
device time (CUDA events on its stream), with CUDA-graph replay for both.

Timing (--time): device time per step and site updates per ns of the cluster
step and of a Metropolis sweep on the same lattices.

Everything runs through the C ABI (libising); this module only orchestrates.
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import ising, workloads

T_CRITICAL = workloads.T_CRITICAL


def _tau(series, c=6.0):
    taus = []
    for x in series:
        try:
            taus.append(ising.ising_tau_int(x, c)[0])
        except ising.IsingError:
            taus.append(float("nan"))
    t = np.array(taus)
    return float(np.nanmean(t)), float(np.nanstd(t) / math.sqrt(max(1, np.isfinite(t).sum())))


def _device_time(stream, fn):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def run_temperature(T: float, L: int = 256, replicas: int = 64, burn: int = 2000, units: int = 20000,
                    sw_units: int = 5000, sw_burn: int = 500, wolff_units: int = 20000, seed: int = 2024,
                    verbose: bool = True) -> dict:
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    s = torch.cuda.Stream(dev)
    N = L * L
    res = {"T": T, "L": L, "replicas": replicas}
    with torch.cuda.stream(s):
        plain = ising.IsingSim(L, [T] * replicas, seed, trace_cap=units, stream=s)
        plain.set_graph(True)
        plain.sw_sweep(sw_burn)                   # cluster steps equilibrate fast at and below T_c
        plain.sweep(burn)
        state = ising.ising_save(plain.h)
        cluster = ising.IsingSim(L, [T] * replicas, seed, trace_cap=sw_units, stream=s)
        ising.ising_load(cluster.h, state)
        cluster.set_graph(True)
        plain.autotune(probe_sweeps=20)
        t_plain = _device_time(s, lambda: plain.sweep(units))
        cluster.sw_sweep(1)                       # scratch allocation and graph capture outside the timing
        ising.ising_load(cluster.h, state)
        t_sw = _device_time(s, lambda: cluster.sw_sweep(sw_units))
        wolff = ising.IsingSim(L, [T] * replicas, seed, trace_cap=wolff_units, stream=s)
        ising.ising_load(wolff.h, state)
        wolff.wolff_sweep(1)                      # scratch allocation outside the timing
        ising.ising_load(wolff.h, state)
        t_wolff = _device_time(s, lambda: wolff.wolff_sweep(wolff_units))
        Ep, Mp = plain.trace(units)
        Es, Ms = cluster.trace(sw_units)
        Ew, Mw = wolff.trace(wolff_units)
    for name, E, M, secs, n in (("plain", Ep, Mp, t_plain, units), ("cluster", Es, Ms, t_sw, sw_units),
                                ("wolff", Ew, Mw, t_wolff, wolff_units)):
        tm, tm_err = _tau(np.abs(M).astype(np.float64))
        te, te_err = _tau(E.astype(np.float64))
        m_abs = np.abs(M).mean(axis=1) / N
        e = E.mean(axis=1) / N
        res[name] = {"units": n, "seconds": secs, "ms_per_unit": 1e3 * secs / n,
                     "tau_int_absM": tm, "tau_int_absM_err": tm_err, "tau_int_E": te, "tau_int_E_err": te_err,
                     "mean_abs_m": float(m_abs.mean()), "mean_abs_m_err": float(m_abs.std(ddof=1) / math.sqrt(replicas)),
                     "mean_e": float(e.mean()), "mean_e_err": float(e.std(ddof=1) / math.sqrt(replicas)),
                     "eff_samples_per_s_absM": replicas * n / (2 * tm) / secs,
                     "eff_samples_per_s_E": replicas * n / (2 * te) / secs}
    p, q, w = res["plain"], res["cluster"], res["wolff"]
    res["gain_eff_samples_absM"] = q["eff_samples_per_s_absM"] / p["eff_samples_per_s_absM"]
    res["gain_eff_samples_E"] = q["eff_samples_per_s_E"] / p["eff_samples_per_s_E"]
    res["wolff_gain_eff_samples_absM"] = w["eff_samples_per_s_absM"] / p["eff_samples_per_s_absM"]
    res["wolff_gain_eff_samples_E"] = w["eff_samples_per_s_E"] / p["eff_samples_per_s_E"]
    # mean cluster size per Wolff step from the magnetization trace (the
    # first step's predecessor is the common starting state's last value)
    dM = np.abs(np.diff(Mw.astype(np.int64), axis=1)) // 2
    w["mean_cluster_fraction"] = float(dM.mean()) / N
    w["agree_abs_m_sigma"] = abs(p["mean_abs_m"] - w["mean_abs_m"]) / math.hypot(p["mean_abs_m_err"], w["mean_abs_m_err"])
    w["agree_e_sigma"] = abs(p["mean_e"] - w["mean_e"]) / math.hypot(p["mean_e_err"], w["mean_e_err"])
    res["agree_abs_m_sigma"] = abs(p["mean_abs_m"] - q["mean_abs_m"]) / math.hypot(p["mean_abs_m_err"], q["mean_abs_m_err"])
    res["agree_e_sigma"] = abs(p["mean_e"] - q["mean_e"]) / math.hypot(p["mean_e_err"], q["mean_e_err"])
    if verbose:
        print(json.dumps(res), flush=True)
    plain.close()
    cluster.close()
    wolff.close()
    return res


def time_steps(name: str, Ls, temps, seeds, steps: int = 50) -> dict:
    """Device time per cluster step and per Metropolis sweep (graphs on)."""
    import torch
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        sim = ising.IsingSim(Ls=list(Ls), temps=list(temps), seeds=list(seeds), stream=s)
        sim.set_graph(True)
        sim.sw_sweep(steps)                        # capture + warm-up
        t_sw = _device_time(s, lambda: sim.sw_sweep(steps)) / steps
        sim.sweep(steps)
        t_mp = _device_time(s, lambda: sim.sweep(steps)) / steps
        sim.wolff_sweep(steps)
        t_w = _device_time(s, lambda: sim.wolff_sweep(steps)) / steps
    sites = sum(int(L) * int(L) for L in Ls)
    out = {"case": name, "lattices": len(Ls), "sites": sites,
           "cluster_ms_per_step": 1e3 * t_sw, "cluster_site_updates_per_ns": sites / t_sw / 1e9,
           "metropolis_ms_per_sweep": 1e3 * t_mp, "metropolis_flip_per_ns": sites / t_mp / 1e9,
           "wolff_ms_per_step": 1e3 * t_w}
    print(json.dumps(out), flush=True)
    sim.close()
    return out


def timing_cases():
    tc = T_CRITICAL
    b = workloads.binder_scan()
    return [
        ("64 x 256^2, T_c", [256] * 64, [tc] * 64, list(range(1, 65)), 50),
        ("4096^2, T_c", [4096], [tc], [1], 50),
        ("4096^2, T = 1.5", [4096], [1.5], [1], 50),
        ("4096^2, T = 3.0", [4096], [3.0], [1], 50),
        ("144 lattices 1024^2-4096^2 (Binder scan)", b.Ls, b.temps, b.seeds, 20),
        ("16384^2, T_c", [16384], [tc], [1], 10),
    ]


def timing_suite(only: int = -1, steps: int = 0) -> list:
    out = []
    for i, (name, Ls, temps, seeds, n) in enumerate(timing_cases()):
        if only < 0 or i == only:
            out.append(time_steps(name, Ls, temps, seeds, steps=steps or n))
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--temps", type=float, nargs="*", default=[2.20, T_CRITICAL, 2.35])
    ap.add_argument("--L", type=int, default=256)
    ap.add_argument("--replicas", type=int, default=64)
    ap.add_argument("--burn", type=int, default=2000)
    ap.add_argument("--units", type=int, default=20000)
    ap.add_argument("--sw-units", type=int, default=5000)
    ap.add_argument("--wolff-units", type=int, default=20000)
    ap.add_argument("--time", action="store_true", help="only the step timings")
    ap.add_argument("--case", type=int, default=-1, help="with --time: only this timing case")
    ap.add_argument("--steps", type=int, default=0, help="with --time: steps per timed call")
    args = ap.parse_args()
    if args.time:
        print(json.dumps({"cluster_timing": timing_suite(args.case, args.steps)}))
        return
    out = [run_temperature(T, L=args.L, replicas=args.replicas, burn=args.burn, units=args.units,
                           sw_units=args.sw_units, wolff_units=args.wolff_units) for T in args.temps]
    print(json.dumps({"cluster_study": out}))


if __name__ == "__main__":
    main()
