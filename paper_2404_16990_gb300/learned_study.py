"""Plain sweeps vs the learned patch proposal near T_c: training on plain-
sampler snapshots, then integrated autocorrelation times and effective
independent samples per second of |M| and E at equal observables.

Workload (per temperature): `replicas` lattices of side L (defaults 64 x
256^2) from random starts, equilibrated by `sw_burn` Swendsen-Wang steps and
`burn` plain sweeps; `n_snap` snapshots (one every `snap_every` sweeps, all
replicas at once) form the training pool; the net is
trained with Adam on random 10x10 windows of the pool; then two chains start
from the same equilibrated state:
  plain    one unit = one checkerboard sweep
  learned  one unit = one learned patch round (a quarter of the lattice
           proposed as 8x8 patches) followed by one checkerboard sweep
E and M are recorded after every unit; tau_int of |M| and E comes from the
Madras-Sokal window per replica (averaged); effective samples per second =
replicas * units / (2 tau_int) / seconds, the seconds being the chain's own
device time (CUDA events).

Everything runs through the C ABI (libising); this module only orchestrates.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import ising

T_CRITICAL = 2.269185


def default_params(seed: int, gain: float = 1.0) -> np.ndarray:
    """Seeded initial weights: N(0, gain^2 / fan_in) for the used weights,
    small biases, zero for the three padding features."""
    rng = np.random.default_rng(seed)
    parts = []
    w1 = np.zeros((16, 16))
    w1[:13] = rng.standard_normal((13, 16)) * gain / math.sqrt(13)
    parts += [w1.ravel(), rng.standard_normal(16) * 0.05]
    for _ in range(2):
        parts += [(rng.standard_normal((5, 16, 16)) * gain / math.sqrt(80)).ravel(), rng.standard_normal(16) * 0.05]
    parts += [(rng.standard_normal((5, 16)) * gain / math.sqrt(80)).ravel(), np.zeros(1)]
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == ising.ISING_NET_PARAMS
    return p


def _tau(series, c=6.0):
    taus = []
    for x in series:
        try:
            taus.append(ising.ising_tau_int(x, c)[0])
        except ising.IsingError:
            taus.append(float("nan"))
    t = np.array(taus)
    return float(np.nanmean(t)), float(np.nanstd(t) / math.sqrt(max(1, np.isfinite(t).sum())))


def _obs_stats(E, M, N):
    m_abs = np.abs(M).mean(axis=1) / N        # per replica
    e = E.mean(axis=1) / N
    return (float(m_abs.mean()), float(m_abs.std(ddof=1) / math.sqrt(len(m_abs))),
            float(e.mean()), float(e.std(ddof=1) / math.sqrt(len(e))))


def run_temperature(T: float, L: int = 256, replicas: int = 64, burn: int = 2000, n_snap: int = 20000,
                    snap_every: int = 10, train_steps: int = 1500, batch: int = 512, lr: float = 3e-3,
                    units: int = 20000, sw_burn: int = 500, seed: int = 2024, verbose: bool = True) -> dict:
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(dev)
    N = L * L
    res = {"T": T, "L": L, "replicas": replicas}
    with torch.cuda.stream(stream):
        sim = ising.IsingSim(L, [T] * replicas, seed, trace_cap=units, stream=stream)
        sim.sw_sweep(sw_burn)                           # cluster steps equilibrate fast at and below T_c
        sim.sweep(burn)
        per = L * L // 8
        sets = max(1, n_snap // replicas)
        pool = torch.empty(sets * replicas * per, dtype=torch.uint8, device=dev)
        for k in range(sets):
            sim.sweep(snap_every)
            ising.ising_snapshot(sim.h, pool.data_ptr() + k * replicas * per, replicas * per)
        torch.cuda.synchronize(dev)
        res["train_pool"] = sets * replicas
        n_win = max(batch, replicas * (L // 16) ** 2)
        net = ising.IsingNet(max_windows=n_win, max_lattices=replicas, stream=stream, max_batch=batch)
        net.set_params(default_params(seed))
        t0 = time.perf_counter()
        losses = net.train(pool.data_ptr(), sets * replicas, L, train_steps, batch, lr, seed)
        res["train_seconds"] = time.perf_counter() - t0
        res["loss_first"] = float(losses[:10].mean())
        res["loss_last"] = float(losses[-50:].mean())
        res["loss_per_site_last"] = res["loss_last"] / 64.0
        sim.set_graph(True)
        sim.autotune(probe_sweeps=20)                   # fastest plan for the plain chain
        state = ising.ising_save(sim.h)
        learned = ising.IsingSim(L, [T] * replicas, seed, trace_cap=units, stream=stream)
        ising.ising_load(learned.h, state)
        learned.set_graph(True)
        learned.autotune(probe_sweeps=20)
        res["plain_plan"] = ising.ising_get_plan(sim.h)
        # what training buys: acceptance of the untrained initial net
        untrained = ising.IsingNet(max_windows=n_win, max_lattices=replicas, stream=stream, max_batch=batch)
        untrained.set_params(default_params(seed))
        probe = ising.IsingSim(L, [T] * replicas, seed, stream=stream)
        ising.ising_load(probe.h, state)
        acc0 = sum(int(probe.learned_round(untrained, r).sum()) for r in range(8))
        res["acceptance_untrained"] = acc0 / (8 * replicas * (L // 16) ** 2)
        probe.close()
        untrained.close()
        # plain chain
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.sweep(units)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        t_plain = e0.elapsed_time(e1) / 1e3
        Ep, Mp = sim.trace(units)
        # learned chain: round r, then one sweep
        learned.learned_round(net, 0, sync=True)      # uploads the lattice table once
        ising.ising_load(learned.h, state)
        net.accepted(replicas, reset=True)
        e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        for u in range(units):
            learned.learned_round(net, u, sync=False)
            learned.sweep(1)
        e3.record(stream)
        torch.cuda.synchronize(dev)
        acc = net.accepted(replicas)
        t_learned = e2.elapsed_time(e3) / 1e3
        El, Ml = learned.trace(units)
    patches = units * replicas * (L // 16) ** 2
    res["acceptance"] = float(acc.sum() / patches)
    res["learned_unit_ms"] = 1e3 * t_learned / units
    res["plain_sweep_ms"] = 1e3 * t_plain / units
    for name, E, M, secs in (("plain", Ep, Mp, t_plain), ("learned", El, Ml, t_learned)):
        tm, tm_err = _tau(np.abs(M).astype(np.float64))
        te, te_err = _tau(E.astype(np.float64))
        m, dm, e, de = _obs_stats(E, M, N)
        res[name] = {"units": units, "seconds": secs, "units_per_s": units / secs,
                     "tau_int_absM": tm, "tau_int_absM_err": tm_err, "tau_int_E": te, "tau_int_E_err": te_err,
                     "mean_abs_m": m, "mean_abs_m_err": dm, "mean_e": e, "mean_e_err": de,
                     "eff_samples_per_s_absM": replicas * units / (2 * tm) / secs,
                     "eff_samples_per_s_E": replicas * units / (2 * te) / secs}
    p, q = res["plain"], res["learned"]
    res["gain_eff_samples_absM"] = q["eff_samples_per_s_absM"] / p["eff_samples_per_s_absM"]
    res["gain_eff_samples_E"] = q["eff_samples_per_s_E"] / p["eff_samples_per_s_E"]
    res["agree_abs_m_sigma"] = abs(p["mean_abs_m"] - q["mean_abs_m"]) / math.hypot(p["mean_abs_m_err"], q["mean_abs_m_err"])
    res["agree_e_sigma"] = abs(p["mean_e"] - q["mean_e"]) / math.hypot(p["mean_e_err"], q["mean_e_err"])
    if verbose:
        print(json.dumps(res), flush=True)
    sim.close()
    learned.close()
    net.close()
    return res


def effective_samples(T: float = T_CRITICAL, L: int = 256, replicas: int = 64, units: int = 20000,
                      sw_steps: int = 5000, train_steps: int = 1500, n_snap: int = 20000, burn: int = 2000,
                      seed: int = 2024) -> dict:
    """Effective independent |M| (and E) samples per second of three chains
    from one equilibrated state: plain sweeps, the learned proposal (one
    patch round + one sweep per unit) and Swendsen-Wang steps; tau_int by the
    library's Madras-Sokal window per replica, seconds by CUDA events on the
    chains' stream.  Returns the learned-vs-plain record of run_temperature
    with a "swendsen_wang" entry and the two ratios added."""
    import torch
    res = run_temperature(T, L=L, replicas=replicas, burn=burn, n_snap=n_snap, train_steps=train_steps,
                          units=units, seed=seed, verbose=False)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(dev)
    N = L * L
    with torch.cuda.stream(stream):
        sim = ising.IsingSim(L, [T] * replicas, seed, trace_cap=sw_steps, stream=stream)
        sim.sw_sweep(500)
        sim.sweep(burn)
        sim.set_graph(True)
        sim.sw_sweep(10)                                 # scratch and graph set up outside the timed region
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.sw_sweep(sw_steps)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        secs = e0.elapsed_time(e1) / 1e3
        E, M = sim.trace(sw_steps)
    tm, tm_err = _tau(np.abs(M).astype(np.float64))
    te, te_err = _tau(E.astype(np.float64))
    m, dm, e, de = _obs_stats(E, M, N)
    res["swendsen_wang"] = {"units": sw_steps, "seconds": secs, "units_per_s": sw_steps / secs,
                            "tau_int_absM": tm, "tau_int_absM_err": tm_err, "tau_int_E": te, "tau_int_E_err": te_err,
                            "mean_abs_m": m, "mean_abs_m_err": dm, "mean_e": e, "mean_e_err": de,
                            "eff_samples_per_s_absM": replicas * sw_steps / (2 * tm) / secs,
                            "eff_samples_per_s_E": replicas * sw_steps / (2 * te) / secs}
    p = res["plain"]
    res["gain_sw_eff_samples_absM"] = res["swendsen_wang"]["eff_samples_per_s_absM"] / p["eff_samples_per_s_absM"]
    res["gain_sw_eff_samples_E"] = res["swendsen_wang"]["eff_samples_per_s_E"] / p["eff_samples_per_s_E"]
    sim.close()
    return res


def round_bench(rounds: int = 20, L: int = 256, replicas: int = 64, precision: int = 0, seed: int = 7) -> dict:
    """Device time of learned rounds alone (no training: seeded initial net) on
    `replicas` lattices of side L at T_c."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    s = torch.cuda.Stream(dev)
    with torch.cuda.stream(s):
        sim = ising.IsingSim(L, [T_CRITICAL] * replicas, seed, stream=s)
        sim.sweep(100)
        net = ising.IsingNet(max_windows=replicas * (L // 16) ** 2, max_lattices=replicas, stream=s, max_batch=512)
        net.set_params(default_params(1))
        net.set_precision(precision)
        sim.learned_round(net, 0)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for r in range(rounds):
            sim.learned_round(net, r + 1, sync=False)
        e1.record(s)
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / max(1, rounds)
    out = {"round_ms": ms, "patches": replicas * (L // 16) ** 2, "precision": "fp8" if precision else "bf16",
           "accepted_fraction": float(net.accepted(replicas).sum()) / (rounds * replicas * (L // 16) ** 2)}
    print(json.dumps(out), flush=True)
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--temps", type=float, nargs="*", default=[2.20, T_CRITICAL, 2.35])
    ap.add_argument("--L", type=int, default=256)
    ap.add_argument("--replicas", type=int, default=64)
    ap.add_argument("--burn", type=int, default=2000)
    ap.add_argument("--snapshots", type=int, default=20000)
    ap.add_argument("--train-steps", type=int, default=1500)
    ap.add_argument("--units", type=int, default=20000)
    ap.add_argument("--round-bench", type=int, default=0, help="only time this many learned rounds")
    ap.add_argument("--fp8", action="store_true", help="with --round-bench: FP8 inference")
    args = ap.parse_args()
    if args.round_bench:
        round_bench(args.round_bench, L=args.L, replicas=args.replicas, precision=1 if args.fp8 else 0)
        return
    out = [run_temperature(T, L=args.L, replicas=args.replicas, burn=args.burn, n_snap=args.snapshots,
                           train_steps=args.train_steps, units=args.units) for T in args.temps]
    print(json.dumps({"learned_study": out}))


if __name__ == "__main__":
    main()
