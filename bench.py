#!/usr/bin/env python3
"""Throughput benchmark: spin-flip attempts per ns on one GB300 (and N GPUs
as independent replicas).

Workload (default, the 16384^2 configuration): six 16384 x 16384 periodic
lattices, T in {1.5, 2.269185, 3.0} x {cold start, random start from seed 2};
one step = 1000 checkerboard sweeps of all six, with E and M recorded every
sweep.  The six lattices (192 MiB packed) are larger than L2; L2 is also
flushed between timed steps.  Flip attempts per step = 6 * 16384^2 * 1000.

Prints one JSON line (see the keys below).  --impl reference times the CPU
oracle (the slow reference definition of the same sweep) on the host cores on
a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

T_RUNS = (1.5, 2.269185, 3.0)
L256_SEED = 2024   # seed of the 64-lattice 256^2 workload (simulations 0 .. 63)
# algorithmic integer ops per site update: a quarter Philox4x32-10 block (15),
# the accept decision (3), the bitsliced neighbour count (0.5)
OPS_PER_SITE = 18.5
SINGLE_THREAD_L = 4096   # lattice of the single-thread oracle figure
# the paper's own figures, for context only (other hardware and workloads)
PAPER_CONTEXT = {
    "paper": "61,853 flip/ns aggregate on a Cerebras CS-2 (WSE-2) for 754 simulations (Section 3.2, Table 1)",
    "paper_gpu": "Romero et al.'s code as the paper quotes it: 880.6 flip/ns on one H100, 585.8 on one A100, "
                 "459 on one V100",
    "note": "other hardware and workloads: context, not a target",
}
# 32-bit integer lanes per SM of compute capability 10.x (Blackwell); the
# device query below supplies the SM count and the maximum SM clock
INT_LANES_PER_SM = {(10, 0): 128, (10, 3): 128}
# (workload, kernel, sites per launch) -> dram__bytes_read.sum +
# dram__bytes_write.sum of one launch of that kernel build, from an ncu full
# capture (first captured launch); other pairings report null
MEASURED_TRAFFIC = {("l16384", "stream_half_kernel<4>", 3 * 16384 * 16384 // 2): 110_270_720}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["l16384", "batch754", "l256x64"], default="l16384")
    ap.add_argument("--L", type=int, default=16384)
    ap.add_argument("--sweeps", type=int, default=0, help="sweeps per step (default 1000; 10000 for batch754 and l256x64)")
    ap.add_argument("--autotune", action="store_true",
                    help="(the default) autotune the plan before timing, outside the timed region")
    ap.add_argument("--no-autotune", action="store_true", help="time the library's default plan instead")
    ap.add_argument("--plan", choices=["tuned", "auto", "resident", "stream", "persist", "cluster"],
                    default="tuned",
                    help="force a plan instead of autotuning")
    ap.add_argument("--threads", type=int, default=0, help="with a forced plan: threads per block (0 = default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the effective-samples comparison (plain / learned / Swendsen-Wang)")
    ap.add_argument("--learned-units", type=int, default=20000)
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, device=None) -> float:
    """The largest x of all ranks (the slowest rank's time); x itself when not
    distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world_size: int, seconds_max: float) -> float:
    """Weak scaling: every rank processes units_per_rank; the job's rate is all
    ranks' units over the slowest rank's time (per ns)."""
    return units_per_rank * world_size / (seconds_max * 1e9)


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []
        self.err = None

    def __enter__(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception as e:  # nvidia-smi missing
            self.err = str(e)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=2)
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0,
                    "note": self.err or "no nvidia-smi samples"}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def device_figures(dev, uuid: str | None) -> dict:
    """SM count and compute capability from the device, the maximum SM clock
    from nvidia-smi (the GPU's own report; 2070 MHz, the GB300 maximum, if
    nvidia-smi is unavailable)."""
    import torch
    p = torch.cuda.get_device_properties(dev)
    cc = (p.major, p.minor)
    mhz, src = 2070.0, "GB300 maximum (nvidia-smi unavailable)"
    try:
        cmd = ["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"]
        if uuid:
            cmd += ["-i", uuid]
        out = subprocess.run(cmd, capture_output=True, text=True, timeout=20).stdout.strip().splitlines()
        if out:
            mhz, src = float(out[0]), "nvidia-smi clocks.max.sm"
    except (OSError, subprocess.SubprocessError, ValueError):
        pass
    return {"sms": p.multi_processor_count, "cc": cc, "int_lanes_per_sm": INT_LANES_PER_SM.get(cc, 128),
            "sm_max_mhz": mhz, "clock_source": src}


def workload_sweeps(args) -> int:
    return args.sweeps or (1000 if args.workload == "l16384" else 10000)


def workload_config(args, rank: int = 0) -> dict:
    """The `config` block both arms print for the workload: what is swept,
    its sizes and the flip attempts of one step on one GPU."""
    n_sw = workload_sweeps(args)
    if args.workload == "l16384":
        L = args.L
        return {"workload": f"six {L}x{L} periodic lattices, T in {{1.5, 2.269185, 3.0}} x "
                            f"{{cold, random seed 2}}, {n_sw} checkerboard sweeps per step, "
                            f"E/M recorded every sweep",
                "lattices_per_gpu": 6, "L": L, "sweeps_per_step": n_sw,
                "flips_per_step_per_gpu": 6 * L * L * n_sw,
                "l2": f"flushed between timed steps; working set {6 * L * L // 8 / 2**20:g} MiB "
                      f"({'>' if 6 * L * L // 8 > 129e6 else '<'} 129 MB L2)"}
    if args.workload == "l256x64":
        return {"workload": f"64 lattices of 256x256 at T=2.269185 (the learned-proposal study's plain chain), "
                            f"random starts (seed {L256_SEED + 1000 * rank}, simulations 0..63), {n_sw} sweeps "
                            f"per step, one launch per step",
                "lattices_per_gpu": 64, "L": 256, "sweeps_per_step": n_sw,
                "flips_per_step_per_gpu": 64 * 256 * 256 * n_sw, "l2": "flushed between timed steps"}
    from paper_2404_16990_gb300 import workloads
    wl = workloads.batch754(master_seed=20240426 + rank)
    sites = sum(L * L for L in wl.Ls)
    return {"workload": f"754 lattices, L in {{128,256,512,1024}} log-uniform, T ~ U[1.8,2.8], "
                        f"random starts, {n_sw} sweeps per step, one persistent launch per step",
            "lattices_per_gpu": 754, "spins_per_gpu": sites, "sweeps_per_step": n_sw,
            "flips_per_step_per_gpu": sites * n_sw, "l2": "flushed between timed steps"}


# ---------------------------------------------------------------------------
# CPU oracle timing (the reference arm and the cpu_baseline object)
# ---------------------------------------------------------------------------
def host_cpu_model() -> str:
    """The host CPU's model name as lscpu reports it (else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.machine() or "unknown"


def time_oracle(L: int, seconds: float, max_sweeps: int | None = None, threads: int | None = None):
    import oracle
    cores = threads or os.cpu_count() or 1
    lat = oracle.init(L, 2, 0, n_threads=cores)
    done, t_total = 0, 0.0
    n = 1
    while (t_total < seconds or done == 0) and (max_sweeps is None or done < max_sweeps):
        if max_sweeps is not None:
            n = min(n, max_sweeps - done)
        t0 = time.perf_counter()
        oracle.sweeps(lat, 2.269185, 2, 0, done, n, n_threads=cores)
        t_total += time.perf_counter() - t0
        done += n
        n = min(n * 2, 64)
    flips = done * L * L
    return {"value": flips / (t_total * 1e9), "unit": "flip/ns", "cores": cores, "kind": "oracle",
            "sample": f"{done} sweep{'s' if done != 1 else ''} of one {L}x{L} lattice (random start seed 2, "
                      f"T=2.269185, E/M each sweep), oracle on "
                      + ("1 host thread" if cores == 1 else
                         f"{cores} host threads (rows of one colour split across threads)"),
            "seconds": t_total}


def cpu_baseline(L: int, seconds: float) -> dict:
    """The `cpu_baseline` object: the oracle on every host thread for about
    `seconds` on one L x L lattice, plus a single-thread figure on a lattice of
    at most 4096^2 (one 16384^2 sweep on one thread would take tens of
    seconds) and the host CPU's model."""
    cpu = time_oracle(L, seconds)
    cpu.pop("seconds", None)
    one = time_oracle(min(L, SINGLE_THREAD_L), seconds / 4, threads=1)
    cpu["single_thread"] = {"value": one["value"], "unit": "flip/ns", "sample": one["sample"]}
    cpu["cpu_model"] = host_cpu_model()
    return cpu


def time_oracle_batch(workload: str, rank: int = 0):
    """One sweep of every lattice of a batch workload (754 lattices, or 64 of
    256^2) by the oracle, lattices spread over the host threads."""
    import oracle
    from paper_2404_16990_gb300 import workloads
    cores = os.cpu_count() or 1
    if workload == "l256x64":
        Ls, temps, seeds = [256] * 64, [T_RUNS[1]] * 64, [L256_SEED + 1000 * rank] * 64
        what = "64 lattices of 256x256"
    else:
        wl = workloads.batch754(master_seed=20240426 + rank)
        Ls, temps, seeds = wl.Ls, wl.temps, wl.seeds
        what = "754 lattices"
    sig = [oracle.init(L, sd, i) for i, (L, sd) in enumerate(zip(Ls, seeds))]
    t0 = time.perf_counter()
    oracle.sweeps_batch(sig, temps, seeds, list(range(len(sig))), 0, 1, n_threads=cores)
    secs = time.perf_counter() - t0
    flips = sum(L * L for L in Ls)
    return {"value": flips / (secs * 1e9), "unit": "flip/ns", "cores": cores, "kind": "oracle",
            "sample": f"1 sweep of all {what} (random starts), oracle on "
                      f"{cores} host threads (one lattice per thread at a time)",
            "seconds": secs, "flips": flips}


def reference_arm(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    per_step = []
    for i in range(args.warmup + args.steps):
        if args.workload == "l16384":
            r = time_oracle(args.L, 0.0, max_sweeps=1)
            r["flips"] = args.L * args.L
        else:
            r = time_oracle_batch(args.workload)
        if i >= args.warmup:
            per_step.append(r)
    secs = sum(r["seconds"] for r in per_step)
    value = sum(r["flips"] for r in per_step) / (secs * 1e9)
    cb = dict(per_step[0])
    cb["value"] = value
    if args.workload == "l16384":
        cb["sample"] = (f"each step: 1 sweep of one {args.L}x{args.L} lattice (random start seed 2, "
                        f"T=2.269185) by the CPU oracle on {cb['cores']} threads")
    else:
        cb["sample"] = "each step: " + cb["sample"]
    cb.pop("seconds", None)
    cb.pop("flips", None)
    cb["cpu_model"] = host_cpu_model()
    line = {"impl": "reference", "metric": "spin-flip attempts/ns", "value": value, "unit": "flip/ns",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": secs / len(per_step) * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int8", "data": "synthetic",
            "config": workload_config(args),
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "flip/ns", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "context": PAPER_CONTEXT}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the metric's second half: effective samples per second, learned vs plain
# ---------------------------------------------------------------------------
def learned_vs_plain(units: int = 20000) -> dict:
    """Effective independent |M| and E samples per second of plain sweeps,
    the learned patch proposal (trained on the GPU on plain-sampler
    snapshots) and Swendsen-Wang steps, on the learned-proposal workload at
    T_c: 64 replicas of 256^2, one equilibrated start, `units` units per
    chain; tau_int from the library's Madras-Sokal window, seconds from CUDA
    events.  A failure is reported in the record, not raised."""
    try:
        from paper_2404_16990_gb300 import learned_study
        r = learned_study.effective_samples(T=T_RUNS[1], units=units)
    except Exception as e:  # the throughput line stands on its own
        return {"error": f"{type(e).__name__}: {e}"}
    chains = {"plain": r["plain"], "learned": r["learned"], "swendsen_wang": r["swendsen_wang"]}
    return {
        "workload": f"64 replicas of 256x256 at T={T_RUNS[1]}, random start equilibrated by 500 Swendsen-Wang "
                    f"steps and 2000 sweeps; learned net trained 1500 Adam steps on {r['train_pool']} plain-sampler "
                    f"snapshots; {units} units per chain (learned unit = patch round + sweep)",
        "metric": "effective independent |M| samples/s (tau_int, Madras-Sokal window)",
        "eff_samples_per_s_absM": {k: v["eff_samples_per_s_absM"] for k, v in chains.items()},
        "eff_samples_per_s_E": {k: v["eff_samples_per_s_E"] for k, v in chains.items()},
        "learned_over_plain_absM": r["gain_eff_samples_absM"],
        "sw_over_plain_absM": r["gain_sw_eff_samples_absM"],
        "tau_int_absM": {k: v["tau_int_absM"] for k, v in chains.items()},
        "units_per_s": {k: v["units_per_s"] for k, v in chains.items()},
        "acceptance": r["acceptance"], "acceptance_untrained": r["acceptance_untrained"],
        "agree_sigma_learned_vs_plain": {"abs_m": r["agree_abs_m_sigma"], "e": r["agree_e_sigma"]},
        "timing": "CUDA events on the chains' stream; training and set-up outside the timed chains",
    }


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def ours(args):
    import torch
    from paper_2404_16990_gb300 import ising

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    L = args.L
    sims = []
    tuned = None
    if args.workload == "l16384":
        n_sw = workload_sweeps(args)
        seed = 2 + 1000 * rank  # independent replicas per rank; rank 0 is the configured seed 2
        with torch.cuda.stream(stream):
            for cold in (True, False):
                s = ising.IsingSim(Ls=[L] * 3, temps=list(T_RUNS), seeds=[seed] * 3, cold=cold,
                                   trace_cap=n_sw, stream=stream, device=dev)
                sims.append(s)
    elif args.workload == "l256x64":
        n_sw = workload_sweeps(args)
        with torch.cuda.stream(stream):
            sims.append(ising.IsingSim(256, [T_RUNS[1]] * 64, L256_SEED + 1000 * rank, trace_cap=0, stream=stream,
                                       device=dev))
    else:
        from paper_2404_16990_gb300 import workloads
        n_sw = workload_sweeps(args)
        wl = workloads.batch754(master_seed=20240426 + rank)
        with torch.cuda.stream(stream):
            s = ising.IsingSim(Ls=wl.Ls, temps=wl.temps, seeds=wl.seeds, trace_cap=0, stream=stream, device=dev)
            sims.append(s)
    if args.plan != "tuned":
        code = {"auto": ising.ISING_PLAN_AUTO, "resident": ising.ISING_PLAN_RESIDENT,
                "stream": ising.ISING_PLAN_STREAM, "persist": ising.ISING_PLAN_PERSIST,
                "cluster": ising.ISING_PLAN_CLUSTER}[args.plan]
        for s in sims:
            s.set_plan(code, threads=args.threads)
    for s in sims:
        s.set_graph(True)
    if args.plan == "tuned" and not args.no_autotune:
        # the library's autotuner picks the plan (saves and restores the
        # lattices and the sweep counter: no result changes)
        tuned = [s.autotune(probe_sweeps=5 if args.workload == "l16384" else 20) for s in sims]
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    sites = sum(sum(int(ising.ising_lattice_size(s.h, i)) ** 2 for i in range(s.n)) for s in sims)
    flips_per_step = sites * n_sw

    def step():
        for s in sims:
            s.sweep(n_sw)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if ws > 1:
        dist.barrier()

    launches0 = sum(ising.ising_kernel_launches(s.h) for s in sims)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = None
    torch.cuda.synchronize(dev)
    with ClockSampler(uuid) as clk:
        time.sleep(0.3)
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(i & 0xFF)            # L2 flush between timed steps
                ev[i][0].record(stream)
                step()
                ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
        time.sleep(0.3)
    launches = sum(ising.ising_kernel_launches(s.h) for s in sims) - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), dev)
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(flips_per_step, ws, ms_per_step / 1e3)

    # dominant kernel, from the plan in use: streaming half-sweeps (two
    # launches per sweep per handle), the cooperative persistent streaming
    # kernel or the resident kernel (one launch per sweep call per handle),
    # the cluster-resident kernel (one launch per lattice side per sweep call);
    # either way the algorithmic ops of the timed region over its duration
    plan = ising.ising_get_plan(sims[0].h)
    V = plan["words_per_thread"]
    if plan["plan"] == ising.ISING_PLAN_RESIDENT:
        kname, n_launch = "resident_kernel", len(sims) * args.steps
    elif plan["plan"] == ising.ISING_PLAN_CLUSTER:
        sides = [len({int(ising.ising_lattice_size(s.h, i)) for i in range(s.n)}) for s in sims]
        kname, n_launch = "cluster_resident_kernel", sum(sides) * args.steps
    elif plan["plan"] == ising.ISING_PLAN_PERSIST:
        kname, n_launch = f"stream_persist_kernel<{V}>", len(sims) * args.steps
    else:
        kname, n_launch = f"stream_half_kernel<{V}>", 2 * n_sw * len(sims) * args.steps
    avg_launch_s = (sum(step_ms) / 1e3) / n_launch
    sites_per_launch = flips_per_step * args.steps / n_launch
    achieved = OPS_PER_SITE * sites_per_launch / avg_launch_s / 1e12
    devf = device_figures(dev, uuid)
    peak = devf["sms"] * devf["int_lanes_per_sm"] * devf["sm_max_mhz"] * 1e6 / 1e12
    # DRAM bytes (read + write) per launch from the ncu capture of this kernel
    # on this workload; null for any other kernel / workload pairing
    traffic = None
    cap = MEASURED_TRAFFIC.get((args.workload, kname, int(round(sites_per_launch))))
    if cap is not None:
        traffic = cap

    # end-to-end through the public API: host checkpoint in (pinned), sweeps,
    # E/M traces and observables out, every step
    e2e = None
    if not args.no_e2e:
        nbytes = [ising.ising_state_bytes(s.h) for s in sims]
        host = [torch.empty(nb, dtype=torch.uint8, pin_memory=True) for nb in nbytes]
        for s, hb, nb in zip(sims, host, nbytes):
            ising.ising_save_to(s.h, hb.data_ptr(), nb)
        d2h = 0
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            d2h = 0
            for s, hb, nb in zip(sims, host, nbytes):
                ising.ising_load_from(s.h, hb.data_ptr(), nb)
                s.sweep(n_sw)
            for s in sims:
                E, M = s.trace(n_sw)
                Eo, Mo = s.observables()
                d2h += E.nbytes + M.nbytes + Eo.nbytes + Mo.nbytes
        torch.cuda.synchronize(dev)
        wall = max_over_ranks(time.perf_counter() - t0, dev)
        e2e_val = whole_job_rate(flips_per_step * args.e2e_steps, ws, wall)
        e2e = {"value": e2e_val, "unit": "flip/ns", "h2d_bytes_per_step": int(sum(nbytes)),
               "d2h_bytes_per_step": int(d2h)}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and args.workload == "l16384":
        cpu = cpu_baseline(L, args.cpu_seconds)
    learned = None
    if rank == 0 and ws == 1 and not args.no_learned and args.workload == "l16384":
        learned = learned_vs_plain(args.learned_units)

    if rank == 0:
        cfg = workload_config(args, rank)
        assert cfg["flips_per_step_per_gpu"] == flips_per_step
        cfg.update({"kernel": kname + ", CUDA graph", "plan": plan, "autotune_probe_flip_per_ns": tuned})
        line = {
            "metric": "spin-flip attempts/ns", "value": value, "unit": "flip/ns", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": cfg,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": kname, "ops_per_site": OPS_PER_SITE,
                         "peak_basis": f"{devf['sms']} SMs x {devf['int_lanes_per_sm']} int32 lanes x "
                                       f"{devf['sm_max_mhz']:.0f} MHz ({devf['clock_source']}; SM count from the "
                                       f"device)"},
            "cpu_baseline": cpu,
            "learned_vs_plain": learned,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
            "context": PAPER_CONTEXT,
        }
        print(json.dumps(line), flush=True)
    for s in sims:
        s.close()
    if ws > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
