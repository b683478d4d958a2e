"""bench.py's reference arm on CPU: it times the oracle on a bounded sample
and prints the contract's JSON line with the same workload `config` as the
GPU arm."""
from __future__ import annotations

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*argv):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *argv], capture_output=True, text=True,
                         timeout=600, cwd=ROOT, check=True).stdout.strip().splitlines()
    assert len(out) == 1
    return json.loads(out[0])


def test_reference_line_keys_and_config():
    import argparse
    import bench
    line = _run("--impl", "reference", "--L", "512", "--steps", "2", "--warmup", "1")
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 1
    assert line["metric"] == "spin-flip attempts/ns" and line["unit"] == "flip/ns" and line["higher_is_better"]
    assert line["value"] > 0 and line["ms_per_step"] > 0
    want = bench.workload_config(argparse.Namespace(workload="l16384", L=512, sweeps=0))
    assert line["config"] == want
    assert want["flips_per_step_per_gpu"] == 6 * 512 * 512 * 1000
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    assert cb["cpu_model"]
    assert "61,853 flip/ns" in line["context"]["paper"]
    assert line["e2e"] == {"value": line["value"], "unit": "flip/ns", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_batch_workload_config():
    import argparse
    import bench
    cfg = bench.workload_config(argparse.Namespace(workload="batch754", L=16384, sweeps=0))
    assert cfg["lattices_per_gpu"] == 754 and cfg["sweeps_per_step"] == 10000
    assert cfg["flips_per_step_per_gpu"] == cfg["spins_per_gpu"] * 10000


def test_small_lattice_workload_reference_line():
    """The 64-lattice 256^2 workload (the learned-proposal study's plain
    chain): the reference arm sweeps all 64 lattices once per step."""
    import argparse
    import bench
    cfg = bench.workload_config(argparse.Namespace(workload="l256x64", L=16384, sweeps=0))
    assert cfg["lattices_per_gpu"] == 64 and cfg["L"] == 256 and cfg["sweeps_per_step"] == 10000
    assert cfg["flips_per_step_per_gpu"] == 64 * 256 * 256 * 10000
    line = _run("--impl", "reference", "--workload", "l256x64", "--steps", "1", "--warmup", "0")
    assert line["config"] == cfg and line["value"] > 0
    assert line["cpu_baseline"]["sample"].startswith("each step: 1 sweep of all 64 lattices of 256x256")


def test_oracle_timing_on_one_thread():
    import bench
    r = bench.time_oracle(256, 0.0, threads=1)              # no time budget: one sweep
    assert r["cores"] == 1 and r["value"] > 0 and r["sample"].startswith("1 sweep of one 256x256")
    assert r["sample"].endswith("oracle on 1 host thread")
    r = bench.time_oracle(256, 10.0, max_sweeps=3, threads=2)  # the sweep cap ends it first
    assert r["cores"] == 2 and r["sample"].startswith("3 sweeps of one 256x256")
    assert bench.host_cpu_model()


def test_cpu_baseline_object():
    import bench
    cb = bench.cpu_baseline(512, 0.0)
    assert cb["kind"] == "oracle" and cb["unit"] == "flip/ns" and cb["value"] > 0 and cb["cores"] >= 1
    assert "seconds" not in cb and cb["cpu_model"]
    st = cb["single_thread"]
    assert st["value"] > 0 and st["unit"] == "flip/ns" and st["sample"].endswith("on 1 host thread")


def test_reference_arm_under_torchrun_prints_once():
    # two ranks on one node: rank 0 alone times the oracle and prints one line,
    # the other rank exits 0 without work
    import socket
    import sys
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
                        "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--L", "256"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
