"""The plain-C example of the ABI (paper_2404_16990_gb300/examples/sweep.c),
built against the in-tree libising.so and run on the GPU: its printed E/N and
M/N after 1000 sweeps of a 256^2 lattice at T_c equal the oracle's for the
same lattice (seed 1, simulation 0, random start), to the six printed
digits -- and so does the output its header records."""
from __future__ import annotations

import os
import re
import subprocess

import pytest

import oracle
from paper_2404_16990_gb300 import ising

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def test_c_example_runs_and_matches_the_oracle(tmp_path):
    lib_path = ising._build.build()
    lib_dir = os.path.dirname(lib_path)
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    src = os.path.join(ROOT, "paper_2404_16990_gb300", "examples", "sweep.c")
    exe = str(tmp_path / "sweep")
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", src, "-I" + os.path.join(ROOT, "include"),
                        "-I" + os.path.join(cuda, "include"), "-L" + lib_dir, "-lising",
                        "-L" + os.path.join(cuda, "lib64"), "-lcudart", "-Wl,-rpath," + lib_dir, "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    env = dict(os.environ)
    env["LD_LIBRARY_PATH"] = os.path.join(cuda, "lib64") + os.pathsep + env.get("LD_LIBRARY_PATH", "")
    run = subprocess.run([exe], capture_output=True, text=True, timeout=300, env=env)
    assert run.returncode == 0, run.stderr
    got = re.search(r"E/N = (-?[0-9.]+), M/N = (-?[0-9.]+)", run.stdout)
    assert got, run.stdout
    sigma = oracle.init(256, 1, 0)
    E, M = oracle.sweeps(sigma, 2.269185, 1, 0, 0, 1000, n_threads=max(1, min(16, os.cpu_count() or 1)))
    want = (f"{E[-1] / 65536:.6f}", f"{M[-1] / 65536:.6f}")
    assert (got.group(1), got.group(2)) == want
    recorded = re.search(r"E/N = (-?[0-9.]+), M/N = (-?[0-9.]+)", open(src).read())
    assert (recorded.group(1), recorded.group(2)) == want
