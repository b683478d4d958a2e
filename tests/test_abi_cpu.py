"""C-ABI checks that need no GPU: the library builds, loads and exports every
function include/*.h declares; workspace sizes follow the documented layout;
invalid arguments are rejected with ISING_EINVAL before any device work."""
from __future__ import annotations

import ctypes
import glob
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2404_16990_gb300 import ising

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b([A-Za-z_][A-Za-z0-9_]*)\s*\([^;{)]*\)\s*;", text):
            name = m.group(1)
            if name not in ("if", "while", "for", "return", "sizeof"):
                names.add(name)
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("ising_create", "ising_sweep", "ising_observables", "ising_create_batch",
                     "ising_workspace_bytes", "ising_destroy", "ising_last_error"):
        assert required in names


@pytest.mark.parametrize("lang,compiler,std", [("c", "gcc", "-std=c99"), ("c++", "g++", "-std=c++17")])
def test_headers_compile_cleanly_as_c_and_cxx(lang, compiler, std, tmp_path):
    # a plain C ABI: every header compiles alone, warning-free, in C and C++
    for hdr in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        src = tmp_path / ("use." + ("c" if lang == "c" else "cpp"))
        src.write_text(f'#include "{os.path.basename(hdr)}"\nint main(void) {{ return 0; }}\n')
        r = subprocess.run([compiler, std, "-Wall", "-Wextra", "-Werror", "-pedantic", "-fsyntax-only",
                            "-I" + os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
        assert r.returncode == 0, (hdr, r.stderr)


def test_plain_c_example_builds_against_the_library(tmp_path):
    # paper_2404_16990_gb300/examples/sweep.c uses the ABI from C alone: it
    # compiles warning-free and links against libising.so (not run: no GPU here)
    lib_path = ising._build.build()
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    src = os.path.join(ROOT, "paper_2404_16990_gb300", "examples", "sweep.c")
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", src, "-I" + os.path.join(ROOT, "include"),
                        "-I" + os.path.join(cuda, "include"), "-L" + os.path.dirname(lib_path), "-lising",
                        "-L" + os.path.join(cuda, "lib64"), "-lcudart", "-o", str(tmp_path / "sweep")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_c_example_recorded_output_is_the_oracles():
    # the E/N and M/N that sweep.c's header records from a GB300 run equal the
    # oracle's for the same lattice (256^2, seed 1, sim 0, T = 2.269185, 1000 sweeps)
    import oracle
    text = open(os.path.join(ROOT, "paper_2404_16990_gb300", "examples", "sweep.c")).read()
    m = re.search(r"E/N = (-?[0-9.]+), M/N = (-?[0-9.]+)", text)
    sigma = oracle.init(256, 1, 0)
    E, M = oracle.sweeps(sigma, 2.269185, 1, 0, 0, 1000, n_threads=max(1, min(8, os.cpu_count() or 1)))
    assert m and m.group(1) == f"{E[-1] / 65536:.6f}" and m.group(2) == f"{M[-1] / 65536:.6f}"


def test_library_exports_every_declared_symbol():
    lib_path = ising._build.build()
    lib = ctypes.CDLL(lib_path)
    for name in _declared_functions():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert set(_declared_functions()) <= exported


def test_python_constants_match_the_header():
    """Every integer #define ISING_* of include/ising.h that the binding
    mirrors has the same value there (the binding passes them to the ABI)."""
    defines = {}
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        for m in re.finditer(r"^#define\s+(ISING_[A-Z0-9_]+)\s+\(?(-?[0-9]+)\)?\s*$", open(hdr).read(), flags=re.M):
            defines[m.group(1)] = int(m.group(2))
    mirrored = {k: v for k, v in vars(ising).items() if k.startswith("ISING_") and isinstance(v, int)}
    assert mirrored, "the binding mirrors no constants"
    for name, value in mirrored.items():
        if name in defines:
            assert defines[name] == value, (name, defines[name], value)
    for name in ("ISING_PLAN_AUTO", "ISING_PLAN_RESIDENT", "ISING_PLAN_STREAM", "ISING_PLAN_PERSIST",
                 "ISING_PLAN_MIXED", "ISING_NET_BF16", "ISING_NET_FP8"):
        assert name in defines and name in mirrored, name


def test_library_has_no_oracle_dependency():
    # the product library links nothing from oracle/
    lib_path = ising._build.build()
    out = subprocess.run(["nm", "-D", lib_path], capture_output=True, text=True).stdout
    assert "oracle_" not in out
    for src in glob.glob(os.path.join(ROOT, "paper_2404_16990_gb300", "**", "*.*"), recursive=True):
        if src.endswith((".py", ".cu", ".h", ".cuh", ".cpp")):
            text = open(src).read()
            assert "import oracle" not in text and "from oracle" not in text, src


def test_version_string():
    assert "sm_103a" in ising.ising_version()


def test_workspace_bytes_layout():
    b1 = ising.ising_workspace_bytes(64, 1, 0)
    b2 = ising.ising_workspace_bytes(64, 2, 0)
    assert b2 - b1 >= 64 * 64 // 8
    big = ising.ising_workspace_bytes(16384, 1, 1000)
    assert big >= 16384 * 16384 // 8 + 1000 * 2 * 8
    assert ising.ising_workspace_bytes(65536, 1, 0) >= 65536 * 65536 // 8
    assert ising.ising_batch_workspace_bytes([64, 128], 0) >= (64 * 64 + 128 * 128) // 8
    assert ising.ising_batch_workspace_bytes([], 0) > 0   # control block only
    assert ising.ising_workspace_bytes(64, 0, 0) == ising.ising_batch_workspace_bytes([], 0)


@pytest.mark.parametrize("L", [0, 2, 32, 63, 96, 100, 65600, -64])
def test_invalid_sizes_rejected(L):
    with pytest.raises(ising.IsingError) as e:
        ising.ising_workspace_bytes(L, 1, 0)
    assert e.value.code == ising.ISING_EINVAL
    assert "L=" in ising.ising_last_error()


def test_invalid_create_arguments_rejected_before_device_work():
    fake = 1 << 40  # never dereferenced: validation fails first
    for L, temps in [(64, [0.0]), (64, [-1.0]), (64, [float("nan")]), (64, [float("inf")]), (60, [2.0])]:
        with pytest.raises(ising.IsingError) as e:
            ising.ising_create(L, 1, temps, 1, 0, 0, fake, 1 << 30, 0)
        assert e.value.code == ising.ISING_EINVAL
    with pytest.raises(ising.IsingError) as e:
        ising.ising_create(64, 1, [2.0], 1, 7, 0, fake, 1 << 30, 0)       # bad init mode
    assert e.value.code == ising.ISING_EINVAL
    need = ising.ising_workspace_bytes(64, 1, 0)
    with pytest.raises(ising.IsingError) as e:
        ising.ising_create(64, 1, [2.0], 1, 0, 0, fake, need - 1, 0)      # workspace too small
    assert e.value.code == ising.ISING_ENOMEM
    with pytest.raises(ising.IsingError) as e:
        ising.ising_create(64, 1, [2.0], 1, 0, 0, fake + 8, need, 0)      # misaligned
    assert e.value.code == ising.ISING_EINVAL
    with pytest.raises(ising.IsingError) as e:
        ising.ising_create(64, 1, [2.0], 1, 0, -1, fake, need, 0)         # negative trace
    assert e.value.code == ising.ISING_EINVAL
    with pytest.raises(ising.IsingError) as e:
        ising.ising_create_batch([64, 96], [2.0, 2.0], [1, 2], 0, 0, fake, 1 << 30, 0)
    assert e.value.code == ising.ISING_EINVAL


def test_null_handle_calls_fail_cleanly():
    lib = ising._load()
    assert lib.ising_sweep(None, 1) == ising.ISING_EINVAL
    assert lib.ising_sweeps_done(None) == -1
    assert lib.ising_num_sims(None) == 0
    lib.ising_destroy(None)
    sz = ctypes.c_size_t()
    assert lib.ising_sw_scratch_bytes(None, ctypes.byref(sz)) == ising.ISING_EINVAL
    assert lib.ising_sw_sweep(None, 1, None, 0) == ising.ISING_EINVAL
    assert lib.ising_wolff_sweep(None, 1, None, 0) == ising.ISING_EINVAL
    assert lib.ising_sw_labels(None, 0, None, 0, None) == ising.ISING_EINVAL
    assert lib.ising_sw_get_thresholds(None, None) == ising.ISING_EINVAL


def test_no_fallback_when_the_library_cannot_be_built():
    # with the build failing (as without nvcc), every entry point raises, the
    # host-only statistics too: there is no CPU path to fall back to
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "from paper_2404_16990_gb300 import build, ising\n"
        "def boom(*a, **k): raise RuntimeError('nvcc failed')\n"
        "build.build = boom\n"
        "ising._lib = None\n"
        "for call in (ising.ising_version, lambda: ising.ising_workspace_bytes(64, 1),\n"
        "             lambda: ising.ising_tau_int([1.0, 2.0, 3.0])):\n"
        "    try:\n"
        "        call()\n"
        "    except Exception as e:\n"
        "        print('raised', type(e).__name__)\n"
        "    else:\n"
        "        print('returned')\n" % ROOT)
    import sys
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300).stdout.split("\n")
    assert [ln.split()[0] for ln in out if ln] == ["raised"] * 3, out
