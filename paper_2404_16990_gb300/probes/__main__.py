"""Build and run the integer-pipe throughput probe (needs a GPU)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))


def main():
    out_dir = os.path.join(ROOT, "_build", "probes")
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "int_pipes")
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                           os.path.join(HERE, "int_pipes.cu")])
    sys.exit(subprocess.call([exe]))


if __name__ == "__main__":
    main()
