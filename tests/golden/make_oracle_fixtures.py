"""Write oracle_regression.txt: digests of small oracle runs (the 64^2
configuration at T_c, a Swendsen-Wang run, a Wolff run, a 3D run), so that
any later change to the oracle's arithmetic shows up as a failing test and
has to be made on purpose.  Calls only oracle/.

    python tests/golden/make_oracle_fixtures.py
"""
from __future__ import annotations

import hashlib
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402

OUT = os.path.join(HERE, "oracle_regression.txt")


def _digest(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()[:32]


def cases():
    """(name, final E, final M, digest of lattice and traces) of each run."""
    out = []
    s = oracle.init(64, 1, 0)                                   # 64^2, T_c, random start seed 1, 1000 sweeps
    E, M = oracle.sweeps(s, 2.269185, 1, 0, 0, 1000)
    out.append(("metropolis_L64_Tc_seed1_1000", int(E[-1]), int(M[-1]), _digest(s, E, M)))
    s = oracle.init(128, 7, 2)                                  # 128^2, T = 2.0, 50 Swendsen-Wang steps
    E, M = oracle.sw_sweeps(s, 2.0, 7, 2, 0, 50)
    out.append(("swendsen_wang_L128_T2_seed7_50", int(E[-1]), int(M[-1]), _digest(s, E, M)))
    s = oracle.init(64, 11, 1)                                  # 64^2, T_c, 200 Wolff steps
    E, M, C = oracle.wolff_sweeps(s, 2.269185, 11, 1, 0, 200)
    out.append(("wolff_L64_Tc_seed11_200", int(E[-1]), int(M[-1]), _digest(s, E, M, C)))
    s = oracle.init3d(16, 5, 0)                                 # 16^3, T = 4.5115, 100 sweeps
    E, M = oracle.sweeps3d(s, 4.5115, 5, 0, 0, 100)
    out.append(("cubic_L16_T4.5115_seed5_100", int(E[-1]), int(M[-1]), _digest(s, E, M)))
    return out


def main():
    with open(OUT, "w") as f:
        f.write("# Digests of small oracle runs, written by make_oracle_fixtures.py (oracle only).\n")
        f.write("# name final_E final_M sha256(lattice, traces)[:32]\n")
        for name, e, m, d in cases():
            f.write(f"{name} {e} {m} {d}\n")
    print(OUT)


if __name__ == "__main__":
    main()
