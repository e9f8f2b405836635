"""Write tests/golden/fullsize_erk3u3_4096x16384.txt from the oracle alone.

The benchmark's headline problem at its full size (ERK3+U3, nx = 4096,
nt = 16384, c = 0.85 * 1.62589, Fourier-field u0 with seed 2, zero initial
iterate, V-cycle with 4 levels and m = 8, auto-width least-squares Psi, FP64,
tol 1e-10), solved by the oracle's MGRIT (Section 2.2) in FP64: its iteration
count, initial residual norm, residual history and a sample of its converged
C-points (C-points j = 1, 64, 512, 1024 and 2048, every 8th point).  The
oracle needs a few minutes for this size, so the GPU test reads the stored
values instead of recomputing them.

    python tests/golden/make_fullsize_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402
from oracle import mgrit as omg  # noqa: E402
from oracle import psi as opsi  # noqa: E402
from oracle import stepping  # noqa: E402

NX, NT, M, L, P = 4096, 16384, 8, 4, 3
CFL = 0.85 * 1.62589
ROWS = (1, 64, 512, 1024, 2048)
EVERY = 8


def main():
    st = stepping.FineStep("ERK", P, CFL, NX)
    ops = opsi.build_hierarchy("ERK", P, CFL, NX, NT, M, L, rule="auto")
    U = omg.zero_iterate(workloads.fourier_field(NX), NT)
    hist = []
    r0 = float(np.linalg.norm(omg.spacetime_residual(U, np.zeros_like(U), st)))
    it, rel = omg.solve(omg.make_levels(st, M, [o.diag for o in ops]), U, tol=1e-10, history=hist)
    path = os.path.join(HERE, "fullsize_erk3u3_4096x16384.txt")
    with open(path, "w") as f:
        f.write("# Oracle MGRIT (FP64) of the headline problem at full size; written by make_fullsize_golden.py\n")
        f.write("# ERK3+U3 nx=4096 nt=16384 c=0.85*1.62589, fourier_field(4096) seed 2, zero iterate,\n")
        f.write("# V-cycle L=4 m=8, auto-width LSQ Psi, tol 1e-10 (Section 2.2)\n")
        f.write(f"iterations {it}\n")
        f.write(f"r0_norm {r0:.17e}\n")
        f.write("history " + " ".join(f"{h:.17e}" for h in hist) + "\n")
        f.write("psi_nnz " + " ".join(str(len(o.diag)) for o in ops) + "\n")
        for j in ROWS:
            f.write(f"cpoint {j} {EVERY} " + " ".join(f"{v:.17e}" for v in U[j * M, ::EVERY]) + "\n")
    print(path, it, rel)


if __name__ == "__main__":
    main()
