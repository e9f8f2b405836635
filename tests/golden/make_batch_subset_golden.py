"""Write tests/golden/batch_subset64.txt from the oracle alone.

The first 64 solves of the uneven batch (workloads.batch_specs, seed 4: nx in
2^8..2^12, nt in 2^10..2^14, order p in 1..5 with ERKp+Up at 85% of Table 1's
CFL limit and the auto-width Psi, or SDIRKp+Up at c = 4 with the threshold Psi
of Section 4.6; m in {4, 8, 16}; Fourier-field u0 with each solve's own seed),
each a two-level FCF-MGRIT solve (Section 2.2) from the zero iterate to a
1e-10 relative residual in FP64.  Per solve: its specification, the oracle's
iteration count, initial residual norm, the 2-norm of the final time level
and 32 of its values (every nx/32-th point).  The oracle needs minutes for
the 64 solves, so the GPU test reads the stored values.

    python tests/golden/make_batch_subset_golden.py [processes]
"""
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

CMAX = {1: 1.0, 2: 0.5, 3: 1.62589, 4: 1.04449, 5: 1.96583}   # Table 1 CFL limits
COUNT = 64
SAMPLES = 32


def solve_one(spec):
    import workloads
    from oracle import mgrit as omg
    from oracle import psi as opsi
    from oracle import stepping
    fam, p, nx, nt, m = spec["family"], spec["p"], spec["nx"], spec["nt"], spec["m"]
    c = 4.0 if fam == "SDIRK" else 0.85 * CMAX[p]
    rule = "threshold" if fam == "SDIRK" else "auto"
    st = stepping.FineStep(fam, p, c, nx)
    ops = opsi.build_hierarchy(fam, p, c, nx, nt, m, 2, rule=rule)
    u0 = workloads.fourier_field(nx, seed=spec["field_seed"])
    U = omg.zero_iterate(u0, nt)
    r0 = float(np.linalg.norm(omg.spacetime_residual(U, np.zeros_like(U), st)))
    it, rel = omg.solve(omg.make_levels(st, m, [o.diag for o in ops]), U, tol=1e-10, max_iter=80)
    fin = U[-1]
    return it, rel, r0, float(np.linalg.norm(fin)), fin[:: nx // SAMPLES].tolist()


def main():
    sys.path.insert(0, ROOT)
    import workloads
    specs = workloads.batch_specs(COUNT)
    procs = int(sys.argv[1]) if len(sys.argv) > 1 else (os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(solve_one, specs, chunksize=1)
    path = os.path.join(HERE, "batch_subset64.txt")
    with open(path, "w") as f:
        f.write("# Oracle two-level FCF-MGRIT (FP64, zero iterate, tol 1e-10) of the first 64 solves of the\n")
        f.write("# uneven batch (workloads.batch_specs seed 4); written by make_batch_subset_golden.py\n")
        f.write("# index family p nx nt m field_seed iterations rel_residual r0_norm final_norm samples...\n")
        for k, (s, (it, rel, r0, fn, smp)) in enumerate(zip(specs, res)):
            f.write(f"{k} {s['family']} {s['p']} {s['nx']} {s['nt']} {s['m']} {s['field_seed']} {it} {rel:.6e} "
                    f"{r0:.17e} {fn:.17e} " + " ".join(f"{v:.17e}" for v in smp) + "\n")
    print(path)


if __name__ == "__main__":
    main()
