"""The uneven batch's first 64 solves (sizes up to 4096 x 16384, ERK and SDIRK
of every order, m = 4..16) through the continuous-batching server against
the oracle's two-level FCF-MGRIT of the same solves (Section 2.2; the values
come from tests/golden/make_batch_subset_golden.py, which calls only the
oracle).  FP64: the same iteration count and initial residual, and the final
time level to 1e-12 plus eight FP64 roundings (2^-53 each) per fine step: the
sample is the last of nt levels, where rounding differences between the two
sides' steps accumulate without growth (|lambda| <= 1), and one step rounds
several times on each side (an SDIRK step chains three to five stages, each
a forward and a backward recurrence on the GPU and an FFT division in the
oracle).  MIXED (FP32 second F-relaxation, as the batch runs): within two
iterations and 1e-9 -- its per-cycle reduction levels off near 1e-2..1e-3,
the accuracy of the FP32 correction pass, so a solve that FP64 finishes in
two or three much faster cycles takes up to two more.  A final level that
the scheme's dissipation has taken down to rounding noise (SDIRK1 over 16384
steps) is compared with an absolute floor of 1e-13 times the initial
residual norm."""
import os
import time

import numpy as np
import pytest

import workloads
from conftest import ROOT

pytestmark = pytest.mark.gpu

CMAX = {1: 1.0, 2: 0.5, 3: 1.62589, 4: 1.04449, 5: 1.96583}


@pytest.fixture(scope="module")
def capi():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1910_03726_gb300 import build
    build.build()
    from paper_1910_03726_gb300 import capi as c
    return c


def golden():
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", "batch_subset64.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = line.split()
            rows.append({"family": v[1], "p": int(v[2]), "nx": int(v[3]), "nt": int(v[4]), "m": int(v[5]),
                         "field_seed": int(v[6]), "iterations": int(v[7]), "r0": float(v[9]),
                         "final_norm": float(v[10]), "samples": np.array([float(x) for x in v[11:]])})
    return rows


def run_server(capi, rows, precision):
    srv = capi.mgrit_server_create(150e9)
    out = []
    try:
        tickets = []
        for g in rows:
            fam, p = g["family"], g["p"]
            c = 4.0 if fam == "SDIRK" else 0.85 * CMAX[p]
            prob = capi.problem(g["nx"], g["nt"], fam, p, p, c)
            opts = capi.mgrit_opts_default(m=g["m"], levels=2, precision=precision, tol=1e-10, max_iter=80,
                                           output=capi.OUT_FINAL,
                                           psi_rule=capi.PSI_THRESHOLD if fam == "SDIRK" else capi.PSI_AUTO)
            tickets.append(capi.mgrit_submit(srv, prob, opts, workloads.fourier_field(g["nx"], seed=g["field_seed"])))
        for g, t in zip(rows, tickets):
            fin = np.zeros(g["nx"])
            t0 = time.time()
            while True:
                st, res = capi.mgrit_poll(srv, t, fin)
                if st != capi.MGRIT_PENDING:
                    break
                assert time.time() - t0 < 300, "request did not finish"
                time.sleep(0.002)
            out.append((st, res, fin))
    finally:
        capi.mgrit_server_destroy(srv)
    return out


def test_batch_subset_fp64_equals_oracle(capi):
    rows = golden()
    assert len(rows) == 64
    specs = workloads.batch_specs(64)
    for g, s in zip(rows, specs):   # the stored specification is the workload's
        assert (g["family"], g["p"], g["nx"], g["nt"], g["m"], g["field_seed"]) == \
               (s["family"], s["p"], s["nx"], s["nt"], s["m"], s["field_seed"])
    for g, (st, res, fin) in zip(rows, run_server(capi, rows, capi.PREC_FP64)):
        assert st == 0 and res.converged == 1
        assert res.iterations == g["iterations"], (g, res.iterations)
        assert abs(res.r0_norm - g["r0"]) <= 1e-12 * g["r0"]
        smp = fin[:: g["nx"] // len(g["samples"])]
        rtol = 1e-12 + 8 * g["nt"] * 2.0 ** -53
        floor = 1e-13 * g["r0"]
        assert np.linalg.norm(smp - g["samples"]) <= rtol * np.linalg.norm(g["samples"]) + floor, g
        assert abs(np.linalg.norm(fin) - g["final_norm"]) <= rtol * g["final_norm"] + floor


def test_batch_subset_mixed_close_to_oracle(capi):
    rows = golden()
    for g, (st, res, fin) in zip(rows, run_server(capi, rows, capi.PREC_MIXED)):
        assert st == 0 and res.converged == 1
        assert -1 <= res.iterations - g["iterations"] <= 2, (g, res.iterations)
        smp = fin[:: g["nx"] // len(g["samples"])]
        assert np.linalg.norm(smp - g["samples"]) <= 1e-9 * np.linalg.norm(g["samples"]) + 1e-13 * g["r0"], g
