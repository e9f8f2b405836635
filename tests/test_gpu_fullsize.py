"""Parity on the paths the benchmark times, at the benchmark's sizes.

* The headline problem at full size (ERK3+U3, 4096 x 16384, V-cycle L = 4,
  m = 8) in the benchmark's launch configuration (one CUDA graph per solve,
  queued, autotuned level-1 launch shape, Fourier-space coarsest level):
  - FP64 against the oracle's own MGRIT of the same problem (iterations,
    initial residual, history, and sampled converged C-points; the values
    come from tests/golden/make_fullsize_golden.py, which calls only the
    oracle, because the oracle needs minutes at this size);
  - every precision against the oracle's sequential stepping u^{n+1} = Phi u^n
    (Eq. 3; the fixed point MGRIT converges to) at every C-point.
* The level-1 FCF shapes the autotuner picks at nx = 4096 (collapsed Phi^m
  chunked at 256 threads, with the 16-byte pair loads of nx % 512 == 0) and
  the coarsest level in Fourier space at nx = 4096, each forced, against the
  oracle's MGRIT at nt = 1024 (FP64 to 1e-12, the same iterations).
* SDIRK3+U5 at nx = 8192 with m = 16 (the SDIRK benchmark's kernel instance)
  against the oracle's MGRIT (nt = 256), and its full 8192 x 8192 solve
  against the oracle's sequential stepping.
* The server with requests of nx = 512..4096: each result equals the same
  solve alone.
"""
import os

import numpy as np
import pytest

import workloads
from conftest import ROOT
from oracle import mgrit as omg
from oracle import psi as opsi
from oracle import schemes, stepping

pytestmark = pytest.mark.gpu

NX, NT, M, L = 4096, 16384, 8, 4
CFL3 = 0.85 * 1.62589


@pytest.fixture(scope="module")
def capi():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1910_03726_gb300 import build
    build.build()
    from paper_1910_03726_gb300 import capi as c
    return c


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def read_golden():
    g = {"cpoints": {}}
    with open(os.path.join(ROOT, "tests", "golden", "fullsize_erk3u3_4096x16384.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, *vals = line.split()
            if key == "cpoint":
                g["cpoints"][int(vals[0])] = (int(vals[1]), np.array([float(v) for v in vals[2:]]))
            elif key == "iterations":
                g["iterations"] = int(vals[0])
            elif key == "r0_norm":
                g["r0_norm"] = float(vals[0])
            else:
                g[key] = [float(v) for v in vals]
    return g


@pytest.fixture(scope="module")
def sequential_cpoints():
    """The oracle's sequential stepping of the headline problem at the C-points."""
    st = stepping.FineStep("ERK", 3, CFL3, NX)
    u = workloads.fourier_field(NX)
    out = np.empty((NT // M + 1, NX))
    out[0] = u
    for n in range(1, NT + 1):
        u = st(u)
        if n % M == 0:
            out[n // M] = u
    return out


def headline_solve(capi, precision, queued=True):
    import torch
    o = capi.mgrit_opts_default(m=M, levels=L, precision=precision, tol=1e-10, output=capi.OUT_CPOINTS,
                                max_iter=100)
    h = capi.mgrit_setup(capi.problem(NX, NT, "ERK", 3, 3, CFL3), o)
    try:
        u0 = torch.tensor(workloads.fourier_field(NX), device="cuda")
        out = torch.empty((NT // M + 1, NX), dtype=torch.float64, device="cuda")
        if queued:
            for _ in range(2):
                capi.mgrit_solve_async(h, u0, out)
            res = [capi.mgrit_solve_wait(h)[0] for _ in range(2)][-1]
        else:
            res, _ = capi.mgrit_solve(h, u0, out)
        return res, out.cpu().numpy()
    finally:
        capi.mgrit_destroy(h)


def test_headline_fp64_full_size_equals_oracle_mgrit(capi):
    g = read_golden()
    res, cp = headline_solve(capi, capi.PREC_FP64)
    assert res.iterations == g["iterations"]
    assert abs(res.r0_norm - g["r0_norm"]) <= 1e-12 * g["r0_norm"]
    hist = list(res.history[: res.n_history])
    assert len(hist) == len(g["history"])
    for a, b in zip(hist, g["history"]):
        assert abs(a - b) <= 1e-6 * b + 1e-13, (hist, g["history"])
    for j, (every, vals) in g["cpoints"].items():
        assert rel(cp[j, ::every], vals) <= 1e-12, j


@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (1, 1e-10), (2, 1e-10)])
def test_headline_full_size_reaches_sequential_stepping(capi, sequential_cpoints, precision, tol):
    """The bench's solve (queued graph launches) against the plain definition:
    MGRIT's fixed point is sequential stepping, and a 1e-10 relative residual
    leaves C-point errors of about 1e-12 on this problem (bound used: 1e-11
    in FP64, the stopping tolerance 1e-10 in the mixed modes); the iterations
    of the mixed modes lie within one of FP64's."""
    res, cp = headline_solve(capi, precision)
    assert res.converged == 1 and res.rel_residual <= 1e-10
    assert rel(cp, sequential_cpoints) <= tol
    assert abs(res.iterations - read_golden()["iterations"]) <= (0 if precision == 0 else 1)


_ORACLE = {}


def oracle_erk3(nt, levels):
    key = (nt, levels)
    if key not in _ORACLE:
        st = stepping.FineStep("ERK", 3, CFL3, NX)
        ops = opsi.build_hierarchy("ERK", 3, CFL3, NX, nt, M, levels, rule="auto")
        U = omg.zero_iterate(workloads.fourier_field(NX), nt)
        it, _ = omg.solve(omg.make_levels(st, M, [o.diag for o in ops]), U, tol=1e-10)
        _ORACLE[key] = (it, U[::M].copy())
    return _ORACLE[key]


def gpu_erk3(capi, nt, levels, precision=0):
    o = capi.mgrit_opts_default(m=M, levels=levels, precision=precision, tol=1e-10, output=capi.OUT_CPOINTS)
    h = capi.mgrit_setup(capi.problem(NX, nt, "ERK", 3, 3, CFL3), o)
    try:
        out = np.zeros((nt // M + 1, NX))
        res, _ = capi.mgrit_solve(h, workloads.fourier_field(NX), out)
    finally:
        capi.mgrit_destroy(h)
    return res, out


@pytest.mark.parametrize("shape", ["98,256,1", "98,512,1", "99,256,0", "8,256,0", None])
@pytest.mark.parametrize("levels", [3, 4])
def test_level1_shapes_at_4096_match_oracle(capi, monkeypatch, shape, levels):
    """98,256,1: the headline's pick (collapsed 73-tap Phi^8, chunked, 256
    threads: pairs of points per 16-byte access since 4096 % 512 == 0); None:
    whatever the autotuner picks here."""
    if shape:
        monkeypatch.setenv("MGRIT_FCF_SHAPE", shape)
    it, ref = oracle_erk3(1024, levels)
    res, out = gpu_erk3(capi, 1024, levels)
    if shape:
        got = f"{res.fine_tile},{res.fine_threads},{res.fine_collapsed}"
        assert got == shape
    assert res.iterations == it
    assert rel(out, ref) <= 1e-12


@pytest.mark.parametrize("fourier", ["0", "1"])
def test_headline_full_size_fourier_fcf_forms(capi, monkeypatch, sequential_cpoints, fourier):
    """The headline in MIXED with the level-1 FCF's FP64 pass in Fourier space
    (forced on) and as the collapsed stencil (forced off): both reach the
    oracle's sequential stepping to the stopping tolerance, with FP64's
    iterations within one."""
    monkeypatch.setenv("MGRIT_FCF_FOURIER", fourier)
    res, cp = headline_solve(capi, 1)
    assert res.fine_fourier == int(fourier)
    assert res.converged == 1 and res.rel_residual <= 1e-10
    assert rel(cp, sequential_cpoints) <= 1e-10
    assert abs(res.iterations - read_golden()["iterations"]) <= 1


@pytest.mark.parametrize("threads", ["256", "128"])
@pytest.mark.parametrize("levels", [3, 4])
def test_fourier_fcf_at_4096_matches_oracle(capi, monkeypatch, threads, levels):
    """nx = 4096: the MIXED level-1 FCF with its FP64 pass in Fourier space
    (2048-point half-length FFTs) against the oracle's MGRIT at nt = 1024."""
    monkeypatch.setenv("MGRIT_FCF_SHAPE", "98,256,1," + threads)
    it, ref = oracle_erk3(1024, levels)
    res, out = gpu_erk3(capi, 1024, levels, precision=1)
    assert res.fine_fourier == 1
    assert abs(res.iterations - it) <= 1
    assert rel(out, ref) <= 1e-9


@pytest.mark.parametrize("coarse", ["fft", "march"])
@pytest.mark.parametrize("levels", [2, 3])
def test_coarsest_level_at_4096_matches_oracle(capi, monkeypatch, coarse, levels):
    """nx = 4096: the Fourier-space coarsest level (a half-length complex FFT
    of 2048 points per slab) over 128 (two-level) and 16 (L = 3) coarse
    steps, and the cluster march, each forced; FP64 and MIXED."""
    monkeypatch.setenv("MGRIT_COARSE", coarse)
    it, ref = oracle_erk3(1024, levels)
    res, out = gpu_erk3(capi, 1024, levels)
    assert res.iterations == it
    assert rel(out, ref) <= 1e-12
    res_m, out_m = gpu_erk3(capi, 1024, levels, precision=1)
    assert abs(res_m.iterations - it) <= 1
    assert rel(out_m, ref) <= 1e-9


def oracle_sdirk35(nx, nt, m, u0):
    st = stepping.FineStep("SDIRK", 3, 4.0, nx, q=5)
    ops = opsi.build_hierarchy("SDIRK", 3, 4.0, nx, nt, m, 2, rule="threshold", q=5)
    U = omg.zero_iterate(u0, nt)
    it, _ = omg.solve(omg.make_levels(st, m, [o.diag for o in ops]), U, tol=1e-10)
    return it, U[::m], ops[0]


def test_sdirk3_u5_8192_m16_matches_oracle(capi):
    nx, nt, m = 8192, 256, 16
    u0 = workloads.wave_packet(nx)
    it, ref, op = oracle_sdirk35(nx, nt, m, u0)
    for prec, tol in ((0, 1e-12), (1, 1e-9)):
        o = capi.mgrit_opts_default(m=m, levels=2, precision=prec, tol=1e-10, output=capi.OUT_CPOINTS,
                                    psi_rule=capi.PSI_THRESHOLD)
        h = capi.mgrit_setup(capi.problem(nx, nt, "SDIRK", 3, 5, 4.0), o)
        try:
            out = np.zeros((nt // m + 1, nx))
            res, _ = capi.mgrit_solve(h, u0, out)
            offs, cfs = capi.mgrit_psi_info(h, 2)
        finally:
            capi.mgrit_destroy(h)
        assert sorted(offs) == sorted(op.diag)
        assert res.iterations == it if prec == 0 else abs(res.iterations - it) <= 1
        assert rel(out, ref) <= tol


def test_sdirk3_u5_full_size_reaches_sequential_stepping(capi):
    """The SDIRK benchmark's solve (8192 x 8192, c = 4, two-level m = 16,
    MIXED) against the oracle's sequential stepping at sampled C-points."""
    nx = nt = 8192
    m = 16
    u0 = workloads.wave_packet(nx)
    st = stepping.FineStep("SDIRK", 3, 4.0, nx, q=5)
    rows = (1, 16, 128, 511, 512)
    want = {}
    u = u0.copy()
    for n in range(1, nt + 1):
        u = st(u)
        if n % m == 0 and n // m in rows:
            want[n // m] = u.copy()
    o = capi.mgrit_opts_default(m=m, levels=2, precision=capi.PREC_MIXED, tol=1e-10, output=capi.OUT_CPOINTS,
                                psi_rule=capi.PSI_THRESHOLD)
    h = capi.mgrit_setup(capi.problem(nx, nt, "SDIRK", 3, 5, 4.0), o)
    try:
        out = np.zeros((nt // m + 1, nx))
        res, _ = capi.mgrit_solve(h, u0, out)
    finally:
        capi.mgrit_destroy(h)
    assert res.converged == 1
    for j in rows:
        assert rel(out[j], want[j]) <= 1e-9, j


def test_server_mix_of_large_requests_equals_alone(capi, monkeypatch):
    """Requests of nx = 512..4096 (ERK and SDIRK, every order, m = 4..16,
    FP64 and MIXED) batched together: each equals the same solve alone with
    the server's kernels (the server marches its coarsest levels and applies
    Phi^m as a stencil in its batched FCF, so alone marches too and keeps the
    Fourier-space FP64 pass off), and the FP64 ERK ones equal the oracle."""
    import time
    mix = [("ERK", 3, 4096, 1024, 8, 0), ("ERK", 1, 2048, 2048, 4, 1), ("SDIRK", 2, 1024, 1024, 16, 1),
           ("ERK", 5, 512, 2048, 8, 0), ("ERK", 2, 1024, 4096, 16, 1), ("SDIRK", 4, 2048, 512, 4, 0),
           ("ERK", 4, 4096, 512, 4, 1), ("ERK", 3, 512, 1024, 4, 2)]
    specs = []
    for fam, p, nx, nt, m, prec in mix:
        c = 4.0 if fam == "SDIRK" else schemes.cfl_number("ERK", p)
        rule = capi.PSI_THRESHOLD if fam == "SDIRK" else capi.PSI_AUTO
        specs.append((capi.problem(nx, nt, fam, p, p, c),
                      capi.mgrit_opts_default(m=m, levels=2, precision=prec, output=capi.OUT_CPOINTS, psi_rule=rule),
                      workloads.fourier_field(nx, seed=300 + nx + p)))
    monkeypatch.setenv("MGRIT_COARSE", "march")
    monkeypatch.setenv("MGRIT_FCF_FOURIER", "0")
    alone = []
    for prob, opts, u0 in specs:
        h = capi.mgrit_setup(prob, opts)
        try:
            out = np.zeros((prob.nt // opts.m + 1, prob.nx))
            alone.append((capi.mgrit_solve(h, u0, out)[0], out))
        finally:
            capi.mgrit_destroy(h)
    srv = capi.mgrit_server_create(20e9)
    try:
        tickets = [capi.mgrit_submit(srv, *sp) for sp in specs]
        for (prob, opts, u0), t, (ares, aout) in zip(specs, tickets, alone):
            out = np.zeros((prob.nt // opts.m + 1, prob.nx))
            t0 = time.time()
            while True:
                st, res = capi.mgrit_poll(srv, t, out)
                if st != capi.MGRIT_PENDING:
                    break
                assert time.time() - t0 < 120
                time.sleep(0.002)
            assert st == 0 and res.iterations == ares.iterations
            assert float(np.max(np.abs(out - aout)) / np.max(np.abs(aout))) <= 1e-14
    finally:
        capi.mgrit_server_destroy(srv)
    for (fam, p, nx, nt, m, prec), (ares, aout), (prob, opts, u0) in zip(mix, alone, specs):
        if fam == "ERK" and prec == 0:
            st = stepping.FineStep("ERK", p, prob.cfl, nx)
            ops = opsi.build_hierarchy("ERK", p, prob.cfl, nx, nt, m, 2, rule="auto")
            U = omg.zero_iterate(u0, nt)
            it, _ = omg.solve(omg.make_levels(st, m, [o.diag for o in ops]), U, tol=1e-10)
            assert ares.iterations == it and rel(aout, U[::m]) <= 1e-12
