"""SDIRK fine steps on the GPU (stage form, periodic banded stage solves by
factored parallel recurrences) against the oracle (stage form, circulant solves
by FFT division): single steps, MGRIT parity, mixed precision, sequential
stepping and the FULL output (Section 2.1, Appendix A, Section 4.6)."""
import numpy as np
import pytest

import workloads
from oracle import mgrit as omg
from oracle import psi as opsi
from oracle import stepping

pytestmark = pytest.mark.gpu

TOL = 1e-12


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


@pytest.mark.parametrize("p,q,nx", [(1, 1, 64), (2, 2, 96), (3, 3, 256), (4, 4, 128), (3, 5, 8192),
                                    (1, 5, 512), (2, 5, 1024), (4, 5, 4096), (3, 5, 160)])
def test_sdirk_steps_match_oracle(capi, p, q, nx):
    import torch
    k, count = 3, 3
    h = capi.mgrit_setup(capi.problem(nx, 8, "SDIRK", p, q, 4.0), capi.mgrit_opts_default(m=2, levels=2))
    try:
        x = np.random.default_rng(p * 10 + q).standard_normal((count, nx))
        xin = torch.tensor(x, device="cuda")
        yout = torch.zeros_like(xin)
        capi.mgrit_propagate(h, 1, k, count, xin, yout)
    finally:
        capi.mgrit_destroy(h)
    st = stepping.FineStep("SDIRK", p, 4.0, nx, q=q)
    ref = x.copy()
    for _ in range(k):
        ref = st(ref)
    assert rel(yout.cpu().numpy(), ref) <= TOL


def _oracle(p, nx, nt, m, L, u0, cycle="V", relax="FCF"):
    st = stepping.FineStep("SDIRK", p, 4.0, nx)
    ops = opsi.build_hierarchy("SDIRK", p, 4.0, nx, nt, m, L, rule="threshold")
    lev = omg.make_levels(st, m, [o.diag for o in ops])
    U = omg.zero_iterate(u0, nt)
    it, r = omg.solve(lev, U, tol=1e-10, cycle=cycle, relax=relax)
    return it, U


@pytest.mark.parametrize("p,nx,nt,m,L", [(1, 256, 256, 4, 2), (2, 128, 256, 8, 2), (3, 256, 512, 16, 2),
                                         (4, 128, 256, 4, 2), (3, 256, 1024, 4, 3)])
def test_sdirk_mgrit_parity(capi, p, nx, nt, m, L):
    u0 = workloads.wave_packet(nx)
    it, U = _oracle(p, nx, nt, m, L, u0)
    opts = capi.mgrit_opts_default(m=m, levels=L, psi_rule=capi.PSI_THRESHOLD)
    h = capi.mgrit_setup(capi.problem(nx, nt, "SDIRK", p, p, 4.0), opts)
    try:
        out = np.zeros((nt // m + 1, nx))
        res, _ = capi.mgrit_solve(h, u0, out)
    finally:
        capi.mgrit_destroy(h)
    assert res.iterations == it
    assert rel(out, U[::m]) <= TOL


def test_sdirk_mixed_precision_and_full_output(capi):
    p, nx, nt, m = 3, 256, 512, 16
    u0 = workloads.wave_packet(nx)
    ref = stepping.sequential(stepping.FineStep("SDIRK", p, 4.0, nx), u0, nt)
    opts = capi.mgrit_opts_default(m=m, levels=2, precision=capi.PREC_MIXED, output=capi.OUT_FULL)
    h = capi.mgrit_setup(capi.problem(nx, nt, "SDIRK", p, p, 4.0), opts)
    try:
        out = np.zeros((nt + 1, nx))
        res, _ = capi.mgrit_solve(h, u0, out)
        seq = np.zeros((nt + 1, nx))
        capi.mgrit_sequential(h, u0, seq)
    finally:
        capi.mgrit_destroy(h)
    assert res.converged == 1 and res.rel_residual <= 1e-10
    assert rel(out, ref) <= 1e-9
    assert rel(seq, ref) <= TOL


def test_sdirk_in_the_server_mix(capi):
    import time
    specs = [("SDIRK", 3, 3, 256, 512, 16), ("ERK", 3, 3, 256, 512, 8), ("SDIRK", 1, 1, 128, 256, 4)]
    from oracle import schemes
    srv = capi.mgrit_server_create(4e9)
    try:
        tickets, alone = [], []
        for fam, p, q, nx, nt, m in specs:
            c = 4.0 if fam == "SDIRK" else schemes.cfl_number(fam, p)
            prob = capi.problem(nx, nt, fam, p, q, c)
            opts = capi.mgrit_opts_default(m=m, levels=2)
            u0 = workloads.fourier_field(nx)
            h = capi.mgrit_setup(prob, opts)
            a = np.zeros((nt // m + 1, nx))
            r, _ = capi.mgrit_solve(h, u0, a)
            capi.mgrit_destroy(h)
            alone.append((r.iterations, a))
            tickets.append((capi.mgrit_submit(srv, prob, opts, u0), nt // m + 1, nx))
        for (t, rows, nx), (it, a) in zip(tickets, alone):
            out = np.zeros((rows, nx))
            t0 = time.time()
            while True:
                st, res = capi.mgrit_poll(srv, t, out)
                if st != 1:
                    break
                assert time.time() - t0 < 120
                time.sleep(0.002)
            assert st == 0 and res.iterations == it
            assert float(np.max(np.abs(out - a))) <= 1e-14 * float(np.max(np.abs(a)))
    finally:
        capi.mgrit_server_destroy(srv)


@pytest.mark.parametrize("p,nx,nt,m,L,cycle,relax", [(3, 256, 512, 16, 2, "V", "F"), (2, 128, 1024, 4, 3, "F", "FCF"),
                                                     (1, 128, 512, 4, 3, "F", "F")])
def test_sdirk_fcycle_and_f_relaxation_parity(capi, p, nx, nt, m, L, cycle, relax):
    u0 = workloads.wave_packet(nx)
    it, U = _oracle(p, nx, nt, m, L, u0, cycle, relax)
    opts = capi.mgrit_opts_default(m=m, levels=L, psi_rule=capi.PSI_THRESHOLD, cycle=0 if cycle == "V" else 1,
                                   relax=0 if relax == "FCF" else 1)
    h = capi.mgrit_setup(capi.problem(nx, nt, "SDIRK", p, p, 4.0), opts)
    try:
        out = np.zeros((nt // m + 1, nx))
        res, _ = capi.mgrit_solve(h, u0, out)
    finally:
        capi.mgrit_destroy(h)
    assert res.iterations == it
    assert rel(out, U[::m]) <= TOL


@pytest.mark.parametrize("p,m", [(1, 2), (2, 4), (3, 2), (4, 4)])
def test_rediscretised_coarse_step_matches_oracle(capi, p, m):
    """PSI_REDISC (Table 2): the coarse propagator is one SDIRKp+Up step at
    m dt, i.e. CFL number m c."""
    import torch
    nx, k, count = 256, 2, 3
    opts = capi.mgrit_opts_default(m=m, levels=2, psi_rule=capi.PSI_REDISC)
    h = capi.mgrit_setup(capi.problem(nx, 64, "SDIRK", p, p, 4.0), opts)
    try:
        x = np.random.default_rng(p + m).standard_normal((count, nx))
        xin = torch.tensor(x, device="cuda")
        yout = torch.zeros_like(xin)
        capi.mgrit_propagate(h, 2, k, count, xin, yout)
    finally:
        capi.mgrit_destroy(h)
    st = stepping.FineStep("SDIRK", p, 4.0 * m, nx)
    ref = x.copy()
    for _ in range(k):
        ref = st(ref)
    assert rel(yout.cpu().numpy(), ref) <= TOL


@pytest.mark.parametrize("p,q,nx,nt,m,L,prec,relax", [
    (3, 5, 8192, 256, 16, 2, 1, 0), (3, 5, 8192, 256, 16, 2, 0, 0), (1, 1, 2048, 512, 4, 2, 0, 0),
    (2, 2, 4096, 256, 8, 3, 1, 0), (2, 3, 2048, 512, 8, 2, 0, 1), (4, 4, 4096, 512, 16, 2, 1, 1),
    (3, 5, 1024, 1024, 4, 3, 0, 0), (3, 5, 2048, 800, 4, 2, 1, 0), (2, 3, 1024, 1216, 4, 2, 0, 0)])
def test_sdirk_fcf_split_over_a_cluster_agrees(capi, monkeypatch, p, q, nx, nt, m, L, prec, relax):
    """The level-1 SDIRK FCF with each interval's slab split over a cluster of
    two CTAs (the scans' warp totals exchanged through distributed shared
    memory; automatic at nx = 8192; with more intervals than SMs the whole
    waves and the tail go in separate launches, N = 200 and 304 here) gives
    bitwise the C-points and the iterations of one CTA per interval, for
    every recurrence-order pair
    (U1..U5), FP64 and MIXED, FCF- and F-relaxation.  The norms are the same
    sums in another order: in FP64 to rounding, in MIXED to the FP32 rounding
    of the per-thread sums (a thread of the split form sums other points)."""
    import torch
    u0 = torch.tensor(workloads.fourier_field(nx), device="cuda")
    got = {}
    for split in ("0", "1"):
        monkeypatch.setenv("MGRIT_SDIRK_SPLIT", split)
        o = capi.mgrit_opts_default(m=m, levels=L, precision=prec, relax=relax, output=1, tol=1e-10,
                                    psi_rule=2, max_iter=60)
        h = capi.mgrit_setup(capi.problem(nx, nt, "SDIRK", p, q, 4.0), o)
        try:
            out = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
            r, _ = capi.mgrit_solve(h, u0, out)
            assert r.converged == 1
            got[split] = (r.iterations, r.rel_residual, out.cpu().numpy())
        finally:
            capi.mgrit_destroy(h)
    a, b = got["1"], got["0"]
    assert a[0] == b[0]
    np.testing.assert_array_equal(a[2], b[2])
    assert abs(a[1] - b[1]) <= (1e-12 if prec == 0 else 1e-6) * b[1]
