"""Continuous-batching server through the C ABI: every result equals the same
solve run alone (same iterations, C-points identical to 1e-14), requests that
arrive while others run are admitted as memory frees up, and failures are
reported per request."""
import time

import numpy as np
import pytest

import workloads
from oracle import schemes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1910_03726_gb300 import build
    build.build()
    from paper_1910_03726_gb300 import capi as c
    return c


MIX = [  # (p, nx, nt, m, levels, precision)
    (1, 64, 512, 8, 2, 0), (3, 128, 1024, 4, 2, 1), (2, 96, 768, 4, 3, 0), (5, 128, 512, 4, 2, 1),
    (3, 256, 2048, 8, 2, 0), (4, 128, 1024, 16, 2, 1), (1, 256, 1024, 4, 3, 1), (3, 64, 256, 4, 2, 0),
    (2, 128, 2048, 8, 2, 1), (5, 256, 1024, 8, 3, 0), (3, 128, 512, 8, 2, 1), (1, 128, 4096, 16, 2, 0),
    # MIXED_DF (float-float C-points): two-level (batched march adds into the
    # pairs) and V-cycle (float-float add of the coarse correction)
    (3, 128, 1024, 4, 2, 2), (1, 256, 1024, 4, 3, 2), (2, 128, 1024, 8, 2, 2),
]


def _spec(capi, p, nx, nt, m, levels, prec):
    c = schemes.cfl_number("ERK", p)
    prob = capi.problem(nx, nt, "ERK", p, p, c)
    opts = capi.mgrit_opts_default(m=m, levels=levels, precision=prec, output=capi.OUT_CPOINTS)
    u0 = workloads.fourier_field(nx, seed=100 + p * 7 + nx)
    return prob, opts, u0


def _alone(capi, prob, opts, u0):
    h = capi.mgrit_setup(prob, opts)
    try:
        out = np.zeros((prob.nt // opts.m + 1, prob.nx))
        res, _ = capi.mgrit_solve(h, u0, out)
    finally:
        capi.mgrit_destroy(h)
    return res, out


def _wait(capi, srv, ticket, rows, nx, timeout=120.0):
    out = np.zeros((rows, nx))
    t0 = time.time()
    while True:
        st, res = capi.mgrit_poll(srv, ticket, out)
        if st != capi.MGRIT_PENDING:
            return st, res, out
        assert time.time() - t0 < timeout, "request did not finish"
        time.sleep(0.002)


@pytest.mark.parametrize("budget_solves", [100, 3])
def test_batch_results_equal_alone(capi, budget_solves, monkeypatch):
    """Each result equals the same solve alone.  The server's two-level
    coarse levels march in its batched march, or, in cycles where few solves
    need a coarse solve, in Fourier space (its counters say how many solves
    switched); "alone" marches (MGRIT_COARSE=march): equal to 1e-14 where
    every solve marched, else to rounding (1e-12, the FP64 parity tolerance,
    as between the two coarse solves of single solves), with the same
    iteration count."""
    specs = [_spec(capi, *s) for s in MIX]
    fourier = [_alone(capi, *sp) for sp in specs]
    monkeypatch.setenv("MGRIT_COARSE", "march")
    alone = [_alone(capi, *sp) for sp in specs]
    monkeypatch.delenv("MGRIT_COARSE")
    for (fres, fout), (ares, aout) in zip(fourier, alone):
        assert fres.iterations == ares.iterations
        assert float(np.max(np.abs(fout - aout)) / np.max(np.abs(aout))) <= 1e-12
    from paper_1910_03726_gb300.capi import _lib  # noqa: F401
    max_bytes = max(sp[0].nx * (sp[0].nt // sp[1].m + 1) * 8 * 6 for sp in specs)
    srv = capi.mgrit_server_create(budget_solves * max_bytes)
    try:
        tickets = [capi.mgrit_submit(srv, *sp) for sp in specs]
        errs = []
        for (prob, opts, u0), t, (ares, aout) in zip(specs, tickets, alone):
            st, res, out = _wait(capi, srv, t, prob.nt // opts.m + 1, prob.nx)
            assert st == 0, capi.mgrit_last_error()
            assert res.iterations == ares.iterations
            assert res.converged == 1
            errs.append(float(np.max(np.abs(out - aout)) / np.max(np.abs(aout))))
        switched = capi.mgrit_server_stats(srv)["fft_coarse_solves"]
        assert max(errs) <= (1e-14 if switched == 0 else 1e-12), (errs, switched)
        # a released ticket is gone
        st, _ = capi.mgrit_poll(srv, tickets[0])
        assert st == -11
    finally:
        capi.mgrit_server_destroy(srv)


def test_requests_join_while_others_run(capi):
    specs = [_spec(capi, *s) for s in MIX[:6]]
    srv = capi.mgrit_server_create(8e9, max_active=2)
    try:
        first = [capi.mgrit_submit(srv, *sp) for sp in specs[:3]]
        time.sleep(0.01)
        later = [capi.mgrit_submit(srv, *sp) for sp in specs[3:]]
        for (prob, opts, u0), t in zip(specs, first + later):
            st, res, out = _wait(capi, srv, t, prob.nt // opts.m + 1, prob.nx)
            assert st == 0 and res.converged == 1
    finally:
        capi.mgrit_server_destroy(srv)


def test_failures_are_per_request(capi):
    """Over-budget requests are refused at submit; a NaN initial condition
    diverges without disturbing its neighbours; max_iter = 0 reports
    NOT_CONVERGED with the relaxed iterate."""
    good = _spec(capi, 3, 128, 512, 4, 2, 0)
    srv = capi.mgrit_server_create(1e8)
    try:
        big = capi.problem(4096, 16384, "ERK", 3, 3, schemes.cfl_number("ERK", 3))
        with pytest.raises(capi.MgritError) as ei:
            capi.mgrit_submit(srv, big, capi.mgrit_opts_default(m=2), workloads.sin4(4096))
        assert ei.value.status == -6
        bad_u0 = workloads.sin4(128)
        bad_u0[5] = np.nan
        t_bad = capi.mgrit_submit(srv, good[0], good[1], bad_u0)
        t_good = capi.mgrit_submit(srv, *good)
        o0 = capi.mgrit_opts_default(m=4, levels=2, max_iter=0)
        t_cap = capi.mgrit_submit(srv, good[0], o0, good[2])
        st, res, _ = _wait(capi, srv, t_bad, 129, 128)
        assert st == -5
        st, res, _ = _wait(capi, srv, t_good, 129, 128)
        assert st == 0 and res.converged == 1
        st, res, _ = _wait(capi, srv, t_cap, 129, 128)
        assert st == -4 and res.iterations == 0
    finally:
        capi.mgrit_server_destroy(srv)


def test_fcycle_and_f_relaxation_requests_equal_alone(capi):
    specs = []
    for (p, nx, nt, m, L, prec), cyc, rlx in [((1, 64, 1024, 2, 6, 0), 1, 0), ((3, 256, 2048, 8, 2, 1), 0, 1),
                                              ((3, 128, 2048, 4, 4, 1), 1, 1)]:
        prob, opts, u0 = _spec(capi, p, nx, nt, m, L, prec)
        opts.cycle, opts.relax = cyc, rlx
        specs.append((prob, opts, u0))
    alone = [_alone(capi, *sp) for sp in specs]
    srv = capi.mgrit_server_create(4e9)
    try:
        tickets = [capi.mgrit_submit(srv, *sp) for sp in specs]
        for (prob, opts, u0), t, (ares, aout) in zip(specs, tickets, alone):
            st, res, out = _wait(capi, srv, t, prob.nt // opts.m + 1, prob.nx)
            assert st == 0 and res.iterations == ares.iterations
            assert float(np.max(np.abs(out - aout)) / np.max(np.abs(aout))) <= 1e-14
    finally:
        capi.mgrit_server_destroy(srv)


@pytest.mark.parametrize("prec", ["FP64", "MIXED", "MIXED_DF"])
def test_few_two_level_solves_switch_to_the_fourier_coarse_solve(capi, monkeypatch, prec):
    """One long two-level solve alone in the server (1024 coarse steps): its
    batched march would cost 1024 dependent steps per cycle, so the server
    switches it to the Fourier-space coarse solve (counted), and the result
    equals the single solve's, which takes the same coarse solve, with the
    same iterations: to 1e-12 in FP64, and to 1e-10 in MIXED and MIXED_DF
    (float-float C-points: the inverse transform's epilogue adds e in FP64 and
    splits back).  MGRIT_COARSE=march keeps it on the march."""
    nx, nt, m = 1024, 8192, 8
    tol = 1e-12 if prec == "FP64" else 1e-10
    prob = capi.problem(nx, nt, "ERK", 3, 3, 0.85 * 1.62589)
    opts = capi.mgrit_opts_default(m=m, levels=2, precision=getattr(capi, "PREC_" + prec), output=capi.OUT_CPOINTS,
                                   tol=1e-10)
    u0 = workloads.fourier_field(nx, seed=9)
    ares, aout = _alone(capi, prob, opts, u0)
    for env, want in ((None, 1), ("march", 0)):
        if env:
            monkeypatch.setenv("MGRIT_COARSE", env)
        srv = capi.mgrit_server_create(50e9)
        try:
            st, res, out = _wait(capi, srv, capi.mgrit_submit(srv, prob, opts, u0), nt // m + 1, nx)
            assert st == 0 and res.converged == 1 and res.iterations == ares.iterations
            assert float(np.max(np.abs(out - aout)) / np.max(np.abs(aout))) <= tol
            assert capi.mgrit_server_stats(srv)["fft_coarse_solves"] == want
        finally:
            capi.mgrit_server_destroy(srv)
