"""Queued solves (mgrit_solve_async / mgrit_solve_wait) and the random initial
iterate (MGRIT_INIT_RANDOM) through the C ABI.

* A queued solve runs the same graph as mgrit_solve: several solves queued back
  to back on one handle give bitwise the results of the same solves one at a
  time, in every precision and for FINAL and CPOINTS output.
* Section 2.2's random initial iterate drawn on the device equals the oracle's
  (its own Philox4x32-10) in FP64: the same initial residual norm (the full
  space-time residual, F-points included), the same iteration count and the
  oracle's converged C-points to 1e-12.
"""
import numpy as np
import pytest

import workloads
from oracle import mgrit as omg
from oracle import philox
from oracle import psi as opsi
from oracle import schemes, stepping

pytestmark = pytest.mark.gpu


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


ASYNC_CASES = [("ERK", 3, 256, 512, 8, 3, 0, 1), ("ERK", 3, 256, 512, 8, 3, 1, 1), ("ERK", 3, 256, 512, 8, 3, 2, 1),
               ("ERK", 1, 512, 1024, 4, 4, 2, 0), ("SDIRK", 3, 256, 256, 16, 2, 1, 1), ("ERK", 2, 128, 2048, 16, 2, 0, 0)]


@pytest.mark.parametrize("case", ASYNC_CASES)
def test_queued_solves_equal_solves_one_at_a_time(capi, case):
    import torch
    fam, p, nx, nt, m, L, prec, output = case
    c = schemes.cfl_number(fam, p)
    opts = capi.mgrit_opts_default(m=m, levels=L, precision=prec, output=output, tol=1e-10)
    h = capi.mgrit_setup(capi.problem(nx, nt, fam, p, p, c), opts)
    try:
        rows = nt // m + 1 if output == 1 else 1
        u0s = [torch.tensor(workloads.fourier_field(nx, seed=20 + k), device="cuda") for k in range(5)]
        want = []
        for u0 in u0s:
            out = torch.empty((rows, nx), dtype=torch.float64, device="cuda")
            r, _ = capi.mgrit_solve(h, u0, out)
            want.append((r.iterations, r.rel_residual, r.r0_norm, out.cpu().numpy()))
        outs = [torch.full((rows, nx), float("nan"), dtype=torch.float64, device="cuda") for _ in u0s]
        for u0, out in zip(u0s, outs):
            capi.mgrit_solve_async(h, u0, out)
        for k, out in enumerate(outs):
            r, st = capi.mgrit_solve_wait(h)
            it, rr, r0, ref = want[k]
            assert st == 0 and r.converged == 1 and r.graph == 1
            assert (r.iterations, r.rel_residual, r.r0_norm) == (it, rr, r0)
            np.testing.assert_array_equal(out.cpu().numpy(), ref)
            assert r.launches > 0
    finally:
        capi.mgrit_destroy(h)


def test_queued_solve_errors(capi):
    import torch
    nx, nt, m = 64, 256, 8
    u0 = torch.tensor(workloads.sin4(nx), device="cuda")
    h = capi.mgrit_setup(capi.problem(nx, nt, "ERK", 1, 1, 0.85), capi.mgrit_opts_default(m=m, output=1))
    try:
        with pytest.raises(capi.MgritError) as e:
            capi.mgrit_solve_wait(h)
        assert e.value.status == -1
        with pytest.raises(capi.MgritError) as e:
            capi.mgrit_solve_async(h, u0, np.zeros((nt // m + 1, nx)))  # host output
        assert e.value.status == -1
        out = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
        for _ in range(capi.MAX_INFLIGHT):
            capi.mgrit_solve_async(h, u0, out)
        with pytest.raises(capi.MgritError) as e:
            capi.mgrit_solve_async(h, u0, out)
        assert e.value.status == -1
        its = {capi.mgrit_solve_wait(h)[0].iterations for _ in range(capi.MAX_INFLIGHT)}
        assert len(its) == 1
    finally:
        capi.mgrit_destroy(h)
    h = capi.mgrit_setup(capi.problem(nx, nt, "ERK", 1, 1, 0.85), capi.mgrit_opts_default(m=m, output=2))
    try:
        with pytest.raises(capi.MgritError) as e:
            capi.mgrit_solve_async(h, u0, None)
        assert e.value.status == -10
    finally:
        capi.mgrit_destroy(h)


RANDOM_CASES = [("ERK", 1, 64, 1024, 8, 2, "halfwidth", 11), ("ERK", 3, 128, 512, 4, 3, "auto", 12),
                ("ERK", 5, 128, 512, 8, 2, "auto", 2 ** 40 + 3), ("SDIRK", 3, 128, 256, 16, 2, "threshold", 14),
                ("SDIRK", 2, 96, 384, 4, 3, "threshold", 15)]
RULE = {"halfwidth": 1, "auto": 0, "threshold": 2}


def oracle_random(fam, p, c, nx, nt, m, L, rule, u0, seed):
    st = stepping.FineStep(fam, p, c, nx)
    ops = [o.diag for o in opsi.build_hierarchy(fam, p, c, nx, nt, m, L, rule=rule, halfwidth=3)]
    U = philox.random_iterate(u0, nt, seed)
    r0 = float(np.linalg.norm(omg.spacetime_residual(U, np.zeros_like(U), st)))
    it, _ = omg.solve(omg.make_levels(st, m, ops), U, tol=1e-10)
    return it, r0, U[::m]


@pytest.mark.parametrize("case", RANDOM_CASES)
def test_random_initial_iterate_matches_oracle(capi, case):
    import torch
    fam, p, nx, nt, m, L, rule, seed = case
    c = schemes.cfl_number(fam, p)
    u0 = workloads.fourier_field(nx, seed=3)
    it, r0, cref = oracle_random(fam, p, c, nx, nt, m, L, rule, u0, seed)
    prob = capi.problem(nx, nt, fam, p, p, c)
    results = []
    for flags in (0, capi.FLAG_HOST_LOOP):
        opts = capi.mgrit_opts_default(m=m, levels=L, psi_rule=RULE[rule], psi_halfwidth=3, output=1, tol=1e-10,
                                       init_guess=capi.INIT_RANDOM, seed=seed, flags=flags)
        h = capi.mgrit_setup(prob, opts)
        try:
            out = np.zeros((nt // m + 1, nx))
            res, _ = capi.mgrit_solve(h, u0, out)
            results.append((res.iterations, res.r0_norm, out))
            if flags == 0:
                dout = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
                capi.mgrit_solve_async(h, torch.tensor(u0, device="cuda"), dout)
                ra, _ = capi.mgrit_solve_wait(h)
                assert ra.iterations == res.iterations and ra.r0_norm == res.r0_norm
                np.testing.assert_array_equal(dout.cpu().numpy(), out)
        finally:
            capi.mgrit_destroy(h)
    for gi, gr0, out in results:
        assert gi == it, (gi, it)
        assert abs(gr0 - r0) <= 1e-12 * r0, (gr0, r0)
        assert rel(out, cref) <= 1e-12


def test_random_iterate_differs_from_zero_iterate_and_depends_on_seed(capi):
    """The random start needs more iterations than the zero start on config 1
    (the paper's tables count from it), and a new seed changes ||r^(0)||."""
    nx, nt, m = 64, 1024, 8
    u0 = workloads.sin4(nx)
    r = {}
    for init, seed in ((0, 0), (1, 1), (1, 2)):
        opts = capi.mgrit_opts_default(m=m, levels=2, psi_rule=1, psi_halfwidth=3, init_guess=init, seed=seed)
        h = capi.mgrit_setup(capi.problem(nx, nt, "ERK", 1, 1, 0.85), opts)
        try:
            r[(init, seed)] = capi.mgrit_solve(h, u0, None)[0]
        finally:
            capi.mgrit_destroy(h)
    assert r[(1, 1)].r0_norm != r[(1, 2)].r0_norm
    assert r[(1, 1)].iterations >= r[(0, 0)].iterations


def test_result_reports_physical_spacings(capi):
    """Eq. 1: dx = (xmax - xmin)/nx and dt = c dx / alpha; the discrete
    solve depends on c only, so alpha and the domain leave it unchanged."""
    nx, nt, m, c = 64, 256, 8, 0.85
    u0 = workloads.sin4(nx)
    outs = []
    for alpha, lo, hi in ((1.0, -1.0, 1.0), (2.5, 0.0, 10.0)):
        h = capi.mgrit_setup(capi.problem(nx, nt, "ERK", 1, 1, c, alpha=alpha, xmin=lo, xmax=hi),
                             capi.mgrit_opts_default(m=m))
        try:
            out = np.zeros((nt // m + 1, nx))
            res, _ = capi.mgrit_solve(h, u0, out)
        finally:
            capi.mgrit_destroy(h)
        assert abs(res.dx - (hi - lo) / nx) <= 1e-15 * res.dx
        assert abs(res.dt - c * res.dx / alpha) <= 1e-15 * res.dt
        outs.append(out)
    np.testing.assert_array_equal(outs[0], outs[1])
