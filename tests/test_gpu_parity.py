"""GPU vs. oracle parity through the C ABI (FP64 relative L2 <= 1e-12 and the
same iteration count; Section 2.2's MGRIT, Eq. 3's sequential stepping)."""
import numpy as np
import pytest

import workloads
from oracle import mgrit as omg
from oracle import psi as opsi
from oracle import schemes, stepping

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


RULE = {"halfwidth": 1, "auto": 0, "threshold": 2, "ideal": 4}


def oracle_run(fam, p, c, nx, nt, m, L, rule, u0, tol=1e-10, psi_ops=None, cycle="V", relax="FCF"):
    st = stepping.FineStep(fam, p, c, nx)
    if psi_ops is None:
        ops = [o.diag for o in opsi.build_hierarchy(fam, p, c, nx, nt, m, L, rule=rule, halfwidth=3)]
    else:
        ops = [dict(zip(o, v)) for o, v in psi_ops]
    lev = omg.make_levels(st, m, ops)
    U = omg.zero_iterate(u0, nt)
    hist = []
    it, r = omg.solve(lev, U, tol=tol, history=hist, cycle=cycle, relax=relax)
    return it, r, U, hist


def gpu_run(capi, fam, p, c, nx, nt, m, L, rule, u0, precision=0, output=1, tol=1e-10, user=None, cycle="V",
            relax="FCF", flags=0):
    opts = capi.mgrit_opts_default(m=m, levels=L, psi_rule=RULE[rule], psi_halfwidth=3, precision=precision,
                                   output=output, tol=tol, cycle=0 if cycle == "V" else 1,
                                   relax=0 if relax == "FCF" else 1, flags=flags)
    keep = capi.user_psi(opts, user) if user is not None else None
    h = capi.mgrit_setup(capi.problem(nx, nt, fam, p, p, c), opts)
    try:
        nrow = {0: 1, 1: nt // m + 1, 2: nt + 1}[output]
        out = np.zeros((nrow, nx))
        res, st = capi.mgrit_solve(h, np.ascontiguousarray(u0), out)
        ops = [capi.mgrit_psi_info(h, l) for l in range(2, L + 1)]
    finally:
        capi.mgrit_destroy(h)
    del keep
    return res, out, ops


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_fine_step_matches_stage_form(capi, p):
    """A1: the collapsed ERK stencil applied k times equals k stage-wise steps."""
    import torch
    nx, k, count = 200, 3, 7           # nx not a power of two: ragged tiles
    c = schemes.cfl_number("ERK", p)
    h = capi.mgrit_setup(capi.problem(nx, 8, "ERK", p, p, c), capi.mgrit_opts_default(m=2, levels=2))
    try:
        x = np.random.default_rng(p).standard_normal((count, nx))
        xin = torch.tensor(x, device="cuda")
        yout = torch.zeros_like(xin)
        capi.mgrit_propagate(h, 1, k, count, xin, yout)
    finally:
        capi.mgrit_destroy(h)
    st = stepping.FineStep("ERK", p, c, nx)
    ref = x.copy()
    for _ in range(k):
        ref = st(ref)
    assert rel(yout.cpu().numpy(), ref) <= TOL


def test_config1_two_level_parity(capi):
    """ERK1+U1, nx=64, nt=1024, m=8, Psi half-width 3, sin^4, zero guess."""
    nx, nt, m = 64, 1024, 8
    u0 = workloads.sin4(nx)
    it, r, U, hist = oracle_run("ERK", 1, 0.85, nx, nt, m, 2, "halfwidth", u0)
    res, out, ops = gpu_run(capi, "ERK", 1, 0.85, nx, nt, m, 2, "halfwidth", u0)
    assert res.iterations == it
    assert res.converged == 1
    assert rel(out, U[::m]) <= TOL
    # relative residuals carry rounding of about eps absolute (they are
    # norms of r over ||r0||): 1e-6 relative above 1e-9, 1e-15 absolute below
    np.testing.assert_allclose(res.history[: res.n_history], hist, rtol=1e-6, atol=1e-15)


@pytest.mark.parametrize("case", [
    ("ERK", 3, 256, 2048, 4, 2), ("ERK", 3, 256, 2048, 8, 3), ("ERK", 3, 256, 2048, 4, 4),
    ("ERK", 5, 128, 1024, 4, 3), ("ERK", 2, 96, 768, 4, 3), ("ERK", 4, 128, 512, 16, 2),
])
def test_mgrit_parity_fp64(capi, case):
    """Two-level and V-cycle MGRIT, own Psi on each side (same pattern; fitted
    coefficients agree to ~1e-10, which the iteration damps)."""
    fam, p, nx, nt, m, L = case
    c = schemes.cfl_number(fam, p)
    u0 = workloads.fourier_field(nx)
    it, r, U, _ = oracle_run(fam, p, c, nx, nt, m, L, "auto", u0)
    res, out, _ = gpu_run(capi, fam, p, c, nx, nt, m, L, "auto", u0)
    assert res.iterations == it
    assert rel(out, U[::m]) <= TOL


def test_mgrit_parity_shared_psi_full_output(capi):
    """Same Psi on both sides (oracle's fit passed through PSI_USER); FULL
    output = C-points plus F-points by ideal interpolation."""
    fam, p, nx, nt, m, L = "ERK", 3, 128, 512, 4, 3
    c = schemes.cfl_number(fam, p)
    ops = opsi.build_hierarchy(fam, p, c, nx, nt, m, L, rule="auto")
    user = [(o.offsets, [o.diag[i] for i in o.offsets]) for o in ops]
    u0 = workloads.sin4(nx)
    it, r, U, _ = oracle_run(fam, p, c, nx, nt, m, L, "auto", u0, psi_ops=user)
    res, out, got_ops = gpu_run(capi, fam, p, c, nx, nt, m, L, "auto", u0, output=2, user=user)
    assert [o for o, _ in got_ops] == [o for o, _ in user]
    assert res.iterations == it
    assert rel(out, U) <= TOL


def test_mixed_precision_reaches_the_fp64_fixed_point(capi):
    """MIXED: FP32 second F-relaxation; the FP64 residual drives the iteration
    to the same discrete solution; iterations equal FP64's (within 1)."""
    fam, p, nx, nt, m, L = "ERK", 3, 256, 2048, 8, 2
    c = schemes.cfl_number(fam, p)
    u0 = workloads.fourier_field(nx)
    it, r, U, _ = oracle_run(fam, p, c, nx, nt, m, L, "auto", u0)
    ref = stepping.sequential(stepping.FineStep(fam, p, c, nx), u0, nt)
    res, out, _ = gpu_run(capi, fam, p, c, nx, nt, m, L, "auto", u0, precision=1)
    assert abs(res.iterations - it) <= 1
    assert res.rel_residual <= 1e-10
    assert rel(out, ref[::m]) <= 1e-9


@pytest.mark.parametrize("output", [0, 1, 2])
def test_sequential_stepping_matches_oracle(capi, output):
    nx, nt, m = 96, 240, 8
    c = schemes.cfl_number("ERK", 3)
    u0 = workloads.fourier_field(nx)
    ref = stepping.sequential(stepping.FineStep("ERK", 3, c, nx), u0, nt)
    h = capi.mgrit_setup(capi.problem(nx, nt, "ERK", 3, 3, c), capi.mgrit_opts_default(m=m, output=output))
    try:
        rows = {0: 1, 1: nt // m + 1, 2: nt + 1}[output]
        out = np.zeros((rows, nx))
        capi.mgrit_sequential(h, u0, out)
    finally:
        capi.mgrit_destroy(h)
    want = {0: ref[-1:], 1: ref[::m], 2: ref}[output]
    assert rel(out, want) <= TOL


def test_edge_cases_small_and_ragged(capi):
    """Smallest grids (nx = 8), m = 2 with two intervals, non-power-of-two nx,
    and max_iter = 0 (returns NOT_CONVERGED with the relaxed iterate)."""
    for (nx, nt, m, L) in [(8, 4, 2, 2), (24, 48, 2, 3), (40, 64, 4, 2)]:
        u0 = workloads.sin4(nx)
        it, r, U, _ = oracle_run("ERK", 1, 0.85, nx, nt, m, L, "auto", u0)
        res, out, _ = gpu_run(capi, "ERK", 1, 0.85, nx, nt, m, L, "auto", u0)
        assert res.iterations == it, (nx, nt, m, L)
        assert rel(out, U[::m]) <= TOL
    opts = capi.mgrit_opts_default(m=8, levels=2, max_iter=0)
    h = capi.mgrit_setup(capi.problem(64, 256, "ERK", 1, 1, 0.85), opts)
    try:
        res, st = capi.mgrit_solve(h, workloads.sin4(64), None, allow_not_converged=True)
        assert st == -4 and res.iterations == 0 and res.converged == 0
    finally:
        capi.mgrit_destroy(h)


def test_nonfinite_initial_condition_reports_divergence(capi):
    u0 = workloads.sin4(64)
    u0[3] = np.inf
    h = capi.mgrit_setup(capi.problem(64, 256, "ERK", 1, 1, 0.85), capi.mgrit_opts_default(m=8))
    try:
        with pytest.raises(capi.MgritError) as ei:
            capi.mgrit_solve(h, u0, None)
        assert ei.value.status == -5
    finally:
        capi.mgrit_destroy(h)


@pytest.mark.parametrize("precision,L", [(1, 3), (2, 2), (2, 4)])
def test_mixed_modes_reach_the_fp64_fixed_point(capi, precision, L):
    """MIXED (FP32 coarse levels) and MIXED_DF (float-float C-point pass):
    the FP64 stopping test is met and the solution agrees with FP64
    sequential stepping to the accuracy the tolerance implies."""
    fam, p, nx, nt, m = "ERK", 3, 256, 4096, 8 if L < 4 else 4
    c = schemes.cfl_number(fam, p)
    u0 = workloads.fourier_field(nx)
    ref = stepping.sequential(stepping.FineStep(fam, p, c, nx), u0, nt)
    it64 = gpu_run(capi, fam, p, c, nx, nt, m, L, "auto", u0, precision=0)[0].iterations
    res, out, _ = gpu_run(capi, fam, p, c, nx, nt, m, L, "auto", u0, precision=precision)
    assert res.converged == 1 and res.rel_residual <= 1e-10
    assert abs(res.iterations - it64) <= 1
    assert rel(out, ref[::m]) <= 1e-9


@pytest.mark.parametrize("L,precision", [(2, 0), (3, 0), (4, 1), (2, 2)])
def test_graph_solve_equals_host_loop(capi, L, precision):
    """The whole solve as one CUDA graph (on-device stopping test driving the
    WHILE/IF nodes) gives the host-driven loop's iterations and C-points."""
    fam, p, nx, nt, m = "ERK", 3, 128, 2048, 4
    c = schemes.cfl_number(fam, p)
    u0 = workloads.fourier_field(nx)
    outs = []
    for flags in (capi.FLAG_HOST_LOOP, 0):
        opts = capi.mgrit_opts_default(m=m, levels=L, precision=precision, flags=flags)
        h = capi.mgrit_setup(capi.problem(nx, nt, fam, p, p, c), opts)
        try:
            out = np.zeros((nt // m + 1, nx))
            res, _ = capi.mgrit_solve(h, u0, out)
            res2, _ = capi.mgrit_solve(h, u0, out)  # the graph is reused
        finally:
            capi.mgrit_destroy(h)
        assert res.iterations == res2.iterations
        outs.append((res, out))
    (r0, o0), (r1, o1) = outs
    assert r1.graph == 1 and r0.graph == 0
    assert r1.iterations == r0.iterations
    np.testing.assert_allclose(r1.history[: r1.n_history], r0.history[: r0.n_history], rtol=1e-14)
    assert rel(o1, o0) <= 1e-15


@pytest.mark.parametrize("shape", ["99,256,0", "8,256,1", "4,512,1", "0,128,0", "8,128,0", "98,256,1", "98,512,0"])
def test_every_fine_launch_shape_matches_oracle(capi, shape, monkeypatch):
    """Each level-1 FCF launch shape the autotuner may pick (step by step with
    Phi or one application of the collapsed Phi^m per pass; fixed-span,
    sliding-window or one-tap-at-a-time stencil) gives the oracle's
    iterations and C-points."""
    monkeypatch.setenv("MGRIT_FCF_SHAPE", shape)
    fam, p, nx, nt, m, L = "ERK", 3, 256, 2048, 8, 3
    c = schemes.cfl_number(fam, p)
    u0 = workloads.fourier_field(nx)
    it, r, U, _ = oracle_run(fam, p, c, nx, nt, m, L, "auto", u0)
    res, out, _ = gpu_run(capi, fam, p, c, nx, nt, m, L, "auto", u0)
    tile, th, col = (int(v) for v in shape.split(","))
    assert (res.fine_tile, res.fine_threads, res.fine_collapsed) == (tile, th, col)
    assert res.iterations == it
    assert rel(out, U[::m]) <= TOL


@pytest.mark.parametrize("precision,relax", [(0, "FCF"), (1, "FCF"), (2, "FCF"), (0, "F")])
def test_relax_sweeps_match_oracle(capi, precision, relax):
    """mgrit_relax: FCF- (or F-) relaxation sweeps without coarse correction
    from the iterate a solve left (here: the paper's random iterate after the
    one relaxation of a max_iter = 0 solve), against the same sweeps in the
    oracle: the relative residual after k sweeps agrees (FP64: to 1e-12;
    mixed modes: to their FP32 second pass).  F-relaxation leaves the
    C-points alone, so its residual stays put."""
    fam, p, nx, nt, m = "ERK", 3, 128, 512, 4
    c = schemes.cfl_number(fam, p)
    st = stepping.FineStep(fam, p, c, nx)
    U = workloads.random_iterate(nt, nx, workloads.sin4(nx), 3)
    r0 = float(np.linalg.norm(omg.spacetime_residual(U, np.zeros_like(U), st)))
    opts = capi.mgrit_opts_default(m=m, levels=2, max_iter=0, precision=precision,
                                   relax=0 if relax == "FCF" else 1)
    h = capi.mgrit_setup(capi.problem(nx, nt, fam, p, p, c), opts)
    try:
        res, status = capi.mgrit_solve_from(h, np.ascontiguousarray(U[::m]), r0, allow_not_converged=True)
        assert status == -4 and res.iterations == 0
        got = [capi.mgrit_relax(h, 1) for _ in range(3)] + [capi.mgrit_relax(h, 4)]
    finally:
        capi.mgrit_destroy(h)
    G = np.zeros_like(U)
    want = []
    for k in range(1 + 3 + 4):
        omg.f_relax(U, G, st, m)
        if relax == "FCF":
            omg.c_relax(U, G, st, m)
            omg.f_relax(U, G, st, m)
        if k >= 1 and k <= 3 or k == 7:
            want.append(float(np.linalg.norm(omg.c_residual(U, G, st, m))) / r0)
    tol = 1e-12 if precision == 0 else 1e-6
    np.testing.assert_allclose(got, want, rtol=tol)
    if relax == "F":
        assert got[0] == got[-1]


@pytest.mark.parametrize("case", [("ERK", 3, 256, 2048, 4, 2), ("ERK", 3, 256, 2048, 8, 3), ("ERK", 1, 64, 1024, 2, 6),
                                  ("ERK", 5, 128, 1024, 4, 3)])
@pytest.mark.parametrize("coarse", ["fft", "march"])
@pytest.mark.parametrize("precision", [0, 1])
def test_coarse_solver_parity(capi, monkeypatch, case, coarse, precision):
    """The coarsest level solved in Fourier space (per-mode recurrences with
    Psi's symbol between forward and inverse FFTs) and by the cluster march,
    forced either way for long and short coarsest levels: FP64 gives the
    oracle's iterations and C-points; MIXED the oracle's C-points to 1e-9."""
    monkeypatch.setenv("MGRIT_COARSE", coarse)
    fam, p, nx, nt, m, L = case
    c = schemes.cfl_number(fam, p)
    u0 = workloads.fourier_field(nx)
    it, r, U, _ = oracle_run(fam, p, c, nx, nt, m, L, "auto", u0)
    res, out, _ = gpu_run(capi, fam, p, c, nx, nt, m, L, "auto", u0, precision=precision)
    assert res.converged == 1
    if precision == 0:
        assert res.iterations == it
        assert rel(out, U[::m]) <= TOL
    else:
        assert abs(res.iterations - it) <= 1
        assert rel(out, U[::m]) <= 1e-9


@pytest.mark.parametrize("p,m", [(1, 4), (2, 4), (1, 16)])
@pytest.mark.parametrize("precision", [0, 1, 2])
def test_collapsed_fixed_span_shape(capi, monkeypatch, p, m, precision):
    """The fixed-span path applied to Phi^m when its span is one the kernels
    are compiled for (ERK1 m = 4: 5; ERK2 m = 4 and ERK1 m = 16: 17): FP64
    gives the oracle's iterations and C-points, the mixed modes FP64
    sequential stepping's C-points."""
    monkeypatch.setenv("MGRIT_FCF_SHAPE", "99,256,1")
    fam, nx, nt, L = "ERK", 256, 4096, 3
    c = schemes.cfl_number(fam, p)
    u0 = workloads.fourier_field(nx)
    it, r, U, _ = oracle_run(fam, p, c, nx, nt, m, L, "auto", u0)
    res, out, _ = gpu_run(capi, fam, p, c, nx, nt, m, L, "auto", u0, precision=precision)
    assert (res.fine_tile, res.fine_threads, res.fine_collapsed) == (99, 256, 1)
    assert res.converged == 1
    if precision == 0:
        assert res.iterations == it
        assert rel(out, U[::m]) <= TOL
    else:
        assert abs(res.iterations - it) <= 1
        assert rel(out, U[::m]) <= 1e-9


@pytest.mark.parametrize("case", [("ERK", 1, 64, 1024, 2, 6), ("ERK", 3, 128, 2048, 4, 4), ("ERK", 5, 128, 1024, 4, 3)])
@pytest.mark.parametrize("flags", [0, 4])
def test_fcycle_parity(capi, case, flags):
    """F-cycles (graph and host-driven loop): the oracle's iterations and
    C-points; on ERK1 m = 2, six levels, fewer iterations than V-cycles."""
    fam, p, nx, nt, m, L = case
    c = schemes.cfl_number(fam, p)
    u0 = workloads.fourier_field(nx)
    it, r, U, _ = oracle_run(fam, p, c, nx, nt, m, L, "auto", u0, cycle="F")
    res, out, _ = gpu_run(capi, fam, p, c, nx, nt, m, L, "auto", u0, cycle="F", flags=flags)
    assert res.iterations == it
    assert rel(out, U[::m]) <= TOL
    if L == 6:
        itv = gpu_run(capi, fam, p, c, nx, nt, m, L, "auto", u0, flags=flags)[0].iterations
        assert res.iterations < itv


@pytest.mark.parametrize("case", [("ERK", 3, 256, 2048, 8, 2), ("ERK", 1, 128, 1024, 4, 3), ("ERK", 4, 128, 512, 4, 2)])
@pytest.mark.parametrize("flags", [0, 4])
def test_f_relaxation_parity(capi, case, flags):
    """F-relaxation only on level 1 (two levels: Parareal): the oracle's
    iterations and C-points."""
    fam, p, nx, nt, m, L = case
    c = schemes.cfl_number(fam, p)
    u0 = workloads.fourier_field(nx)
    it, r, U, _ = oracle_run(fam, p, c, nx, nt, m, L, "auto", u0, relax="F")
    res, out, _ = gpu_run(capi, fam, p, c, nx, nt, m, L, "auto", u0, relax="F", flags=flags)
    assert res.iterations == it
    assert rel(out, U[::m]) <= TOL


def test_f_relaxation_mixed_reaches_the_fp64_fixed_point(capi):
    fam, p, nx, nt, m, L = "ERK", 3, 256, 2048, 8, 2
    c = schemes.cfl_number(fam, p)
    u0 = workloads.fourier_field(nx)
    ref = stepping.sequential(stepping.FineStep(fam, p, c, nx), u0, nt)
    it64 = gpu_run(capi, fam, p, c, nx, nt, m, L, "auto", u0, relax="F")[0].iterations
    for prec in (1, 2):
        res, out, _ = gpu_run(capi, fam, p, c, nx, nt, m, L, "auto", u0, precision=prec, relax="F")
        assert res.converged == 1 and abs(res.iterations - it64) <= 1
        assert rel(out, ref[::m]) <= 1e-9


@pytest.mark.parametrize("nx,nt,m,L", [(4096, 16384, 4, 4), (512, 2048, 4, 2), (8192, 1024, 4, 3), (1024, 64, 4, 2),
                                       (2048, 8192, 4, 3)])
def test_fused_float_float_fcf_forms_agree(capi, monkeypatch, nx, nt, m, L):
    """The fused float-float FCF (ERK1+U1, m = 4: collapsed Phi^4 of 5 taps) in
    its five forms -- the slab in shared memory, one interval per CTA (0);
    register-resident runs of intervals per CTA with the next slab prefetched
    (1, the default); runs with the slabs in shared memory, streamed through
    registers (2) or with cp.async copies (3); register-resident, one interval
    per CTA (4) -- give the same solve
    (bitwise C-points, the same iterations) and the same relaxation sweeps,
    from the zero iterate (zero slabs) and from a converged one; grids from
    one interval per CTA (nt/m = 16) to runs of about 14."""
    import torch
    u0 = torch.tensor(workloads.fourier_field(nx), device="cuda")
    got = {}
    for stream in ("0", "1", "2", "3", "4"):
        monkeypatch.setenv("MGRIT_FCF_STREAM", stream)
        monkeypatch.setenv("MGRIT_FCF_SHAPE", "99,256,1")
        o = capi.mgrit_opts_default(m=m, levels=L, precision=capi.PREC_MIXED_DF, output=capi.OUT_CPOINTS,
                                    tol=1e-10)
        h = capi.mgrit_setup(capi.problem(nx, nt, "ERK", 1, 1, 0.85), o)
        try:
            out = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
            r, _ = capi.mgrit_solve(h, u0, out)
            rel_sweeps = capi.mgrit_relax(h, 3)
            out2 = torch.empty_like(out)
            capi.mgrit_solve(h, u0, out2)
            got[stream] = (r.iterations, out.cpu().numpy(), rel_sweeps, out2.cpu().numpy())
        finally:
            capi.mgrit_destroy(h)
    b = got["0"]
    assert np.isfinite(b[2]) and b[2] > 0
    for mode in ("1", "2", "3", "4"):
        a = got[mode]
        assert a[0] == b[0], mode
        np.testing.assert_array_equal(a[1], b[1])
        np.testing.assert_array_equal(a[3], b[3])
        assert abs(a[2] - b[2]) <= 1e-6 * b[2], mode


@pytest.mark.parametrize("nx,nt,m,L", [(4096, 16384, 4, 4), (512, 2048, 4, 2), (8192, 1024, 4, 3), (256, 4096, 4, 3),
                                       (1024, 64, 4, 2)])
def test_mixed_fcf_register_run_agrees(capi, monkeypatch, nx, nt, m, L):
    """MIXED (FP64 C-point update, FP32 second pass) on ERK1+U1, m = 4: the
    collapsed Phi^4 of 5 taps with one interval per CTA and the slab in shared
    memory (form 0) and as register-resident runs of intervals with the next
    slab prefetched (form 1, the default) give bitwise the same C-points and
    iterations, and the same relaxation sweeps; where the oracle's sequential
    stepping (Eq. 3) is small enough, the solve reaches its C-points to 1e-9."""
    import torch
    u0h = workloads.fourier_field(nx)
    u0 = torch.tensor(u0h, device="cuda")
    got = {}
    for stream in ("0", "1"):
        monkeypatch.setenv("MGRIT_FCF_STREAM", stream)
        monkeypatch.setenv("MGRIT_FCF_SHAPE", "99,256,1")
        o = capi.mgrit_opts_default(m=m, levels=L, precision=capi.PREC_MIXED, output=capi.OUT_CPOINTS, tol=1e-10)
        h = capi.mgrit_setup(capi.problem(nx, nt, "ERK", 1, 1, 0.85), o)
        try:
            out = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
            r, _ = capi.mgrit_solve(h, u0, out)
            assert r.converged == 1
            rel_sweeps = capi.mgrit_relax(h, 3)
            out2 = torch.empty_like(out)
            capi.mgrit_solve(h, u0, out2)
            got[stream] = (r.iterations, out.cpu().numpy(), rel_sweeps, out2.cpu().numpy())
        finally:
            capi.mgrit_destroy(h)
    a, b = got["1"], got["0"]
    assert a[0] == b[0]
    np.testing.assert_array_equal(a[1], b[1])
    np.testing.assert_array_equal(a[3], b[3])
    assert np.isfinite(b[2]) and b[2] > 0 and abs(a[2] - b[2]) <= 1e-6 * b[2]
    if nx * nt <= 2 ** 21:
        ref = stepping.sequential(stepping.FineStep("ERK", 1, 0.85, nx), u0h, nt)[::m]
        assert rel(a[1], ref) <= 1e-9


@pytest.mark.parametrize("nx,nt,m,L,prec", [(4096, 16384, 8, 4, 1), (4096, 1024, 8, 2, 0), (2048, 2048, 4, 3, 0),
                                            (8192, 512, 16, 2, 1), (2048, 1024, 8, 2, 2)])
def test_coarsest_fourier_solve_split_over_a_cluster_agrees(capi, monkeypatch, nx, nt, m, L, prec):
    """The coarsest level in Fourier space with each slab's transforms split
    over a cluster of four CTAs (automatic when the level has fewer slabs
    than SMs) gives bitwise the C-points and iterations of one CTA per slab:
    the same butterflies in the same order, the last two passes across the
    CTAs' blocks."""
    import torch
    u0 = torch.tensor(workloads.fourier_field(nx), device="cuda")
    got = {}
    for split in ("0", "1"):
        monkeypatch.setenv("MGRIT_FFT_SPLIT", split)
        monkeypatch.setenv("MGRIT_COARSE", "fft")
        o = capi.mgrit_opts_default(m=m, levels=L, precision=prec, output=capi.OUT_CPOINTS, tol=1e-10)
        h = capi.mgrit_setup(capi.problem(nx, nt, "ERK", 3, 3, 0.85 * 1.62589), o)
        try:
            out = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
            r, _ = capi.mgrit_solve(h, u0, out)
            assert r.converged == 1
            got[split] = (r.iterations, r.rel_residual, out.cpu().numpy())
        finally:
            capi.mgrit_destroy(h)
    assert got["1"][0] == got["0"][0] and got["1"][1] == got["0"][1]
    np.testing.assert_array_equal(got["1"][2], got["0"][2])


def test_integer_pipe_conversion_matches_the_conversion_instruction(capi):
    """The kernels' binary32 -> binary64 conversion built from the IEEE 754
    bit fields (the level-1 correction, the coarse march's FP32 right-hand
    side) gives bitwise the GPU's conversion instruction's result on 2^25
    hashed patterns, zeros, subnormals, infinities and NaNs among them, for
    two seeds."""
    for seed in (1, 2 ** 40 + 7):
        assert capi.mgrit_check_conversions(1 << 24, seed) == 0


@pytest.mark.parametrize("nx,p,L", [(12231, 1, 2), (12231, 3, 3), (12224, 2, 2)])
def test_largest_slab_matches_oracle(capi, nx, p, L):
    """The largest slab a CTA holds (nx = 12231: two padded FP64 slabs and up
    to 12 KiB of static shared memory in 227 KiB; odd, so every loop takes
    its ragged tail): FP64 the oracle's iterations and C-points to 1e-12,
    MIXED at sequential stepping to 1e-9; and the server (whose batched FCF
    keeps its stencil in shared memory too) gives the same solve."""
    nt, m = 256, 4
    c = schemes.cfl_number("ERK", p)
    u0 = workloads.fourier_field(nx)
    it, r, U, _ = oracle_run("ERK", p, c, nx, nt, m, L, "auto", u0)
    res, out, _ = gpu_run(capi, "ERK", p, c, nx, nt, m, L, "auto", u0)
    assert res.iterations == it
    assert rel(out, U[::m]) <= TOL
    ref = stepping.sequential(stepping.FineStep("ERK", p, c, nx), u0, nt)
    res, out, _ = gpu_run(capi, "ERK", p, c, nx, nt, m, L, "auto", u0, precision=1)
    assert res.converged == 1 and rel(out, ref[::m]) <= 1e-9
    srv = capi.mgrit_server_create(20e9)
    try:
        opts = capi.mgrit_opts_default(m=m, levels=L, psi_rule=RULE["auto"], psi_halfwidth=3, precision=0,
                                       output=1, tol=1e-10)
        t = capi.mgrit_submit(srv, capi.problem(nx, nt, "ERK", p, p, c), opts, np.ascontiguousarray(u0))
        sout = np.zeros((nt // m + 1, nx))
        import time
        t0 = time.time()
        while True:
            st, sres = capi.mgrit_poll(srv, t, sout)
            if st != capi.MGRIT_PENDING:
                break
            assert time.time() - t0 < 120, "request did not finish"
            time.sleep(0.002)
        assert st == 0 and sres.iterations == it and rel(sout, U[::m]) <= TOL
    finally:
        capi.mgrit_server_destroy(srv)


@pytest.mark.parametrize("nx,L", [(131, 2), (1001, 2), (1001, 3), (4099, 2)])
@pytest.mark.parametrize("precision", [0, 1])
def test_ragged_cluster_march_matches_oracle(capi, monkeypatch, nx, L, precision):
    """The march's cluster need not divide nx: CTAs own ceil(nx / cs) points
    and the last one the rest (131 on 2 CTAs: 66 + 65; 1001 on 8: 7 x 126 +
    119; the prime 4099 on 16: 15 x 257 + 244).  The coarsest level forced
    onto the march gives the oracle's iterations and C-points (FP64, 1e-12),
    MIXED the oracle's C-points to 1e-9."""
    monkeypatch.setenv("MGRIT_COARSE", "march")
    nt, m = 512, 4
    c = schemes.cfl_number("ERK", 3)
    u0 = workloads.fourier_field(nx)
    it, r, U, _ = oracle_run("ERK", 3, c, nx, nt, m, L, "auto", u0)
    res, out, _ = gpu_run(capi, "ERK", 3, c, nx, nt, m, L, "auto", u0, precision=precision)
    assert res.converged == 1
    if precision == 0:
        assert res.iterations == it
        assert rel(out, U[::m]) <= TOL
    else:
        assert abs(res.iterations - it) <= 1
        assert rel(out, U[::m]) <= 1e-9


def test_ragged_cluster_batched_march_matches_oracle(capi, monkeypatch):
    """The server's batched march on clusters that do not divide nx (1001 and
    131 points, two-level solves in one mix): each result is the oracle's."""
    monkeypatch.setenv("MGRIT_COARSE", "march")
    nt, m = 512, 4
    c = schemes.cfl_number("ERK", 3)
    srv = capi.mgrit_server_create(20e9)
    try:
        opts = capi.mgrit_opts_default(m=m, levels=2, psi_rule=RULE["auto"], psi_halfwidth=3, precision=0,
                                       output=1, tol=1e-10)
        cases = []
        for nx in (1001, 131, 1001):
            u0 = np.ascontiguousarray(workloads.fourier_field(nx))
            t = capi.mgrit_submit(srv, capi.problem(nx, nt, "ERK", 3, 3, c), opts, u0)
            cases.append((nx, u0, t, np.zeros((nt // m + 1, nx))))
        import time
        for nx, u0, t, sout in cases:
            t0 = time.time()
            while True:
                st, sres = capi.mgrit_poll(srv, t, sout)
                if st != capi.MGRIT_PENDING:
                    break
                assert time.time() - t0 < 120, "request did not finish"
                time.sleep(0.002)
            it, r, U, _ = oracle_run("ERK", 3, c, nx, nt, m, 2, "auto", u0)
            assert st == 0 and sres.iterations == it and rel(sout, U[::m]) <= TOL
    finally:
        capi.mgrit_server_destroy(srv)


@pytest.mark.parametrize("p,nx,m,L", [(1, 256, 4, 3), (2, 512, 8, 2), (3, 1024, 8, 3), (4, 256, 4, 2), (5, 512, 4, 3),
                                      (3, 8192, 8, 2)])
@pytest.mark.parametrize("shape", ["1", "8,256,1,128"])
def test_fourier_fcf_matches_oracle(capi, monkeypatch, p, nx, m, L, shape):
    """MIXED level-1 FCF with the FP64 pass Phi^m c_{j-1} taken in Fourier
    space (half-length complex FFT of the slab, product with the collapsed
    stencil's symbol, inverse FFT; Lemma 1's diagonalisation of a circulant),
    forced on (256 threads, or pinned at 128): the oracle's C-points to 1e-9
    and its iterations within one, from nx = 256 (fewer butterflies per pass
    than threads) to 8192."""
    if shape == "1":
        monkeypatch.setenv("MGRIT_FCF_FOURIER", "1")
    else:
        monkeypatch.setenv("MGRIT_FCF_SHAPE", shape)
    nt = 512 if nx <= 1024 else 256
    c = schemes.cfl_number("ERK", p)
    u0 = workloads.fourier_field(nx)
    it, r, U, _ = oracle_run("ERK", p, c, nx, nt, m, L, "auto", u0)
    res, out, _ = gpu_run(capi, "ERK", p, c, nx, nt, m, L, "auto", u0, precision=1)
    assert res.fine_fourier == 1
    assert res.converged == 1 and abs(res.iterations - it) <= 1
    assert rel(out, U[::m]) <= 1e-9


def test_fourier_fcf_off_and_other_precisions(capi, monkeypatch):
    """MGRIT_FCF_FOURIER=0 keeps the stencil form; FP64 and MIXED_DF never
    take the Fourier form (their FP64 pass is the exact-cancellation value
    form, or float-float)."""
    nx, nt, m, L = 512, 512, 8, 2
    c = schemes.cfl_number("ERK", 3)
    u0 = workloads.fourier_field(nx)
    monkeypatch.setenv("MGRIT_FCF_FOURIER", "0")
    res, _, _ = gpu_run(capi, "ERK", 3, c, nx, nt, m, L, "auto", u0, precision=1)
    assert res.fine_fourier == 0
    monkeypatch.setenv("MGRIT_FCF_FOURIER", "1")
    for prec in (0, 2):
        res, _, _ = gpu_run(capi, "ERK", 3, c, nx, nt, m, L, "auto", u0, precision=prec)
        assert res.fine_fourier == 0


def test_fourier_fcf_relax_sweeps_match_stencil_form(capi, monkeypatch):
    """FCF sweeps without coarse correction from the paper's random iterate:
    the Fourier form's relative residuals after 1, 2, 3 and 7 sweeps equal
    the oracle's to the FP32 second pass (1e-6), as the stencil form's do."""
    fam, p, nx, nt, m = "ERK", 3, 256, 512, 4
    c = schemes.cfl_number(fam, p)
    st = stepping.FineStep(fam, p, c, nx)
    U = workloads.random_iterate(nt, nx, workloads.sin4(nx), 3)
    r0 = float(np.linalg.norm(omg.spacetime_residual(U, np.zeros_like(U), st)))
    got = {}
    for fourier in ("0", "1"):
        monkeypatch.setenv("MGRIT_FCF_FOURIER", fourier)
        opts = capi.mgrit_opts_default(m=m, levels=2, max_iter=0, precision=1)
        h = capi.mgrit_setup(capi.problem(nx, nt, fam, p, p, c), opts)
        try:
            res, status = capi.mgrit_solve_from(h, np.ascontiguousarray(U[::m]), r0, allow_not_converged=True)
            assert status == -4 and res.fine_fourier == int(fourier)
            got[fourier] = [capi.mgrit_relax(h, 1) for _ in range(3)] + [capi.mgrit_relax(h, 4)]
        finally:
            capi.mgrit_destroy(h)
    G = np.zeros_like(U)
    want = []
    for k in range(1 + 3 + 4):
        omg.f_relax(U, G, st, m)
        omg.c_relax(U, G, st, m)
        omg.f_relax(U, G, st, m)
        if 1 <= k <= 3 or k == 7:
            want.append(float(np.linalg.norm(omg.c_residual(U, G, st, m))) / r0)
    np.testing.assert_allclose(got["1"], want, rtol=1e-6)
    np.testing.assert_allclose(got["0"], want, rtol=1e-6)
