"""Inflow/outflow boundaries (Section 4.5) on the GPU against the oracle
(oracle/boundaries.py): single steps of Phi and of the truncated Psi,
sequential stepping, MGRIT parity (FP64 relative L2 <= 1e-12 and the same
iteration count) over cycles, relaxations and precisions, the server, and
Table 5's iteration counts from the paper's random initial iterate."""
import time

import numpy as np
import pytest

import workloads
from conftest import golden
from oracle import boundaries as bd
from oracle import mgrit as omg
from oracle import psi as opsi
from oracle import schemes

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


def sin4(nx):
    return np.sin(np.pi * bd.grid(nx)) ** 4


def prob(capi, p, nx, nt, c=None):
    c = schemes.cfl_number("ERK", p) if c is None else c
    return capi.problem(nx, nt, "ERK", p, p, c, boundary="inflow")


def oracle_levels(p, nx, nt, m, L, c=None):
    c = schemes.cfl_number("ERK", p) if c is None else c
    st = bd.InflowStep(p, c, nx)
    ops = opsi.build_hierarchy("ERK", p, c, nx, nt, m, L, rule="auto")
    return st, omg.make_levels(st, m, [bd.truncated(o.diag) for o in ops])


def gpu_solve(capi, p, nx, nt, m, L, u0, precision=0, output=1, cycle=0, relax=0, tol=1e-10):
    opts = capi.mgrit_opts_default(m=m, levels=L, precision=precision, output=output, tol=tol, cycle=cycle,
                                   relax=relax)
    h = capi.mgrit_setup(prob(capi, p, nx, nt), opts)
    try:
        rows = {0: 1, 1: nt // m + 1, 2: nt + 1}[output]
        out = np.zeros((rows, nx))
        res, _ = capi.mgrit_solve(h, np.ascontiguousarray(u0), out)
    finally:
        capi.mgrit_destroy(h)
    return res, out


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_fine_step_matches_stage_form(capi, p):
    """Phi with the closures, k steps, on a ragged nx: the circulant stencil
    plus the recomputed boundary rows equal the oracle's stage-wise step."""
    import torch
    nx, k, count = 200, 5, 3
    c = schemes.cfl_number("ERK", p)
    h = capi.mgrit_setup(prob(capi, p, nx, 8), capi.mgrit_opts_default(m=2, levels=2))
    try:
        x = np.random.default_rng(p).standard_normal((count, nx))
        xin = torch.tensor(x, device="cuda")
        yout = torch.zeros_like(xin)
        capi.mgrit_propagate(h, 1, k, count, xin, yout)
    finally:
        capi.mgrit_destroy(h)
    st = bd.InflowStep(p, c, nx)
    ref = x.copy()
    for _ in range(k):
        ref = st(ref)
    assert rel(yout.cpu().numpy(), ref) <= TOL


def test_coarse_step_is_truncated_psi(capi):
    """Psi_l (levels 2 and 3) applied k times on the GPU = the truncated
    Toeplitz Psi of the oracle, with the handle's own fitted taps."""
    import torch
    p, nx, nt, m, L, k = 3, 160, 256, 4, 3, 4
    h = capi.mgrit_setup(prob(capi, p, nx, nt), capi.mgrit_opts_default(m=m, levels=L))
    try:
        x = np.random.default_rng(7).standard_normal((2, nx))
        for lev in (2, 3):
            offs, cfs = capi.mgrit_psi_info(h, lev)
            xin = torch.tensor(x, device="cuda")
            yout = torch.zeros_like(xin)
            capi.mgrit_propagate(h, lev, k, 2, xin, yout)
            T = bd.truncated(dict(zip(offs, cfs)))
            ref = x.copy()
            for _ in range(k):
                ref = T(ref)
            assert rel(yout.cpu().numpy(), ref) <= TOL, lev
    finally:
        capi.mgrit_destroy(h)


@pytest.mark.parametrize("output", [0, 1, 2])
def test_sequential_stepping(capi, output):
    p, nx, nt, m = 3, 136, 320, 8
    c = schemes.cfl_number("ERK", p)
    u0 = sin4(nx)
    st = bd.InflowStep(p, c, nx)
    ref = [u0]
    for _ in range(nt):
        ref.append(st(ref[-1]))
    ref = np.array(ref)
    h = capi.mgrit_setup(prob(capi, p, nx, nt), capi.mgrit_opts_default(m=m, output=output))
    try:
        rows = {0: 1, 1: nt // m + 1, 2: nt + 1}[output]
        out = np.zeros((rows, nx))
        capi.mgrit_sequential(h, u0, out)
    finally:
        capi.mgrit_destroy(h)
    want = {0: ref[-1:], 1: ref[::m], 2: ref}[output]
    assert rel(out, want) <= TOL


CASES = [  # p, nx, nt, m, L, cycle, relax
    (3, 256, 1024, 4, 2, "V", "FCF"), (3, 256, 1024, 4, 3, "V", "FCF"), (3, 256, 1024, 4, 4, "F", "FCF"),
    (1, 200, 1600, 16, 2, "V", "FCF"), (5, 160, 512, 4, 3, "V", "FCF"), (2, 128, 512, 8, 2, "V", "F"),
    (4, 192, 768, 4, 3, "V", "F"),
    (1, 256, 4096, 4, 5, "V", "FCF"),  # level-5 Psi shifted by most of the domain: mostly zero rows
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "-".join(map(str, c)))
def test_mgrit_parity_fp64(capi, case):
    p, nx, nt, m, L, cycle, relax = case
    u0 = workloads.fourier_field(nx)
    st, lev = oracle_levels(p, nx, nt, m, L)
    U = omg.zero_iterate(u0, nt)
    it, _ = omg.solve(lev, U, tol=1e-10, cycle=cycle, relax=relax)
    res, out = gpu_solve(capi, p, nx, nt, m, L, u0, cycle=0 if cycle == "V" else 1, relax=0 if relax == "FCF" else 1)
    assert res.converged == 1
    assert res.iterations == it
    assert rel(out, U[::m]) <= TOL


@pytest.mark.parametrize("shape", ["98,256,1", "98,512,1", "8,256,1", "99,256,0", "98,256,0", "8,256,0", "0,128,0"])
@pytest.mark.parametrize("precision", [0, 1, 2])
def test_launch_shapes(capi, monkeypatch, shape, precision):
    """Every level-1 launch shape with the boundary rows: step by step (the
    rows of Phi after each step) or the collapsed Phi^m (the rows of Phi^m
    after each pass), in each precision; FP64 gives the oracle's iterations
    and C-points, the mixed modes FP64 sequential stepping's C-points."""
    monkeypatch.setenv("MGRIT_FCF_SHAPE", shape)
    p, nx, nt, m, L = 3, 256, 1024, 8, 3
    u0 = workloads.fourier_field(nx)
    st, lev = oracle_levels(p, nx, nt, m, L)
    U = omg.zero_iterate(u0, nt)
    it, _ = omg.solve(lev, U, tol=1e-10)
    res, out = gpu_solve(capi, p, nx, nt, m, L, u0, precision=precision)
    tile, th, col = (int(v) for v in shape.split(","))
    assert (res.fine_tile, res.fine_threads, res.fine_collapsed) == (tile, th, col)
    assert res.converged == 1
    if precision == 0:
        assert res.iterations == it
        assert rel(out, U[::m]) <= TOL
    else:
        ref = [u0]
        for _ in range(nt):
            ref.append(st(ref[-1]))
        assert abs(res.iterations - it) <= 1
        assert rel(out, np.array(ref)[::m]) <= 1e-9


def test_full_output_interpolates_with_the_closures(capi):
    p, nx, nt, m, L = 3, 144, 384, 4, 3
    u0 = sin4(nx)
    st, lev = oracle_levels(p, nx, nt, m, L)
    U = omg.zero_iterate(u0, nt)
    it, _ = omg.solve(lev, U, tol=1e-10)
    res, out = gpu_solve(capi, p, nx, nt, m, L, u0, output=2)
    assert res.iterations == it
    assert rel(out, U) <= TOL


@pytest.mark.parametrize("precision,L", [(1, 2), (1, 3), (2, 3)])
def test_mixed_modes_reach_sequential_stepping(capi, precision, L):
    """MIXED (FP32 second pass and coarse levels, FP32 boundary rows there)
    and MIXED_DF: the FP64 test is met and the C-points agree with FP64
    sequential stepping of the closed problem."""
    p, nx, nt, m = 3, 256, 2048, 4
    c = schemes.cfl_number("ERK", p)
    u0 = workloads.fourier_field(nx)
    st = bd.InflowStep(p, c, nx)
    ref = [u0]
    for _ in range(nt):
        ref.append(st(ref[-1]))
    ref = np.array(ref)
    it64 = gpu_solve(capi, p, nx, nt, m, L, u0)[0].iterations
    res, out = gpu_solve(capi, p, nx, nt, m, L, u0, precision=precision)
    assert res.converged == 1 and res.rel_residual <= 1e-10
    assert abs(res.iterations - it64) <= 1
    assert rel(out, ref[::m]) <= 1e-9


def test_server_inflow_requests_match_single_solves(capi, monkeypatch):
    """Periodic and inflow/outflow requests in one server: each result equals
    its single solve (the batched FCF launch carries each solve's boundary
    rows; here every coarsest level marches, in the server and alone)."""
    monkeypatch.setenv("MGRIT_COARSE", "march")
    nx, nt, m = 256, 1024, 4
    reqs = [("inflow", 3, 2), ("periodic", 3, 2), ("inflow", 3, 3), ("inflow", 5, 2)]
    singles = []
    for bc, p, L in reqs:
        c = schemes.cfl_number("ERK", p)
        u0 = workloads.fourier_field(nx, seed=p + L)
        opts = capi.mgrit_opts_default(m=m, levels=L)
        h = capi.mgrit_setup(capi.problem(nx, nt, "ERK", p, p, c, boundary=bc), opts)
        try:
            out = np.zeros((nt // m + 1, nx))
            res, _ = capi.mgrit_solve(h, u0, out)
        finally:
            capi.mgrit_destroy(h)
        singles.append((res.iterations, out, u0, opts, capi.problem(nx, nt, "ERK", p, p, c, boundary=bc)))
    srv = capi.mgrit_server_create(4e9)
    try:
        tickets = [capi.mgrit_submit(srv, pr, o, u0) for (_, _, u0, o, pr) in singles]
        for t, (it, out, *_rest) in zip(tickets, singles):
            got = np.zeros_like(out)
            t0 = time.time()
            while True:
                st, res = capi.mgrit_poll(srv, t, got)
                if st != capi.MGRIT_PENDING:
                    break
                assert time.time() - t0 < 120.0, "request did not finish"
                time.sleep(0.002)
            assert st == 0 and res.iterations == it
            assert rel(got, out) <= 1e-14
    finally:
        capi.mgrit_server_destroy(srv)


def test_rejections(capi):
    for (nx, p) in [(40, 5), (16, 3)]:
        with pytest.raises(capi.MgritError) as ei:
            capi.mgrit_setup(prob(capi, p, nx, 64), capi.mgrit_opts_default(m=4))
        assert ei.value.status == -10
    with pytest.raises(capi.MgritError) as ei:
        capi.mgrit_setup(capi.problem(128, 64, "SDIRK", 2, 2, 2.0, boundary="inflow"),
                         capi.mgrit_opts_default(m=4))
    assert ei.value.status == -10


def _table5(nx_rows):
    rows = []
    for r in golden("table5_inflow.txt"):
        p, nx, nt = int(r[0]), int(r[1]), int(r[2])
        if nx not in nx_rows:
            continue
        two = dict(zip((2, 4, 8, 16, 32, 64), (int(v) for v in r[3:9])))
        multi = {L: int(v) for L, v in zip(range(2, 8), r[9:15]) if v != "-"}
        rows.append((p, nx, nt, two, multi))
    return rows


@pytest.mark.parametrize("row", _table5((256, 1024)), ids=lambda r: f"ERK{r[0]}-{r[1]}")
def test_table5(capi, row):
    """Table 5 from the paper's random initial iterate: two-level counts per m
    and V-cycle counts (m = 4) per number of levels within one of the printed
    ones on the 2^8 grids and within two on the 2^10 grids (the paper's
    patterns for Table 5 are not printed; the auto-width rule's Psi needs up
    to two fewer iterations at m = 16, 32 for ERK1 there, and the oracle's
    counts on the same iterate differ from the printed ones by the same
    amounts), ERK1 with m = 2 excepted (the width rule takes all of Phi^2
    there: one iteration).  On the 2^8 grids the GPU's counts equal the
    oracle's on the same iterate."""
    p, nx, nt, two, multi = row
    slack = 1 if nx == 256 else 2
    c = schemes.cfl_number("ERK", p)
    st = bd.InflowStep(p, c, nx)
    U = workloads.random_iterate(nt, nx, sin4(nx), 1)
    r0 = float(np.linalg.norm(omg.spacetime_residual(U, np.zeros_like(U), st)))
    pr = prob(capi, p, nx, nt, c)

    def run(m, L):
        h = capi.mgrit_setup(pr, capi.mgrit_opts_default(m=m, levels=L, min_coarse=2))
        try:
            res, _ = capi.mgrit_solve_from(h, np.ascontiguousarray(U[::m]), r0)
        finally:
            capi.mgrit_destroy(h)
        return res

    for m, v in two.items():
        res = run(m, 2)
        assert res.converged == 1
        if not (p == 1 and m == 2):
            assert abs(res.iterations - v) <= slack, (m, res.iterations, v)
        if nx == 256:
            ops = opsi.build_hierarchy("ERK", p, c, nx, nt, m, 2, rule="auto")
            it, _ = omg.solve(omg.make_levels(st, m, [bd.truncated(ops[0].diag)]), U.copy())
            assert res.iterations == it, (m, res.iterations, it)
    for L, v in multi.items():
        res = run(4, L)
        assert res.converged == 1 and abs(res.iterations - v) <= slack, (L, res.iterations, v)
        if nx == 256:
            ops = opsi.build_hierarchy("ERK", p, c, nx, nt, 4, L, rule="auto")
            it, _ = omg.solve(omg.make_levels(st, 4, [bd.truncated(o.diag) for o in ops]), U.copy())
            assert res.iterations == it, (L, res.iterations, it)
