"""C-ABI checks that need no GPU: the library loads, exports every entry point
declared in include/mgrit.h, validates its inputs, and its host-side FP64 setup
(collapsed ERK propagator, Corollary 1; least-squares Psi, Eq. 6) agrees with
the oracle's."""
import os
import re

import numpy as np
import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def capi():
    from paper_1910_03726_gb300 import build
    build.build()
    from paper_1910_03726_gb300 import capi as c
    return c


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mgrit.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mgrit_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_entry_point(capi):
    names = declared_functions()
    assert "mgrit_setup" in names and "mgrit_poll" in names
    missing = [n for n in names if not hasattr(capi._lib, n)]
    assert not missing, missing
    assert capi.mgrit_abi_version() == 6


def test_struct_layouts_match_the_header(capi):
    """mgrit_opts_default writes every field of the C struct: the binding's
    fields after the ones added in ABI 5 (init_guess, seed) read back the
    documented defaults only if both sides agree on the layout."""
    o = capi.mgrit_opts_default()
    assert (o.m, o.levels, o.max_iter, o.psi_halfwidth, o.min_coarse) == (8, 2, 100, 3, 2)
    assert (o.init_guess, o.seed, o.tol, o.psi_rho) == (0, 0, 1e-10, 0.15)
    assert not o.psi_user_nnz and not o.psi_user_offsets and not o.psi_user_coeffs
    import ctypes as C
    assert C.sizeof(capi.MgritProblem) == 56 and C.sizeof(capi.MgritOpts) == 104
    assert C.sizeof(capi.MgritServerStats) == 17 * 8   # ABI 6: fft_coarse_solves last


@pytest.mark.parametrize("alpha,xmin,xmax,status", [(-1.0, -1.0, 1.0, -10), (1.0, 1.0, -1.0, -1),
                                                     (float("nan"), -1.0, 1.0, -1), (0.0, 0.0, 0.0, 0),
                                                     (2.5, 0.0, 10.0, 0)])
def test_problem_validation_of_wave_speed_and_domain(capi, alpha, xmin, xmax, status):
    """Eq. 1's alpha and domain: U_p is upwind for alpha > 0 (a left-moving
    wave is unsupported), xmin < xmax, and zeros select alpha = 1 on [-1, 1]."""
    prob = capi.problem(64, 64, "ERK", 1, 1, 0.85, alpha=alpha, xmin=xmin, xmax=xmax)
    import ctypes as C
    n = C.c_int32()
    offs = (C.c_int32 * 16)()
    cfs = (C.c_double * 16)()
    assert capi._lib.mgrit_phi_taps(C.byref(prob), 16, C.byref(n), offs, cfs) == status


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_phi_taps_match_oracle_first_column(capi, p):
    from oracle import psi, schemes, stepping
    c = schemes.cfl_number("ERK", p)
    offs, cfs = capi.mgrit_phi_taps(capi.problem(64, 64, "ERK", p, p, c))
    col = psi.phi_m_column_by_stepping(stepping.FineStep("ERK", p, c, 64), 64, 1)
    d = psi.column_to_diagonals(col)
    assert sorted(offs) == sorted(i for i, v in d.items() if v != 0.0)
    for o, v in zip(offs, cfs):
        assert abs(v - d[o]) <= 4e-16 * max(1.0, abs(d[o]))


CASES = [("ERK", 1, 64, 1024, 8, 2, "halfwidth"), ("ERK", 3, 256, 512, 8, 2, "auto"),
         ("ERK", 3, 256, 512, 4, 4, "auto"), ("ERK", 5, 256, 512, 4, 3, "auto"),
         ("ERK", 2, 128, 2048, 16, 2, "auto"), ("SDIRK", 3, 256, 256, 16, 2, "threshold"),
         ("SDIRK", 1, 256, 256, 4, 2, "threshold"), ("ERK", 2, 64, 256, 4, 2, "ideal")]


@pytest.mark.parametrize("case", CASES)
def test_psi_plan_matches_oracle(capi, case):
    """Same sparsity pattern (bit-exact integers) and coefficients within 1e-9
    relative: the two sides solve Eq. 6 by different factorisations (LAPACK
    SVD least squares vs. Householder QR) of a problem whose row weights span
    12 orders of magnitude."""
    from oracle import psi, schemes
    fam, p, nx, nt, m, L, rule = case
    c = schemes.cfl_number(fam, p)
    rules = {"halfwidth": capi.PSI_HALFWIDTH, "auto": capi.PSI_AUTO, "threshold": capi.PSI_THRESHOLD,
             "ideal": capi.PSI_IDEAL}
    opts = capi.mgrit_opts_default(m=m, levels=L, psi_rule=rules[rule], psi_halfwidth=3)
    got, diag = capi.mgrit_psi_plan(capi.problem(nx, nt, fam, p, p, c), opts)
    ref = psi.build_hierarchy(fam, p, c, nx, nt, m, L, rule=rule, halfwidth=3)
    assert len(got) == len(ref)
    for (offs, cfs), op in zip(got, ref):
        assert offs == op.offsets
        ref_c = np.array([op.diag[i] for i in offs])
        err = np.max(np.abs(np.array(cfs) - ref_c)) / np.max(np.abs(ref_c))
        assert err < 1e-9, err
    for (im, bound, mumax), op in zip(diag, ref):
        assert im <= 1e-8
        if rule != "ideal":
            assert abs(bound - op.bound_max) <= 1e-6 * max(1.0, op.bound_max)


def test_setup_rejects_invalid_requests_before_touching_the_gpu(capi):
    opts = capi.mgrit_opts_default(m=8, levels=2)
    bad = [
        (capi.problem(64, 1024, "ERK", 1, 1, 1.2), opts, -2),            # CFL above Table 1
        (capi.problem(64, 1020, "ERK", 1, 1, 0.85), opts, -1),           # nt % m != 0
        (capi.problem(4, 1024, "ERK", 1, 1, 0.85), opts, -1),            # nx too small
        (capi.problem(64, 1024, "ERK", 6, 6, 0.85), opts, -1),           # no ERK6
        (capi.problem(64, 64, "ERK", 1, 1, 0.85), capi.mgrit_opts_default(m=8, levels=3), -1),
    ]
    for prob, o, code in bad:
        with pytest.raises(capi.MgritError) as ei:
            capi.mgrit_setup(prob, o)
        assert ei.value.status == code
        assert capi.mgrit_last_error()


def test_server_host_side_without_gpu(capi):
    """Admission control and ticket bookkeeping run on the host: an oversize
    request is refused at submit, an unknown ticket is reported, and the server
    shuts down cleanly (no GPU work is needed for any of this)."""
    import workloads
    srv = capi.mgrit_server_create(1e6)
    try:
        prob = capi.problem(1024, 4096, "ERK", 1, 1, 0.85)
        with pytest.raises(capi.MgritError) as ei:
            capi.mgrit_submit(srv, prob, capi.mgrit_opts_default(m=4), workloads.sin4(1024))
        assert ei.value.status == -6
        st, _ = capi.mgrit_poll(srv, 12345)
        assert st == -11
        with pytest.raises(capi.MgritError) as ei:
            capi.mgrit_submit(srv, capi.problem(64, 1020, "ERK", 1, 1, 0.85), capi.mgrit_opts_default(m=8),
                              workloads.sin4(64))
        assert ei.value.status == -1
    finally:
        capi.mgrit_server_destroy(srv)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_phi_boundary_rows_match_oracle(capi, p):
    """Inflow/outflow Phi (Section 4.5): the library's boundary rows equal the
    oracle's stage-wise Phi with the same closures, and every other row is the
    interior stencil of mgrit_phi_taps."""
    from oracle import boundaries as bd
    from oracle import schemes
    nx = 96
    c = schemes.cfl_number("ERK", p)
    prob = capi.problem(nx, 64, "ERK", p, p, c, boundary="inflow")
    left, right = capi.mgrit_phi_boundary(prob)
    P = bd.dense_phi(bd.InflowStep(p, c, nx))
    nl, cl = left.shape
    nr, cr = right.shape
    assert nl > 0 and (nr > 0) == (max(schemes.dtL_taps(p, c)) > 0)  # outflow ghosts only if the stencil reaches right
    # same stage-wise arithmetic, other summation orders
    assert np.max(np.abs(left - P[:nl, :cl])) < 2e-14
    assert np.all(np.abs(right - P[nx - nr:, nx - cr:]) < 2e-14)
    # outside the blocks the boundary rows are zero
    assert np.all(P[:nl, cl:] == 0.0) and np.all(P[nx - nr:, : nx - cr] == 0.0)
    offs, cfs = capi.mgrit_phi_taps(prob)
    Q = np.zeros((nx, nx))
    for r in range(nl, nx - nr):
        for o, v in zip(offs, cfs):
            Q[r, r + o] += v
    assert np.max(np.abs(Q[nl: nx - nr] - P[nl: nx - nr])) < 1e-14


def test_inflow_validation(capi):
    prob = capi.problem(96, 64, "SDIRK", 2, 2, 1.0, boundary="inflow")
    ok = capi.problem(96, 64, "ERK", 3, 3, 1.0, boundary="inflow")
    assert capi._lib.mgrit_phi_boundary(capi.C.byref(prob), 1, 0, None, None) == -10  # ERK only
    small = capi.problem(40, 64, "ERK", 5, 5, 1.5, boundary="inflow")
    assert capi._lib.mgrit_phi_boundary(capi.C.byref(small), 1, 0, None, None) == -10  # ends too close
    bad = capi.problem(96, 64, "ERK", 3, 3, 1.0)
    bad.boundary = 7
    assert capi._lib.mgrit_phi_boundary(capi.C.byref(bad), 1, 0, None, None) == -1
    opts = capi.mgrit_opts_default(m=4, levels=2, psi_rule=capi.PSI_IDEAL)
    L = 1
    nnz = (capi.C.c_int32 * L)()
    assert capi._lib.mgrit_psi_plan(capi.C.byref(ok), capi.C.byref(opts), 0, nnz, None, None, None) == -10


@pytest.mark.parametrize("p,m,nx", [(1, 16, 700), (3, 4, 700), (3, 8, 160), (5, 4, 900)])
def test_phi_power_boundary_rows_match_oracle(capi, p, m, nx):
    """Boundary rows of Phi^m (the collapsed path's): the oracle's dense
    stage-wise Phi to the m-th power on the whole domain, also where the
    library builds them on a shorter domain (nx = 700, 900)."""
    from oracle import boundaries as bd
    from oracle import schemes
    c = schemes.cfl_number("ERK", p)
    left, right = capi.mgrit_phi_boundary(capi.problem(nx, 64, "ERK", p, p, c, boundary="inflow"), m)
    Pm = np.linalg.matrix_power(bd.dense_phi(bd.InflowStep(p, c, nx)), m)
    nl, cl = left.shape
    nr, cr = right.shape
    s = {1: 1, 2: 2, 3: 3, 4: 4, 5: 6}[p]
    lo, hi = min(schemes.dtL_taps(p, c)), max(schemes.dtL_taps(p, c))
    assert (nl, nr) == (m * s * -lo, m * s * hi)
    assert np.max(np.abs(left - Pm[:nl, :cl])) < 1e-13
    assert np.all(np.abs(right - Pm[nx - nr:, nx - cr:]) < 1e-13)
    assert np.all(Pm[:nl, cl:] == 0.0) and np.all(Pm[nx - nr:, : nx - cr] == 0.0)


def test_static_entry_point_checks_the_shared_memory_bound(capi):
    """The FCF keeps two padded FP64 slabs (nx + nx/8 + 1 values each) in one
    CTA's 227 KiB of shared memory, beside up to 12 KiB of static shared memory
    (the server's batched FCF copies its stencil there), so nx <= 12231; the
    check runs before any device call (null buffers are rejected next, still
    on the host)."""
    import ctypes as C
    offs = (C.c_int32 * 2)(0, -1)
    cfs = (C.c_double * 2)(0.15, 0.85)
    lib = capi._lib
    st = lib.mgrit_fcf_residual_static(None, None, None, None, 12232, 4, 8, 2, offs, cfs, 0, None)
    assert st == -1 and "8..12231" in capi.mgrit_last_error()
    st = lib.mgrit_fcf_residual_static(None, None, None, None, 12231, 4, 8, 2, offs, cfs, 0, None)
    assert st == -1 and "device pointers" in capi.mgrit_last_error()
