"""Pins of the oracle's time stepping (Section 2.1, Eq. 3, Figure 1)."""
import numpy as np
import pytest

import workloads
from oracle import schemes, stepping


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_sdirk_stage_solve_residual(p):
    nx = 256
    st = stepping.FineStep("SDIRK", p, 4.0, nx)
    rng = np.random.default_rng(0)
    rhs = rng.standard_normal((3, nx))
    a = st.A[0, 0]
    K = st.stage_solve(a, rhs)
    res = K - a * st.dtL(K) - rhs
    assert np.max(np.abs(res)) < 1e-13 * np.max(np.abs(rhs))


def test_erk1_u1_is_the_printed_two_point_update():
    """ERK1+U1: u_i <- (1 - c) u_i + c u_{i-1} (Euler + first-order upwind)."""
    nx, c = 32, 0.85
    u = np.random.default_rng(1).standard_normal(nx)
    got = stepping.FineStep("ERK", 1, c, nx)(u)
    np.testing.assert_allclose(got, (1 - c) * u + c * np.roll(u, 1), rtol=0, atol=1e-15)


@pytest.mark.parametrize("fam,p", [("ERK", 2), ("SDIRK", 3)])
def test_linear_and_shift_equivariant(fam, p):
    nx = 64
    st = stepping.FineStep(fam, p, schemes.cfl_number(fam, p), nx)
    rng = np.random.default_rng(2)
    u, v = rng.standard_normal(nx), rng.standard_normal(nx)
    np.testing.assert_allclose(st(2.0 * u - 3.0 * v), 2.0 * st(u) - 3.0 * st(v), atol=1e-13)
    np.testing.assert_allclose(st(np.roll(u, 5)), np.roll(st(u), 5), atol=1e-13)


def _sin4(x):
    return np.sin(np.pi * x) ** 4


@pytest.mark.parametrize("fam,p", [("ERK", 1), ("ERK", 2), ("ERK", 3), ("ERK", 4), ("ERK", 5),
                                   ("SDIRK", 2), ("SDIRK", 3), ("SDIRK", 4)])
def test_order_of_accuracy(fam, p):
    """Figure 1: the space-time error against u0(x - t) falls at order p under
    refinement at fixed CFL number (discrete L2 norm, final time T)."""
    c = schemes.cfl_number(fam, p)
    base = 128 if fam == "ERK" else 256
    T = 1.0 if fam == "ERK" else 2.0
    errs = []
    for nx in (base, 2 * base):
        dx = 2.0 / nx
        nt = int(round(T / (c * dx)))
        dt = T / nt                      # land exactly on T
        cc = dt / dx
        st = stepping.FineStep(fam, p, cc, nx)
        u = stepping.sequential(st, workloads.sin4(nx), nt, keep_all=False)
        ex = stepping.exact_solution(_sin4, nx, T)
        errs.append(np.sqrt(dx) * np.linalg.norm(u - ex))
    rate = np.log2(errs[0] / errs[1])
    assert rate > p - 0.35, (errs, rate)
