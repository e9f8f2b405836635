"""Pins of the oracle's discretisation against what the paper fixes
(Section 2.1, Lemma 1, Table 1, Appendix A)."""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

from conftest import golden
from oracle import schemes, stepping


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_upwind_exact_on_polynomials(p):
    """U_p differentiates x^q exactly for q <= p and not for q = p + 1."""
    s, a = schemes.UPWIND[p]
    dx = Fr(1, 7)
    x0 = Fr(3, 5)
    for q in range(0, p + 2):
        approx = sum(Fr(ak) * (x0 + k * dx) ** q for k, ak in a.items()) / (s * dx)
        exact = q * x0 ** (q - 1) if q > 0 else 0
        if q <= p:
            assert approx == exact, (p, q)
        else:
            assert approx != exact, (p, q)


def test_upwind_stencils_are_upwind_biased():
    """Wave speed > 0: every stencil reaches further upwind (k < 0) than downwind."""
    for p, (s, a) in schemes.UPWIND.items():
        assert min(a) < 0 and max(a) <= min(-min(a), 2)
        assert sum(a.values()) == 0          # annihilates constants


ABSC = {("ERK", p): schemes.ERK_ABSCISSAE[p] for p in range(1, 6)}
ABSC.update({("SDIRK", p): schemes.SDIRK_ABSCISSAE[p] for p in range(1, 5)})


@pytest.mark.parametrize("fam,p", sorted(ABSC))
def test_tableau_row_sums_equal_printed_abscissae(fam, p):
    A, b = schemes.tableau(fam, p)
    np.testing.assert_allclose(A.sum(axis=1), ABSC[(fam, p)], rtol=0, atol=1e-15)
    assert abs(b.sum() - 1.0) < 1e-15
    if fam == "SDIRK":
        d = np.diag(A)
        assert np.all(d == d[0])                       # singly diagonal
        np.testing.assert_array_equal(A[-1], b)        # stiffly accurate


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_erk_linear_order_conditions_exact(p):
    """b^T A^{k-1} 1 = 1/k! for k <= p (R(z) = e^z + O(z^{p+1})), exact rationals."""
    A, b = schemes.erk_tableau_exact(p)
    s = len(b)
    v = [Fr(1)] * s
    for k in range(1, p + 1):
        coef = sum(bi * vi for bi, vi in zip(b, v))
        assert coef == Fr(1, math.factorial(k)), (p, k)
        v = [sum(A[i][j] * v[j] for j in range(s)) for i in range(s)]


@pytest.mark.parametrize("fam,p", [("ERK", q) for q in range(1, 6)] + [("SDIRK", q) for q in range(1, 5)])
def test_stability_function_order(fam, p):
    """|R(z) - e^z| scales like |z|^{p+1} for small z."""
    z1, z2 = 2e-2, 1e-2
    e1 = abs(schemes.stability(fam, p, -z1)[0] - math.exp(-z1))
    e2 = abs(schemes.stability(fam, p, -z2)[0] - math.exp(-z2))
    slope = math.log(e1 / e2) / math.log(z1 / z2)
    assert abs(slope - (p + 1)) < 0.15, slope


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_sdirk_is_l_stable(p):
    """L-stability (Section 2.1): |R| <= 1 on the left half-plane and R(-inf) = 0."""
    assert abs(schemes.stability("SDIRK", p, -1e9)[0]) < 1e-7
    y = np.linspace(-50, 50, 2001)
    for x in (0.0, -0.5, -5.0):
        assert np.max(np.abs(schemes.stability("SDIRK", p, x + 1j * y))) <= 1.0 + 1e-12


def test_sdirk3_zeta_root_of_cubic():
    """zeta of Appendix A is the root in (0, 1) of x^3 - 3x^2 + 3x/2 - 1/6."""
    z = schemes.SDIRK3_ZETA
    assert abs(z ** 3 - 3 * z ** 2 + 1.5 * z - 1.0 / 6.0) < 1e-16
    roots = np.roots([1, -3, 1.5, -1.0 / 6.0])
    real = sorted(r.real for r in roots if abs(r.imag) < 1e-12)
    assert any(abs(r - z) < 1e-14 for r in real)


def test_table1_cfl_limits():
    """Table 1.  ERK1..3 hold with |R| <= 1 strictly; ERK4 and ERK5 exceed 1
    by less than 1e-6 at low frequencies below their printed limit, so the
    printed values are the limits for |R| <= 1 + 1e-6 (a reading)."""
    for p, cmax in ((int(r[0]), float(r[1])) for r in golden("table1_cfl_limits.txt")):
        digits = 5 if cmax not in (1.0, 0.5) else 9
        c = schemes.erk_cfl_limit(p, slack=1e-6 if p >= 4 else 0.0, ntheta=2048)
        assert abs(c - cmax) < 0.6 * 10.0 ** (-digits) * max(1.0, cmax) + 1e-6, (p, c, cmax)


@pytest.mark.parametrize("fam,p", [("ERK", 3), ("ERK", 5), ("SDIRK", 3), ("SDIRK", 4)])
def test_fourier_mode_multiplied_by_symbol(fam, p):
    """Lemma 1: Phi acts on exp(i j theta) as multiplication by R(z(theta))."""
    nx = 64
    c = schemes.cfl_number(fam, p)
    step = stepping.FineStep(fam, p, c, nx)
    lam = schemes.phi_symbol(fam, p, c, nx)
    j = np.arange(nx)
    for k in (0, 1, 5, 17, 32, 40):
        th = 2 * np.pi * k / nx
        out = step(np.cos(th * j)) + 1j * step(np.sin(th * j))
        np.testing.assert_allclose(out, lam[k] * np.exp(1j * th * j), atol=1e-13)
