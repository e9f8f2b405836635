"""Pins of the oracle's coarse-operator construction (Section 4, Eq. 4-6,
Remark 1, Lemma 2, Figures 3-4)."""
import numpy as np
import pytest

from oracle import psi, schemes, stepping


@pytest.mark.parametrize("fam,p,m", [("ERK", 1, 8), ("ERK", 3, 4), ("ERK", 5, 16), ("SDIRK", 2, 8), ("SDIRK", 3, 16)])
def test_phi_m_column_stepping_equals_inverse_dft(fam, p, m):
    nx = 128
    c = schemes.cfl_number(fam, p)
    st = stepping.FineStep(fam, p, c, nx)
    lam = schemes.phi_symbol(fam, p, c, nx)
    a = psi.phi_m_column_by_stepping(st, nx, m)
    b = psi.phi_m_column_by_symbol(lam, m)
    np.testing.assert_allclose(a, b, atol=1e-13)


def test_erk_phi_nnz_matches_corollary1():
    """Corollary 1: ERK Phi is one circulant stencil with s(w-1)+1 diagonals."""
    w = {1: 2, 2: 3, 3: 4, 4: 5, 5: 6}
    s = {1: 1, 2: 2, 3: 3, 4: 4, 5: 6}
    for p in range(1, 6):
        st = stepping.FineStep("ERK", p, schemes.cfl_number("ERK", p), 64)
        assert len(psi.phi_m_column_nonzeros(st, 64)) == s[p] * (w[p] - 1) + 1


@pytest.mark.parametrize("fam,p,m", [("ERK", 1, 16), ("ERK", 3, 16), ("ERK", 5, 64), ("SDIRK", 3, 16)])
def test_phi_m_peaks_at_characteristic_departure_point(fam, p, m):
    """Figures 3-4 and 7: the largest entries of Phi^m sit near diagonal -m c
    (within the phase lag of the scheme: 5% of m c)."""
    nx = 512
    c = schemes.cfl_number(fam, p)
    col = psi.phi_m_column_by_symbol(schemes.phi_symbol(fam, p, c, nx), m)
    assert abs(psi.argmax_offset(col) + m * c) <= max(1.5, 0.05 * m * c)


def test_unit_weight_gives_truncation():
    """Remark 1: with W = I the fit is the restriction of phi~^m."""
    nx, m = 128, 8
    c = schemes.cfl_number("ERK", 3)
    lam = schemes.phi_symbol("ERK", 3, c, nx)
    col = psi.phi_m_column_by_symbol(lam, m)
    offs = psi.best_window(col, 9)
    d, imag = psi.lsq_fit(lam, np.fft.fft(col), offs, unit_weight=True)
    diag_all = psi.column_to_diagonals(col)
    for i in offs:
        assert abs(d[i] - diag_all[i]) < 1e-13
    assert imag < 1e-12


@pytest.mark.parametrize("fam,p,m,rule", [("ERK", 1, 8, "halfwidth"), ("ERK", 3, 8, "auto"),
                                           ("ERK", 5, 4, "auto"), ("SDIRK", 3, 16, "threshold"),
                                           ("SDIRK", 1, 4, "threshold")])
def test_fit_is_real_and_matches_the_constant_mode(fam, p, m, rule):
    """Lemma 2 (real solution, imaginary part below the 1e-8 flag); the weight
    w(1) = 1e12 pins mu(0) to lambda(0)^m = 1, and the fit beats the truncation
    of Phi^m to the same pattern in the weighted norm (it is the minimiser)."""
    nx = 256
    nt = 8 * nx
    ops = psi.build_hierarchy(fam, p, schemes.cfl_number(fam, p), nx, nt, m, 2, rule=rule)
    op = ops[0]
    assert op.imag <= psi.IMAG_FLAG
    assert abs(op.mu[0] - 1.0) < 1e-5
    assert np.max(np.abs(op.mu)) <= 1.0 + 1e-9
    c = schemes.cfl_number(fam, p)
    lam = schemes.phi_symbol(fam, p, c, nx)
    sw = np.sqrt(psi.weights(lam))
    col = psi.phi_m_column_by_symbol(lam, m)
    trunc = {i: psi.column_to_diagonals(col)[i] for i in op.offsets}
    r_fit = np.linalg.norm(sw * (lam ** m - op.mu))
    r_trunc = np.linalg.norm(sw * (lam ** m - psi.symbol(trunc, nx)))
    assert r_fit <= r_trunc * (1 + 1e-9)


def test_halfwidth_pattern_erk1_m8():
    """ERK1+U1, c = 0.85, m = 8: Phi^8 has binomial entries C(8,k) c^k (1-c)^(8-k)
    on diagonal -k, largest at k = 7, so half-width 3 gives offsets -10..-4."""
    nx = 64
    st = stepping.FineStep("ERK", 1, 0.85, nx)
    col = psi.phi_m_column_by_stepping(st, nx, 8)
    from math import comb
    d = psi.column_to_diagonals(col)
    for k in range(9):
        assert abs(d[-k] - comb(8, k) * 0.85 ** k * 0.15 ** (8 - k)) < 1e-15
    assert psi.halfwidth_pattern(col, 3) == list(range(-10, -3))


def test_bound_is_zero_for_ideal_and_operator_complexity():
    nx, m = 64, 4
    c = schemes.cfl_number("ERK", 2)
    lam = schemes.phi_symbol("ERK", 2, c, nx)
    assert np.max(psi.two_level_bound(lam, lam ** m, m, 256)) < 1e-13
    # Eq. 5 with nnz(Psi) = nnz(Phi) on every level gives 1 + 1/m (+ ...)
    assert abs(psi.operator_complexity([5, 5], 4) - 1.25) < 1e-15
    assert abs(psi.operator_complexity([5] * 30, 4) - 4.0 / 3.0) < 1e-12


def test_bound_matches_geometric_sum_form():
    """Eq. 4's last factor (1 - |mu|^{N-1})/(1 - |mu|) is the geometric sum."""
    lam = np.array([0.9 + 0.1j, 0.5j])
    mu = np.array([0.8, 0.3 + 0.1j])
    m, nt = 4, 40
    N = nt // m
    b = psi.two_level_bound(lam, mu, m, nt)
    ref = [np.sqrt(m) * abs(l) ** m * abs(l ** m - u) * sum(abs(u) ** i for i in range(N - 1))
           for l, u in zip(lam, mu)]
    np.testing.assert_allclose(b, ref, rtol=1e-14)
