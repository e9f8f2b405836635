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


@pytest.mark.parametrize("fam,p,q,m", [("SDIRK", 3, 5, 16), ("SDIRK", 1, 5, 4), ("ERK", 2, 4, 8)])
def test_phi_m_column_with_another_upwind_order(fam, p, q, m):
    """Lemma 1 with U_q in place of U_p: stepping and the inverse DFT of
    R(z)^m built from U_q's symbol give the same first column of Phi^m."""
    nx = 256
    c = 4.0 if fam == "SDIRK" else 0.5 * schemes.cfl_number("ERK", p)
    st = stepping.FineStep(fam, p, c, nx, q=q)
    lam = schemes.phi_symbol(fam, p, c, nx, q=q)
    np.testing.assert_allclose(psi.phi_m_column_by_stepping(st, nx, m), psi.phi_m_column_by_symbol(lam, m),
                               atol=1e-13)
    assert not np.allclose(lam, schemes.phi_symbol(fam, p, c, nx))


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


# ---------------------------------------------------------------------------
# Eq. 4 against the two-level error propagator of the oracle's own iteration
# ---------------------------------------------------------------------------
#
# Section 3.1: Phi and Psi are circulant, so one MGRIT iteration acts on each
# Fourier mode k separately; E_k is that action on the space-time error of the
# mode, ||E||_2 = max_k ||E_k||_2, Eq. 4 bounds ||E_k||_2 from above, and the
# bound is sharp up to O(m/n_t).  Below, E_k is formed column by column by
# running one two-level FCF iteration of the oracle (oracle.mgrit.vcycle on a
# homogeneous error with u^0 fixed) on unit errors at x = 0 and transforming
# the result in x.  Three facts of the mathematics then pin the bound:
#
#  * identity: the C-point block of E_k is lambda^m (lambda^m - mu) times a
#    lower-triangular Toeplitz matrix of powers of mu, so its induced l1 norm
#    (largest column sum of moduli) times sqrt(m) is Eq. 4's right-hand side
#    exactly.  The paper's coarse system counts the initial C-point as an
#    unknown; the oracle keeps u^0 fixed, so the oracle's problem with
#    n_t + m steps has the unknown C-points of the paper's at n_t.  This fixes
#    the factor |lambda|^m, the difference |lambda^m - mu| and the exponent
#    n_t/m - 1 of the last factor;
#  * upper bound: ||E_k||_2 <= bound_k for every mode of the paper's schemes
#    with their least-squares Psi (a dropped sqrt(m) fails here);
#  * sharpness: ideal interpolation puts |lambda|^i e_j on the F-points of
#    interval j, so the F-points multiply the norm by sqrt(s_k),
#    s_k = sum_{i<m} |lambda_k|^{2i} <= m; with that factor the bound is
#    attained as n_t/m grows: 1 <= sqrt(s_k/m) bound_k / ||E_k||_2 <= 1 + 2 m/n_t
#    at n_t/m = 256 (a |lambda| in place of |lambda|^m fails here).

from oracle import mgrit as omg  # noqa: E402


def mode_propagators(phi_diag, psi_diag, nx, m, nt):
    """E_k (n_t x n_t, complex) for every mode k, from one oracle iteration per
    unit error (batched along a middle axis: the oracle acts on the last)."""
    levels = omg.make_levels(omg.stencil_step(phi_diag), m, [psi_diag])
    U = np.zeros((nt + 1, nt, nx))
    for n in range(1, nt + 1):
        U[n, n - 1, 0] = 1.0
    omg.vcycle(levels, 0, U, np.zeros_like(U))
    return np.transpose(np.fft.fft(U[1:], axis=-1), (2, 0, 1))


def synthetic_circulant(nx, values):
    """Real circulant whose symbol takes the given values on modes k (and
    their conjugates on -k): first column = inverse DFT of the symbol."""
    sym = np.zeros(nx, complex)
    for k, v in values.items():
        sym[k] = v
        sym[(-k) % nx] = np.conj(v)
    assert np.allclose(sym[0].imag, 0) and (nx % 2 or abs(sym[nx // 2].imag) < 1e-15)
    d = psi.column_to_diagonals(np.real(np.fft.ifft(sym)))
    return d, psi.symbol(d, nx)


SYNTH_LAM = {0: 1.0, 1: (1 - 1e-9) * np.exp(0.3j), 2: 0.9 * np.exp(1.0j), 3: 0.6 * np.exp(2.0j), 4: 0.5}


def synth_mu(m):
    return {0: 1.0, 1: 0.8 * np.exp(0.3j * m + 0.05j), 2: 0.85 * np.exp(1.0j * m - 0.1j),
            3: 0.2 * np.exp(2.0j * m + 0.3j), 4: -0.1}


def scheme_case(fam, p, m, rule, nx):
    c = schemes.cfl_number(fam, p)
    st = stepping.FineStep(fam, p, c, nx)
    col = psi.phi_m_column_by_stepping(st, nx, 1)
    phi_d = {i: v for i, v in psi.column_to_diagonals(col).items() if v != 0.0}
    ops = psi.build_hierarchy(fam, p, c, nx, 64 * m, m, 2, rule=rule, halfwidth=3)
    return phi_d, psi.symbol(phi_d, nx), ops[0].diag, ops[0].mu


@pytest.mark.parametrize("m,N", [(2, 5), (4, 12), (8, 3), (8, 30)])
def test_bound_is_sqrt_m_times_l1_norm_of_cpoint_propagator(m, N):
    nx = 8
    phi_d, lam = synthetic_circulant(nx, SYNTH_LAM)
    psi_d, mu = synthetic_circulant(nx, synth_mu(m))
    Ek = mode_propagators(phi_d, psi_d, nx, m, (N + 1) * m)
    b = psi.two_level_bound(lam, mu, m, N * m)
    for k in range(1, nx // 2 + 1):
        C = Ek[k][m - 1::m, m - 1::m]               # C-point rows and columns
        l1 = np.max(np.sum(np.abs(C), axis=0))
        assert abs(np.sqrt(m) * l1 - b[k]) <= 1e-12 * b[k], (k, np.sqrt(m) * l1, b[k])


@pytest.mark.parametrize("fam,p,m,rule", [("ERK", 1, 8, "halfwidth"), ("ERK", 3, 4, "auto"),
                                           ("ERK", 2, 8, "auto"), ("SDIRK", 3, 4, "threshold")])
def test_bound_dominates_the_propagator_norm_of_the_paper_schemes(fam, p, m, rule):
    nx, N = 32, 24
    phi_d, lam, psi_d, mu = scheme_case(fam, p, m, rule, nx)
    Ek = mode_propagators(phi_d, psi_d, nx, m, N * m)
    b = psi.two_level_bound(lam, mu, m, N * m)
    checked = 0
    for k in range(nx):
        if abs(lam[k]) < 1 - 1e-12 and abs(mu[k]) < 1 - 1e-12:
            n2 = np.linalg.norm(Ek[k], 2)
            assert n2 <= b[k] * (1 + 1e-10) + 1e-15, (k, n2, b[k])
            checked += 1
    assert checked >= nx - 2


@pytest.mark.parametrize("m", [2, 4, 8])
def test_bound_is_sharp_with_the_interpolation_factor(m):
    nx, N = 8, 256
    phi_d, lam = synthetic_circulant(nx, SYNTH_LAM)
    psi_d, mu = synthetic_circulant(nx, synth_mu(m))
    Ek = mode_propagators(phi_d, psi_d, nx, m, N * m)
    b = psi.two_level_bound(lam, mu, m, N * m)
    for k in range(1, nx // 2 + 1):
        s = sum(abs(lam[k]) ** (2 * i) for i in range(m))
        ratio = np.sqrt(s / m) * b[k] / np.linalg.norm(Ek[k], 2)
        assert 1 - 1e-12 <= ratio <= 1 + 2.0 * m / (N * m), (k, ratio)
    # the mode with |lambda| -> 1 attains Eq. 4 itself, without the factor
    assert b[1] / np.linalg.norm(Ek[1], 2) <= 1 + 2.0 / N
