"""Coarse-grid operators Psi (oracle; test infrastructure only).

Follows Section 4: Psi is a sparse circulant whose nonzero diagonals are fitted
by the weighted linear least-squares problem of Eq. 6,

    psi = argmin || W^{1/2} F (phi~^m - R^T psi^) ||_2^2 ,
    w_k = w(|lambda_k|),  w(z) = 1 / (1 - z + eps)^2,  eps = 1e-6,

with F the DFT, phi~^m the first column of Phi^m and R the restriction onto
the chosen nonzero pattern.  The complex problem is solved with LAPACK
(``numpy.linalg.lstsq``); its imaginary part is dropped (Lemma 2) and a
solution whose imaginary part exceeds 1e-8 is flagged as not acceptable
(Section 4.1).  Also here: the two-level convergence bound (Eq. 4), operator
complexity (Eq. 5), and the sparsity-pattern rules of Sections 4.2-4.4 and 4.6.

Diagonal index (Section 4.2): i = 0 on the main diagonal, negative below it.
For a circulant the entry on diagonal i is the first-column entry in row
(-i) mod nx, and applying the matrix is the stencil (Psi v)_r = sum_i psi_i
v_{r+i}.  Patterns and coefficients are therefore stored as (offset i, value).

Pins (tests/test_oracle_psi.py): the first column of Phi^m by stepping equals
the inverse DFT of lambda^m; unit weights give the truncation of Phi^m (Remark
1); the fitted psi is real to within the flag and its symbol reproduces
lambda^m at theta = 0; Psi = Phi^m gives one-iteration convergence; the
thresholded SDIRK operators reproduce Table 6 iteration counts.  The
two-level bound (Eq. 4) is pinned to the error propagator E_k of one oracle
iteration per Fourier mode: sqrt(m) times the induced l1 norm of its C-point
block equals the bound exactly (the paper's coarse system counts the initial
C-point as an unknown, so the oracle's problem with n_t + m steps is compared);
||E_k||_2 never exceeds it; and with the ideal-interpolation factor
sqrt(sum_{i<m} |lambda_k|^{2i} / m) it is attained as n_t/m grows (Section 3.1).

Readings (where the paper is silent):
* ERK pattern ("contiguous subset of the largest entries of Phi^m, widened
  until scalable", Section 4.3): among all contiguous windows of width W the
  one holding the largest sum of |phi~^m_i|^2; W starts at nnz(Phi) and grows
  until the fit is acceptable (imaginary part <= 1e-8, max |mu_k| <= 1 + 1e-12)
  and max_k of the bound (Eq. 4, at the level's own n_t, over the modes with
  |lambda_k| < 1) is <= rho_target = 0.15.
* Half-width rule: 2h+1 contiguous offsets centred on argmax |phi~^m_i|
  (ties to the smaller |i|).
"""
from __future__ import annotations

import numpy as np

from . import schemes, stepping

EPS_WEIGHT = 1e-6       # epsilon of the weight function, Section 4
IMAG_FLAG = 1e-8        # imaginary-part acceptance limit, Section 4.1


# ---------------------------------------------------------------------------
# Sparse circulant operators as {offset: coefficient}
# ---------------------------------------------------------------------------

def column_to_diagonals(col: np.ndarray) -> dict:
    """First column -> {diagonal index i: entry}, i in (-nx/2, nx/2]."""
    nx = len(col)
    out = {}
    for i in range(-(nx // 2) + 1, nx // 2 + 1):
        out[i] = float(col[(-i) % nx])
    return out


def diagonals_to_column(diag: dict, nx: int) -> np.ndarray:
    col = np.zeros(nx)
    for i, v in diag.items():
        col[(-i) % nx] += v
    return col


def symbol(diag: dict, nx: int) -> np.ndarray:
    """Eigenvalues mu_k of the circulant with these diagonals (DFT of the
    first column, numpy ordering)."""
    return np.fft.fft(diagonals_to_column(diag, nx))


# ---------------------------------------------------------------------------
# First column of Phi^m
# ---------------------------------------------------------------------------

def phi_m_column_by_stepping(step, nx: int, m: int) -> np.ndarray:
    """Apply the fine step m times to e_0 (works for any linear step)."""
    e = np.zeros(nx)
    e[0] = 1.0
    for _ in range(m):
        e = step(e)
    return e


def phi_m_column_by_symbol(lam: np.ndarray, m: int) -> np.ndarray:
    """Inverse DFT of lambda^m (Section 4.6, used for the dense SDIRK Phi^m)."""
    return np.real(np.fft.ifft(lam ** m))


def stencil_power_column(diag: dict, nx: int, m: int) -> np.ndarray:
    """First column of (sparse circulant)^m by repeated application."""
    e = np.zeros(nx)
    e[0] = 1.0
    for _ in range(m):
        e = stepping.apply_taps(e, diag)
    return e


# ---------------------------------------------------------------------------
# Weighted least squares, Eq. 6
# ---------------------------------------------------------------------------

def weights(lam: np.ndarray, eps: float = EPS_WEIGHT) -> np.ndarray:
    return 1.0 / (1.0 - np.abs(lam) + eps) ** 2


def lsq_fit(lam: np.ndarray, lam_m: np.ndarray, offsets, unit_weight: bool = False):
    """Solve Eq. 6 for the nonzeros on the given diagonal offsets.

    lam   eigenvalues of the level's operator (they set the weights)
    lam_m eigenvalues of the ideal coarse operator (= F phi~^m)
    Returns (diag dict, max |imag part| of the complex solution).
    """
    nx = len(lam)
    offsets = list(offsets)
    k = np.arange(nx)
    # column for offset i: F e_{(-i) mod nx} = exp(+2 pi i_ i k / nx)
    M = np.exp(2j * np.pi * np.outer(k, offsets) / nx)
    w = np.ones(nx) if unit_weight else weights(lam)
    sw = np.sqrt(w)
    sol, *_ = np.linalg.lstsq(sw[:, None] * M, sw * lam_m, rcond=None)
    imag = float(np.max(np.abs(sol.imag))) if len(sol) else 0.0
    return {i: float(v.real) for i, v in zip(offsets, sol)}, imag


# ---------------------------------------------------------------------------
# Two-level bound (Eq. 4) and operator complexity (Eq. 5)
# ---------------------------------------------------------------------------

def two_level_bound(lam: np.ndarray, mu: np.ndarray, m: int, nt: int | None) -> np.ndarray:
    """Per-mode bound sqrt(m) |lam|^m |lam^m - mu| (1 - |mu|^{N-1}) / (1 - |mu|),
    N = nt/m; nt None means the nt -> infinity limit (last factor 1).
    (1 - x^{N-1})/(1 - x) is evaluated as the geometric sum when x ~ 1."""
    a = np.abs(lam) ** m * np.abs(lam ** m - mu)
    am = np.abs(mu)
    if nt is None:
        with np.errstate(divide="ignore", invalid="ignore"):
            g = np.where(am < 1.0, 1.0 / (1.0 - am), np.inf)
        g = np.where(a == 0.0, 0.0, g)
    else:
        N = nt // m
        with np.errstate(divide="ignore", invalid="ignore"):
            g = np.where(np.abs(1.0 - am) > 1e-8, (1.0 - am ** (N - 1)) / (1.0 - am), N - 1.0)
    return np.sqrt(m) * a * g


def operator_complexity(nnz_per_level, m: int) -> float:
    """Eq. 5: (1/nnz(Phi_1)) sum_l m^{1-l} nnz(Phi_l)."""
    return sum(m ** (-l) * n for l, n in enumerate(nnz_per_level)) / nnz_per_level[0]


# ---------------------------------------------------------------------------
# Sparsity patterns
# ---------------------------------------------------------------------------

def argmax_offset(col: np.ndarray) -> int:
    d = column_to_diagonals(col)
    best = max(d.items(), key=lambda kv: (abs(kv[1]), -abs(kv[0])))
    return best[0]


def halfwidth_pattern(col: np.ndarray, h: int):
    """2h+1 contiguous offsets centred on argmax |phi~^m_i|."""
    i0 = argmax_offset(col)
    return list(range(i0 - h, i0 + h + 1))


def best_window(col: np.ndarray, width: int):
    """Contiguous window of `width` offsets holding the most |phi~^m|^2
    (ties: the window whose first offset is smallest)."""
    d = column_to_diagonals(col)
    nx = len(col)
    lo_all = -(nx // 2) + 1
    best, best_start = -1.0, None
    for start in range(lo_all, nx // 2 + 2 - width):
        e = sum(d[i] ** 2 for i in range(start, start + width))
        if e > best * (1.0 + 1e-13):
            best, best_start = e, start
    return list(range(best_start, best_start + width))


def threshold_pattern(col: np.ndarray, eta: float):
    """Offsets with |phi~^m_i| >= eta max |phi~^m| (Section 4.6)."""
    d = column_to_diagonals(col)
    mx = max(abs(v) for v in d.values())
    return sorted(i for i, v in d.items() if abs(v) >= eta * mx)


# eta_tol per (p, m) for SDIRKp+Up, Section 4.6
ETA_TOL = {
    1: {2: .1, 4: .125, 8: .25, 16: .5, 32: .5, 64: .6},
    2: {2: .05, 4: .1, 8: .1, 16: .2, 32: .2, 64: .2},
    3: {2: .005, 4: .01, 8: .02, 16: .02, 32: .02, 64: .04},
    4: {2: .005, 4: .01, 8: .01, 16: .01, 32: .02, 64: .02},
}

DEFAULT_RHO_TARGET = 0.15


class CoarseOp:
    """A fitted coarse operator: diagonals, eigenvalues and diagnostics."""

    def __init__(self, diag, mu, imag, bound_max):
        self.diag = diag
        self.mu = mu
        self.imag = imag
        self.bound_max = bound_max

    @property
    def offsets(self):
        return sorted(self.diag)

    @property
    def nnz(self):
        return len(self.diag)

    def acceptable(self) -> bool:
        return self.imag <= IMAG_FLAG


def fit(lam, col_m, offsets, m, nt=None, unit_weight=False) -> CoarseOp:
    lam_m = np.fft.fft(col_m)
    diag, imag = lsq_fit(lam, lam_m, offsets, unit_weight=unit_weight)
    mu = symbol(diag, len(lam))
    return CoarseOp(diag, mu, imag, max_bound(lam, mu, m, nt))


def max_bound(lam, mu, m, nt=None) -> float:
    """max_k of Eq. 4 over the modes with |lambda_k| < 1 (the bound does not
    apply to |lambda_k| = 1, i.e. the constant mode theta = 0)."""
    keep = np.abs(lam) < 1.0 - 1e-14
    if not np.any(keep):
        return 0.0
    return float(np.max(two_level_bound(lam[keep], mu[keep], m, nt)))


def auto_width_fit(lam, col_m, m, nt, w0: int, rho_target=DEFAULT_RHO_TARGET, wmax=None) -> CoarseOp:
    """ERK rule: grow a best contiguous window from width w0 until the fit is
    acceptable, stable (max |mu| <= 1 + 1e-12) and its bound (Eq. 4 at this
    level's nt) is below rho_target."""
    nx = len(lam)
    wmax = wmax or min(nx - 1, 8 * w0 + 64)
    last = None
    for W in range(w0, wmax + 1):
        op = fit(lam, col_m, best_window(col_m, W), m, nt)
        last = op
        if op.acceptable() and np.max(np.abs(op.mu)) <= 1.0 + 1e-12 and op.bound_max <= rho_target:
            return op
    return last


def build_hierarchy(family: str, p: int, c: float, nx: int, nt: int, m: int, levels: int,
                    rule: str = "auto", halfwidth: int = 3, eta=None,
                    rho_target: float = DEFAULT_RHO_TARGET, q: int | None = None):
    """Coarse operators Phi_2..Phi_L (Section 4.4: each level fits Phi_l^m).

    rule: 'halfwidth' | 'auto' | 'threshold' | 'ideal'.  Returns a list of
    CoarseOp (one per coarse level).  For 'ideal' the list holds the dense
    first-column diagonals of Phi^m (two levels only).  q: order of the
    upwind stencil (default p); the threshold rule keeps the eta_tol row of
    the Runge-Kutta order p."""
    step = stepping.FineStep(family, p, c, nx, q=q)
    lam = schemes.phi_symbol(family, p, c, nx, q=q)
    if family == "ERK":
        nnz_fine = len(phi_m_column_nonzeros(step, nx))
    ops = []
    cur_lam = lam
    cur_diag = None
    for lvl in range(1, levels):
        lvl_nt = nt // m ** (lvl - 1)
        if cur_diag is None:
            col = (phi_m_column_by_stepping(step, nx, m) if family == "ERK"
                   else phi_m_column_by_symbol(lam, m))
        else:
            col = stencil_power_column(cur_diag, nx, m)
        if rule == "ideal":
            d = {i: v for i, v in column_to_diagonals(col).items() if v != 0.0}
            mu = symbol(d, nx)
            ops.append(CoarseOp(d, mu, 0.0, 0.0))
            cur_lam, cur_diag = mu, d
            continue
        if rule == "halfwidth":
            op = fit(cur_lam, col, halfwidth_pattern(col, halfwidth), m, lvl_nt)
        elif rule == "threshold":
            e = eta if eta is not None else ETA_TOL[p][m]
            op = fit(cur_lam, col, threshold_pattern(col, e), m, lvl_nt)
        elif rule == "auto":
            w0 = nnz_fine if (family == "ERK" and cur_diag is None) else (ops[-1].nnz if ops else 1)
            op = auto_width_fit(cur_lam, col, m, lvl_nt, w0, rho_target)
        else:
            raise ValueError(rule)
        ops.append(op)
        cur_lam, cur_diag = op.mu, op.diag
    return ops


def phi_m_column_nonzeros(step, nx: int):
    """Nonzero diagonals of Phi itself (nnz(Phi) of Corollary 1 for ERK)."""
    col = phi_m_column_by_stepping(step, nx, 1)
    d = column_to_diagonals(col)
    return sorted(i for i, v in d.items() if v != 0.0)
