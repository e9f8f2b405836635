"""Spatial stencils, Runge-Kutta tableaux, stability functions and Fourier
symbols (oracle; test infrastructure only).

Follows Section 2.1 (U1..U5 upwind differences, Lemma 1, Corollary 1, the CFL
number and Table 1) and Appendix A (Butcher tableaux).

Pins (tests/test_oracle_schemes.py): U_p is exact on polynomials of degree
<= p; tableau row sums equal the printed abscissae; the stability function
matches exp(z) to order p; the SDIRK3 constant zeta solves its defining cubic;
the CFL limits of Table 1; stepping a Fourier mode multiplies it by lambda.
"""
from __future__ import annotations

import math
from fractions import Fraction as Fr

import numpy as np

# ---------------------------------------------------------------------------
# U_p upwind differences, Section 2.1:  v'_i ~ (1/(s dx)) * sum_k a_k v_{i+k}.
# Stored as (s, {k: a_k}); k > 0 is downwind, k < 0 upwind (wave speed > 0).
# ---------------------------------------------------------------------------
UPWIND = {
    1: (1, {0: 1, -1: -1}),
    2: (2, {0: 3, -1: -4, -2: 1}),
    3: (6, {1: 2, 0: 3, -1: -6, -2: 1}),
    4: (12, {1: 3, 0: 10, -1: -18, -2: 6, -3: -1}),
    5: (60, {2: -3, 1: 30, 0: 20, -1: -60, -2: 15, -3: -2}),
}


def dtL_taps(p: int, c: float) -> dict:
    """Taps of dt*L where L discretises -alpha d/dx with U_p (Eq. 2):
    (dt L v)_i = -(c/s) sum_k a_k v_{i+k},  c = alpha dt / dx (Eq. 3's CFL)."""
    s, a = UPWIND[p]
    return {k: -c * ak / s for k, ak in a.items()}


def stencil_symbol(taps: dict, theta: np.ndarray) -> np.ndarray:
    """Eigenvalue of the circulant operator v_i -> sum_k t_k v_{i+k} on the
    Fourier mode exp(i j theta): sum_k t_k exp(i k theta)."""
    theta = np.asarray(theta, dtype=np.float64)
    out = np.zeros(theta.shape, dtype=np.complex128)
    for k, t in taps.items():
        out += t * np.exp(1j * k * theta)
    return out


# ---------------------------------------------------------------------------
# Butcher tableaux, Appendix A.  Exact rationals where the paper prints them.
# ---------------------------------------------------------------------------

def _erk_tableaux():
    z = Fr(0)
    t = {}
    t[1] = ([[z]], [Fr(1)])
    t[2] = ([[z, z], [Fr(1), z]], [Fr(1, 2), Fr(1, 2)])
    t[3] = ([[z, z, z], [Fr(1), z, z], [Fr(1, 4), Fr(1, 4), z]], [Fr(1, 6), Fr(1, 6), Fr(2, 3)])
    t[4] = ([[z, z, z, z], [Fr(1, 2), z, z, z], [z, Fr(1, 2), z, z], [z, z, Fr(1), z]],
            [Fr(1, 6), Fr(1, 3), Fr(1, 3), Fr(1, 6)])
    t[5] = ([[z] * 6,
             [Fr(1, 4), z, z, z, z, z],
             [Fr(1, 8), Fr(1, 8), z, z, z, z],
             [z, z, Fr(1, 2), z, z, z],
             [Fr(3, 16), Fr(-3, 8), Fr(3, 8), Fr(9, 16), z, z],
             [Fr(-3, 7), Fr(8, 7), Fr(6, 7), Fr(-12, 7), Fr(8, 7), z]],
            [Fr(7, 90), z, Fr(32, 90), Fr(12, 90), Fr(32, 90), Fr(7, 90)])
    return t


ERK_ABSCISSAE = {1: [0], 2: [0, 1], 3: [0, 1, 0.5], 4: [0, 0.5, 0.5, 1],
                 5: [0, 0.25, 0.25, 0.5, 0.75, 1]}

# SDIRK3 constant printed in Appendix A (20 significant digits).
SDIRK3_ZETA = 0.43586652150845899942


def _sdirk_tableaux():
    t = {}
    t[1] = (np.array([[1.0]]), np.array([1.0]))
    g = 1.0 - math.sqrt(2.0) / 2.0
    t[2] = (np.array([[g, 0.0], [math.sqrt(2.0) / 2.0, g]]), np.array([math.sqrt(2.0) / 2.0, g]))
    zt = SDIRK3_ZETA
    beta = (1.0 - zt) / 2.0
    gam = -1.5 * zt * zt + 4.0 * zt - 0.25
    eps = 1.5 * zt * zt - 5.0 * zt + 1.25
    t[3] = (np.array([[zt, 0, 0], [beta, zt, 0], [gam, eps, zt]]), np.array([gam, eps, zt]))
    q = 0.25
    a4 = [[q, 0, 0, 0, 0],
          [Fr(1, 2), q, 0, 0, 0],
          [Fr(17, 50), Fr(-1, 25), q, 0, 0],
          [Fr(371, 1360), Fr(-137, 2720), Fr(15, 544), q, 0],
          [Fr(25, 24), Fr(-49, 48), Fr(125, 16), Fr(-85, 12), q]]
    A = np.array([[float(v) for v in row] for row in a4])
    t[4] = (A, A[-1].copy())
    return t


SDIRK_ABSCISSAE = {1: [1.0], 2: [1.0 - math.sqrt(2.0) / 2.0, 1.0],
                   3: [SDIRK3_ZETA, (1.0 + SDIRK3_ZETA) / 2.0, 1.0],
                   4: [0.25, 0.75, 11.0 / 20.0, 0.5, 1.0]}


def tableau(family: str, p: int):
    """(A, b) as float64 arrays for ERKp or SDIRKp (Appendix A)."""
    if family == "ERK":
        A, b = _erk_tableaux()[p]
        return (np.array([[float(v) for v in row] for row in A]), np.array([float(v) for v in b]))
    if family == "SDIRK":
        return _sdirk_tableaux()[p]
    raise ValueError(family)


def erk_tableau_exact(p: int):
    """ERK tableau as exact rationals (for order-condition pins)."""
    return _erk_tableaux()[p]


# ---------------------------------------------------------------------------
# Stability function R(z) = 1 + z b^T (I - z A)^{-1} 1  (Lemma 1).
# ---------------------------------------------------------------------------

def stability(family: str, p: int, z) -> np.ndarray:
    A, b = tableau(family, p)
    z = np.atleast_1d(np.asarray(z, dtype=np.complex128))
    s = len(b)
    zf = z.reshape(-1)
    mats = np.eye(s)[None, :, :] - zf[:, None, None] * A[None, :, :]
    y = np.linalg.solve(mats, np.ones((len(zf), s, 1), dtype=np.complex128))[..., 0]
    return (1.0 + zf * (y @ b)).reshape(z.shape)


def thetas(nx: int) -> np.ndarray:
    """Fourier frequencies theta_k = 2 pi k / nx, k = 0..nx-1."""
    return 2.0 * np.pi * np.arange(nx) / nx


def phi_symbol(family: str, p: int, c: float, nx: int, q: int | None = None) -> np.ndarray:
    """Eigenvalues lambda_k of the fine propagator Phi (Lemma 1, Corollary 1):
    lambda_k = R(z_k), z_k the eigenvalue of dt*L on mode theta_k.  Ordered as
    numpy's DFT of the first column of Phi.  q: order of the upwind stencil
    (default p, the paper's pairing)."""
    z = stencil_symbol(dtL_taps(q or p, c), thetas(nx))
    return stability(family, p, z)


# ---------------------------------------------------------------------------
# CFL (Eq. 3) and the ERK limits of Table 1.
# ---------------------------------------------------------------------------

CMAX_TABLE1 = {1: 1.0, 2: 0.5, 3: 1.62589, 4: 1.04449, 5: 1.96583}


def max_amplification(p: int, c: float, ntheta: int = 4096) -> float:
    th = np.linspace(0.0, np.pi, ntheta + 1)
    z = stencil_symbol(dtL_taps(p, c), th)
    return float(np.max(np.abs(stability("ERK", p, z))))


def erk_cfl_limit(p: int, slack: float = 0.0, ntheta: int = 4096) -> float:
    """Largest c with max_theta |R(z_c(theta))| <= 1 + slack (bisection)."""
    lo, hi = 0.0, 3.0
    # the stable set is [0, cmax]; bisect on its right end
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if max_amplification(p, mid, ntheta) <= 1.0 + slack:
            lo = mid
        else:
            hi = mid
    return lo


def cfl_number(family: str, p: int, cfl_fraction: float = 0.85) -> float:
    """CFL number used by the paper's experiments (Section 2.1): ERK runs at
    c = 0.85 c_max with the printed c_max of Table 1, SDIRK at c = 4."""
    if family == "ERK":
        return cfl_fraction * CMAX_TABLE1[p]
    return 4.0
