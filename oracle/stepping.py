"""The fine time-stepping operator Phi and sequential time stepping (oracle;
test infrastructure only).

Follows Section 2.1: method of lines with U_p in space (Eq. 2) and an s-stage
Runge-Kutta method in time, giving the one-step form u^{n+1} = Phi u^n (Eq. 3).
Each step is taken stage by stage from the Butcher tableau:

    K_i = dt L (u + sum_{j<i} a_ij K_j)           (ERK, a_ii = 0)
    (I - a_ii dt L) K_i = dt L (u + sum_{j<i} a_ij K_j)   (SDIRK)
    u_new = u + sum_i b_i K_i

where K_i = dt k_i.  Periodic shifts are ``np.roll``; the implicit stage
matrix is circulant, so its solve is an exact division in Fourier space
(numpy FFT).  All arrays may carry leading batch axes: the last axis is x.

Pins (tests/test_oracle_stepping.py): a Fourier mode is multiplied by
R(z(theta)) (Lemma 1); the SDIRK stage solve leaves a residual at rounding
level; the discrete solution converges at order p to the exact solution
u0(x - alpha t) (Figure 1); sequential stepping is linear and periodic-shift
equivariant.
"""
from __future__ import annotations

import numpy as np

from . import schemes


def apply_taps(v: np.ndarray, taps: dict) -> np.ndarray:
    """(T v)_i = sum_k t_k v_{(i+k) mod nx}, along the last axis."""
    out = np.zeros_like(v)
    for k, t in taps.items():
        out += t * np.roll(v, -k, axis=-1)
    return out


class FineStep:
    """u -> Phi u for a family/order pair at CFL number c on nx points."""

    def __init__(self, family: str, p: int, c: float, nx: int, q: int | None = None):
        """q: order of the upwind stencil (default p, the paper's pairing)."""
        self.family, self.p, self.c, self.nx = family, p, c, nx
        self.A, self.b = schemes.tableau(family, p)
        self.taps = schemes.dtL_taps(q or p, c)
        if family == "SDIRK":
            sym = schemes.stencil_symbol(self.taps, schemes.thetas(nx))
            # one divisor per distinct diagonal entry (all equal for SDIRK)
            self._div = {float(a): 1.0 - a * sym for a in np.diag(self.A)}

    def dtL(self, v: np.ndarray) -> np.ndarray:
        return apply_taps(v, self.taps)

    def stage_solve(self, a_ii: float, rhs: np.ndarray) -> np.ndarray:
        """Solve (I - a_ii dt L) K = rhs exactly (circulant: divide the DFT)."""
        return np.real(np.fft.ifft(np.fft.fft(rhs, axis=-1) / self._div[float(a_ii)], axis=-1))

    def __call__(self, u: np.ndarray) -> np.ndarray:
        s = len(self.b)
        K = []
        for i in range(s):
            y = u.copy()
            for j in range(i):
                if self.A[i, j] != 0.0:
                    y += self.A[i, j] * K[j]
            rhs = self.dtL(y)
            if self.family == "SDIRK":
                K.append(self.stage_solve(self.A[i, i], rhs))
            else:
                K.append(rhs)
        out = u.copy()
        for i in range(s):
            if self.b[i] != 0.0:
                out += self.b[i] * K[i]
        return out


def sequential(step, u0: np.ndarray, nt: int, keep_all: bool = True):
    """Sequential time stepping u^{n+1} = Phi u^n, n = 0..nt-1 (Eq. 3).
    Returns all nt+1 time levels (keep_all) or only u^{nt}."""
    if keep_all:
        U = np.empty((nt + 1,) + u0.shape)
        U[0] = u0
        for n in range(nt):
            U[n + 1] = step(U[n])
        return U
    u = u0.copy()
    for n in range(nt):
        u = step(u)
    return u


def exact_solution(u0_func, nx: int, t: float, alpha: float = 1.0) -> np.ndarray:
    """Exact solution u0(x - alpha t) of Eq. 1 on the periodic grid, with x
    wrapped back into [-1, 1)."""
    x = -1.0 + 2.0 * np.arange(nx) / nx
    xs = np.mod(x - alpha * t + 1.0, 2.0) - 1.0
    return u0_func(xs)
