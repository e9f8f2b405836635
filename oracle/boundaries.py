"""Inflow/outflow boundaries (oracle; test infrastructure only).

Follows Section 4.5: u_t + u_x = 0 on [-1, 1] with an inflow condition at
x = -1 and no condition at the outflow x = 1; the same ERKp+Up schemes as the
periodic problem, ghost values at the outflow by p-th order extrapolation from
inside the domain, and coarse operators Psi fitted for the analogous periodic
problem and truncated at the boundaries (Toeplitz, no longer circulant).

Readings (where Section 4.5 leaves the details to its references):
  * Grid: x_i = -1 + i dx, dx = 2/nx, unknowns i = 1..nx (x_0 = -1 carries
    the inflow value, x_nx = 1 is the outflow point).
  * The operators act on the homogeneous problem (inflow data zero): the
    inflow value and the inflow-side ghost values of every Runge-Kutta stage
    are zero.  MGRIT's convergence on a linear problem does not depend on the
    right-hand side that non-zero inflow data would add, which is what the
    iteration counts of Table 5 measure.
  * Outflow ghosts x_{nx+j}, j = 1..hi: the degree-p polynomial through the
    last p+1 unknowns u_{nx-p}..u_{nx}, evaluated at x_{nx+j}, applied to every
    stage input.
  * Truncated Psi: (Psi v)_r = sum_i psi_i v_{r+i} over r+i in 1..nx only.

Pins (tests/test_oracle_boundaries.py): the extrapolation reproduces
polynomials of degree p; the scheme converges at order p to the exact
solution u0(x - t) (zero behind the characteristic from x = -1); no
eigenvalue of Phi exceeds 1 in modulus at 85% of Table 1's limit; MGRIT with
the truncated Psi converges to sequential stepping and terminates after
n_t/(2m) iterations for any Psi; Table 5's iteration counts (soft).
"""
from __future__ import annotations

import numpy as np

from . import schemes


def grid(nx: int) -> np.ndarray:
    """Unknown positions x_i = -1 + i dx, i = 1..nx."""
    return -1.0 + 2.0 * np.arange(1, nx + 1, dtype=np.float64) / nx


def extrapolation_weights(p: int, j: int) -> np.ndarray:
    """Weights w_q, q = 0..p, with u_{nx+j} = sum_q w_q u_{nx-q}: the Lagrange
    polynomial of degree p through the nodes -q, evaluated at j."""
    nodes = -np.arange(p + 1, dtype=np.float64)
    w = np.ones(p + 1)
    for q in range(p + 1):
        for r in range(p + 1):
            if r != q:
                w[q] *= (j - nodes[r]) / (nodes[q] - nodes[r])
    return w


class InflowStep:
    """u -> Phi u for ERKp+Uq with homogeneous inflow at x = -1 and p-th order
    extrapolation at the outflow, stage by stage (Section 2.1's stage form)."""

    def __init__(self, p: int, c: float, nx: int, q: int | None = None):
        self.p, self.c, self.nx = p, c, nx
        self.q = q or p
        self.A, self.b = schemes.tableau("ERK", p)
        self.taps = schemes.dtL_taps(self.q, c)
        self.lo = min(min(self.taps), 0)
        self.hi = max(max(self.taps), 0)
        self.ext_w = [extrapolation_weights(self.q, j) for j in range(1, self.hi + 1)]

    def extend(self, v: np.ndarray) -> np.ndarray:
        """[inflow ghosts (zero) | v | outflow ghosts (extrapolated)] along x."""
        left = np.zeros(v.shape[:-1] + (-self.lo,))
        tail = v[..., ::-1][..., : self.q + 1]  # u_nx, u_{nx-1}, ..., u_{nx-q}
        right = [np.tensordot(tail, w, axes=([-1], [0])) for w in self.ext_w]
        right = np.stack(right, axis=-1) if right else np.zeros(v.shape[:-1] + (0,))
        return np.concatenate([left, v, right], axis=-1)

    def dtL(self, v: np.ndarray) -> np.ndarray:
        ext = self.extend(v)
        nx = v.shape[-1]
        out = np.zeros_like(v)
        for k, t in self.taps.items():
            s = k - self.lo  # ext index of u_{i+k} for i = 1 is (i - 1) + (k - lo)
            out += t * ext[..., s: s + nx]
        return out

    def __call__(self, u: np.ndarray) -> np.ndarray:
        s = len(self.b)
        K = []
        for i in range(s):
            y = u.copy()
            for j in range(i):
                if self.A[i, j] != 0.0:
                    y += self.A[i, j] * K[j]
            K.append(self.dtL(y))
        out = u.copy()
        for i in range(s):
            if self.b[i] != 0.0:
                out += self.b[i] * K[i]
        return out


def truncated(diag: dict):
    """(Psi v)_r = sum_i psi_i v_{r+i} over r+i inside the domain (Toeplitz)."""
    def apply(v: np.ndarray) -> np.ndarray:
        nx = v.shape[-1]
        out = np.zeros_like(v)
        for i, t in diag.items():
            if i >= 0:
                if i < nx:
                    out[..., : nx - i] += t * v[..., i:]
            elif -i < nx:
                out[..., -i:] += t * v[..., : nx + i]
        return out
    return apply


def exact_solution(nx: int, t: float) -> np.ndarray:
    """u(x, t) = sin^4(pi (x - t)) for x - t >= -1, 0 behind the characteristic
    that leaves x = -1 at t = 0 (homogeneous inflow, alpha = 1)."""
    s = grid(nx) - t
    return np.where(s >= -1.0, np.sin(np.pi * s) ** 4, 0.0)


def dense_phi(step: InflowStep) -> np.ndarray:
    """Phi as a dense matrix (column j = Phi e_j)."""
    return step(np.eye(step.nx)).T
