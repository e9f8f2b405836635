"""Two-level and multilevel MGRIT (FCF- or F-relaxation, V- or F-cycles) with
full space-time storage (oracle; test infrastructure only).

Follows Section 2.2.  On level l the time grid has N_l + 1 points; every
m-th point is a C-point.  With operator Phi_l and right-hand side g:

  F-relaxation   from each C-point, step across the following F-interval:
                 u_{jm+i} = Phi_l u_{jm+i-1} + g_{jm+i},  i = 1..m-1
  C-relaxation   u_{jm} = Phi_l u_{jm-1} + g_{jm}
  FCF            F, then C, then F
  residual       r_j = g_{jm} + Phi_l u_{jm-1} - u_{jm} at the C-points
                 (zero at F-points after F-relaxation)
  coarse system  e_{j} = Phi_{l+1} e_{j-1} + r_j, e_0 = 0 (Eq. 5), solved
                 sequentially on the coarsest level, otherwise by a recursive
                 V-cycle on the coarse problem (Section 2.2, Section 4.4)
  correction     u_{jm} += e_j, then F-relaxation (ideal interpolation)

Level 1 has g = 0 and u_0 fixed to the initial condition.  The stopping test
compares the space-time residual 2-norm after FCF-relaxation on level 1 with
the residual of the initial iterate (Section 2.2); iterations are counted as
the number of coarse-grid corrections applied before the test passes.

Pins (tests/test_oracle_mgrit.py): the converged iterate equals sequential
stepping; for any Psi, after k iterations C-points 0..2k are exact and the
solve terminates after n_t/(2m) iterations (finite termination, Section 1 and
the right-hand side of Table 2); Psi = Phi^m converges in one iteration;
iteration counts of Tables 2 and 6 (exact) and Tables 3 and 4 (soft).
"""
from __future__ import annotations

import numpy as np

from . import stepping


class Level:
    """One level of the hierarchy: its propagator and its coarsening factor."""

    def __init__(self, step, m: int | None):
        self.step = step          # callable, acts on the last axis (batched)
        self.m = m                # None on the coarsest level


def stencil_step(diag: dict):
    return lambda v: stepping.apply_taps(v, diag)


def f_relax(U, G, step, m):
    N = U.shape[0] - 1
    starts = np.arange(0, N, m)
    v = U[starts]
    for i in range(1, m):
        v = step(v) + G[starts + i]
        U[starts + i] = v


def c_relax(U, G, step, m):
    N = U.shape[0] - 1
    cpts = np.arange(m, N + 1, m)
    U[cpts] = step(U[cpts - 1]) + G[cpts]


def c_residual(U, G, step, m):
    """r_j at C-points j = 1..N/m (index 0 holds 0)."""
    N = U.shape[0] - 1
    cpts = np.arange(m, N + 1, m)
    r = np.zeros((N // m + 1,) + U.shape[1:])
    r[1:] = G[cpts] + step(U[cpts - 1]) - U[cpts]
    return r


def spacetime_residual(U, G, step):
    """r_n = g_n + Phi u_{n-1} - u_n for n = 1..N (full space-time residual)."""
    return G[1:] + step(U[:-1]) - U[1:]


def sequential_solve(U, G, step):
    for n in range(1, U.shape[0]):
        U[n] = step(U[n - 1]) + G[n]


def vcycle(levels, l, U, G):
    """One V-cycle on level l >= 1 of the error/residual equation (l >= 1 here
    means a coarse level of the recursion; level 0 is driven by `solve`).
    U is the level's current iterate (zero on the first visit)."""
    lev = levels[l]
    if lev.m is None:
        sequential_solve(U, G, lev.step)
        return
    m = lev.m
    f_relax(U, G, lev.step, m)
    c_relax(U, G, lev.step, m)
    f_relax(U, G, lev.step, m)
    r = c_residual(U, G, lev.step, m)
    E = np.zeros_like(r)
    vcycle(levels, l + 1, E, r)
    U[m::m] += E[1:]
    f_relax(U, G, lev.step, m)


def fcycle(levels, l, U, G):
    """One F-cycle on level l >= 1 (multigrid F-cycle, the cycle Section 4.4 and
    Section 5 compare with V-cycles): relax, then solve the coarse error
    equation by an F-cycle from zero followed by a V-cycle from that result
    (one exact solve when the coarse level is the coarsest), correct, and
    F-relax."""
    lev = levels[l]
    if lev.m is None:
        sequential_solve(U, G, lev.step)
        return
    m = lev.m
    f_relax(U, G, lev.step, m)
    c_relax(U, G, lev.step, m)
    f_relax(U, G, lev.step, m)
    r = c_residual(U, G, lev.step, m)
    E = np.zeros_like(r)
    fcycle(levels, l + 1, E, r)
    if levels[l + 1].m is not None:
        vcycle(levels, l + 1, E, r)
    U[m::m] += E[1:]
    f_relax(U, G, lev.step, m)


def solve(levels, U, tol=1e-10, max_iter=200, history=None, r0_norm=None, cycle="V", relax="FCF"):
    """MGRIT on level 0 (g = 0, U[0] = initial condition).

    cycle: "V" or "F" (the coarse error equation is solved by a V-cycle or by
    an F-cycle, see fcycle).  relax: "FCF" (the paper's choice) or "F"
    (F-relaxation only; with two levels this is Parareal, Section 2.2).
    U: (nt+1, nx) initial space-time iterate, modified in place.
    Returns (iterations, final relative residual).
    """
    lev = levels[0]
    m = lev.m
    G = np.zeros_like(U)
    if r0_norm is None:
        r0_norm = float(np.linalg.norm(spacetime_residual(U, G, lev.step)))
    coarse = fcycle if cycle == "F" else vcycle
    it = 0
    while True:
        f_relax(U, G, lev.step, m)
        if relax == "FCF":
            c_relax(U, G, lev.step, m)
            f_relax(U, G, lev.step, m)
        r = c_residual(U, G, lev.step, m)
        rel = float(np.linalg.norm(r)) / r0_norm if r0_norm > 0 else 0.0
        if history is not None:
            history.append(rel)
        if rel <= tol or it >= max_iter:
            return it, rel
        E = np.zeros_like(r)
        coarse(levels, 1, E, r)
        U[m::m] += E[1:]
        f_relax(U, G, lev.step, m)
        it += 1


def make_levels(fine_step, m: int, coarse_ops):
    """Level list for a fine step and fitted coarse operators (diag dicts or
    callables).  Two-level = one coarse operator."""
    levels = [Level(fine_step, m)]
    for k, op in enumerate(coarse_ops):
        st = op if callable(op) else stencil_step(op)
        levels.append(Level(st, m if k < len(coarse_ops) - 1 else None))
    return levels


def zero_iterate(u0: np.ndarray, nt: int) -> np.ndarray:
    U = np.zeros((nt + 1, len(u0)))
    U[0] = u0
    return U
