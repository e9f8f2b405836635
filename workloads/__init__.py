"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the solver: it only draws initial
conditions, random initial iterates and request mixes from fixed seeds, with
the shapes and value distributions of the runs in the paper (Section 2.1,
Section 2.2) and of the benchmark workloads built on it.  Both the CPU oracle
and the GPU path receive the arrays produced here as plain inputs.

Grid convention (Section 2.1): the periodic domain [-1, 1) is sampled at
``x_i = -1 + i*dx``, ``dx = 2/nx``, ``i = 0..nx-1``; the point ``x = 1`` is the
periodic image of ``x = -1`` and is not stored.
"""
from __future__ import annotations

import numpy as np

# Seeds of the synthetic workloads (fixed so that every run sees the same data).
SEED_FOURIER_FIELD = 2      # ERK3+U3 4096 x 16384 field
SEED_WAVE_PACKET = 3        # SDIRK3+U5 8192 x 8192 packet noise
SEED_BATCH = 4              # 4096-solve batch: sizes and fields
SEED_ARRIVALS = 5           # serving stream arrivals


def grid(nx: int) -> np.ndarray:
    """Periodic grid points x_i = -1 + 2 i / nx (Section 2.1)."""
    return -1.0 + 2.0 * np.arange(nx, dtype=np.float64) / nx


def sin4(nx: int) -> np.ndarray:
    """The paper's initial condition u(x, 0) = sin^4(pi x) (Eq. 1)."""
    return np.sin(np.pi * grid(nx)) ** 4


def fourier_coefficients(seed: int = SEED_FOURIER_FIELD, modes: int = 64):
    """The (a_k, b_k), k = 1..modes, of the random Fourier field."""
    rng = np.random.Generator(np.random.PCG64(seed))
    a = rng.standard_normal(modes)
    b = rng.standard_normal(modes)
    return a, b


def fourier_field(nx: int, seed: int = SEED_FOURIER_FIELD, modes: int = 64, shift: float = 0.0) -> np.ndarray:
    """Random smooth periodic field: sum over k = 1..modes of
    (a_k cos(k pi x) + b_k sin(k pi x)) / k^2 with a_k, b_k ~ N(0, 1),
    sampled at x_i - shift (shift = alpha t gives the exact solution of Eq. 1
    at time t for this initial condition).

    The period-2 domain makes k*pi the k-th wavenumber.
    """
    a, b = fourier_coefficients(seed, modes)
    x = grid(nx) - shift
    u = np.zeros(nx)
    for k in range(1, modes + 1):
        u += (a[k - 1] * np.cos(k * np.pi * x) + b[k - 1] * np.sin(k * np.pi * x)) / (k * k)
    return u


def wave_packet(nx: int, seed: int = SEED_WAVE_PACKET, noise: float = 1e-3) -> np.ndarray:
    """Gaussian wave packet exp(-100 x^2) cos(20 pi x) plus noise * N(0, 1) per point."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = grid(nx)
    return np.exp(-100.0 * x * x) * np.cos(20.0 * np.pi * x) + noise * rng.standard_normal(nx)


def random_iterate(nt: int, nx: int, u0: np.ndarray, seed: int) -> np.ndarray:
    """Space-time initial iterate of Section 2.2: U[0, 1) random at every time
    level except t = 0, where it equals the initial condition."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.random((nt + 1, nx))
    u[0] = u0
    return u


# ---------------------------------------------------------------------------
# Batch and serving mixes
# ---------------------------------------------------------------------------

NX_CHOICES = (256, 512, 1024, 2048, 4096)
NT_CHOICES = (1024, 2048, 4096, 8192, 16384)
M_CHOICES = (4, 8, 16)


def batch_specs(count: int, seed: int = SEED_BATCH):
    """Draw ``count`` independent solve specifications.

    nx and nt uniform over powers of two, order p uniform in 1..5, m uniform in
    {4, 8, 16}; for p <= 4 the scheme family is ERK or SDIRK with probability
    1/2 each, p = 5 is always ERK5 (the paper has no fifth-order SDIRK).
    Returns a list of dicts with keys nx, nt, p, family ('ERK'|'SDIRK'), m and
    field_seed (the seed of the solve's Fourier-field initial condition).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    specs = []
    for i in range(count):
        nx = int(rng.choice(NX_CHOICES))
        nt = int(rng.choice(NT_CHOICES))
        p = int(rng.integers(1, 6))
        m = int(rng.choice(M_CHOICES))
        fam = "ERK" if (p == 5 or rng.random() < 0.5) else "SDIRK"
        specs.append(dict(nx=nx, nt=nt, p=p, family=fam, m=m, field_seed=int(seed * 1_000_003 + i)))
    return specs


def arrivals(rate_per_s: float, count: int, seed: int = SEED_ARRIVALS):
    """Poisson arrival times (seconds) and a per-request tolerance drawn from
    {1e-8, 1e-10} with probability 1/2 each."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_per_s, size=count)
    tols = np.where(rng.random(count) < 0.5, 1e-8, 1e-10)
    return np.cumsum(gaps), tols
