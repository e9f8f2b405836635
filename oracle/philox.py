"""Counter-based uniform draws for the paper's random initial iterate (oracle;
test infrastructure only).

Section 2.2: the tests start from a space-time iterate that is uniformly
random except at t = 0.  The library draws it on the device, so both sides
implement one counter-based generator from its published definition:
Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
as 1, 2, 3", SC'11).  A 4 x 32-bit counter and a 2 x 32-bit key pass through
ten rounds; each round multiplies counter words 0 and 2 by fixed 32-bit
constants, keeps the high and low halves of the 64-bit products, and XORs the
high halves with words 1 and 3 and the key; the key grows by two Weyl
constants between rounds.

Point i of time level n uses counter (i, n, 0, 0) and key (seed mod 2^32,
seed div 2^32); its value in [0, 1) joins the top 27 bits of output word 0 and
the top 26 bits of word 1 into a 53-bit integer and scales it by 2^-53.

Pins (tests/test_oracle_philox.py): the published known-answer vectors of
Philox4x32-10; the draws are uniform on [0, 1) (mean, variance and a
chi-square test on a million values).
"""
from __future__ import annotations

import numpy as np

MULT = (0xD2511F53, 0xCD9E8D57)
WEYL = (0x9E3779B9, 0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)


def _mulhilo(a: int, x: np.ndarray):
    p = np.uint64(a) * x                       # < 2^64: both factors < 2^32
    return p >> np.uint64(32), p & MASK


def philox4x32_10(ctr, key):
    """ctr: four uint64 arrays (values < 2^32), key: two ints < 2^32.
    Returns the four output words as uint64 arrays."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & MASK for c in ctr)
    k0, k1 = int(key[0]), int(key[1])
    for _ in range(10):
        hi0, lo0 = _mulhilo(MULT[0], c0)
        hi1, lo1 = _mulhilo(MULT[1], c2)
        c0, c1, c2, c3 = hi1 ^ c1 ^ np.uint64(k0), lo1, hi0 ^ c3 ^ np.uint64(k1), lo0
        k0 = (k0 + WEYL[0]) & 0xFFFFFFFF
        k1 = (k1 + WEYL[1]) & 0xFFFFFFFF
    return c0, c1, c2, c3


def uniform(seed: int, i, n):
    """Draw of point i at time level n (arrays broadcast), in [0, 1)."""
    i, n = np.broadcast_arrays(np.asarray(i, dtype=np.uint64), np.asarray(n, dtype=np.uint64))
    zero = np.zeros_like(i)
    w0, w1, _, _ = philox4x32_10((i, n, zero, zero), (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF))
    bits = ((w0 >> np.uint64(5)) << np.uint64(26)) | (w1 >> np.uint64(6))
    return bits.astype(np.float64) * 2.0 ** -53


def random_iterate(u0: np.ndarray, nt: int, seed: int) -> np.ndarray:
    """(nt+1, nx) iterate: u0 at t = 0, the draws of every later point."""
    nx = len(u0)
    U = uniform(seed, np.arange(nx)[None, :], np.arange(nt + 1)[:, None])
    U[0] = u0
    return U
