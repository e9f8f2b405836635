"""Pins of the oracle's Philox4x32-10 (the random initial iterate of Section
2.2): the published known-answer vectors, and uniformity of the draws."""
import numpy as np

from oracle import philox

# Known-answer vectors of Philox4x32-10 published with the generator (counter
# words, key words, output words; hexadecimal).
KAT = [
    ((0x00000000, 0x00000000, 0x00000000, 0x00000000), (0x00000000, 0x00000000),
     (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF), (0xFFFFFFFF, 0xFFFFFFFF),
     (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


def test_known_answer_vectors():
    for ctr, key, want in KAT:
        got = philox.philox4x32_10(tuple(np.array([c], dtype=np.uint64) for c in ctr), key)
        assert tuple(int(w[0]) for w in got) == want


def test_draws_are_uniform_on_unit_interval():
    n = 1 << 20
    u = philox.uniform(12345, np.arange(n) % 4096, np.arange(n) // 4096)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 5e-4
    counts = np.bincount((u * 64).astype(int), minlength=64)
    chi2 = float(np.sum((counts - n / 64) ** 2 / (n / 64)))
    assert chi2 < 120.0   # 63 degrees of freedom: p ~ 1e-5


def test_iterate_keeps_u0_and_depends_on_seed_and_position():
    u0 = np.linspace(0, 1, 16)
    a = philox.random_iterate(u0, 32, 7)
    b = philox.random_iterate(u0, 32, 8)
    np.testing.assert_array_equal(a[0], u0)
    assert not np.array_equal(a[1:], b[1:])
    assert len(np.unique(a[1:])) == a[1:].size
    np.testing.assert_array_equal(a[5, 3], philox.uniform(7, 3, 5))
