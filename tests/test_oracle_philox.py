"""Pins of the oracle's Philox4x32-10 against the published known-answer vectors of the
Random123 distribution (Salmon et al., SC'11), which both the initial-state perturbation
(App. A) and the Metropolis tests draw from."""
import numpy as np

from oracle import philox

KAT = [  # (counter, key, output) -- philox4x32, 10 rounds
    ((0, 0, 0, 0), (0, 0), (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
    ((0xffffffff,) * 4, (0xffffffff,) * 2, (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
    ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
     (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1)),
]


def test_known_answers():
    for ctr, key, out in KAT:
        got = tuple(int(x) for x in philox.philox4x32_10(ctr, key))
        assert got == out


def test_vectorised_matches_scalar():
    c0 = np.arange(17, dtype=np.uint64)
    v = philox.uniform(12345, c0, c0 * 3, np.zeros_like(c0), philox.TAG_MC)
    for k in range(17):
        assert v[k] == philox.uniform(12345, int(k), int(3 * k), 0, philox.TAG_MC)


def test_uniform_range_and_moments():
    c0 = np.arange(200000, dtype=np.uint64)
    u = philox.uniform(7, c0, np.zeros_like(c0), np.zeros_like(c0), philox.TAG_INIT)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / u.size)
    assert abs(u.var() - 1 / 12) < 1e-3
