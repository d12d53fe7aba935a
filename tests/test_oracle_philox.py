"""Pins the oracle's Philox4x32-10 to the published known-answer vectors."""

import numpy as np

from oracle.philox import philox4x32_10, seed_key


def test_known_answers(golden):
    rows = golden("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for row in rows:
        vals = [int(t, 16) for t in row]
        out = philox4x32_10(*vals[:6])
        assert [int(w) for w in out] == vals[6:]


def test_vectorised_matches_scalar():
    c0 = np.arange(17, dtype=np.uint64)
    vec = philox4x32_10(c0, 3, 1, 0, 0xDEADBEEF, 7)
    for i in range(17):
        sc = philox4x32_10(i, 3, 1, 0, 0xDEADBEEF, 7)
        assert [int(w[i]) for w in vec] == [int(w) for w in sc]


def test_seed_split():
    assert seed_key(0x0123456789ABCDEF) == (0x89ABCDEF, 0x01234567)
    assert seed_key(42) == (42, 0)
