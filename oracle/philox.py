"""Philox4x32-10 in plain numpy (test infrastructure; see ``oracle/__init__``).

Definition (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11, Sec. 3 "Philox"): a 128-bit counter (c0, c1, c2, c3) and a
64-bit key (k0, k1) go through 10 rounds. One round multiplies c0 and c2 by
the two published multipliers, keeps both halves of each 64-bit product and
mixes the high halves with the other two counter words and the key:

    (hi0, lo0) = M0 * c0          (hi1, lo1) = M1 * c2
    c <- (hi1 ^ c1 ^ k0,  lo1,  hi0 ^ c3 ^ k1,  lo0)

Between rounds the key is bumped by the two Weyl constants. The paper of the
method uses Murmurhash as its hash (Sec. "McKernel", item "Binary B"); any
counter-based hash satisfies it, and Philox is the one this library uses.

Pinned by: the Random123 known-answer vectors (tests/golden/philox4x32_10_kat.txt).
"""

import numpy as np

PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
MASK32 = 0xFFFFFFFF


def _u32(a):
    return np.asarray(a, dtype=np.uint64) & np.uint64(MASK32)


def _mulhilo(m, c):
    p = np.uint64(m) * c  # both < 2**32, product fits in 64 bits
    return p >> np.uint64(32), p & np.uint64(MASK32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Return the four uint32 output words for counters (c0..c3) and key (k0, k1).

    All arguments broadcast against each other; the result is a tuple of four
    uint32 arrays of the broadcast shape.
    """
    c0, c1, c2, c3, k0, k1 = np.broadcast_arrays(
        _u32(c0), _u32(c1), _u32(c2), _u32(c3), _u32(k0), _u32(k1))
    c0, c1, c2, c3 = c0.copy(), c1.copy(), c2.copy(), c3.copy()
    k0, k1 = k0.copy(), k1.copy()
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + np.uint64(PHILOX_W0)) & np.uint64(MASK32)
            k1 = (k1 + np.uint64(PHILOX_W1)) & np.uint64(MASK32)
        hi0, lo0 = _mulhilo(PHILOX_M0, c0)
        hi1, lo1 = _mulhilo(PHILOX_M1, c2)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return tuple(w.astype(np.uint32) for w in (c0, c1, c2, c3))


def seed_key(seed):
    """Split a 64-bit seed into the Philox key (low word, high word)."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & MASK32, seed >> 32
