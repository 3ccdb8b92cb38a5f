"""Philox-4x32-10, the counter-based generator behind every random draw.

Oracle (test infrastructure; see ``oracle/__init__.py``).

The paper draws its hash, signs and Gaussians from per-thread STL engines
(Sec. 5.1), so its results depend on the thread count, and it names the
Random123 counter-based generators (Salmon, Moraes, Dror & Shaw, "Parallel
random numbers: as easy as 1, 2, 3", SC'11) as the planned replacement.  This
module is Philox-4x32 with 10 rounds as defined in that paper: a 128-bit
counter (c0..c3) and a 64-bit key (k0, k1); each round multiplies c0 and c2
by the two Philox multipliers, recombines the high/low halves with the other
two words and the key, and the key is advanced by the two Weyl constants
between rounds.  Pinned by the published known-answer vectors
(``tests/golden/philox4x32_10_kat.txt``).
"""
import numpy as np

PHILOX_M4x32_0 = 0xD2511F53
PHILOX_M4x32_1 = 0xCD9E8D57
PHILOX_W32_0 = 0x9E3779B9
PHILOX_W32_1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)
_SHIFT32 = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Return the four 32-bit output words of Philox-4x32-10.

    All arguments broadcast (numpy arrays or Python ints, taken mod 2**32).
    Output: tuple of four uint32 arrays.
    """
    c = [np.asarray(x, dtype=np.uint64) & _MASK32 for x in (c0, c1, c2, c3)]
    c = np.broadcast_arrays(*c)
    c = [x.copy() for x in c]
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK32
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK32
    m0 = np.uint64(PHILOX_M4x32_0)
    m1 = np.uint64(PHILOX_M4x32_1)
    for rnd in range(10):
        if rnd > 0:  # key schedule: bump by the Weyl constants between rounds
            k0 = (k0 + np.uint64(PHILOX_W32_0)) & _MASK32
            k1 = (k1 + np.uint64(PHILOX_W32_1)) & _MASK32
        p0 = c[0] * m0  # 32x32 -> 64-bit product, exact in uint64
        p1 = c[2] * m1
        hi0, lo0 = p0 >> _SHIFT32, p0 & _MASK32
        hi1, lo1 = p1 >> _SHIFT32, p1 & _MASK32
        c = [(hi1 ^ c[1] ^ k0) & _MASK32, lo1, (hi0 ^ c[3] ^ k1) & _MASK32, lo0]
    return tuple(x.astype(np.uint32) for x in c)


def split_seed(seed):
    """64-bit seed -> Philox key (k0 = low word, k1 = high word)."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32
