"""Philox4x32-10 and Box-Muller normals (oracle side).

Philox4x32-R is the counter-based generator of Salmon, Moraes, Dror & Shaw,
"Parallel random numbers: as easy as 1, 2, 3" (SC'11): a 4 x 32-bit counter is
mixed with a 2 x 32-bit key by R rounds of two 32x32->64 multiplications, the
key being bumped by the Weyl constants between rounds.  Written here from that
published definition with plain numpy uint64 arithmetic.

The paper draws its Brownian increments with MATLAB randn (Section 3,
"Implementation"); a counter-based generator replaces it so that every path is
a pure function of (seed, global path index, fine index) on both sides.

Counter layout used by this project (both sides implement it independently):
    key     = (seed & 0xffffffff, seed >> 32)
    counter = (pair index j, path & 0xffffffff, path >> 32, stream tag)
One call gives four words (x0, x1, x2, x3) -> two 52-bit uniforms
    u1 = ((x1:x0 >> 12) + 0.5) * 2^-52,   u2 = ((x3:x2 >> 12) + 0.5) * 2^-52
on the lattice (k + 1/2) 2^-52, k = 0..2^52-1, strictly inside (0, 1) and
computed without rounding in float64, and Box-Muller turns them into the standard
normals of fine indices 2j and 2j+1:
    z_{2j}   = sqrt(-2 log u1) cos(2 pi u2)
    z_{2j+1} = sqrt(-2 log u1) sin(2 pi u2)
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)

STREAM_BROWNIAN = 0


def philox4x32(ctr, key, rounds: int = 10):
    """Philox4x32-`rounds` bijection.

    ctr: tuple of four uint32 arrays (broadcastable), key: tuple of two uint32.
    Returns a tuple of four uint32 arrays.
    """
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & MASK32 for c in ctr)
    k0, k1 = (np.asarray(k, dtype=np.uint64) & MASK32 for k in key)
    for r in range(rounds):
        if r > 0:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = M0 * c0            # full 64-bit product (both factors < 2^32)
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)
    return tuple(c.astype(np.uint32) for c in (c0, c1, c2, c3))


def brownian_words(seed: int, path: int, pairs, tag: int = STREAM_BROWNIAN):
    """Raw Philox words for pair indices `pairs` of global path `path`."""
    j = np.asarray(pairs, dtype=np.uint64)
    key = (np.uint64(seed & 0xFFFFFFFF), np.uint64((seed >> 32) & 0xFFFFFFFF))
    ctr = (j, np.uint64(path & 0xFFFFFFFF), np.uint64((path >> 32) & 0xFFFFFFFF),
           np.uint64(tag))
    return philox4x32(ctr, key)


def uniform52(lo, hi):
    """Two 32-bit words -> uniform in (0, 1) from the top 52 bits of hi:lo."""
    u = (np.asarray(hi, dtype=np.uint64) << np.uint64(32)) | np.asarray(lo, dtype=np.uint64)
    return ((u >> np.uint64(12)).astype(np.float64) + 0.5) * 2.0 ** -52


def standard_normals(seed: int, path: int, n: int, tag: int = STREAM_BROWNIAN):
    """First n standard normals of a path's stream (Box-Muller on Philox pairs)."""
    npairs = (n + 1) // 2
    x0, x1, x2, x3 = brownian_words(seed, path, np.arange(npairs), tag)
    u1 = uniform52(x0, x1)
    u2 = uniform52(x2, x3)
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * npairs)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:n]
