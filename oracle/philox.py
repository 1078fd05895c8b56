"""Philox4x32-10 and the draw conventions of the sparse FFT (oracle side).

Philox4x32-10 follows its published definition (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11): a 4x32-bit counter and
a 2x32-bit key; each of the 10 rounds multiplies words 0 and 2 by the round
multipliers, XORs the high halves with the other words and the key, and the
key is bumped by the Weyl constants between rounds.

Draw conventions (shared, by specification, with the CUDA library; the two
implementations share no code):

  key     = (seed mod 2^32, floor(seed / 2^32) mod 2^32)
  counter = (c0, c1, c2, purpose * 2^24 + t)
  out     = 4 words x0..x3;  u64a = x0 + 2^32 x1,  u64b = x2 + 2^32 x3

  uniform in [0,1)          : (u64a >> 11) * 2^-53
  generating vector entry   : 1 + (u64a mod (M - 1))       (in [1, M-1])
  normal pair (Box-Muller)  : u1 = ((u64a >> 11) + 1) 2^-53, u2 = (u64b >> 11) 2^-53,
                              R = sqrt(-2 ln u1), g1 = R cos(2 pi u2), g2 = R sin(2 pi u2)

Purposes (t is the 1-based dimension increment, i the 0-based repetition):
  1 anchor of a 1-D detection line   c0 = component j (0-based), c1 = 0, c2 = i
  2 anchor of a lattice pass         c0 = component j (0-based), c1 = 0, c2 = i
  3 generating-vector entry          c0 = component j, c1 = lattice l (0-based), c2 = attempt
  4 noise of a 1-D line sample       c0 = node, c1 = 0, c2 = i
  5 noise of a lattice sample        c0 = node j, c1 = l (0 for the shared node 0), c2 = i
"""

from __future__ import annotations

import numpy as np

MASK32 = np.uint64(0xFFFFFFFF)
ROUND_MUL0 = np.uint64(0xD2511F53)
ROUND_MUL1 = np.uint64(0xCD9E8D57)
WEYL0 = np.uint64(0x9E3779B9)
WEYL1 = np.uint64(0xBB67AE85)

ANCHOR_LINE = 1
ANCHOR_LAT = 2
ZVEC = 3
NOISE_LINE = 4
NOISE_LAT = 5

TWO_M53 = 2.0 ** -53


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10 block function; arguments are array-likes of
    32-bit values (held in uint64), returns the four output words."""
    c0 = np.asarray(c0, dtype=np.uint64) & MASK32
    c1 = np.asarray(c1, dtype=np.uint64) & MASK32
    c2 = np.asarray(c2, dtype=np.uint64) & MASK32
    c3 = np.asarray(c3, dtype=np.uint64) & MASK32
    k0 = np.asarray(k0, dtype=np.uint64) & MASK32
    k1 = np.asarray(k1, dtype=np.uint64) & MASK32
    c0, c1, c2, c3, k0, k1 = np.broadcast_arrays(c0, c1, c2, c3, k0, k1)
    for rnd in range(10):
        if rnd:
            k0 = (k0 + WEYL0) & MASK32
            k1 = (k1 + WEYL1) & MASK32
        p0 = ROUND_MUL0 * c0          # < 2^64: exact in uint64
        p1 = ROUND_MUL1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def _u64pair(seed: int, purpose: int, t: int, c0, c1, c2):
    k0 = seed & 0xFFFFFFFF
    k1 = (seed >> 32) & 0xFFFFFFFF
    c3 = (purpose << 24) | (t & 0xFFFFFF)
    x0, x1, x2, x3 = philox4x32_10(c0, c1, c2, c3, k0, k1)
    a = x0 | (x1 << np.uint64(32))
    b = x2 | (x3 << np.uint64(32))
    return a, b


def uniform(seed: int, purpose: int, t: int, c0, c1, c2) -> np.ndarray:
    a, _ = _u64pair(seed, purpose, t, c0, c1, c2)
    return (a >> np.uint64(11)).astype(np.float64) * TWO_M53


def zvec(seed: int, t: int, lattice: int, attempt: int, M: int, redraw: int = 0) -> np.ndarray:
    """Generating vector z in [1, M-1]^t of lattice `lattice` (0-based) of the
    given attempt at dimension increment t (Algorithm 1, random choice of z).
    redraw r > 0 is the r-th replacement draw of the redraw rule (the remark
    after Algorithm 1): counter word c2 = attempt + r 2^16."""
    j = np.arange(t, dtype=np.uint64)
    a, _ = _u64pair(seed, ZVEC, t, j, lattice, attempt + (redraw << 16))
    return (np.uint64(1) + a % np.uint64(M - 1)).astype(np.int64)


def normal_pairs(seed: int, purpose: int, t: int, c0, c1, c2):
    a, b = _u64pair(seed, purpose, t, c0, c1, c2)
    u1 = ((a >> np.uint64(11)).astype(np.float64) + 1.0) * TWO_M53
    u2 = (b >> np.uint64(11)).astype(np.float64) * TWO_M53
    R = np.sqrt(-2.0 * np.log(u1))
    return R * np.cos(2.0 * np.pi * u2), R * np.sin(2.0 * np.pi * u2)
