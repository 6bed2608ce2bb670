"""Counter-based random draws of the method, restated from their published
definitions.  TEST INFRASTRUCTURE ONLY.

Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
easy as 1, 2, 3", SC'11): a 4-word 64-bit counter and a 2-word key; each
of the 10 rounds multiplies counter words 0 and 2 by two fixed odd
constants, mixes the high/low halves of the 128-bit products with the
other counter words and the key, and then bumps the key by two Weyl
constants.  All arithmetic here is on Python integers.

Draws used by the method (the paper's randomized HSS needs random vectors,
Section 1 and Section 3.1; the two-means seeding needs one uniform pick and
one distance-weighted pick, Section 4.3):

* random block R (n x r, N(0,1)): key = (seed, STREAM_R), counter =
  (row j, column group c // 4, 0, 0); the four output words give columns
  4g..4g+3 by two Box-Muller pairs (w0, w1) and (w2, w3).
* two-means seeding of the node covering rows [b, b + m): key =
  (seed, STREAM_CLUSTER), counter = (b, m, 0, 0); words w0 and w1.
"""
from __future__ import annotations

import math

import numpy as np

MASK64 = (1 << 64) - 1
# Philox4x64 round multipliers and Weyl key increments (Salmon et al. 2011).
PHILOX_M0 = 0xD2E7470EE14C6C93
PHILOX_M1 = 0xCA5A826395121157
PHILOX_W0 = 0x9E3779B97F4A7C15
PHILOX_W1 = 0xBB67AE8584CAA73B

STREAM_R = 0x52
STREAM_CLUSTER = 0x43


def philox4x64(counter, key, rounds: int = 10):
    c0, c1, c2, c3 = (int(v) & MASK64 for v in counter)
    k0, k1 = (int(v) & MASK64 for v in key)
    for _ in range(rounds):
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> 64, p0 & MASK64
        hi1, lo1 = p1 >> 64, p1 & MASK64
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + PHILOX_W0) & MASK64
        k1 = (k1 + PHILOX_W1) & MASK64
    return c0, c1, c2, c3


def mulhi64(a: int, b: int) -> int:
    """floor(a * b / 2^64): maps a uniform 64-bit word onto [0, b)."""
    return (int(a) * int(b)) >> 64


def u01(w: int) -> float:
    """Uniform in (0, 1) from the top 53 bits of a 64-bit word."""
    return ((int(w) >> 11) + 0.5) * (2.0 ** -53)


def box_muller(w_a: int, w_b: int):
    """Two independent N(0,1) values from two uniform words (Box-Muller)."""
    u1, u2 = u01(w_a), u01(w_b)
    rho = math.sqrt(-2.0 * math.log(u1))
    th = 2.0 * math.pi * u2
    return rho * math.cos(th), rho * math.sin(th)


def gaussian_block(n: int, r: int, seed: int, col0: int = 0) -> np.ndarray:
    """Columns [col0, col0 + r) of the method's random block R, in FP64.

    col0 must be a multiple of 4 (columns come in groups of four).
    """
    assert col0 % 4 == 0
    out = np.empty((n, r))
    g0, g1 = col0 // 4, (col0 + r + 3) // 4
    for j in range(n):
        for g in range(g0, g1):
            w = philox4x64((j, g, 0, 0), (seed, STREAM_R))
            z = box_muller(w[0], w[1]) + box_muller(w[2], w[3])
            for t in range(4):
                c = 4 * g + t - col0
                if 0 <= c < r:
                    out[j, c] = z[t]
    return out


def cluster_words(seed: int, begin: int, m: int):
    w = philox4x64((begin, m, 0, 0), (seed, STREAM_CLUSTER))
    return w[0], w[1]
