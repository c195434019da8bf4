"""Counter-based generators and the mini-batch order, written from their
published definitions (oracle side; test infrastructure only).

* SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15, then two
  xor-shift-multiply mixing rounds.
* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
  as 1, 2, 3", SC 2011): ten rounds of two 32x32->64 multiplies on a 128-bit
  counter under a 64-bit key with Weyl key bumps.
* Box-Muller transform (Box and Muller, 1958).

The paper draws each mini-batch "without replacement from {1,...,N}" (Sec. 3,
after eq. approx-grad) and appends whole mini-batches cumulatively (Sec. 3,
"append one full MB").  Reading: one permutation of the training set is drawn
once; D_k is its first M_k entries.  The permutation is a Fisher-Yates shuffle
driven by SplitMix64, with the bounded draw j = floor(r * (i + 1) / 2^64).
"""
from __future__ import annotations

import math

import numpy as np

MASK64 = (1 << 64) - 1
MASK32 = (1 << 32) - 1


class SplitMix64:
    """Sequential SplitMix64 stream (Steele et al. 2014)."""

    GAMMA = 0x9E3779B97F4A7C15

    def __init__(self, seed: int):
        self.state = int(seed) & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + self.GAMMA) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def next_double(self) -> float:
        """Uniform double in [0, 1): the top 53 bits times 2^-53."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))


def fisher_yates_permutation(n: int, seed: int) -> np.ndarray:
    """Uniform random permutation of 0..n-1 (Durstenfeld's Fisher-Yates):
    for i = n-1 down to 1 swap a[i] with a[j], j uniform on 0..i.  The bounded
    draw is j = floor(r * (i+1) / 2^64) for a SplitMix64 output r."""
    a = list(range(n))
    g = SplitMix64(seed)
    for i in range(n - 1, 0, -1):
        r = g.next_u64()
        j = (r * (i + 1)) >> 64
        a[i], a[j] = a[j], a[i]
    return np.asarray(a, dtype=np.int32)


# ---------------------------------------------------------------- Philox4x32-10
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85


def philox4x32_10(counter, key):
    """One Philox4x32-10 block.  counter: four u32 words, key: two u32 words.
    Returns four u32 words."""
    c0, c1, c2, c3 = (int(v) & MASK32 for v in counter)
    k0, k1 = (int(v) & MASK32 for v in key)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> 32, p0 & MASK32
        hi1, lo1 = p1 >> 32, p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & MASK32, lo1, (hi0 ^ c3 ^ k1) & MASK32, lo0
    return (c0, c1, c2, c3)


def box_muller(x0: int, x1: int):
    """Two standard normals from two u32 words: u1 = (x0 + 1) 2^-32 in (0, 1],
    u2 = x1 2^-32 in [0, 1); r = sqrt(-2 ln u1); (r cos 2 pi u2, r sin 2 pi u2)."""
    u1 = (x0 + 1.0) * 2.0 ** -32
    u2 = x1 * 2.0 ** -32
    r = math.sqrt(-2.0 * math.log(u1))
    return r * math.cos(2.0 * math.pi * u2), r * math.sin(2.0 * math.pi * u2)


def philox_normals(seed: int, stream: int, iteration: int, n: int, offset: int = 0):
    """Normals number offset..offset+n-1 of the (seed, stream, iteration)
    sequence.  Normal e comes from block q = e // 4 with counter
    (q mod 2^32, q >> 32, iteration, stream) and key (seed mod 2^32, seed >> 32);
    words (x0, x1) give normals 4q and 4q+1, words (x2, x3) give 4q+2, 4q+3."""
    out = np.empty(n, dtype=np.float64)
    key = (seed & MASK32, (seed >> 32) & MASK32)
    cache_q, cache = -1, None
    for t in range(n):
        e = offset + t
        q, r = divmod(e, 4)
        if q != cache_q:
            x = philox4x32_10((q & MASK32, (q >> 32) & MASK32, iteration, stream), key)
            cache = box_muller(x[0], x[1]) + box_muller(x[2], x[3])
            cache_q = q
        out[t] = cache[r]
    return out
