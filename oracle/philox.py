"""Philox4x32-10 counter-based generator and the Box-Muller map, in numpy,
written from the published definition (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11).  TEST
INFRASTRUCTURE ONLY: the reference for the library's Gaussian test matrix
Omega (Algorithm 4, line 1).

Round: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2 (32 x 32 -> 64 bit),
c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); between rounds the key is
bumped by the Weyl constants (W0, W1).  Ten rounds.
Pinned by the published known-answer vectors (tests/golden/philox_kat.json).
"""
import numpy as np

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """ctr: (N, 4) uint32-valued array; key: (k0, k1).  Returns (N, 4) uint32."""
    c = np.asarray(ctr, dtype=np.uint64).reshape(-1, 4)
    c0, c1, c2, c3 = (c[:, i].copy() for i in range(4))
    k0, k1 = np.uint64(key[0] & MASK), np.uint64(key[1] & MASK)
    for _ in range(10):
        p0 = c0 * np.uint64(M0)
        p1 = c2 * np.uint64(M1)
        hi0, lo0 = p0 >> np.uint64(32), p0 & np.uint64(MASK)
        hi1, lo1 = p1 >> np.uint64(32), p1 & np.uint64(MASK)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + np.uint64(W0)) & np.uint64(MASK)
        k1 = (k1 + np.uint64(W1)) & np.uint64(MASK)
    return np.stack([c0, c1, c2, c3], axis=1).astype(np.uint32)


def gaussian(rows, cols, seed):
    """The library's Omega: element e uses counter (e // 4, 0, 0, 0) (64-bit
    index split low/high into the first two words), key (seed low, seed
    high), word e % 4 -> u = ((w >> 8) + 1) / 2^24 in (0, 1]; words (0, 1)
    and (2, 3) form Box-Muller pairs r cos(2 pi u'), r sin(2 pi u'),
    r = sqrt(-2 ln u).  Returned in float64."""
    total = rows * cols
    groups = (total + 3) // 4
    g = np.arange(groups, dtype=np.uint64)
    ctr = np.zeros((groups, 4), dtype=np.uint64)
    ctr[:, 0] = g & np.uint64(MASK)
    ctr[:, 1] = g >> np.uint64(32)
    w = philox4x32_10(ctr, (seed & MASK, (seed >> 32) & MASK)).astype(np.float64)
    u = (np.floor(w / 256.0) + 1.0) / 16777216.0
    r0 = np.sqrt(-2.0 * np.log(u[:, 0]))
    r1 = np.sqrt(-2.0 * np.log(u[:, 2]))
    t0 = 2 * np.pi * u[:, 1]
    t1 = 2 * np.pi * u[:, 3]
    z = np.stack([r0 * np.cos(t0), r0 * np.sin(t0), r1 * np.cos(t1), r1 * np.sin(t1)], axis=1)
    return z.reshape(-1)[:total].reshape(rows, cols)
