"""Philox4x32-10 counter-based generator, written from its published definition
(Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11).

TEST INFRASTRUCTURE: part of the FP64 CPU oracle.  Only tests, the smoke check
and the CPU-baseline leg of the benchmark may use it.

The white-noise orbitals of the stochastic resolution of the identity (Sec. 2.1:
the zeta-bar and eta-bar start orbitals) are drawn from this generator on both
sides of the parity check, so that runs at equal seeds see the same noise.

Definition (per the SC'11 paper): a 4-word counter (c0,c1,c2,c3) and a 2-word key
(k0,k1) of W-bit words go through R rounds.  One round multiplies c0 and c2 by the
round multipliers, keeping both halves of each double-width product, and mixes
    (c0,c1,c2,c3) <- (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0))
and between rounds the key is bumped by the Weyl constants (k0 += W0, k1 += W1).
"""
import numpy as np

# Multipliers and Weyl constants of the published 32-bit and 64-bit variants.
PHILOX_CONST = {
    32: dict(M0=0xD2511F53, M1=0xCD9E8D57, W0=0x9E3779B9, W1=0xBB67AE85),
    64: dict(M0=0xD2E7470EE14C6C93, M1=0xCA5A826395121157,
             W0=0x9E3779B97F4A7C15, W1=0xBB67AE8584CAA73B),
}


def philox_scalar(ctr, key, rounds=10, width=32):
    """Philox4xW-R on one counter with Python integers (any word width).

    Slow and obviously correct; used to pin the vectorised 32-bit version and,
    at width 64, to check the round structure against an independent
    implementation of the 64-bit variant.
    """
    c = PHILOX_CONST[width]
    mask = (1 << width) - 1
    c0, c1, c2, c3 = [int(x) & mask for x in ctr]
    k0, k1 = [int(x) & mask for x in key]
    for r in range(rounds):
        if r > 0:
            k0 = (k0 + c['W0']) & mask
            k1 = (k1 + c['W1']) & mask
        p0 = c['M0'] * c0
        p1 = c['M1'] * c2
        hi0, lo0 = p0 >> width, p0 & mask
        hi1, lo1 = p1 >> width, p1 & mask
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return (c0, c1, c2, c3)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10 over uint32 arrays (broadcasting).  Returns 4 uint32 arrays."""
    M0 = np.uint64(PHILOX_CONST[32]['M0'])
    M1 = np.uint64(PHILOX_CONST[32]['M1'])
    W0 = PHILOX_CONST[32]['W0']
    W1 = PHILOX_CONST[32]['W1']
    m32 = np.uint64(0xFFFFFFFF)
    s32 = np.uint64(32)
    c0, c1, c2, c3 = [np.asarray(x, dtype=np.uint64) & m32 for x in (c0, c1, c2, c3)]
    k0 = int(k0) & 0xFFFFFFFF
    k1 = int(k1) & 0xFFFFFFFF
    for r in range(10):
        if r > 0:
            k0 = (k0 + W0) & 0xFFFFFFFF
            k1 = (k1 + W1) & 0xFFFFFFFF
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> s32, p0 & m32
        hi1, lo1 = p1 >> s32, p1 & m32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1,
                          hi0 ^ c3 ^ np.uint64(k1), lo0)
    return tuple(x.astype(np.uint32) for x in (c0, c1, c2, c3))


def rademacher_words(seed, stream, sample, vector, n_points):
    """Sign bits for one white-noise vector.

    Point g of vector `vector` of Monte-Carlo sample `sample` uses counter
    (g // 4, vector, sample, stream) and key (seed mod 2^32, seed div 2^32); the
    sign is taken from the top bit of output word g mod 4 (bit set -> -1).
    Returns an int8 array of +1/-1.
    """
    blk = np.arange((n_points + 3) // 4, dtype=np.uint64)
    out = philox4x32_10(blk, np.uint64(vector), np.uint64(sample), np.uint64(stream),
                        seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    words = np.stack(out, axis=-1)  # [nblk, 4]
    g = np.arange(n_points)
    w = words[g // 4, g % 4]
    return np.where((w >> np.uint32(31)) != 0, -1, 1).astype(np.int8)
