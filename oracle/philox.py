"""Oracle: Philox4x32-10 counter-based RNG and the Gaussian test matrix of App. A.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

App. A (Alg. randomized_nystrom, first step) draws Omega = randn(p, ell).  The
paper does not name a generator; both this oracle and the CUDA library draw it
from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
as 1, 2, 3", SC'11), each side written from that published definition:

  one round:  (hi0, lo0) = M0 * c0,  (hi1, lo1) = M1 * c2   (32x32 -> 64-bit products)
              c <- (hi1 ^ c1 ^ k0,  lo1,  hi0 ^ c3 ^ k1,  lo0)
  key schedule between rounds: k0 += W0, k1 += W1 (mod 2^32)
  M0 = 0xD2511F53, M1 = 0xCD9E8D57, W0 = 0x9E3779B9, W1 = 0xBB67AE85, 10 rounds.

Counter layout of the test matrix (a reading; the paper is silent): entry
Omega[i, j] of column j, row i belongs to the row pair m = i // 2; the block
    counter = (m, j, step mod 2^32, step >> 32),  key = (seed mod 2^32, seed >> 32)
gives four words x0..x3.  Two 52-bit uniforms
    u1 = ((x0 << 20) ^ (x1 >> 12) + 1/2) 2^-52,  u2 = ((x2 << 20) ^ (x3 >> 12) + 1/2) 2^-52
(every value of (m + 1/2) 2^-52 with m < 2^52 is exact and lies strictly in (0, 1))
feed Box-Muller (Box & Muller 1958):
    Omega[2m, j] = sqrt(-2 ln u1) cos(2 pi u2),   Omega[2m+1, j] = sqrt(-2 ln u1) sin(2 pi u2).

The sampling test matrix draws one uniform per parameter index j from the block at
    counter = (j, 2^32 - 1, step mod 2^32, step >> 32),  key as above,
u_j = ((x0 << 20) ^ (x1 >> 12) + 1/2) 2^-52 (column 2^32 - 1 is never a Gaussian column).
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """Philox4x32-10 on arrays: ctr (..., 4) and key (..., 2) of uint32 -> (..., 4) uint32."""
    c = [np.asarray(ctr[..., i], dtype=np.uint64) for i in range(4)]
    k0 = np.asarray(key[..., 0], dtype=np.uint64)
    k1 = np.asarray(key[..., 1], dtype=np.uint64)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = M0 * c[0]
        p1 = M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return np.stack([x.astype(np.uint32) for x in c], axis=-1)


def uniform52(a, b):
    """(0,1) double from two 32-bit words: m = (a << 20) ^ (b >> 12) < 2^52, u = (m + 1/2) 2^-52."""
    m = (np.asarray(a, dtype=np.uint64) << np.uint64(20)) ^ (np.asarray(b, dtype=np.uint64) >> np.uint64(12))
    m = m & np.uint64((1 << 52) - 1)
    return (m.astype(np.float64) + 0.5) * 2.0 ** -52


def box_muller(u1, u2):
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)


def gaussian_test_matrix(p: int, ell: int, seed: int, step: int) -> np.ndarray:
    """Omega (p, ell), standard normal entries from the counter layout above."""
    npairs = (p + 1) // 2
    m = np.arange(npairs, dtype=np.uint64)
    j = np.arange(ell, dtype=np.uint64)
    mm, jj = np.meshgrid(m, j, indexing="ij")
    ctr = np.stack([mm, jj,
                    np.full_like(mm, np.uint64(step) & MASK32),
                    np.full_like(mm, np.uint64(step) >> np.uint64(32))], axis=-1)
    key = np.stack([np.full_like(mm, np.uint64(seed) & MASK32),
                    np.full_like(mm, np.uint64(seed) >> np.uint64(32))], axis=-1)
    x = philox4x32_10(ctr, key)
    z0, z1 = box_muller(uniform52(x[..., 0], x[..., 1]), uniform52(x[..., 2], x[..., 3]))
    out = np.empty((2 * npairs, ell))
    out[0::2] = z0
    out[1::2] = z1
    return out[:p]


def sampling_uniforms(p: int, seed: int, step: int) -> np.ndarray:
    """u_j in (0, 1), j < p, of the sampling test matrix (counter layout above)."""
    j = np.arange(p, dtype=np.uint64)
    ctr = np.stack([j, np.full_like(j, np.uint64(0xFFFFFFFF)),
                    np.full_like(j, np.uint64(step) & MASK32),
                    np.full_like(j, np.uint64(step) >> np.uint64(32))], axis=-1)
    key = np.stack([np.full_like(j, np.uint64(seed) & MASK32),
                    np.full_like(j, np.uint64(seed) >> np.uint64(32))], axis=-1)
    x = philox4x32_10(ctr, key)
    return uniform52(x[..., 0], x[..., 1])


def rpchol_uniforms(p: int, b: int, rnd: int, seed: int, step: int) -> np.ndarray:
    """u (p, b) of round rnd of block RPCholesky: counter (j, 2^30 + rnd b + k, step mod 2^32,
    step >> 32), words (x0, x1) as in sampling_uniforms."""
    j = np.arange(p, dtype=np.uint64)
    k = np.arange(b, dtype=np.uint64)
    jj, kk = np.meshgrid(j, k, indexing="ij")
    ctr = np.stack([jj, np.uint64(1 << 30) + np.uint64(rnd * b) + kk,
                    np.full_like(jj, np.uint64(step) & MASK32),
                    np.full_like(jj, np.uint64(step) >> np.uint64(32))], axis=-1)
    key = np.stack([np.full_like(jj, np.uint64(seed) & MASK32),
                    np.full_like(jj, np.uint64(seed) >> np.uint64(32))], axis=-1)
    x = philox4x32_10(ctr, key)
    return uniform52(x[..., 0], x[..., 1])


def power_start(p: int, seed: int, step: int) -> np.ndarray:
    """Start vector of the power method: the Gaussian column with counter word 2^32 - 2."""
    npairs = (p + 1) // 2
    m = np.arange(npairs, dtype=np.uint64)
    ctr = np.stack([m, np.full_like(m, np.uint64(0xFFFFFFFE)),
                    np.full_like(m, np.uint64(step) & MASK32),
                    np.full_like(m, np.uint64(step) >> np.uint64(32))], axis=-1)
    key = np.stack([np.full_like(m, np.uint64(seed) & MASK32),
                    np.full_like(m, np.uint64(seed) >> np.uint64(32))], axis=-1)
    x = philox4x32_10(ctr, key)
    z0, z1 = box_muller(uniform52(x[..., 0], x[..., 1]), uniform52(x[..., 2], x[..., 3]))
    out = np.empty(2 * npairs)
    out[0::2] = z0
    out[1::2] = z1
    return out[:p]
