"""Counter-based random stream (oracle; test infrastructure).

Alg. 3's randomMatrix draws i.i.d. N(0,1) entries without naming a generator.
Reading: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
as easy as 1, 2, 3", SC'11) followed by the Box-Muller transform, so that the
CPU oracle and the GPU kernels can draw the same matrix independently.

Philox4x32-10, from the published definition: ten rounds of
  (c0, c1, c2, c3) -> (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0))
with M0 = 0xD2511F53, M1 = 0xCD9E8D57, the key bumped by (0x9E3779B9, 0xBB67AE85)
between rounds.

Gaussian entry (i, c) of a sample block: counter (i, c // 2, block_id, pass | attempt << 16),
key (seed mod 2^32, seed >> 32); words (w0, w1) give the even column and (w2, w3)
the odd one, via u1 = (w + 1) 2^-32, u2 = w' 2^-32, z = sqrt(-2 ln u1) cos(2 pi u2).
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """ctr: uint32 array [..., 4]; key: uint32 array [..., 2] (broadcast). Returns uint32 [..., 4]."""
    c = [np.asarray(ctr, dtype=np.uint64)[..., i] for i in range(4)]
    k0 = np.asarray(key, dtype=np.uint64)[..., 0] + np.zeros_like(c[0])
    k1 = np.asarray(key, dtype=np.uint64)[..., 1] + np.zeros_like(c[0])
    for r in range(10):
        if r > 0:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c[0]
        p1 = M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return np.stack(c, axis=-1).astype(np.uint32)


def gaussian_block(m: int, ncols: int, seed: int, block_id: int, pass_: int, attempt: int) -> np.ndarray:
    """m x ncols standard normal matrix (ncols even) of one sample pass."""
    assert ncols % 2 == 0
    i = np.arange(m, dtype=np.uint64)[:, None]
    cp = np.arange(ncols // 2, dtype=np.uint64)[None, :]
    ctr = np.zeros((m, ncols // 2, 4), dtype=np.uint64)
    ctr[..., 0] = i
    ctr[..., 1] = cp
    ctr[..., 2] = np.uint64(block_id)
    ctr[..., 3] = np.uint64(pass_) | (np.uint64(attempt) << np.uint64(16))
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint64)
    w = philox4x32_10(ctr, key).astype(np.float64)
    two32 = 2.0 ** -32
    z_even = np.sqrt(-2.0 * np.log((w[..., 0] + 1.0) * two32)) * np.cos(2.0 * np.pi * (w[..., 1] * two32))
    z_odd = np.sqrt(-2.0 * np.log((w[..., 2] + 1.0) * two32)) * np.cos(2.0 * np.pi * (w[..., 3] * two32))
    out = np.empty((m, ncols))
    out[:, 0::2] = z_even
    out[:, 1::2] = z_odd
    return out
