"""Counter-based Gaussian test matrices: Philox4x32-10 + Box-Muller (FP64).

TEST INFRASTRUCTURE -- part of the FP64 oracle.  Only tests, the smoke check
and the benchmark's CPU-baseline leg use it; the product path never does.

The compression draws a Gaussian test matrix Omega with i.i.d. N(0, 1)
entries (Sec. II, Alg. 1, first step).  So that the oracle and the GPU can
draw the *same* matrix without passing it around, both sides implement one
counter-based generator from its published definition:

* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
  easy as 1, 2, 3", SC'11): a 4 x 32-bit counter and a 2 x 32-bit key; each
  of 10 rounds multiplies counter words 0 and 2 by the constants
  0xD2511F53 and 0xCD9E8D57 (64-bit products split into hi/lo), mixes the
  high halves with the other two words and the key, and bumps the key by the
  Weyl constants 0x9E3779B9, 0xBB67AE85 between rounds.
* Box-Muller (1958): uniforms u1, u2 in (0, 1) give
  z0 = sqrt(-2 ln u1) cos(2 pi u2), z1 = sqrt(-2 ln u1) sin(2 pi u2).

Stream layout (the library's convention, independent of the paper):
  key      = (seed mod 2^32, seed >> 32)
  counter  = (b mod 2^32, b >> 32, stream, 0) for block b = e // 4 of the
             row-major element index e of the matrix
  uniforms u_i = (x_i + 0.5) / 2^32 for the 4 output words x_0..x_3
  normals  (z0, z1) from (u_0, u_1), (z2, z3) from (u_2, u_3);
  element e takes z_{e mod 4}.
Stream 0 draws Omega (n x d, used for the left compression L), stream 1
draws Psi (m x d, used for the right compression R).
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """Philox4x32-10 on arrays of counters.

    ctr: (N, 4) uint32-valued, key: (N, 2) or (2,) uint32-valued.
    Returns (N, 4) uint32.
    """
    c = [np.asarray(ctr[:, i], dtype=np.uint64) for i in range(4)]
    key = np.asarray(key, dtype=np.uint64)
    if key.ndim == 1:
        k0 = np.full_like(c[0], key[0])
        k1 = np.full_like(c[0], key[1])
    else:
        k0 = key[:, 0].copy()
        k1 = key[:, 1].copy()
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c[0]          # < 2^64, exact in uint64
        p1 = M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return np.stack(c, axis=1).astype(np.uint32)


def raw_words(seed: int, stream: int, nblocks: int, first_block: int = 0):
    """The 4 x uint32 outputs of blocks first_block .. first_block+nblocks-1."""
    b = np.arange(first_block, first_block + nblocks, dtype=np.uint64)
    ctr = np.stack([b & MASK, b >> np.uint64(32),
                    np.full_like(b, stream), np.zeros_like(b)], axis=1)
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF],
                   dtype=np.uint64)
    return philox4x32_10(ctr, key)


def gaussian_matrix(seed: int, stream: int, rows: int, cols: int) -> np.ndarray:
    """rows x cols FP64 matrix of N(0, 1) draws on the given stream."""
    count = rows * cols
    nblocks = (count + 3) // 4
    x = raw_words(seed, stream, nblocks).astype(np.float64)
    u = (x + 0.5) * 2.0 ** -32
    rad = np.sqrt(-2.0 * np.log(u[:, 0::2]))        # (nblocks, 2)
    ang = 2.0 * np.pi * u[:, 1::2]
    z = np.empty((nblocks, 4))
    z[:, 0] = rad[:, 0] * np.cos(ang[:, 0])
    z[:, 1] = rad[:, 0] * np.sin(ang[:, 0])
    z[:, 2] = rad[:, 1] * np.cos(ang[:, 1])
    z[:, 3] = rad[:, 1] * np.sin(ang[:, 1])
    return z.reshape(-1)[:count].reshape(rows, cols)


def test_matrices(seed: int, m: int, n: int, d: int):
    """(Omega n x d from stream 0, Psi m x d from stream 1)."""
    return gaussian_matrix(seed, 0, n, d), gaussian_matrix(seed, 1, m, d)
