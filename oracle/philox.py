"""Philox4x32-10 counter-based generator and the Gaussian compression matrix.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper draws a Gaussian i.i.d. (GIID) compression matrix Omega of size
l x m with unit-variance entries (Sec. 3, Alg. 3 and the opening steps of
Alg. 4) but does not name a generator.  Both sides of
this project implement the same published generator independently:

* Philox4x32 with 10 rounds, as defined by Salmon, Moraes, Dror and Shaw,
  "Parallel random numbers: as easy as 1, 2, 3", SC'11: a 4x32-bit counter,
  a 2x32-bit key, each round two 32x32->64-bit multiplications whose high
  halves are xored with the other counter words and the key, followed by a
  key bump by two Weyl constants.
* Two words give one uniform double in (0, 1) from their top 52 bits plus a
  half-step offset, two uniforms give two normals by Box and Muller (1958).

Omega layout contract (shared with the CUDA generator by specification only):
entry Omega[i, r] (row i < l, column r < m) comes from the Philox block with
key (seed mod 2^32, seed >> 32) and counter (r mod 2^32, r >> 32, i // 2,
stream).  Words (x0, x1) give u1 and (x2, x3) give u2; row 2q receives
rho*cos(2*pi*u2) and row 2q+1 receives rho*sin(2*pi*u2) with
rho = sqrt(-2 ln u1).  Rows therefore do not depend on l (prefix-stable).
"""

import numpy as np

# Philox4x32 round multipliers and Weyl key increments, as published by
# Salmon et al. (SC'11), Sec. 4.
PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint64(0x9E3779B9)
PHILOX_W1 = np.uint64(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)

OMEGA_STREAM = 1


def philox4x32_10(ctr, key):
    """Philox4x32-10 on arrays of counters.

    ctr: uint32-valued array of shape (..., 4); key: (..., 2) (broadcastable).
    Returns uint64 array (..., 4) holding the four 32-bit output words.
    """
    ctr = np.asarray(ctr, dtype=np.uint64) & _MASK32
    key = np.asarray(key, dtype=np.uint64) & _MASK32
    c0, c1, c2, c3 = (ctr[..., i].copy() for i in range(4))
    k0 = np.broadcast_to(key[..., 0], c0.shape).copy()
    k1 = np.broadcast_to(key[..., 1], c0.shape).copy()
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + PHILOX_W0) & _MASK32
            k1 = (k1 + PHILOX_W1) & _MASK32
        p0 = c0 * PHILOX_M0  # exact: both factors < 2^32
        p1 = c2 * PHILOX_M1
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return np.stack([c0, c1, c2, c3], axis=-1)


def words_to_unit(lo, hi):
    """Two 32-bit words -> double strictly inside (0,1): the top 52 bits of
    (hi:lo) as an integer t, u = (t + 1/2) * 2^-52 (exact in float64, so
    1 - 2^-53 is the largest value and 2^-53 the smallest)."""
    lo = np.asarray(lo, dtype=np.uint64)
    hi = np.asarray(hi, dtype=np.uint64)
    top52 = (hi << np.uint64(20)) | (lo >> np.uint64(12))
    return (top52.astype(np.float64) + 0.5) * (2.0 ** -52)


def gaussian_block(seed, rows, cols, stream=OMEGA_STREAM):
    """Return the rows x cols block of the seeded GIID matrix (float64).

    Entry (i, r) follows the layout contract in the module docstring.
    """
    rows = int(rows)
    cols = int(cols)
    seed = int(seed)
    npairs = (rows + 1) // 2
    r = np.arange(cols, dtype=np.uint64)
    q = np.arange(npairs, dtype=np.uint64)
    ctr = np.empty((npairs, cols, 4), dtype=np.uint64)
    ctr[..., 0] = (r & _MASK32)[None, :]
    ctr[..., 1] = (r >> np.uint64(32))[None, :]
    ctr[..., 2] = q[:, None]
    ctr[..., 3] = np.uint64(stream)
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint64)
    x = philox4x32_10(ctr, key)
    u1 = words_to_unit(x[..., 0], x[..., 1])
    u2 = words_to_unit(x[..., 2], x[..., 3])
    rho = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    out = np.empty((2 * npairs, cols), dtype=np.float64)
    out[0::2] = rho * np.cos(ang)
    out[1::2] = rho * np.sin(ang)
    return out[:rows]


def gaussian_omega(seed, ell, m):
    """The l x m compression matrix Omega of Alg. 4 (and Alg. 6) for ``seed``."""
    return gaussian_block(seed, ell, m, OMEGA_STREAM)
