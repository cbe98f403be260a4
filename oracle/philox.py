"""Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
easy as 1, 2, 3", SC'11), written from its published definition.

The generator maps a 128-bit counter and a 64-bit key to 128 random bits
with ten rounds of: two 32x32->64 multiplications by the constants M0, M1,
a swap/xor mix of the counter words with the key, and a Weyl bump of the
key by W0, W1 between rounds.

Test infrastructure: part of the oracle package.  The product library
carries its own implementation of the same published definition; the two
are never linked together.

Random block entries.  The paper fills its benchmark H-matrices with random
numbers (Section 5.1) without naming a distribution; here an entry is the
exact dyadic value (w >> 8 - 2^23) * 2^-23, uniform on [-1, 1) and exact
in float32 and float64, so both sides obtain bit-identical blocks.  For the
entry at (row, col) of block kind `kind` between target node `t` and
source node `s` at tree level `level`:

    counter = (row, col >> 2, t, s | level << 24 | kind << 29)
    key     = (seed & 0xffffffff, seed >> 32)
    value   = uniform(word[col & 3])
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)
SHIFT32 = np.uint64(32)

KIND_U, KIND_V, KIND_D, KIND_SKETCH = 0, 1, 2, 3


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox rounds on arrays of 32-bit counter words (broadcastable).

    Returns the four output words as uint64 arrays holding 32-bit values.
    """
    c0 = np.asarray(c0, dtype=np.uint64) & MASK32
    c1 = np.asarray(c1, dtype=np.uint64) & MASK32
    c2 = np.asarray(c2, dtype=np.uint64) & MASK32
    c3 = np.asarray(c3, dtype=np.uint64) & MASK32
    k0 = np.asarray(k0, dtype=np.uint64) & MASK32
    k1 = np.asarray(k1, dtype=np.uint64) & MASK32
    for rnd in range(10):
        if rnd > 0:                       # key schedule: Weyl sequence
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = M0 * c0                      # 64-bit products of 32-bit words
        p1 = M1 * c2
        hi0, lo0 = p0 >> SHIFT32, p0 & MASK32
        hi1, lo1 = p1 >> SHIFT32, p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def uniform_from_word(w) -> np.ndarray:
    """Exact dyadic uniform on [-1, 1) from a 32-bit word: (w>>8 - 2^23)/2^23."""
    w = np.asarray(w, dtype=np.uint64)
    return ((w >> np.uint64(8)).astype(np.int64) - (1 << 23)).astype(np.float64) \
        * (2.0 ** -23)


def block_uniform(seed: int, kind: int, level: int, t: int, s: int,
                  rows, cols) -> np.ndarray:
    """Random entries of one block at the given local rows x cols (float64).

    `rows`, `cols` are 1-D integer arrays of local indices (position inside
    the target / source node in tree order).
    """
    rows = np.asarray(rows, dtype=np.uint64).reshape(-1, 1)
    cols = np.asarray(cols, dtype=np.uint64).reshape(-1)
    if not (0 <= s < (1 << 24) and 0 <= level < 32 and 0 <= kind < 8):
        raise ValueError("block_uniform: node index, level or kind out of range")
    c3 = np.uint64(s | (level << 24) | (kind << 29))
    # one generator call per counter (row, col >> 2) yields the four words
    # of the columns 4 (col >> 2) .. 4 (col >> 2) + 3
    groups, where = np.unique(cols >> np.uint64(2), return_inverse=True)
    words = philox4x32_10(rows, groups.reshape(1, -1), np.uint64(t), c3,
                          np.uint64(seed & 0xFFFFFFFF), np.uint64(seed >> 32))
    stacked = np.stack(np.broadcast_arrays(*words), axis=-1)   # rows x groups x 4
    sel = (cols & np.uint64(3)).astype(np.int64)
    w = stacked[:, where.reshape(-1), sel]
    return uniform_from_word(w)
