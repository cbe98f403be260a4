"""The H-matrix-vector product y = K x (Section 2, eq. (hmat-vec-add)).

Test infrastructure: part of the oracle package.

Start from y = 0; for every block holding data, restricted to its target
rows w_t and source columns w_s:
    dense block:     y_{w_t} += D (x_{w_s})
    low-rank block:  y_{w_t} += U (V^T x_{w_s})
When every block has been visited, y = K x.  Blocks are visited in the
order of Definition def:hmat (root to leaves, child pairs in order); any
order gives the same result up to rounding.  x and y are N x k arrays in
the caller's (original) point order.
"""
from __future__ import annotations

import numpy as np

from .hmatrix import METHOD_RANDOM, HMatrix, fill_block


def _block_data(H: HMatrix, b):
    if b.D is None and b.U is None:
        return fill_block(H, b.kind, b.level, b.t, b.s)
    return b


def hmat_matvec(H: HMatrix, x: np.ndarray) -> np.ndarray:
    """y = K x by eq. (hmat-vec-add), float64, original point order."""
    x = np.asarray(x, dtype=np.float64)
    vec = x.ndim == 1
    X = x.reshape(H.N, -1)
    perm = H.tree.perm
    xt = X[perm]                                   # tree order
    yt = np.zeros_like(xt)
    for b in H.blocks:
        b = _block_data(H, b)
        xs = xt[b.s.begin:b.s.end]
        if b.kind == "dense":
            yt[b.t.begin:b.t.end] += b.D @ xs
        else:
            yt[b.t.begin:b.t.end] += b.U @ (b.V.T @ xs)
    y = np.empty_like(yt)
    y[perm] = yt
    return y.reshape(-1) if vec else y


def hmat_matvec_transpose(H: HMatrix, x: np.ndarray) -> np.ndarray:
    """y = K^T x: every block applied transposed from its target rows to its
    source columns, y_{w_s} += D^T x_{w_t} and y_{w_s} += V (U^T x_{w_t})
    (the transposed product of the NEXT rows; the paper's algorithm is
    stated for K x, and K^T is the H-matrix of the swapped domain trees)."""
    x = np.asarray(x, dtype=np.float64)
    vec = x.ndim == 1
    X = x.reshape(H.N, -1)
    perm = H.tree.perm
    xt = X[perm]
    yt = np.zeros_like(xt)
    for b in H.blocks:
        b = _block_data(H, b)
        xs = xt[b.t.begin:b.t.end]
        if b.kind == "dense":
            yt[b.s.begin:b.s.end] += b.D.T @ xs
        else:
            yt[b.s.begin:b.s.end] += b.V @ (b.U.T @ xs)
    y = np.empty_like(yt)
    y[perm] = yt
    return y.reshape(-1) if vec else y


def hmat_matvec_rows(H: HMatrix, x: np.ndarray, tree_rows) -> np.ndarray:
    """Rows `tree_rows` (tree-order positions) of y = K x, eq. (hmat-vec-add)
    restricted to those target rows; block contents are generated on demand
    (for the random fill only the needed rows of U and D).  Returns
    len(rows) x k."""
    X = np.asarray(x, dtype=np.float64).reshape(H.N, -1)
    xt = X[H.tree.perm]
    rows = np.asarray(tree_rows, dtype=np.int64)
    out = np.zeros((rows.size, X.shape[1]))
    for b in H.blocks:
        hit = np.nonzero((rows >= b.t.begin) & (rows < b.t.end))[0]
        if hit.size == 0:
            continue
        loc = rows[hit] - b.t.begin
        xs = xt[b.s.begin:b.s.end]
        if b.D is None and b.U is None and H.method == METHOD_RANDOM:
            # rows `loc` of D or U only
            b = fill_block(H, b.kind, b.level, b.t, b.s, rows=loc)
            loc = np.arange(loc.size)
        else:
            b = _block_data(H, b)
        if b.kind == "dense":
            out[hit] += b.D[loc] @ xs
        else:
            out[hit] += b.U[loc] @ (b.V.T @ xs)
    return out


def hmat_matvec_transpose_rows(H: HMatrix, x: np.ndarray, tree_rows) -> np.ndarray:
    """Rows `tree_rows` (tree-order positions) of y = K^T x: every block whose
    source range holds a row adds D^T x_{w_t} or V (U^T x_{w_t}) restricted
    to those rows, i.e. columns of D and rows of V (for the random fill only
    those are generated).  Returns len(rows) x k."""
    X = np.asarray(x, dtype=np.float64).reshape(H.N, -1)
    xt = X[H.tree.perm]
    rows = np.asarray(tree_rows, dtype=np.int64)
    out = np.zeros((rows.size, X.shape[1]))
    for b in H.blocks:
        hit = np.nonzero((rows >= b.s.begin) & (rows < b.s.end))[0]
        if hit.size == 0:
            continue
        loc = rows[hit] - b.s.begin
        xs = xt[b.t.begin:b.t.end]
        if b.D is None and b.U is None and H.method == METHOD_RANDOM:
            b = fill_block(H, b.kind, b.level, b.t, b.s, srcs=loc)
            loc = np.arange(loc.size)
        else:
            b = _block_data(H, b)
        if b.kind == "dense":
            out[hit] += b.D[:, loc].T @ xs
        else:
            out[hit] += b.V[loc] @ (b.U.T @ xs)
    return out


def assemble_dense(H: HMatrix) -> tuple[np.ndarray, np.ndarray]:
    """Dense N x N matrix holding every block in place (original order), and
    a coverage count of how many blocks wrote each entry (brute force)."""
    N = H.N
    M = np.zeros((N, N))
    cover = np.zeros((N, N), dtype=np.int64)
    perm = H.tree.perm
    for b in H.blocks:
        b = _block_data(H, b)
        ri = perm[b.t.begin:b.t.end]
        ci = perm[b.s.begin:b.s.end]
        blk = b.D if b.kind == "dense" else b.U @ b.V.T
        M[np.ix_(ri, ci)] += blk
        cover[np.ix_(ri, ci)] += 1
    return M, cover


def entry_counts(H: HMatrix) -> tuple[int, int]:
    """(factor entries, dense entries): sum (|w_t| + |w_s|) r_b over low-rank
    blocks and sum |w_t| |w_s| over dense blocks."""
    fac = 0
    den = 0
    for b in H.blocks:
        if b.kind == "dense":
            den += b.t.size * b.s.size
        else:
            rb = b.rank if (b.U is not None) else min(H.rank, b.t.size, b.s.size)
            fac += (b.t.size + b.s.size) * rb
    return fac, den


def flop_count(H: HMatrix, k: int = 1) -> int:
    """Multiply-add count x 2 of eq. (hmat-vec-add) for k right-hand sides."""
    fac, den = entry_counts(H)
    return 2 * k * (fac + den)
