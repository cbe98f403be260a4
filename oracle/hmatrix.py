"""Block structure and block contents of an H-matrix (Section 2).

Test infrastructure: part of the oracle package.

Structure.  Definition "H-matrix" (def:hmat) walks the child pairs
(w_t, w_s) of a block and checks, in this order:
  1. if w_t or w_s has no children, the block is dense;
  2. else if w_t and w_s are admissible, the block is low-rank, U V^T with
     U of |w_t| x r and V of |w_s| x r;
  3. else the block is itself an H-matrix and is split again.
Weak admissibility (Definition "Weak admissibility condition"): two
domains are admissible iff they are disjoint, i.e. iff they are distinct
nodes of one level.  Starting from (root, root) this yields, under every
diagonal block, the 2^d (2^d - 1) admissible sibling pairs (12 of 16 in 2D,
the walkthrough after the definition), low-rank on levels 1..L-1, and dense
blocks between all sibling leaves (reading A).

Standard admissibility (Definition "Standard admissibility condition",
eq. (standard-ad-cond)): w and v are admissible iff
min(diam w, diam v) <= rho dist(w, v), with rho = sqrt(d) as the paper
adopts; strong admissibility takes the max instead of the min.  Both are
evaluated on the nodes' boxes of the ideal domain (see tree.py), exactly:
the squared diameters and the squared distance are integers in units of
h^2 for two boxes of one level, and rho^2 = d.  The walk of Definition
def:hmat is unchanged; only the admissibility test differs.

Reading B (``leaf_lowrank=True``) checks admissibility before leafness, so
distinct sibling leaves are low-rank too and only diagonal leaf blocks stay
dense ("every sibling off-diagonal block is low-rank").  A tree of depth 0
(N <= leaf size) is a single dense block.

Contents.  The paper leaves construction out of scope (end of Section 2)
and fills its benchmark matrices with random numbers (Section 5.1).  Three
fills are provided, all float64:
  * kernel + truncated SVD: K_b = U~ S V~^T, U = U~_r S_r, V = V~_r
    (numpy.linalg.svd, i.e. LAPACK);
  * kernel + randomized SVD (Halko, Martinsson, Tropp 2011, range finder
    with q power iterations): test matrix Omega of n_s x (r+p) from Philox
    (block kind 3), Y = K_b Omega, Q = orth(Y), q times {Q = orth(K_b
    orth(K_b^T Q))}, B = Q^T K_b = U_B S V_B^T, U = Q U_B,r S_r, V = V_B,r;
  * random: U, V, D entries uniform on [-1,1) from Philox (kinds 0, 1, 2)
    times 2^-e(n), e(n) = ceil(ceil(log2 n) / 2), n = the inner dimension
    of the product the factor takes part in (r for U, |w_s| for V and D).
Rank of a block: min(r, |w_t|, |w_s|) (fixed rank), or with a relative
tolerance the smallest k with sigma_{k+1} <= tol * sigma_1.

Kernels: K(x,y) = -log|x-y| in 2D, 1/(4 pi |x-y|) in 3D, K(x,x) = 1 (the
paper names no kernel; these are the workloads' choice).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .philox import KIND_D, KIND_SKETCH, KIND_U, KIND_V, block_uniform
from .tree import DomainTree, Node, build_tree

KERNEL_LOG2D, KERNEL_INV4PIR3D, KERNEL_RANDOM = 0, 1, 2
METHOD_TSVD, METHOD_RSVD, METHOD_RANDOM = 0, 1, 2


@dataclass
class Block:
    kind: str                 # "dense" or "lowrank"
    level: int                # level of w_t and w_s
    t: Node
    s: Node
    D: np.ndarray | None = None
    U: np.ndarray | None = None
    V: np.ndarray | None = None

    @property
    def rank(self) -> int:
        return 0 if self.U is None else self.U.shape[1]


@dataclass
class HMatrix:
    tree: DomainTree
    points: np.ndarray        # original order, N x d
    kernel: int
    rank: int
    tol: float
    method: int
    seed: int
    oversample: int
    power_iters: int
    leaf_lowrank: bool
    admissibility: str = "weak"
    blocks: list = field(default_factory=list)

    @property
    def N(self) -> int:
        return self.tree.N


def kernel_eval(kernel: int, P: np.ndarray, Q: np.ndarray,
                ip: np.ndarray, iq: np.ndarray) -> np.ndarray:
    """Kernel matrix between point sets P (a x d) and Q (b x d).

    `ip`, `iq` are the original point indices; entries with ip == iq are 1.
    """
    diff = P[:, None, :] - Q[None, :, :]
    r = np.sqrt(np.sum(diff * diff, axis=2))
    same = ip[:, None] == iq[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        if kernel == KERNEL_LOG2D:
            K = -np.log(r)
        elif kernel == KERNEL_INV4PIR3D:
            K = 1.0 / (4.0 * np.pi * r)
        else:
            raise ValueError("kernel_eval: not a kernel function")
    K[same] = 1.0
    if not np.all(np.isfinite(K)):
        raise ValueError("kernel_eval: coincident distinct points")
    return K


def dense_kernel_matrix(points: np.ndarray, kernel: int) -> np.ndarray:
    """The full N x N kernel matrix in original order (small N only)."""
    idx = np.arange(points.shape[0])
    return kernel_eval(kernel, points, points, idx, idx)


def scale_exp(n: int) -> int:
    """e(n) = ceil(ceil(log2 n) / 2): random entries are scaled by 2^-e(n)."""
    return ((max(n, 1) - 1).bit_length() + 1) // 2


ADMISSIBILITY = ("weak", "standard", "strong")


def box_diam2_dist2(t: Node, s: Node) -> tuple[int, int, int]:
    """Squared diameters of the boxes of t and s and their squared distance,
    in units of h^2 (h = 2^-level; both nodes of one level)."""
    d = len(t.coords)
    gaps = [max(0, abs(a - b) - 1) for a, b in zip(t.coords, s.coords)]
    return d, d, sum(g * g for g in gaps)


def admissible(cond: str, t: Node, s: Node) -> bool:
    """Admissibility of two nodes of one level under `cond`."""
    if cond == "weak":                       # disjoint domains
        return t is not s
    diam2_t, diam2_s, dist2 = box_diam2_dist2(t, s)
    rho2 = len(t.coords)                     # rho = sqrt(d)
    side2 = min(diam2_t, diam2_s) if cond == "standard" else max(diam2_t, diam2_s)
    return side2 <= rho2 * dist2             # diam <= rho dist, both sides >= 0 squared


def enumerate_blocks(tree: DomainTree, leaf_lowrank: bool, admissibility: str = "weak") -> list:
    """(kind, level, t, s) for every block holding data, Definition def:hmat."""
    if admissibility not in ADMISSIBILITY:
        raise ValueError("unknown admissibility condition")
    out = []
    root = tree.root
    if root.is_leaf():
        return [("dense", 0, root, root)]

    def split(t: Node, s: Node):
        for ct in t.children:
            for cs in s.children:
                adm = admissible(admissibility, ct, cs)
                if not leaf_lowrank:
                    if ct.is_leaf() or cs.is_leaf():
                        out.append(("dense", ct.level, ct, cs))
                    elif adm:
                        out.append(("lowrank", ct.level, ct, cs))
                    else:
                        split(ct, cs)
                else:
                    if adm:
                        out.append(("lowrank", ct.level, ct, cs))
                    elif ct.is_leaf():
                        out.append(("dense", ct.level, ct, cs))
                    else:
                        split(ct, cs)

    split(root, root)
    return out


def _orth(Y: np.ndarray) -> np.ndarray:
    Q, _ = np.linalg.qr(Y, mode="reduced")
    return Q


def _rank_from(S: np.ndarray, rank: int, tol: float, cap: int) -> int:
    if rank > 0:
        return min(rank, cap)
    if S.size == 0 or S[0] == 0.0:
        return 0
    return int(min(cap, np.count_nonzero(S > tol * S[0])))


def fill_block(H: HMatrix, kind: str, level: int, t: Node, s: Node,
               rows=None, srcs=None) -> Block:
    """Contents of one block (see module docstring).  Random fill only:
    `rows` selects the local target rows generated of D and U, `srcs` the
    local source positions generated of V (its rows) and of D (its
    columns); all of them by default."""
    tr = H.tree
    b = Block(kind, level, t, s)
    nt, ns = t.size, s.size
    if H.method == METHOD_RANDOM:
        trows = np.arange(nt) if rows is None else np.asarray(rows, dtype=np.int64)
        scols = np.arange(ns) if srcs is None else np.asarray(srcs, dtype=np.int64)
        if kind == "dense":
            b.D = block_uniform(H.seed, KIND_D, level, t.index, s.index,
                                trows, scols) * 2.0 ** -scale_exp(ns)
        else:
            rb = min(H.rank, nt, ns)
            b.U = block_uniform(H.seed, KIND_U, level, t.index, s.index,
                                trows, np.arange(rb)) * 2.0 ** -scale_exp(rb)
            b.V = block_uniform(H.seed, KIND_V, level, t.index, s.index,
                                scols, np.arange(rb)) * 2.0 ** -scale_exp(ns)
        return b
    ip = tr.perm[t.begin:t.end]
    iq = tr.perm[s.begin:s.end]
    A = kernel_eval(H.kernel, H.points[ip], H.points[iq], ip, iq)
    if kind == "dense":
        b.D = A
        return b
    cap = min(nt, ns)
    if H.method == METHOD_TSVD:
        Uf, S, Vt = np.linalg.svd(A, full_matrices=False)
        rb = _rank_from(S, H.rank, H.tol, cap)
        b.U = Uf[:, :rb] * S[:rb]
        b.V = Vt[:rb].T.copy()
        return b
    if H.method == METHOD_RSVD:
        ell = min((H.rank if H.rank > 0 else cap) + H.oversample, cap)
        Om = block_uniform(H.seed, KIND_SKETCH, level, t.index, s.index,
                           np.arange(ns), np.arange(ell))
        Q = _orth(A @ Om)
        for _ in range(H.power_iters):
            Q = _orth(A @ _orth(A.T @ Q))
        B = Q.T @ A
        Ub, S, Vbt = np.linalg.svd(B, full_matrices=False)
        rb = _rank_from(S, H.rank, H.tol, min(cap, ell))
        b.U = (Q @ Ub[:, :rb]) * S[:rb]
        b.V = Vbt[:rb].T.copy()
        return b
    raise ValueError("fill_block: unknown method")


def build_hmatrix(points: np.ndarray, kernel: int, leaf_size: int, rank: int,
                  tol: float = 0.0, method: int = METHOD_TSVD, seed: int = 0,
                  oversample: int = 8, power_iters: int = 1,
                  leaf_lowrank: bool = False, materialize: bool = True,
                  admissibility: str = "weak") -> HMatrix:
    """Tree, block list and (if `materialize`) every block's contents."""
    points = np.ascontiguousarray(points, dtype=np.float64)
    if kernel == KERNEL_RANDOM and method != METHOD_RANDOM:
        raise ValueError("random kernel needs the random fill")
    if kernel != KERNEL_RANDOM and method == METHOD_RANDOM:
        raise ValueError("random fill needs the random kernel")
    if rank <= 0 and not (tol > 0.0):
        raise ValueError("need rank > 0 or tol > 0")
    tree = build_tree(points, leaf_size)
    H = HMatrix(tree, points, kernel, rank, tol, method, seed, oversample,
                power_iters, bool(leaf_lowrank), admissibility)
    for kind, level, t, s in enumerate_blocks(tree, H.leaf_lowrank, admissibility):
        if materialize:
            H.blocks.append(fill_block(H, kind, level, t, s))
        else:
            H.blocks.append(Block(kind, level, t, s))
    return H
