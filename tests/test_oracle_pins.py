"""Pins of the FP64 oracle against facts fixed by the paper and by
mathematics (no GPU).  Each test would fail for a plausible mistake in the
oracle: a dropped or duplicated block, a wrong child order or permutation,
a transposed factor, a wrong kernel sign, a broken generator.
"""
import math

import numpy as np
import pytest

import oracle as o
from oracle.hmatrix import (KERNEL_INV4PIR3D, KERNEL_LOG2D, KERNEL_RANDOM,
                            METHOD_RANDOM, METHOD_RSVD, METHOD_TSVD,
                            enumerate_blocks, scale_exp)
from oracle.philox import KIND_U, KIND_V, block_uniform, philox4x32_10
from oracle.tree import build_tree, tree_depth
from tests.conftest import read_golden
import workloads as w


# ---------------------------------------------------------------- generator
def test_philox_known_answers():
    """Published Philox4x32-10 known-answer vectors (Salmon et al., SC'11)."""
    for row in read_golden("philox4x32_10_kat.txt"):
        v = [int(h, 16) for h in row]
        out = philox4x32_10(*v[:6])
        assert [int(a) for a in out] == v[6:]


def test_block_uniform_exact_dyadic_and_keyed():
    a = block_uniform(7, KIND_U, 2, 3, 5, np.arange(40), np.arange(9))
    assert a.shape == (40, 9)
    assert np.all(a >= -1.0) and np.all(a < 1.0)
    assert np.all(a * 2.0 ** 23 == np.round(a * 2.0 ** 23))      # exact dyadic
    assert np.all(a.astype(np.float32).astype(np.float64) == a)  # exact in fp32
    b = block_uniform(7, KIND_U, 2, 5, 3, np.arange(40), np.arange(9))
    c = block_uniform(7, KIND_V, 2, 3, 5, np.arange(40), np.arange(9))
    d = block_uniform(8, KIND_U, 2, 3, 5, np.arange(40), np.arange(9))
    for other in (b, c, d):
        assert not np.allclose(a, other)
    # sub-block extraction agrees with the full block (counter-based)
    sub = block_uniform(7, KIND_U, 2, 3, 5, np.array([4, 17]), np.array([2, 7]))
    assert np.array_equal(sub, a[np.ix_([4, 17], [2, 7])])
    # roughly uniform on [-1, 1): mean ~ 0, variance ~ 1/3
    big = block_uniform(1, KIND_V, 1, 0, 1, np.arange(2000), np.arange(50))
    assert abs(big.mean()) < 0.02 and abs(big.var() - 1 / 3) < 0.01


def test_scale_exponent():
    assert [scale_exp(n) for n in (1, 2, 3, 4, 5, 16, 17, 64, 65536)] == \
        [0, 1, 1, 1, 2, 2, 3, 3, 8]


# --------------------------------------------------------------------- tree
def test_tree_depth_and_leaf_sizes():
    assert tree_depth(4096, 2, 64) == 3
    assert tree_depth(262144, 2, 64) == 6
    assert tree_depth(262144, 3, 64) == 4
    assert tree_depth(1048576, 2, 64) == 7
    assert tree_depth(64, 2, 64) == 0
    assert tree_depth(65, 2, 64) == 1
    P = w.uniform_points(5000, 2, 3)
    T = build_tree(P, 64)
    assert T.depth == 3 or T.depth == 4
    assert sorted(T.perm.tolist()) == list(range(5000))
    leaves = T.levels[T.depth]
    assert max(n.size for n in leaves) <= 64
    assert max(n.size for n in leaves) - min(n.size for n in leaves) <= 1
    for l in range(T.depth):
        for n in T.levels[l]:
            assert [c.begin for c in n.children][0] == n.begin
            assert n.children[-1].end == n.end
            assert sum(c.size for c in n.children) == n.size


@pytest.mark.parametrize("d,n", [(2, 16), (3, 8)])
def test_tree_is_uniform_geometric_partition_on_grids(d, n):
    """On a power-of-two grid every node is the geometric box given by its
    child ids (2^d uniform partition of an ideal domain, Section 2)."""
    P = w.grid_points(n, d)
    T = build_tree(P, 4)
    for level in T.levels:
        for node in level:
            lo = np.zeros(d)
            size = 1.0
            chain = []
            cur = node
            while cur.parent is not None:
                chain.append(cur.child_id)
                cur = cur.parent
            for cid in reversed(chain):
                size /= 2
                for a in range(d):
                    lo[a] += size * ((cid >> a) & 1)
            pts = P[T.perm[node.begin:node.end]]
            assert np.all(pts >= lo) and np.all(pts < lo + size)
            assert node.size == (n ** d) >> (d * node.level)


# ---------------------------------------------------------- block structure
def test_worked_example_2d_level1():
    """Section 2 walkthrough: 16 child pairs at level 1, 12 low-rank."""
    g = {k: int(v) for k, v in read_golden("weak_admissibility_2d_level1.txt")}
    T = build_tree(w.grid_points(32, 2), 16)      # depth 2: level-1 nodes split
    blocks = enumerate_blocks(T, leaf_lowrank=False)
    lvl1 = [b for b in blocks if b[1] == 1]
    assert len(lvl1) == g["lowrank"]
    assert all(kind == "lowrank" for kind, *_ in lvl1)
    assert g["child_pairs"] - len(lvl1) == g["recursed"]
    assert {(b[2].index, b[3].index) for b in lvl1} == \
        {(i, j) for i in range(4) for j in range(4) if i != j}


def closed_form_counts(N, d, m, reading_b=False):
    L = tree_depth(N, d, m)
    nf = L if reading_b else L - 1
    per = (1 << d) * ((1 << d) - 1)
    n_lr = per * sum(1 << (d * (l - 1)) for l in range(1, nf + 1))
    if reading_b:
        n_dense = 1 << (d * L)
    else:
        n_dense = (1 << (d * L)) * (1 << d)   # all sibling leaf pairs
    return L, n_lr, n_dense


@pytest.mark.parametrize("N,d,m,rb", [(4096, 2, 64, False), (4096, 2, 64, True),
                                      (32768, 3, 64, False), (4096, 3, 8, True),
                                      (16384, 2, 16, False)])
def test_block_counts_closed_form(N, d, m, rb):
    n = round(N ** (1 / d))
    T = build_tree(w.grid_points(n, d), m)
    blocks = enumerate_blocks(T, rb)
    L, n_lr, n_dense = closed_form_counts(N, d, m, rb)
    assert T.depth == L
    assert sum(b[0] == "lowrank" for b in blocks) == n_lr
    assert sum(b[0] == "dense" for b in blocks) == n_dense


def test_block_counts_benchmark_sizes():
    """Low-rank block counts 2^d(2^d-1) sum_l 2^{d(l-1)} at the workload sizes."""
    assert closed_form_counts(4096, 2, 64)[1] == 60
    assert closed_form_counts(262144, 2, 64)[1] == 4092
    assert closed_form_counts(262144, 3, 64)[1] == 4088
    assert closed_form_counts(1048576, 2, 64)[1] == 16380
    T = build_tree(w.grid_points(512, 2), 64)
    assert sum(b[0] == "lowrank" for b in enumerate_blocks(T, False)) == 4092


@pytest.mark.parametrize("pts,m,rb", [
    ("g2", 16, False), ("g2", 16, True), ("g3", 8, False), ("u2", 20, False),
    ("u3", 9, True), ("u2tiny", 64, False)])
def test_blocks_cover_every_entry_once(pts, m, rb):
    P = {"g2": w.grid_points(16, 2), "g3": w.grid_points(8, 3),
         "u2": w.uniform_points(700, 2, 5), "u3": w.uniform_points(600, 3, 6),
         "u2tiny": w.uniform_points(50, 2, 7)}[pts]
    H = o.build_hmatrix(P, KERNEL_RANDOM, m, 3, method=METHOD_RANDOM, seed=11,
                        leaf_lowrank=rb)
    _, cover = o.assemble_dense(H)
    assert cover.min() == 1 and cover.max() == 1


# ------------------------------------------------------------ contents/SVD
def test_tsvd_eckart_young_and_structure():
    """Truncated SVD block: V orthonormal, U = K_b V, and the Frobenius error
    equals the tail of the spectrum, sum_{q>r} lambda_q(K_b^T K_b), taken
    from a symmetric eigen-solver (a different algorithm than the SVD)."""
    P = w.grid_points(32, 2)
    H = o.build_hmatrix(P, KERNEL_LOG2D, 16, 6, method=METHOD_TSVD)
    perm = H.tree.perm
    for b in [b for b in H.blocks if b.kind == "lowrank"][:6]:
        ip, iq = perm[b.t.begin:b.t.end], perm[b.s.begin:b.s.end]
        A = o.kernel_eval(KERNEL_LOG2D, P[ip], P[iq], ip, iq)
        assert np.allclose(b.V.T @ b.V, np.eye(b.rank), atol=1e-12)
        assert np.allclose(A @ b.V, b.U, atol=1e-11 * np.abs(A).max())
        lam = np.sort(np.linalg.eigvalsh(A.T @ A))[::-1]
        err2 = np.linalg.norm(A - b.U @ b.V.T) ** 2
        tail = lam[b.rank:].sum()
        assert abs(err2 - tail) <= 1e-9 * lam[0]


def test_oracle_vs_dense_kernel_within_compression_bound():
    """||Hx - Kx|| <= sqrt(sum_blocks sum_{q>r} sigma_q^2) ||x|| (TSVD)."""
    P = w.grid_points(32, 2)
    H = o.build_hmatrix(P, KERNEL_LOG2D, 16, 5, method=METHOD_TSVD)
    K = o.dense_kernel_matrix(P, KERNEL_LOG2D)
    x = w.gaussian_rhs(P.shape[0], 1, 3)[:, 0]
    perm = H.tree.perm
    tail = 0.0
    for b in H.blocks:
        if b.kind == "lowrank":
            ip, iq = perm[b.t.begin:b.t.end], perm[b.s.begin:b.s.end]
            A = o.kernel_eval(KERNEL_LOG2D, P[ip], P[iq], ip, iq)
            tail += np.linalg.norm(A - b.U @ b.V.T) ** 2
    y = o.hmat_matvec(H, x)
    err = np.linalg.norm(y - K @ x)
    assert err <= math.sqrt(tail) * np.linalg.norm(x) * (1 + 1e-9)
    assert err > 0                                     # rank 5 is not exact


@pytest.mark.parametrize("method", [METHOD_TSVD, METHOD_RSVD])
@pytest.mark.parametrize("d,n,m", [(2, 16, 16), (3, 8, 8)])
def test_full_rank_equals_dense_kernel(method, d, n, m):
    """Rank = block size: every low-rank block is exact, so H = K and
    Hx = Kx up to float64 rounding (Definition def:hmat + eq. hmat-vec-add)."""
    P = w.grid_points(n, d)
    kern = KERNEL_LOG2D if d == 2 else KERNEL_INV4PIR3D
    N = P.shape[0]
    H = o.build_hmatrix(P, kern, m, N, method=method, seed=5)
    assert H.tree.depth == 2
    K = o.dense_kernel_matrix(P, kern)
    X = w.gaussian_rhs(N, 3, 9)
    Y = o.hmat_matvec(H, X)
    assert np.linalg.norm(Y - K @ X) <= 1e-13 * np.linalg.norm(K @ X)


def test_pure_dense_case():
    P = w.uniform_points(60, 2, 4)
    H = o.build_hmatrix(P, KERNEL_LOG2D, 64, 8)
    assert len(H.blocks) == 1 and H.blocks[0].kind == "dense"
    K = o.dense_kernel_matrix(P, KERNEL_LOG2D)
    x = w.gaussian_rhs(60, 1, 1)[:, 0]
    assert np.linalg.norm(o.hmat_matvec(H, x) - K @ x) <= 1e-15 * np.linalg.norm(K @ x) * 60


def test_kernel_values():
    p = np.array([[0.1, 0.2], [0.4, 0.6]])
    K = o.dense_kernel_matrix(p, KERNEL_LOG2D)
    assert K[0, 0] == 1.0 and K[1, 1] == 1.0
    assert abs(K[0, 1] - (-math.log(0.5))) < 1e-15 and K[0, 1] == K[1, 0]
    q = np.array([[0.0, 0.0, 0.0], [0.0, 0.3, 0.4]])
    K3 = o.dense_kernel_matrix(q, KERNEL_INV4PIR3D)
    assert abs(K3[0, 1] - 1.0 / (4 * math.pi * 0.5)) < 1e-15


def test_rsvd_close_to_tsvd():
    """Randomized SVD (q=1, p=8) error within a small factor of the optimum."""
    P = w.grid_points(32, 2)
    Ht = o.build_hmatrix(P, KERNEL_LOG2D, 16, 6, method=METHOD_TSVD)
    Hr = o.build_hmatrix(P, KERNEL_LOG2D, 16, 6, method=METHOD_RSVD, seed=3)
    K = o.dense_kernel_matrix(P, KERNEL_LOG2D)
    Mt, _ = o.assemble_dense(Ht)
    Mr, _ = o.assemble_dense(Hr)
    et, er = np.linalg.norm(Mt - K), np.linalg.norm(Mr - K)
    assert et <= er <= 1.5 * et


def test_tolerance_rank_selection():
    P = w.grid_points(32, 2)
    H = o.build_hmatrix(P, KERNEL_LOG2D, 16, 0, tol=1e-6, method=METHOD_TSVD)
    perm = H.tree.perm
    for b in [b for b in H.blocks if b.kind == "lowrank"][:4]:
        ip, iq = perm[b.t.begin:b.t.end], perm[b.s.begin:b.s.end]
        A = o.kernel_eval(KERNEL_LOG2D, P[ip], P[iq], ip, iq)
        lam = np.sort(np.linalg.eigvalsh(A.T @ A))[::-1]
        s = np.sqrt(np.maximum(lam, 0))
        assert s[b.rank] <= 1e-6 * s[0] * (1 + 1e-6)
        assert s[b.rank - 1] > 1e-6 * s[0] * (1 - 1e-6)


# -------------------------------------------------------------- the product
def test_brute_force_assembly():
    P = w.uniform_points(900, 2, 21)
    H = o.build_hmatrix(P, KERNEL_RANDOM, 16, 4, method=METHOD_RANDOM, seed=77)
    M, _ = o.assemble_dense(H)
    X = w.gaussian_rhs(900, 2, 2)
    assert np.linalg.norm(o.hmat_matvec(H, X) - M @ X) <= 1e-14 * np.linalg.norm(M @ X)


def test_linearity_and_columns():
    P = w.grid_points(16, 3)
    H = o.build_hmatrix(P, KERNEL_RANDOM, 64, 8, method=METHOD_RANDOM, seed=5)
    X = w.gaussian_rhs(P.shape[0], 3, 8)
    Y = o.hmat_matvec(H, X)
    for c in range(3):
        assert np.allclose(o.hmat_matvec(H, X[:, c]), Y[:, c], rtol=0, atol=1e-13)
    a, b = 0.75, -2.5
    lhs = o.hmat_matvec(H, a * X[:, 0] + b * X[:, 1])
    assert np.linalg.norm(lhs - (a * Y[:, 0] + b * Y[:, 1])) <= 1e-14 * np.linalg.norm(lhs) * 10


def test_rows_version_matches_full_product():
    P = w.grid_points(32, 2)
    H = o.build_hmatrix(P, KERNEL_RANDOM, 16, 4, method=METHOD_RANDOM, seed=3)
    Hl = o.build_hmatrix(P, KERNEL_RANDOM, 16, 4, method=METHOD_RANDOM, seed=3,
                         materialize=False)
    X = w.gaussian_rhs(1024, 2, 4)
    Y = o.hmat_matvec(H, X)
    rows = np.array([0, 5, 511, 1023])
    Yt = Y[H.tree.perm]
    assert np.allclose(o.hmat_matvec_rows(Hl, X, rows), Yt[rows], rtol=0, atol=1e-13)


def test_permutation_equivariance():
    """Relabelling the points relabels y (TSVD blocks do not depend on the
    order of points inside a node)."""
    P = w.grid_points(32, 2)
    rng = np.random.default_rng(0)
    q = rng.permutation(P.shape[0])
    x = w.gaussian_rhs(P.shape[0], 1, 5)[:, 0]
    y = o.hmat_matvec(o.build_hmatrix(P, KERNEL_LOG2D, 16, 5), x)
    y2 = o.hmat_matvec(o.build_hmatrix(P[q], KERNEL_LOG2D, 16, 5), x[q])
    assert np.linalg.norm(y2 - y[q]) <= 1e-12 * np.linalg.norm(y)


def test_entry_and_flop_counts_closed_form():
    """Uniform grids: factor entries = 2 s N r (#low-rank levels), dense =
    N 2^d m (reading A); flops = 2 k (factor + dense): O(r N log N)."""
    for n, d, m, r in [(64, 2, 64, 8), (32, 2, 16, 4), (16, 3, 8, 5)]:
        P = w.grid_points(n, d)
        H = o.build_hmatrix(P, KERNEL_RANDOM, m, r, method=METHOD_RANDOM,
                            seed=1, materialize=False)
        N = P.shape[0]
        L = H.tree.depth
        s = (1 << d) - 1
        fac, den = o.entry_counts(H)
        assert fac == 2 * s * N * r * (L - 1)
        assert den == N * (1 << d) * m
        assert o.flop_count(H, 7) == 14 * (fac + den)
    # N log N growth between the 64^2 and 512^2 grids (rank 16): the factor
    # part scales as N (L - 1) with L = log_4(N / 64)
    f1 = 2 * 3 * 4096 * 16 * 2
    f2 = 2 * 3 * 262144 * 16 * 5
    assert f2 / f1 == pytest.approx((262144 * 5) / (4096 * 2))
