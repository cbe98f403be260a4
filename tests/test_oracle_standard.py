"""Pins of the oracle's standard admissibility (Definition "Standard
admissibility condition", eq. (standard-ad-cond), rho = sqrt(d)) and of the
H-matrix it produces through Definition def:hmat, against facts the paper
and geometry fix.  CPU only."""
import itertools
import math

import numpy as np
import pytest

import oracle as o
from oracle.hmatrix import (KERNEL_LOG2D, KERNEL_RANDOM, METHOD_RANDOM, METHOD_TSVD,
                            admissible, enumerate_blocks)
from oracle.tree import build_tree
import workloads as w


def float_geometry_admissible(t, s):
    """eq. (standard-ad-cond) in floating point on the boxes' corners, a
    computation separate from the oracle's integer one."""
    d = len(t.coords)
    h = 2.0 ** -t.level
    lo_t = np.array(t.coords) * h
    lo_s = np.array(s.coords) * h
    gap = np.maximum(0.0, np.maximum(lo_s - (lo_t + h), lo_t - (lo_s + h)))
    dist = math.sqrt(float(np.sum(gap * gap)))
    diam = math.sqrt(d) * h                        # both boxes have side h
    return diam <= math.sqrt(d) * dist


@pytest.mark.parametrize("d,n,level", [(2, 16, 3), (3, 8, 2)])
def test_standard_condition_on_the_boxes(d, n, level):
    """On boxes of one level the condition holds exactly when the boxes do
    not touch (Chebyshev distance of their coordinates >= 2): diam = sqrt(d)
    h and dist >= h iff some gap is at least one box."""
    T = build_tree(w.grid_points(n, d), 1)
    nodes = T.levels[level]
    for t, s in itertools.product(nodes, nodes):
        cheb = max(abs(a - b) for a, b in zip(t.coords, s.coords))
        assert admissible("standard", t, s) == (cheb >= 2)
        assert admissible("standard", t, s) == float_geometry_admissible(t, s)
        assert admissible("strong", t, s) == admissible("standard", t, s)
        assert admissible("weak", t, s) == (t is not s)


def lowrank_partners(blocks, node):
    return sum(1 for kind, lvl, t, s in blocks if kind == "lowrank" and t is node)


@pytest.mark.parametrize("d,n,m,level,center,want_center,want_corner", [
    (2, 64, 4, 3, (3, 3), 3 ** 2 * 2 ** 2 - 3 ** 2, 2 ** 2 * 2 ** 2 - 2 ** 2),
    (3, 32, 8, 3, (3, 3, 3), 3 ** 3 * 2 ** 3 - 3 ** 3, 2 ** 3 * 2 ** 3 - 2 ** 3)])
def test_paper_center_and_corner_counts(d, n, m, level, center, want_center, want_corner):
    """Sec. 3 (load balancing under standard admissibility): at a level that
    is neither among the first two nor the last, a centre subdomain has
    3^d 2^d - 3^d admissible subdomains (27 in 2D, 189 in 3D), a corner one
    2^d 2^d - 2^d (12, 56); their ratio is the load factor (3/2)^d."""
    T = build_tree(w.grid_points(n, d), m)
    assert 2 <= level < T.depth
    blocks = enumerate_blocks(T, False, "standard")
    by_coords = {nd.coords: nd for nd in T.levels[level]}
    c = lowrank_partners(blocks, by_coords[center])
    k = lowrank_partners(blocks, by_coords[(0,) * d])
    assert (c, k) == (want_center, want_corner) == ((27, 12) if d == 2 else (189, 56))
    assert c / k == pytest.approx(1.5 ** d)


@pytest.mark.parametrize("d,n,m", [(2, 32, 4), (3, 16, 8), (2, 16, 16)])
def test_standard_structure_matches_pair_enumeration(d, n, m):
    """Def. def:hmat with standard admissibility, restated without recursion:
    the pairs of one level whose parents touch (or coincide) are the split
    ones; among them the non-touching pairs are low-rank (levels below the
    leaves) and every pair of the leaf level is dense."""
    T = build_tree(w.grid_points(n, d), m)
    L = T.depth
    got = {(kind, lvl, t.coords, s.coords) for kind, lvl, t, s in enumerate_blocks(T, False, "standard")}
    want = set()
    for lvl in range(1, L + 1):
        side = 2 ** lvl
        boxes = list(itertools.product(range(side), repeat=d))
        for a, b in itertools.product(boxes, boxes):
            pa = tuple(q // 2 for q in a)
            pb = tuple(q // 2 for q in b)
            if max(abs(x - y) for x, y in zip(pa, pb)) > 1:
                continue                            # parents admissible: never reached
            if lvl == L:
                want.add(("dense", lvl, a, b))
            elif max(abs(x - y) for x, y in zip(a, b)) >= 2:
                want.add(("lowrank", lvl, a, b))
    assert got == want


@pytest.mark.parametrize("d,n,m", [(2, 32, 4), (3, 8, 2)])
def test_strong_equals_standard_on_ideal_domains(d, n, m):
    """Sec. 2: strong (max) and standard (min) admissibility coincide on
    ideal domains."""
    T = build_tree(w.grid_points(n, d), m)
    a = [(k, l, t.index, s.index) for k, l, t, s in enumerate_blocks(T, False, "standard")]
    b = [(k, l, t.index, s.index) for k, l, t, s in enumerate_blocks(T, False, "strong")]
    assert a == b


@pytest.mark.parametrize("pts,m", [("g2", 4), ("g3", 4), ("u2", 20), ("u3", 9)])
def test_standard_blocks_cover_every_entry_once(pts, m):
    """Every (target, source) pair of points lies in exactly one block."""
    P = {"g2": w.grid_points(16, 2), "g3": w.grid_points(8, 3),
         "u2": w.uniform_points(700, 2, 5), "u3": w.uniform_points(600, 3, 6)}[pts]
    H = o.build_hmatrix(P, KERNEL_RANDOM, m, 3, method=METHOD_RANDOM, seed=11,
                        admissibility="standard", materialize=False)
    cover = np.zeros((H.N, H.N), dtype=np.int64)
    for b in H.blocks:
        cover[b.t.begin:b.t.end, b.s.begin:b.s.end] += 1
    assert cover.min() == 1 and cover.max() == 1
    assert any(b.kind == "lowrank" for b in H.blocks)


def test_standard_product_matches_dense_assembly():
    """Brute force: the product over the blocks equals the assembled dense
    matrix (holding every block in place) times x."""
    P = w.uniform_points(400, 2, 8)
    H = o.build_hmatrix(P, KERNEL_RANDOM, 12, 3, method=METHOD_RANDOM, seed=12,
                        admissibility="standard")
    M, cover = o.assemble_dense(H)
    assert cover.min() == 1 and cover.max() == 1
    X = w.gaussian_rhs(400, 2, 13)
    Y = o.hmat_matvec(H, X)
    assert np.linalg.norm(Y - M @ X) <= 1e-13 * np.linalg.norm(M @ X)


def test_standard_product_within_compression_bound_and_tighter_than_weak():
    """||Hx - Kx|| <= sqrt(sum_blocks sum_{q>r} sigma_q^2) ||x|| under standard
    admissibility (TSVD), and at the same rank the well-separated blocks
    compress far better than weak admissibility's touching siblings."""
    P = w.grid_points(32, 2)
    K = o.dense_kernel_matrix(P, KERNEL_LOG2D)
    x = w.gaussian_rhs(P.shape[0], 1, 3)[:, 0]
    errs = {}
    for cond in ("standard", "weak"):
        H = o.build_hmatrix(P, KERNEL_LOG2D, 4, 3, method=METHOD_TSVD, admissibility=cond)
        perm = H.tree.perm
        tail = 0.0
        for b in H.blocks:
            if b.kind == "lowrank":
                ip, iq = perm[b.t.begin:b.t.end], perm[b.s.begin:b.s.end]
                A = o.kernel_eval(KERNEL_LOG2D, P[ip], P[iq], ip, iq)
                tail += np.linalg.norm(A - b.U @ b.V.T) ** 2
        err = np.linalg.norm(o.hmat_matvec(H, x) - K @ x)
        assert err <= math.sqrt(tail) * np.linalg.norm(x) * (1 + 1e-9)
        errs[cond] = err / np.linalg.norm(K @ x)
    assert errs["standard"] < 0.1 * errs["weak"]


# ------------------------------------------------------ transposed product
@pytest.mark.parametrize("cond", ["weak", "standard"])
def test_transpose_adjoint_identity_and_brute_force(cond):
    """<K x, y> = <x, K^T y> against the forward product, and K^T x against
    the transposed dense assembly of the same blocks."""
    P = w.uniform_points(500, 2, 21)
    H = o.build_hmatrix(P, KERNEL_RANDOM, 16, 4, method=METHOD_RANDOM, seed=22,
                        admissibility=cond)
    X = w.gaussian_rhs(500, 2, 23)
    Y = w.gaussian_rhs(500, 2, 24)
    lhs = np.sum(o.hmat_matvec(H, X) * Y)
    rhs = np.sum(X * o.hmat_matvec_transpose(H, Y))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1.0)
    M, _ = o.assemble_dense(H)
    Z = o.hmat_matvec_transpose(H, X)
    assert np.linalg.norm(Z - M.T @ X) <= 1e-13 * np.linalg.norm(M.T @ X)


def test_transpose_of_symmetric_kernel_with_tsvd():
    """A symmetric kernel compressed by truncated SVD: block (j, i) is the
    SVD of the transpose of block (i, j), so K^T = K up to rounding (random
    points: no ties in the singular values at the truncation)."""
    P = w.uniform_points(600, 2, 25)
    H = o.build_hmatrix(P, KERNEL_LOG2D, 24, 5, method=METHOD_TSVD)
    X = w.gaussian_rhs(600, 1, 26)
    a = o.hmat_matvec(H, X)
    b = o.hmat_matvec_transpose(H, X)
    assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(a)
    # the random fill is not symmetric: the two products differ
    Hr = o.build_hmatrix(P, KERNEL_RANDOM, 24, 5, method=METHOD_RANDOM, seed=27)
    assert np.linalg.norm(o.hmat_matvec(Hr, X) - o.hmat_matvec_transpose(Hr, X)) > 1e-3


@pytest.mark.parametrize("method", [METHOD_RANDOM, METHOD_TSVD])
def test_transpose_rows_version_matches_full_transpose(method):
    """Rows of K^T x restricted to chosen positions (columns of D and rows
    of V generated only where needed for the random fill) equal the same
    rows of the full transposed product; repeated rows included."""
    P = w.grid_points(32, 2)
    kern = KERNEL_RANDOM if method == METHOD_RANDOM else KERNEL_LOG2D
    H = o.build_hmatrix(P, kern, 16, 4, method=method, seed=31)
    Hl = o.build_hmatrix(P, kern, 16, 4, method=method, seed=31, materialize=False)
    X = w.gaussian_rhs(1024, 3, 32)
    Yt = o.hmat_matvec_transpose(H, X)[H.tree.perm]
    rows = np.array([0, 5, 5, 255, 256, 511, 700, 1023])
    got = o.hmat_matvec_transpose_rows(Hl, X, rows)
    assert np.allclose(got, Yt[rows], rtol=0, atol=1e-13)
