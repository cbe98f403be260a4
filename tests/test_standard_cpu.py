"""Standard admissibility (Definition "Standard admissibility condition",
eq. (standard-ad-cond), rho = sqrt(d)) in the C-ABI library's host builder,
against the oracle's block structure and contents (no GPU: host-only
builds).  The library stores each node's interaction list in fixed stencil
slots (offsets of the non-touching children of the parent's touching
neighbours) and the near field of a group as its 3^d touching source
groups; the exported blocks must be the oracle's, bit for bit for the
random fill, to rounding for the compressed kernel blocks."""
import numpy as np
import pytest

import oracle as o
import workloads as w
from oracle.hmatrix import METHOD_RANDOM, METHOD_RSVD, METHOD_TSVD


@pytest.fixture(scope="module")
def hm():
    from paper_2008_12441_gb300 import _build
    _build.build()
    from paper_2008_12441_gb300 import hmat
    return hmat


def host_build(hm, P, kernel, m, r, method, seed, adm=1):
    opts = hm.hmat_default_opts(device=-1, method=method, seed=seed, prec=1, admissibility=adm)
    return hm.hmat_build(P, kernel, m, r, 0.0, opts)


def compare(hm, h, Ho):
    inf = hm.hmat_info(h)
    assert inf.admissibility == 1
    assert inf.partners == (27 if inf.d == 2 else 189)
    assert inf.near_groups == 3 ** inf.d
    fac, den = o.entry_counts(Ho)
    assert inf.factor_entries == fac and inf.dense_entries == den
    assert inf.lowrank_blocks == sum(b.kind == "lowrank" for b in Ho.blocks)
    assert inf.dense_blocks == sum(b.kind == "dense" for b in Ho.blocks)
    worst = 0.0
    for b in Ho.blocks:
        if b.kind != "lowrank":
            continue
        U, V = hm.hmat_export_block(h, b.level, b.t.index, b.s.index,
                                    inf.rank_per_level[b.level])
        A = b.U @ b.V.T
        worst = max(worst, np.abs(U @ V.T - A).max() / max(np.abs(A).max(), 1e-300))
    # the group's near-field block with itself
    nf = inf.lowrank_levels
    for g, node in enumerate(Ho.tree.levels[nf]):
        D = hm.hmat_export_dense(h, g)
        ref = np.zeros_like(D)
        for b in Ho.blocks:
            if (b.kind == "dense" and node.begin <= b.t.begin and b.t.end <= node.end and
                    node.begin <= b.s.begin and b.s.end <= node.end):
                ref[b.t.begin - node.begin:b.t.end - node.begin,
                    b.s.begin - node.begin:b.s.end - node.begin] = b.D
        worst = max(worst, np.abs(D - ref).max() / max(np.abs(ref).max(), 1e-300))
    return worst


@pytest.mark.parametrize("case", ["grid2", "ragged2", "grid3"])
def test_standard_random_fill_bit_identical(hm, case):
    P, m, r = {"grid2": (w.grid_points(64, 2), 16, 4),
               "ragged2": (w.uniform_points(5000, 2, 6), 20, 3),
               "grid3": (w.grid_points(16, 3), 8, 2)}[case]
    Ho = o.build_hmatrix(P, 2, m, r, method=METHOD_RANDOM, seed=77, admissibility="standard")
    h = host_build(hm, P, 2, m, r, METHOD_RANDOM, 77)
    assert compare(hm, h, Ho) == 0.0
    hm.hmat_destroy(h)


@pytest.mark.parametrize("meth", [METHOD_TSVD, METHOD_RSVD])
def test_standard_compression_matches_oracle(hm, meth):
    """Kernel blocks compressed by the library's SVDs against the oracle's
    (rank 6 on a 32^2 grid, leaf 16: well-separated blocks, clear gaps)."""
    P = w.grid_points(32, 2)
    Ho = o.build_hmatrix(P, 0, 16, 6, method=meth, seed=5, admissibility="standard")
    h = host_build(hm, P, 0, 16, 6, meth, 5)
    assert compare(hm, h, Ho) < 1e-9
    hm.hmat_destroy(h)


def test_standard_export_refuses_non_partners(hm):
    P = w.grid_points(64, 2)
    h = host_build(hm, P, 2, 16, 4, METHOD_RANDOM, 3)
    # level 2: node 0 (box (0,0)) and node 1 (box (1,0)) touch: not low-rank
    with pytest.raises(hm.HMatError) as ei:
        hm.hmat_export_block(h, 2, 0, 1, 4)
    assert ei.value.code == hm.HMAT_EINVAL
    # box (2,0) = node 4 does not touch box (0,0) and its parent (1,0) touches (0,0)
    U, V = hm.hmat_export_block(h, 2, 0, 4, 4)
    assert U.shape[1] == 4 and np.abs(U).max() > 0
    hm.hmat_destroy(h)


def test_standard_options_refused(hm):
    P = w.grid_points(32, 2)
    opts = hm.hmat_default_opts(device=-1, method=METHOD_RANDOM, seed=1, admissibility=1,
                                leaf_lowrank=1)
    with pytest.raises(hm.HMatError) as ei:
        hm.hmat_build(P, 2, 16, 4, 0.0, opts)
    assert ei.value.code == hm.HMAT_EUNSUPPORTED
    opts = hm.hmat_default_opts(device=-1, method=METHOD_RANDOM, seed=1, admissibility=5)
    with pytest.raises(hm.HMatError) as ei:
        hm.hmat_build(P, 2, 16, 4, 0.0, opts)
    assert ei.value.code == hm.HMAT_EINVAL


def test_standard_save_load_round_trip(hm, tmp_path):
    P = w.grid_points(64, 2)
    h = host_build(hm, P, 2, 16, 4, METHOD_RANDOM, 8)
    path = str(tmp_path / "s.hmat")
    hm.hmat_save(h, path)
    g = hm.hmat_load(path)
    a, b = hm.hmat_info(h), hm.hmat_info(g)
    assert (a.admissibility, a.partners, a.near_groups) == (b.admissibility, b.partners, b.near_groups)
    Ho = o.build_hmatrix(P, 2, 16, 4, method=METHOD_RANDOM, seed=8, admissibility="standard")
    assert compare(hm, g, Ho) == 0.0
    hm.hmat_destroy(g)
    hm.hmat_destroy(h)
