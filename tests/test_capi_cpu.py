"""C-ABI library on the CPU (no GPU): it loads, exports every entry point
declared in include/*.h, rejects bad arguments, and its host-side builder
(tree, block structure, compression, layout) reproduces the oracle's
blocks.  Builds with device = -1 never touch CUDA."""
import os
import re

import numpy as np
import pytest

import oracle as o
import workloads as w
from oracle.hmatrix import METHOD_RANDOM, METHOD_RSVD, METHOD_TSVD

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hm():
    from paper_2008_12441_gb300 import _build
    _build.build()
    from paper_2008_12441_gb300 import hmat
    hmat.library()
    return hmat


def header_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(hmat_\w+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol(hm):
    declared = header_functions()
    assert {"hmat_build", "hmat_matvec", "hmat_destroy"} <= declared
    lib = hm.library()
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert set(hm.EXPORTED) == declared


def host_build(hm, P, kernel, m, r, method, seed, tol=0.0, lr=0, prec=1):
    opts = hm.hmat_default_opts(device=-1, method=method, seed=seed, leaf_lowrank=lr, prec=prec)
    return hm.hmat_build(P, kernel, m, r, tol, opts)


def test_invalid_arguments(hm):
    P = w.grid_points(8, 2)
    bad = [
        (P[:0], 0, 16, 4),          # N = 0
        (P, 1, 16, 4),              # 3D kernel on 2D points
        (P, 0, 0, 4),               # leaf size 0
        (P, 0, 16, 0),              # no rank and no tolerance
        (P, 7, 16, 4),              # unknown kernel
    ]
    for pts, kern, m, r in bad:
        with pytest.raises(hm.HMatError) as ei:
            host_build(hm, pts, kern, m, r, METHOD_RSVD, 1)
        assert ei.value.code == hm.HMAT_EINVAL
    with pytest.raises(hm.HMatError):
        host_build(hm, P, 2, 16, 4, METHOD_RSVD, 1)    # random kernel needs random fill
    Q = P.copy()
    Q[3] = Q[5]                                          # coincident distinct points
    with pytest.raises(hm.HMatError) as ei:
        host_build(hm, Q, 0, 4, 4, METHOD_RSVD, 1)
    assert "coincide" in str(ei.value)
    h = host_build(hm, P, 0, 16, 4, METHOD_RSVD, 1)
    with pytest.raises(hm.HMatError) as ei:
        hm.hmat_matvec(h, 16, 32, 1, 1, 1, 0, 0)       # host-only handle
    assert ei.value.code == hm.HMAT_EUNSUPPORTED
    with pytest.raises(hm.HMatError) as ei:
        hm.hmat_matvec(h, 16, 32, 0, 1, 1, 0, 0)       # nrhs = 0
    assert ei.value.code == hm.HMAT_EINVAL
    # status word: nothing to read on a host-only handle; no self-test there
    assert hm.hmat_check(h, 0) == (0, 0)
    with pytest.raises(hm.HMatError) as ei:
        hm.hmat_selftest_timeout(h, 5000, 0)
    assert ei.value.code == hm.HMAT_EUNSUPPORTED
    with pytest.raises(hm.HMatError) as ei:
        hm.hmat_selftest_timeout(h, 0, 0)               # limit out of range
    assert ei.value.code == hm.HMAT_EINVAL
    lib = hm.library()
    assert lib.hmat_check(None, None, None) == hm.HMAT_EINVAL
    assert lib.hmat_selftest_timeout(None, 100, None, None) == hm.HMAT_EINVAL
    # GEMV form and workspace clones: argument checks before any CUDA call
    with pytest.raises(hm.HMatError) as ei:
        hm.hmat_gemv(h, 1.0, 16, 0.0, 32, 1, 1, 1, 0, 0)     # host-only handle
    assert ei.value.code == hm.HMAT_EUNSUPPORTED
    with pytest.raises(hm.HMatError) as ei:
        hm.hmat_gemv(h, float("nan"), 16, 0.0, 32, 1, 1, 1, 0, 0)
    assert ei.value.code == hm.HMAT_EINVAL
    with pytest.raises(hm.HMatError) as ei:
        hm.hmat_gemv(h, 1.0, 16, 0.0, 16, 1, 1, 1, 0, 0)     # x and y overlap
    assert ei.value.code in (hm.HMAT_EINVAL, hm.HMAT_EUNSUPPORTED)
    with pytest.raises(hm.HMatError) as ei:
        hm.hmat_gemv(h, 1.0, 16, 0.0, 32, 2, 1, 2, 0, 0)     # ldx < nrhs
    assert ei.value.code == hm.HMAT_EINVAL
    assert lib.hmat_gemv(None, 1.0, None, 0.0, None, 1, 1, 1, 0, None) == hm.HMAT_EINVAL
    with pytest.raises(hm.HMatError) as ei:
        hm.hmat_clone_workspace(h)                          # nothing on a device to share
    assert ei.value.code == hm.HMAT_EUNSUPPORTED
    out = __import__("ctypes").c_void_p()
    assert lib.hmat_clone_workspace(None, __import__("ctypes").byref(out)) == hm.HMAT_EINVAL
    hm.hmat_destroy(h)


def compare_blocks(hm, h, Ho):
    inf = hm.hmat_info(h)
    assert np.array_equal(hm.hmat_get_perm(h, Ho.N), Ho.tree.perm)
    worst = 0.0
    for b in Ho.blocks:
        if b.kind != "lowrank":
            continue
        U, V = hm.hmat_export_block(h, b.level, b.t.index, b.s.index,
                                    inf.rank_per_level[b.level])
        A = b.U @ b.V.T
        worst = max(worst, np.abs(U @ V.T - A).max() / max(np.abs(A).max(), 1e-300))
    nf = inf.lowrank_levels
    for g, node in enumerate(Ho.tree.levels[nf]):
        D = hm.hmat_export_dense(h, g)
        ref = np.zeros_like(D)
        for b in Ho.blocks:
            if b.kind == "dense" and node.begin <= b.t.begin and b.t.end <= node.end:
                ref[b.t.begin - node.begin:b.t.end - node.begin,
                    b.s.begin - node.begin:b.s.end - node.begin] = b.D
        worst = max(worst, np.abs(D - ref).max() / max(np.abs(ref).max(), 1e-300))
    fac, den = o.entry_counts(Ho)
    assert inf.factor_entries == fac and inf.dense_entries == den
    assert inf.lowrank_blocks == sum(b.kind == "lowrank" for b in Ho.blocks)
    assert inf.dense_blocks == sum(b.kind == "dense" for b in Ho.blocks)
    return worst


@pytest.mark.parametrize("case", ["grid2", "ragged2", "ragged3b", "tiny"])
def test_builder_random_fill_bit_identical(hm, case):
    P, m, r, lr = {"grid2": (w.grid_points(32, 2), 16, 6, 0),
                   "ragged2": (w.uniform_points(3000, 2, 4), 32, 5, 0),
                   "ragged3b": (w.uniform_points(1500, 3, 8), 20, 4, 1),
                   "tiny": (w.uniform_points(40, 2, 9), 64, 3, 0)}[case]
    Ho = o.build_hmatrix(P, 2, m, r, method=METHOD_RANDOM, seed=99, leaf_lowrank=bool(lr))
    h = host_build(hm, P, 2, m, r, METHOD_RANDOM, 99, lr=lr)
    assert compare_blocks(hm, h, Ho) == 0.0
    hm.hmat_destroy(h)


@pytest.mark.parametrize("case", ["tsvd2", "rsvd2", "rsvd3", "tol2", "fullrank"])
def test_builder_compression_matches_oracle(hm, case):
    P, kern, m, r, meth, tol = {
        "tsvd2": (w.grid_points(32, 2), 0, 16, 8, METHOD_TSVD, 0.0),
        "rsvd2": (w.grid_points(64, 2), 0, 64, 8, METHOD_RSVD, 0.0),
        "rsvd3": (w.uniform_points(2000, 3, 1), 1, 32, 12, METHOD_RSVD, 0.0),
        "tol2": (w.grid_points(32, 2), 0, 16, 0, METHOD_TSVD, 1e-6),
        "fullrank": (w.grid_points(16, 2), 0, 16, 256, METHOD_TSVD, 0.0)}[case]
    Ho = o.build_hmatrix(P, kern, m, r, tol=tol, method=meth, seed=5)
    h = host_build(hm, P, kern, m, r, meth, 5, tol=tol)
    assert compare_blocks(hm, h, Ho) < 1e-12
    hm.hmat_destroy(h)


def test_save_load_round_trip_host(hm, tmp_path):
    """hmat_save / hmat_load on a host-only handle: the loaded handle has the
    same structure, permutation, low-rank blocks and dense groups, bitwise;
    truncated and foreign files are refused."""
    P = w.uniform_points(900, 2, 31)
    h = host_build(hm, P, 2, 32, 6, METHOD_RANDOM, 17)
    path = str(tmp_path / "h.hmat")
    hm.hmat_save(h, path)
    g = hm.hmat_load(path)
    a, b = hm.hmat_info(h), hm.hmat_info(g)
    for f in ("N", "d", "depth", "lowrank_levels", "leaf_slots", "prec", "padded_N",
              "lowrank_blocks", "dense_blocks", "factor_entries", "dense_entries"):
        assert getattr(a, f) == getattr(b, f), f
    assert list(a.rank_per_level) == list(b.rank_per_level)
    assert np.array_equal(hm.hmat_get_perm(h, 900), hm.hmat_get_perm(g, 900))
    Ho = o.build_hmatrix(P, 2, 32, 6, method=METHOD_RANDOM, seed=17)
    for blk in Ho.blocks:
        if blk.kind != "lowrank":
            continue
        r = a.rank_per_level[blk.level]
        U1, V1 = hm.hmat_export_block(h, blk.level, blk.t.index, blk.s.index, r)
        U2, V2 = hm.hmat_export_block(g, blk.level, blk.t.index, blk.s.index, r)
        assert np.array_equal(U1, U2) and np.array_equal(V1, V2)
    for gi in range(len(Ho.tree.levels[a.lowrank_levels])):
        assert np.array_equal(hm.hmat_export_dense(h, gi), hm.hmat_export_dense(g, gi))
    hm.hmat_destroy(g)
    data = open(path, "rb").read()
    bad = str(tmp_path / "bad.hmat")
    for blob in (data[: len(data) // 2], b"NOTANHMATRIX" + data[12:]):
        open(bad, "wb").write(blob)
        with pytest.raises(hm.HMatError) as ei:
            hm.hmat_load(bad)
        assert ei.value.code == hm.HMAT_EINVAL
    with pytest.raises(hm.HMatError) as ei:
        hm.hmat_load(str(tmp_path / "missing.hmat"))
    assert ei.value.code == hm.HMAT_EINVAL
    hm.hmat_destroy(h)


def test_injected_host_allocation_failure_returns_enomem(hm):
    """Out-of-memory path of a host build: the float64 master arrays are the
    build's host allocations; failing either returns HMAT_ENOMEM (nothing is
    handed out), and with the injection off the same build succeeds."""
    P = w.grid_points(32, 2)
    try:
        for after in (0, 1):
            hm.hmat_inject_alloc_failure(after)
            with pytest.raises(hm.HMatError) as ei:
                host_build(hm, P, 2, 16, 4, METHOD_RANDOM, 3)
            assert ei.value.code == hm.HMAT_ENOMEM
    finally:
        hm.hmat_inject_alloc_failure(-1)
    h = host_build(hm, P, 2, 16, 4, METHOD_RANDOM, 3)
    assert hm.hmat_info(h).lowrank_blocks > 0
    hm.hmat_destroy(h)
    assert hm.hmat_inject_alloc_failure(-1) == -1


@pytest.mark.parametrize("case", ["2d32", "3d16", "fp8_8", "2d64"])
def test_leaf_slot_multiple(hm, case, tmp_path):
    """opts.leaf_slot_multiple pads every leaf to a multiple of q (and of the
    storage's alignment): the structure and the blocks are the oracle's,
    bit for bit (padding adds zero slots only); the setting survives
    hmat_save / hmat_load."""
    P, q, prec, want = {"2d32": (w.uniform_points(3000, 2, 4), 32, 1, 32),
                        "3d16": (w.uniform_points(2500, 3, 5), 16, 2, 16),
                        "fp8_8": (w.uniform_points(2000, 2, 6), 8, 4, 16),
                        "2d64": (w.uniform_points(1200, 2, 7), 64, 3, 64)}[case]
    opts = hm.hmat_default_opts(device=-1, method=METHOD_RANDOM, seed=21, prec=prec,
                                leaf_slot_multiple=q)
    h = hm.hmat_build(P, 2, 64, 6, 0.0, opts)
    inf = hm.hmat_info(h)
    assert inf.leaf_slots % want == 0
    assert inf.padded_N == inf.leaf_slots * (1 << (inf.d * inf.depth))
    Ho = o.build_hmatrix(P, 2, 64, 6, method=METHOD_RANDOM, seed=21)
    assert max(n.end - n.begin for n in Ho.tree.levels[inf.depth]) <= inf.leaf_slots
    assert compare_blocks(hm, h, Ho) == 0.0
    path = str(tmp_path / "q.hmat")
    hm.hmat_save(h, path)
    g = hm.hmat_load(path)
    assert hm.hmat_info(g).leaf_slots == inf.leaf_slots
    assert compare_blocks(hm, g, Ho) == 0.0
    hm.hmat_destroy(g)
    hm.hmat_destroy(h)


def test_leaf_slot_multiple_refused(hm):
    P = w.uniform_points(500, 2, 8)
    for q in (-8, 12, 264, 512):
        opts = hm.hmat_default_opts(device=-1, method=METHOD_RANDOM, seed=1, leaf_slot_multiple=q)
        with pytest.raises(hm.HMatError) as ei:
            hm.hmat_build(P, 2, 64, 4, 0.0, opts)
        assert ei.value.code == hm.HMAT_EINVAL


def test_batch_plan_arguments_refused_on_host(hm):
    """Plan-level argument checks that need no device: both schedule bits at
    once, host-only handles, a repeated handle, null plans for the plan
    calls, a negative or empty right-hand-side count."""
    import ctypes
    lib = hm.library()
    P = w.uniform_points(600, 2, 3)
    h = host_build(hm, P, 2, 64, 4, METHOD_RANDOM, 3)
    g = host_build(hm, P, 2, 64, 4, METHOD_RANDOM, 4)
    with pytest.raises(hm.HMatError) as ei:
        hm.hmat_batch_create([h], [1], hm.HMAT_BATCH_QUEUE | hm.HMAT_BATCH_BRANCHES)
    assert ei.value.code == hm.HMAT_EINVAL
    for flags in (0, hm.HMAT_BATCH_QUEUE, hm.HMAT_BATCH_BRANCHES):
        with pytest.raises(hm.HMatError) as ei:
            hm.hmat_batch_create([h, g], [1, 2], flags)            # not on a device
        assert ei.value.code == hm.HMAT_EINVAL
    with pytest.raises(hm.HMatError) as ei:
        hm.hmat_batch_create([h], [1], 0x4)                         # unknown flag
    assert ei.value.code == hm.HMAT_EINVAL
    out = ctypes.c_void_p()
    assert lib.hmat_batch_create(None, 1, None, 0, ctypes.byref(out)) == hm.HMAT_EINVAL
    code = ctypes.c_int(7)
    assert lib.hmat_batch_check(None, None, ctypes.byref(code)) == hm.HMAT_EINVAL
    assert code.value == 0
    assert lib.hmat_batch_poison_task(None, 0, 0, 0) == hm.HMAT_EINVAL
    assert lib.hmat_batch_matvec(None, None, None, None) == hm.HMAT_EINVAL
    assert lib.hmat_batch_destroy(None) == hm.HMAT_OK
    hm.hmat_destroy(g)
    hm.hmat_destroy(h)
