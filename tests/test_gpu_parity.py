"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.  Error = ||Y_gpu - Y_oracle||_F / ||Y_oracle||_F.
Tolerances: 1e-12 for the FP64 mode, 1e-5 for FP32."""
import numpy as np
import pytest

import oracle as o
import workloads as w
from oracle.hmatrix import METHOD_RANDOM, METHOD_RSVD, METHOD_TSVD

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


@pytest.fixture(scope="module")
def hm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_12441_gb300 import _build
    _build.build()
    from paper_2008_12441_gb300 import hmat
    return hmat


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def gpu_apply(H, X, flags=0, stream=None, path=None):
    """H X through hmat_matvec; `path`: the HMAT_PATH_* bits the product
    must have taken (None: not checked)."""
    import torch
    x = torch.from_numpy(np.ascontiguousarray(X)).to(H.vec_dtype).cuda()
    y = H.matvec(x, flags=flags, stream=stream)
    torch.cuda.synchronize()
    # no bounded device-side wait gave up
    assert H.check() == (0, 0)
    if path is not None:
        assert H.last_path() == path, (H.last_path(), path)
    return y.double().cpu().numpy()


def sm_count():
    import torch
    return torch.cuda.get_device_properties(0).multi_processor_count


def build_pair(hm, P, kern, m, r, meth, seed, prec, lr=0, tol=0.0, max_nrhs=64):
    Ho = o.build_hmatrix(P, kern, m, r, tol=tol, method=meth, seed=seed, leaf_lowrank=bool(lr))
    H = hm.HMatrix(P, kern, m, r, tol, prec=prec, method=meth, seed=seed, leaf_lowrank=lr,
                   max_nrhs=max_nrhs)
    return Ho, H


def test_2d_fp64_tsvd_rank8_n4096(hm):
    """64x64 grid, log kernel, leaf 64, truncated SVD rank 8, FP64, 1 RHS."""
    inst = w.c1_small()
    P = inst.points()
    Ho, H = build_pair(hm, P, inst.kernel, 64, 8, METHOD_TSVD, inst.seed, 0)
    x = inst.rhs()
    y = gpu_apply(H, x)
    yo = o.hmat_matvec(Ho, x)
    assert rel(y, yo) <= TOL[0], rel(y, yo)
    # against the dense kernel matrix: the compression error of rank 8
    K = o.dense_kernel_matrix(P, inst.kernel)
    assert rel(y, K @ x) < 0.05


def test_2d_fp32_rsvd_rank16_n16384(hm):
    P = w.grid_points(128, 2)
    Ho, H = build_pair(hm, P, 0, 64, 16, METHOD_RSVD, 7, 1)
    x = w.gaussian_rhs(P.shape[0], 1, 70)
    e = rel(gpu_apply(H, x, path=hm.PATH_STREAMED), o.hmat_matvec(Ho, x))
    assert e <= TOL[1], e


def test_3d_fp32_rsvd_rank32_32rhs(hm):
    P = w.grid_points(16, 3)
    Ho, H = build_pair(hm, P, 1, 64, 32, METHOD_RSVD, 9, 1)
    X = w.gaussian_rhs(P.shape[0], 32, 71)
    e = rel(gpu_apply(H, X, path=hm.PATH_CACHED), o.hmat_matvec(Ho, X))
    assert e <= TOL[1], e


def test_3d_ragged_grid_padding_fp64(hm):
    """24^3 grid: leaves of 27 points padded to 32 slots, 3 tree levels.
    Random blocks: on this symmetric grid some kernel blocks have
    sigma_6 = sigma_7, where a rank-6 truncation is not unique."""
    P = w.grid_points(24, 3)
    Ho, H = build_pair(hm, P, 2, 64, 6, METHOD_RANDOM, 10, 0)
    assert H.info.leaf_slots == 32 and H.info.depth == 3
    X = w.gaussian_rhs(P.shape[0], 2, 72)
    e = rel(gpu_apply(H, X), o.hmat_matvec(Ho, X))
    assert e <= TOL[0], e


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("k", [1, 3, 64])
def test_rhs_counts_random_fill(hm, prec, k):
    P = w.grid_points(64, 2)
    Ho, H = build_pair(hm, P, 2, 32, 8, METHOD_RANDOM, 11, prec)
    X = w.gaussian_rhs(P.shape[0], k, 73)
    e = rel(gpu_apply(H, X), o.hmat_matvec(Ho, X))
    assert e <= TOL[prec], e


def test_more_rhs_than_one_pass(hm):
    """nrhs above max_nrhs runs in several passes over the same handle."""
    P = w.grid_points(32, 2)
    Ho, H = build_pair(hm, P, 2, 16, 4, METHOD_RANDOM, 12, 1, max_nrhs=8)
    X = w.gaussian_rhs(P.shape[0], 21, 74)
    e = rel(gpu_apply(H, X), o.hmat_matvec(Ho, X))
    assert e <= TOL[1], e


@pytest.mark.parametrize("flags", [0, 1])
def test_ragged_points_and_orders(hm, flags):
    """Uniform random points (uneven leaves, padding); original vs tree order."""
    P = w.uniform_points(5000, 2, 13)
    Ho, H = build_pair(hm, P, 2, 32, 10, METHOD_RANDOM, 13, 0)
    X = w.gaussian_rhs(5000, 2, 75)
    Yo = o.hmat_matvec(Ho, X)
    if flags:
        perm = H.perm()
        assert np.array_equal(perm, Ho.tree.perm)
        e = rel(gpu_apply(H, X[perm], flags=1), Yo[perm])
    else:
        e = rel(gpu_apply(H, X), Yo)
    assert e <= TOL[0], e


def test_leaf_lowrank_reading(hm):
    P = w.grid_points(32, 2)
    Ho, H = build_pair(hm, P, 0, 16, 4, METHOD_TSVD, 14, 0, lr=1)
    assert H.info.lowrank_levels == H.info.depth
    x = w.gaussian_rhs(1024, 1, 76)
    e = rel(gpu_apply(H, x), o.hmat_matvec(Ho, x))
    assert e <= TOL[0], e


def test_pure_dense_and_full_rank(hm):
    P = w.uniform_points(50, 2, 15)
    Ho, H = build_pair(hm, P, 0, 64, 8, METHOD_RSVD, 15, 0)
    assert H.info.depth == 0
    x = w.gaussian_rhs(50, 3, 77)
    K = o.dense_kernel_matrix(P, 0)
    assert rel(gpu_apply(H, x), K @ x) <= 1e-13
    # rank = block size: H = K exactly
    P = w.grid_points(16, 2)
    H2 = hm.HMatrix(P, 0, 16, 64, 0.0, prec=0, method=METHOD_TSVD, seed=1)
    x = w.gaussian_rhs(256, 1, 78)
    K = o.dense_kernel_matrix(P, 0)
    assert rel(gpu_apply(H2, x), K @ x) <= 1e-12


def test_bitwise_determinism_and_stream(hm):
    import torch
    P = w.grid_points(128, 2)
    H = hm.HMatrix(P, 2, 64, 16, 0.0, prec=1, method=METHOD_RANDOM, seed=16)
    x = torch.from_numpy(w.gaussian_rhs(P.shape[0], 1, 79)).float().cuda()
    y1 = H.matvec(x)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        y2 = H.matvec(x, stream=s)
        ev = torch.cuda.Event()
        ev.record(s)
    ev.synchronize()
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)


def sampled_rows_check(hm, grid_n, d, r, k, prec, rows_seed, path):
    """Full-size random-fill H-matrix, in the launch configuration bench.py
    times: the oracle computes output rows one by one (eq. (hmat-vec-add)
    restricted to those rows) at one position in every 256- and 128-slot
    tile and at both ends of every persistent CTA's tile range
    (workloads.covering_rows); the error is the rel-L2 over those rows and
    the worst row's relative error is reported beside it."""
    P = w.grid_points(grid_n, d)
    N = P.shape[0]
    H = hm.HMatrix(P, 2, 64, r, 0.0, prec=prec, method=METHOD_RANDOM, seed=rows_seed,
                   max_nrhs=max(k, 1))
    X = w.gaussian_rhs(N, k, rows_seed + 1)
    Y = gpu_apply(H, X, flags=hm.HMAT_TREE_ORDER, path=path)
    H.close()
    Ho = o.build_hmatrix(P, 2, 64, r, method=METHOD_RANDOM, seed=rows_seed, materialize=False)
    rows = w.covering_rows(N, sm_count(), rows_seed)
    Xo = np.empty_like(X)
    Xo[Ho.tree.perm] = X               # X was passed in tree order
    Yo_rows = o.hmat_matvec_rows(Ho, Xo, rows)
    Yg_rows = Y[rows]
    worst = float(np.max(np.linalg.norm(Yg_rows - Yo_rows, axis=1) /
                         np.maximum(np.linalg.norm(Yo_rows, axis=1), 1e-300)))
    return rel(Yg_rows, Yo_rows), worst


def test_full_size_2d_n262144_rank16_sampled_rows(hm):
    e, worst = sampled_rows_check(hm, 512, 2, 16, 1, 1, 21, hm.PATH_STREAMED)
    assert e <= TOL[1], (e, worst)


def test_full_size_2d_n1048576_rank16_fp32_one_rhs(hm):
    """The headline configuration: 1024^2 grid, rank 16, FP32, one
    right-hand side, through the streamed kernels; 1e-5 against the FP64
    oracle over rows of every tile and every CTA range."""
    e, worst = sampled_rows_check(hm, 1024, 2, 16, 1, 1, 25, hm.PATH_STREAMED)
    assert e <= TOL[1], (e, worst)


def test_full_size_3d_n262144_rank32_32rhs_sampled_rows(hm):
    e, worst = sampled_rows_check(hm, 64, 3, 32, 32, 1, 22, hm.PATH_CACHED)
    assert e <= TOL[1], (e, worst)


def test_gpu_side_builder_against_oracle(hm):
    """Randomized SVD with the kernel-block products on the GPU (float kernel
    evaluation, double chunk sums): the H-matrix differs from the oracle's
    float64 randomized SVD only by the float evaluation of the sketches."""
    P = w.grid_points(128, 2)
    Ho = o.build_hmatrix(P, 0, 64, 16, method=METHOD_RSVD, seed=31)
    H = hm.HMatrix(P, 0, 64, 16, 0.0, prec=0, method=METHOD_RSVD, seed=31, build_gpu=1)
    x = w.gaussian_rhs(P.shape[0], 1, 81)
    e = rel(gpu_apply(H, x), o.hmat_matvec(Ho, x))
    assert e <= 1e-5, e


def test_full_size_2d_kernel_rsvd_vs_dense_kernel_rows(hm):
    """512x512 grid, log kernel, rank 16 (GPU-side sketches): sampled rows
    of Hx against the same rows of the dense kernel matrix times x; the
    difference is the compression error of weak admissibility at rank 16."""
    P = w.grid_points(512, 2)
    H = hm.HMatrix(P, 0, 64, 16, 0.0, prec=1, method=METHOD_RSVD, seed=12442)
    x = w.gaussian_rhs(P.shape[0], 1, 82)
    y = gpu_apply(H, x)[:, 0]
    rows = np.random.default_rng(3).integers(0, P.shape[0], 16)
    Krows = o.kernel_eval(0, P[rows], P, rows, np.arange(P.shape[0]))
    e = rel(y[rows], Krows @ x[:, 0])
    assert e < 1e-2, e


PREC_TOL = {0: 1e-12, 1: 1e-5, 2: 1e-2, 3: 1e-5, 4: 5e-2}


@pytest.fixture(scope="module")
def log2d_16384():
    P = w.grid_points(128, 2)
    Ho = o.build_hmatrix(P, 0, 64, 16, method=METHOD_RSVD, seed=44)
    X = w.gaussian_rhs(P.shape[0], 64, 83)
    return P, Ho, X, o.hmat_matvec(Ho, X)


@pytest.mark.parametrize("prec", [2, 3, 4])
@pytest.mark.parametrize("k", [1, 8, 64])
def test_storage_precisions_against_fp64_oracle(hm, log2d_16384, prec, k):
    """bf16 with block scales, split bf16, e4m3 with column scales (dense
    blocks bf16), float accumulation: error against the float64 oracle on the
    unquantised factors, so the storage rounding counts."""
    P, Ho, X, Y = log2d_16384
    H = hm.HMatrix(P, 0, 64, 16, 0.0, prec=prec, method=METHOD_RSVD, seed=44)
    want = hm.PATH_STREAMED if k == 1 else hm.PATH_TENSOR
    e = rel(gpu_apply(H, X[:, :k], path=want), Y[:, :k])
    assert e <= PREC_TOL[prec], e


@pytest.mark.parametrize("prec", [2, 3, 4])
def test_storage_precisions_ragged_3d(hm, prec):
    """Padded leaves (uniform random points in 3D), random blocks."""
    P = w.uniform_points(6000, 3, 17)
    Ho = o.build_hmatrix(P, 2, 48, 8, method=METHOD_RANDOM, seed=17)
    H = hm.HMatrix(P, 2, 48, 8, 0.0, prec=prec, method=METHOD_RANDOM, seed=17)
    X = w.gaussian_rhs(6000, 3, 84)
    e = rel(gpu_apply(H, X), o.hmat_matvec(Ho, X))
    assert e <= PREC_TOL[prec], e


def test_device_status_word_selftest(hm):
    """The error path of the bounded waits: a kernel whose one wait cannot
    complete gives up after its limit, sets the status word and returns;
    hmat_check reports HMAT_ETIMEOUT once and clears the word, and the
    context stays usable for correct products."""
    import time
    P = w.grid_points(64, 2)
    Ho, H = build_pair(hm, P, 0, 64, 8, METHOD_RSVD, 11, 1)
    x = w.gaussian_rhs(P.shape[0], 1, 12)
    y0 = gpu_apply(H, x)
    t = time.perf_counter()
    assert hm.hmat_selftest_timeout(H.h, 5000) == (hm.HMAT_ETIMEOUT, 1)
    assert time.perf_counter() - t < 5.0
    assert hm.hmat_check(H.h) == (0, 0)
    y1 = gpu_apply(H, x)
    assert np.array_equal(y0, y1)
    assert rel(y1, o.hmat_matvec(Ho, x)) <= TOL[1]


def test_save_load_on_device(hm, tmp_path):
    """A handle written by hmat_save and read by hmat_load onto the GPU gives
    the same FP32 product as the original, bitwise, and in bf16 (storage
    chosen at load) stays within the bf16 tolerance of the oracle."""
    import torch
    P = w.grid_points(64, 2)
    Ho = o.build_hmatrix(P, 2, 64, 8, method=METHOD_RANDOM, seed=23)
    opts = hm.hmat_default_opts(device=0, method=METHOD_RANDOM, seed=23, prec=1, keep_host=1)
    h = hm.hmat_build(P, 2, 64, 8, 0.0, opts)
    path = str(tmp_path / "g.hmat")
    hm.hmat_save(h, path)
    g = hm.hmat_load(path)
    ob = hm.hmat_default_opts(device=0, prec=2)
    gb = hm.hmat_load(path, ob)
    X = w.gaussian_rhs(4096, 3, 24)
    x = torch.from_numpy(X).float().cuda()
    ys = []
    for hh in (h, g, gb):
        y = torch.empty_like(x)
        hm.hmat_matvec(hh, x, y, 3, 3, 3, 0, None)
        torch.cuda.synchronize()
        assert hm.hmat_check(hh) == (0, 0)
        ys.append(y.double().cpu().numpy())
    assert np.array_equal(ys[0], ys[1])
    ref = o.hmat_matvec(Ho, X)
    assert rel(ys[0], ref) <= TOL[1]
    assert rel(ys[2], ref) <= 1e-2
    for hh in (h, g, gb):
        hm.hmat_destroy(hh)
