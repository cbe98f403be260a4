"""GPU parity of the transposed product y = K^T x (HMAT_TRANSPOSE) against the
FP64 oracle's transposed product (every block applied from its target rows
to its source columns).  The same kernels run with U and V swapped and the
near-field blocks transposed (a device copy unless every block is
symmetric); each test asserts the kernel families that ran.  Tolerances as
the forward product: FP64 1e-12, FP32 and split bf16 1e-5, bf16 1e-2,
e4m3 5e-2."""
import numpy as np
import pytest

import oracle as o
import workloads as w
from oracle.hmatrix import METHOD_RANDOM, METHOD_RSVD, METHOD_TSVD

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5, 2: 1e-2, 3: 1e-5, 4: 5e-2}


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


def apply_t(hm, H, X, flags=0, path=None):
    import torch
    x = torch.from_numpy(np.ascontiguousarray(X)).to(H.vec_dtype).cuda()
    y = torch.empty_like(x)
    k = x.shape[1]
    hm.hmat_matvec(H.h, x, y, k, k, k, flags | hm.HMAT_TRANSPOSE, None)
    torch.cuda.synchronize()
    assert H.check() == (0, 0)
    if path is not None:
        assert H.last_path() == path, (H.last_path(), path)
    return y.double().cpu().numpy()


@pytest.mark.parametrize("prec,k", [(0, 1), (0, 3), (1, 1), (1, 64)])
def test_transpose_random_fill_against_oracle(hm, prec, k):
    """Random blocks (near field not symmetric: the transposed copy is used)."""
    P = w.grid_points(128, 2)
    Ho = o.build_hmatrix(P, 2, 64, 8, method=METHOD_RANDOM, seed=41)
    H = hm.HMatrix(P, 2, 64, 8, 0.0, prec=prec, method=METHOD_RANDOM, seed=41)
    X = w.gaussian_rhs(P.shape[0], k, 42)
    want = hm.PATH_STREAMED if k == 1 else hm.PATH_CACHED
    e = rel(apply_t(hm, H, X, path=want), o.hmat_matvec_transpose(Ho, X))
    assert e <= TOL[prec], e
    # the forward product of the same handle is unchanged afterwards
    Yf = H.matvec(__import__("torch").from_numpy(X).to(H.vec_dtype).cuda())
    assert rel(Yf.double().cpu().numpy(), o.hmat_matvec(Ho, X)) <= TOL[prec]


def test_transpose_symmetric_kernel_uses_d_itself(hm):
    """The log kernel's near-field blocks are symmetric: no transposed copy
    is made (device bytes unchanged) and K^T x matches the oracle."""
    P = w.grid_points(64, 2)
    Ho = o.build_hmatrix(P, 0, 64, 8, method=METHOD_TSVD)
    H = hm.HMatrix(P, 0, 64, 8, 0.0, prec=0, method=METHOD_TSVD)
    before = hm.hmat_info(H.h).device_bytes
    hm.hmat_prepare_transpose(H.h)
    after = hm.hmat_info(H.h).device_bytes
    assert after - before < P.shape[0] * 64          # maps only, no G x G copies
    X = w.gaussian_rhs(P.shape[0], 2, 43)
    e = rel(apply_t(hm, H, X), o.hmat_matvec_transpose(Ho, X))
    assert e <= TOL[0], e


@pytest.mark.parametrize("prec", [2, 3, 4])
@pytest.mark.parametrize("k", [1, 16])
def test_transpose_storage_precisions(hm, prec, k):
    """bf16 / split bf16 / e4m3 storage: streamed kernels at one right-hand
    side, tensor cores at 16."""
    P = w.grid_points(128, 2)
    Ho = o.build_hmatrix(P, 2, 64, 16, method=METHOD_RANDOM, seed=44)
    H = hm.HMatrix(P, 2, 64, 16, 0.0, prec=prec, method=METHOD_RANDOM, seed=44, max_nrhs=16)
    X = w.gaussian_rhs(P.shape[0], k, 45)
    want = hm.PATH_STREAMED if k == 1 else hm.PATH_TENSOR
    e = rel(apply_t(hm, H, X, path=want), o.hmat_matvec_transpose(Ho, X))
    assert e <= TOL[prec], e


@pytest.mark.parametrize("flags", [0, 1])
def test_transpose_ragged_points_orders(hm, flags):
    """Uniform random points (padded leaves, CUDA-core kernels), original and
    tree order."""
    P = w.uniform_points(5000, 3, 46)
    Ho = o.build_hmatrix(P, 2, 48, 6, method=METHOD_RANDOM, seed=46)
    H = hm.HMatrix(P, 2, 48, 6, 0.0, prec=0, method=METHOD_RANDOM, seed=46)
    X = w.gaussian_rhs(5000, 2, 47)
    Yo = o.hmat_matvec_transpose(Ho, X)
    if flags:
        perm = H.perm()
        e = rel(apply_t(hm, H, X[perm], flags=hm.HMAT_TREE_ORDER), Yo[perm])
    else:
        e = rel(apply_t(hm, H, X), Yo)
    assert e <= TOL[0], e


def test_transpose_gemv_clone_and_noalloc(hm):
    """y = alpha K^T x + beta y, a workspace clone (sharing the prepared
    transposition) and the allocation-free entry point, against the oracle."""
    import torch
    P = w.grid_points(64, 2)
    Ho = o.build_hmatrix(P, 2, 64, 8, method=METHOD_RANDOM, seed=48)
    H = hm.HMatrix(P, 2, 64, 8, 0.0, prec=1, method=METHOD_RANDOM, seed=48)
    X = w.gaussian_rhs(P.shape[0], 2, 49)
    Y0 = w.gaussian_rhs(P.shape[0], 2, 50)
    ref = o.hmat_matvec_transpose(Ho, X)
    x = torch.from_numpy(X).float().cuda()
    # the allocation-free entry point refuses K^T before the preparation
    y = torch.empty_like(x)
    with pytest.raises(hm.HMatError):
        hm.hmat_matvec_noalloc(H.h, x, y, 2, 2, 2, hm.HMAT_TRANSPOSE, None)
    hm.hmat_prepare_transpose(H.h)
    hm.hmat_matvec_noalloc(H.h, x, y, 2, 2, 2, hm.HMAT_TRANSPOSE, None)
    torch.cuda.synchronize()
    assert rel(y.double().cpu().numpy(), ref) <= 1e-5
    yg = torch.from_numpy(Y0).float().cuda()
    hm.hmat_gemv(H.h, 0.5, x, -2.0, yg, 2, 2, 2, hm.HMAT_TRANSPOSE, None)
    torch.cuda.synchronize()
    assert rel(yg.double().cpu().numpy(), 0.5 * ref - 2.0 * Y0) <= 1e-5
    c = H.clone_workspace()
    yc = torch.empty_like(x)
    hm.hmat_matvec(c.h, x, yc, 2, 2, 2, hm.HMAT_TRANSPOSE, None)
    torch.cuda.synchronize()
    assert rel(yc.double().cpu().numpy(), ref) <= 1e-5
    c.close()
    H.close()


def test_full_size_transpose_n262144_sampled_rows(hm):
    """512^2 grid, random fill rank 16, FP32, one right-hand side through the
    streamed kernels: rows of every tile and CTA range against the oracle's
    transposed rows."""
    import torch
    P = w.grid_points(512, 2)
    N = P.shape[0]
    H = hm.HMatrix(P, 2, 64, 16, 0.0, prec=1, method=METHOD_RANDOM, seed=51)
    X = w.gaussian_rhs(N, 1, 52)
    Y = apply_t(hm, H, X, flags=hm.HMAT_TREE_ORDER, path=hm.PATH_STREAMED)
    H.close()
    Ho = o.build_hmatrix(P, 2, 64, 16, method=METHOD_RANDOM, seed=51, materialize=False)
    rows = w.covering_rows(N, torch.cuda.get_device_properties(0).multi_processor_count, 51)
    Xo = np.empty_like(X)
    Xo[Ho.tree.perm] = X
    e = rel(Y[rows], o.hmat_matvec_transpose_rows(Ho, Xo, rows))
    assert e <= TOL[1], e


def test_adjoint_identity_kernel_operator_full_size(hm):
    """<y, K x> = <K^T y, x> on the 1024^2 log-kernel operator (randomized
    SVD, FP32, one right-hand side): a property of any operator and its
    transpose, checked at the full size without the oracle; the two sides
    differ by FP32 rounding only."""
    import torch
    P = w.grid_points(1024, 2)
    N = P.shape[0]
    H = hm.HMatrix(P, 0, 64, 16, 0.0, prec=1, method=METHOD_RSVD, seed=12444)
    x = torch.from_numpy(w.gaussian_rhs(N, 1, 53)).float().cuda()
    y = torch.from_numpy(w.gaussian_rhs(N, 1, 54)).float().cuda()
    kx = torch.empty_like(x)
    kty = torch.empty_like(y)
    hm.hmat_matvec(H.h, x, kx, 1, 1, 1, hm.HMAT_TREE_ORDER, None)
    hm.hmat_matvec(H.h, y, kty, 1, 1, 1, hm.HMAT_TREE_ORDER | hm.HMAT_TRANSPOSE, None)
    torch.cuda.synchronize()
    assert H.check() == (0, 0)
    assert H.last_path() == hm.PATH_STREAMED
    lhs = float(torch.dot(y[:, 0].double(), kx[:, 0].double()))
    rhs = float(torch.dot(kty[:, 0].double(), x[:, 0].double()))
    scale = float(torch.linalg.norm(y.double()) * torch.linalg.norm(kx.double()))
    assert abs(lhs - rhs) <= 1e-5 * scale, (lhs, rhs, scale)
    H.close()
