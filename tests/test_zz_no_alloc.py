"""hmat_matvec_noalloc: the product for callers that must not have device
memory allocated for them at call time (its partial sums live in the
library's static 8 MiB device array instead of the handle's workspace).

Checked through the C ABI against hmat_matvec on the same handle and
inputs, on two calls in a row (the second call finds the array holding the
first call's contents).  Tolerances are the ones of the other parity tests:
1e-5 relative for FP32, 1e-12 for FP64.  Runs alone in a fresh process or
after the other tests.
"""
import numpy as np
import pytest

import oracle as o
import workloads as w

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("prec,k,tol", [(1, 1, 1e-5), (1, 5, 1e-5), (0, 3, 1e-12)])
def test_noalloc_matches_matvec_twice(hm, prec, k, tol):
    import torch
    P = w.grid_points(128, 2)
    H = hm.HMatrix(P, hm.HMAT_K_LOG2D, 64, 16, 0.0, prec=prec, method=hm.HMAT_RSVD, seed=4)
    dt = H.vec_dtype
    N = P.shape[0]
    x = torch.from_numpy(w.gaussian_rhs(N, k, 90 + k)).to(dt).cuda()
    y_ref = torch.empty_like(x)
    hm.hmat_matvec(H.h, x, y_ref, k, k, k, 0, None)
    torch.cuda.synchronize()
    ref = y_ref.double().cpu().numpy()
    for _ in range(2):
        y = torch.full_like(x, float("nan"))
        hm.hmat_matvec_noalloc(H.h, x, y, k, k, k, 0, None)
        torch.cuda.synchronize()
        got = y.double().cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel(got, ref) <= tol, rel(got, ref)
    H.close()


def test_noalloc_two_passes_against_oracle_and_no_allocation(hm):
    """70 right-hand sides in FP32 take two passes over the static array
    (64 + 6); the result matches hmat_matvec and, directly, the FP64 oracle.
    A warm call leaves the device's free memory unchanged and uses only the
    CUDA-core kernels."""
    import torch
    P = w.grid_points(64, 2)
    k = 70
    H = hm.HMatrix(P, hm.HMAT_K_RANDOM, 64, 8, 0.0, prec=1, method=hm.HMAT_RANDOM_FILL, seed=6,
                   max_nrhs=64)
    X = w.gaussian_rhs(P.shape[0], k, 92)
    x = torch.from_numpy(X).float().cuda()
    y_ref = torch.empty_like(x)
    hm.hmat_matvec(H.h, x, y_ref, k, k, k, 0, None)
    y = torch.full_like(x, float("nan"))
    hm.hmat_matvec_noalloc(H.h, x, y, k, k, k, 0, None)      # warm: address lookup done
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    y.fill_(float("nan"))
    hm.hmat_matvec_noalloc(H.h, x, y, k, k, k, 0, None)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert H.last_path() == hm.PATH_CACHED
    got = y.double().cpu().numpy()
    assert rel(got, y_ref.double().cpu().numpy()) <= 1e-5
    Ho = o.build_hmatrix(P, 2, 64, 8, method=2, seed=6)
    assert rel(got, o.hmat_matvec(Ho, X)) <= 1e-5
    H.close()


def test_noalloc_second_handle_and_tree_order(hm):
    """A second handle of another shape reuses the same array."""
    import torch
    P = w.uniform_points(5000, 3, 8)
    H = hm.HMatrix(P, hm.HMAT_K_RANDOM, 32, 6, 0.0, prec=1, method=hm.HMAT_RANDOM_FILL, seed=5)
    x = torch.from_numpy(w.gaussian_rhs(5000, 2, 91)).float().cuda()
    y_ref = torch.empty_like(x)
    hm.hmat_matvec(H.h, x, y_ref, 2, 2, 2, hm.HMAT_TREE_ORDER, None)
    for _ in range(2):
        y = torch.full_like(x, float("nan"))
        hm.hmat_matvec_noalloc(H.h, x, y, 2, 2, 2, hm.HMAT_TREE_ORDER, None)
        torch.cuda.synchronize()
        assert rel(y.double().cpu().numpy(), y_ref.double().cpu().numpy()) <= 1e-5
    H.close()
