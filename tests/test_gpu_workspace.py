"""The GEMV form y = alpha K x + beta y (the remark closing the algorithm
of Sec. 4.1) against the FP64 oracle, and workspace clones: products on a
clone are bitwise those of the original, clones run concurrently on
separate streams, a product on another stream while the handle's previous
one is in flight is refused, and the destroy order is enforced."""
import numpy as np
import pytest

import oracle as o
import workloads as w
from oracle.hmatrix import KERNEL_RANDOM, METHOD_RANDOM

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


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("k", [1, 3])
def test_gemv_against_oracle(hm, prec, k):
    import torch
    P = w.grid_points(64, 2)
    N = P.shape[0]
    Ho = o.build_hmatrix(P, KERNEL_RANDOM, 32, 8, method=METHOD_RANDOM, seed=31)
    # max_nrhs 2: k = 3 runs in two chunks through the staging buffer
    H = hm.HMatrix(P, KERNEL_RANDOM, 32, 8, 0.0, prec=prec, method=METHOD_RANDOM, seed=31,
                   max_nrhs=2)
    dt = H.vec_dtype
    X = w.gaussian_rhs(N, k, 32)
    Y0 = w.gaussian_rhs(N, k, 33)
    KX = o.hmat_matvec(Ho, X)
    for alpha, beta in [(1.0, 0.0), (2.5, -0.5), (0.0, 1.5), (-1.0, 1.0)]:
        x = torch.from_numpy(X).to(dt).cuda()
        # y is a strided view (leading dimension k + 2); the pad columns stay put
        buf = torch.full((N, k + 2), 7.0, dtype=dt, device="cuda")
        y = buf[:, :k]
        if beta == 0.0:
            y.fill_(float("nan"))        # not read when beta == 0
        else:
            y.copy_(torch.from_numpy(Y0).to(dt))
        H.gemv(alpha, x, beta, y)
        torch.cuda.synchronize()
        assert H.check() == (0, 0)
        got = buf[:, :k].double().cpu().numpy()
        # the y the kernel read: Y0 rounded to the vectors' precision
        y0_used = Y0.astype(np.float32).astype(np.float64) if prec == 1 else Y0
        want = alpha * KX + beta * y0_used if beta != 0.0 else alpha * KX
        assert np.isfinite(got).all()
        e = rel(got, want)
        assert e <= TOL[prec], (alpha, beta, e)
        assert (buf[:, k:] == 7.0).all()
    H.close()


def build_pair(hm, prec, d, n, m, r, max_nrhs=64):
    P = w.grid_points(n, d)
    H = hm.HMatrix(P, KERNEL_RANDOM, m, r, 0.0, prec=prec, method=METHOD_RANDOM, seed=41,
                   max_nrhs=max_nrhs)
    return P, H


@pytest.mark.parametrize("prec,d,n,k", [(1, 2, 128, 1), (1, 2, 128, 5), (2, 3, 16, 32)])
def test_clone_products_bitwise_and_concurrent(hm, prec, d, n, k):
    """(2, 3, 16, 32): bf16 storage, 32 right-hand sides -- the tensor-core
    kernels with the clone's own prepared operands."""
    import torch
    P, H = build_pair(hm, prec, d, n, 64, 8)
    C = H.clone_workspace()
    C2 = C.clone_workspace()                      # a clone of a clone borrows the same factors
    assert C.info.factor_entries == H.info.factor_entries
    assert 0 < C.info.workspace_bytes <= H.info.workspace_bytes
    N = H.N
    xs = [torch.from_numpy(w.gaussian_rhs(N, k, 50 + i)).float().cuda() for i in range(3)]
    ref = []
    for x in xs:
        ref.append(H.matvec(x).clone())
    torch.cuda.synchronize()
    for h in (C, C2):
        for x, r in zip(xs, ref):
            y = h.matvec(x)
            torch.cuda.synchronize()
            assert torch.equal(y, r)
    # the three handles at once on three streams, several rounds each
    streams = [torch.cuda.Stream() for _ in range(3)]
    outs = [[torch.empty_like(ref[i]) for _ in range(4)] for i in range(3)]
    torch.cuda.synchronize()
    for rnd in range(4):
        for i, (h, st) in enumerate(zip((H, C, C2), streams)):
            with torch.cuda.stream(st):
                h.matvec(xs[i], outs[i][rnd], stream=st)
    torch.cuda.synchronize()
    for i in range(3):
        for rnd in range(4):
            assert torch.equal(outs[i][rnd], ref[i]), (i, rnd)
    for h in (H, C, C2):
        assert h.check() == (0, 0)
    # host entry point on a clone: its own staging
    xh = xs[0].cpu().numpy()
    yh = np.empty_like(xh)
    hm.hmat_matvec_host(C.h, xh, yh, k, k, k, 0, None)
    assert np.array_equal(yh, ref[0].cpu().numpy())
    C2.close()
    C.close()
    H.close()


def test_cross_stream_conflict_refused(hm):
    import torch
    P, H = build_pair(hm, 1, 2, 128, 64, 8)
    C = H.clone_workspace()
    x = torch.from_numpy(w.gaussian_rhs(H.N, 1, 60)).float().cuda()
    want = H.matvec(x).clone()
    torch.cuda.synchronize()
    A, B = torch.cuda.Stream(), torch.cuda.Stream()
    ya, yb, yc = torch.empty_like(x), torch.empty_like(x), torch.empty_like(x)
    with torch.cuda.stream(A):
        torch.cuda._sleep(200_000_000)           # stream A busy for a while (bounded spin)
    H.matvec(x, ya, stream=A)                    # queued behind it
    with pytest.raises(hm.HMatError) as ei:
        H.matvec(x, yb, stream=B)                # same workspace, another stream, in flight
    assert ei.value.code == hm.HMAT_EUNSUPPORTED
    C.matvec(x, yc, stream=B)                    # a clone has its own workspace
    H.matvec(x, ya, stream=A)                    # the same stream is always fine
    A.synchronize()
    H.matvec(x, yb, stream=B)                    # A is done: B may take the handle
    torch.cuda.synchronize()
    for y in (ya, yb, yc):
        assert torch.equal(y, want)
    assert H.check() == (0, 0) and C.check() == (0, 0)
    # destroy order: the original cannot go while a clone borrows its factors
    with pytest.raises(hm.HMatError) as ei:
        H.close()
    assert ei.value.code == hm.HMAT_EINVAL
    C.close()
    H.close()
