"""GPU parity of the product under standard admissibility (Definition
"Standard admissibility condition", eq. (standard-ad-cond), rho = sqrt(d))
against the FP64 oracle's standard block structure: interaction lists of
27 (2D) / 189 (3D) nodes routed by the expand kernel's stencil table, near
field over the 3^d touching groups.  Streamed kernels only (each test
asserts it), one right-hand side per pass.  Tolerances: FP64 1e-12, FP32
and split bf16 1e-5, bf16 1e-2, e4m3 5e-2."""
import numpy as np
import pytest

import oracle as o
import workloads as w
from oracle.hmatrix import METHOD_RANDOM, METHOD_RSVD

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


def build(hm, P, kern, m, r, meth, seed, prec):
    return hm.HMatrix(P, kern, m, r, 0.0, prec=prec, method=meth, seed=seed,
                      admissibility=hm.HMAT_ADM_STANDARD)


def apply(hm, H, X, flags=0):
    import torch
    x = torch.from_numpy(np.ascontiguousarray(X)).to(H.vec_dtype).cuda()
    y = H.matvec(x, flags=flags)
    torch.cuda.synchronize()
    assert H.check() == (0, 0)
    assert H.last_path() == hm.PATH_STREAMED, H.last_path()
    return y.double().cpu().numpy()


def test_standard_2d_fp64_rsvd_full_vector(hm):
    """128^2 grid, log kernel, randomized SVD rank 8 (the same seeded sketches
    on both sides), FP64: every output against the oracle; and the kernel
    rows show the smaller compression error of standard admissibility."""
    P = w.grid_points(128, 2)
    Ho = o.build_hmatrix(P, 0, 64, 8, method=METHOD_RSVD, seed=60, admissibility="standard")
    H = build(hm, P, 0, 64, 8, METHOD_RSVD, 60, 0)
    assert H.info.admissibility == 1 and H.info.partners == 27
    x = w.gaussian_rhs(P.shape[0], 1, 61)
    ys = apply(hm, H, x)
    e = rel(ys, o.hmat_matvec(Ho, x))
    assert e <= TOL[0], e
    rows = np.arange(0, P.shape[0], 97)
    Krows = o.kernel_eval(0, P[rows], P, rows, np.arange(P.shape[0]))
    Hw = hm.HMatrix(P, 0, 64, 8, 0.0, prec=0, method=METHOD_RSVD, seed=60)
    yw = apply(hm, Hw, x)
    ew = rel(yw[rows, 0], Krows @ x[:, 0])
    es = rel(ys[rows, 0], Krows @ x[:, 0])
    assert es < ew, (es, ew)


@pytest.mark.parametrize("prec,k", [(1, 1), (1, 3), (0, 2)])
def test_standard_2d_random_fill(hm, prec, k):
    P = w.grid_points(128, 2)
    Ho = o.build_hmatrix(P, 2, 64, 8, method=METHOD_RANDOM, seed=62, admissibility="standard")
    H = build(hm, P, 2, 64, 8, METHOD_RANDOM, 62, prec)
    X = w.gaussian_rhs(P.shape[0], k, 63)
    e = rel(apply(hm, H, X), o.hmat_matvec(Ho, X))
    assert e <= TOL[prec], e


@pytest.mark.parametrize("prec", [2, 3, 4])
def test_standard_storage_precisions(hm, prec):
    P = w.grid_points(128, 2)
    Ho = o.build_hmatrix(P, 2, 64, 16, method=METHOD_RANDOM, seed=64, admissibility="standard")
    H = build(hm, P, 2, 64, 16, METHOD_RANDOM, 64, prec)
    x = w.gaussian_rhs(P.shape[0], 1, 65)
    e = rel(apply(hm, H, x), o.hmat_matvec(Ho, x))
    assert e <= TOL[prec], e


def sampled(hm, P, m, r, seed, prec=1):
    import torch
    N = P.shape[0]
    H = build(hm, P, 2, m, r, METHOD_RANDOM, seed, prec)
    X = w.gaussian_rhs(N, 1, seed + 1)
    Y = apply(hm, H, X, flags=hm.HMAT_TREE_ORDER)
    H.close()
    Ho = o.build_hmatrix(P, 2, m, r, method=METHOD_RANDOM, seed=seed, materialize=False,
                         admissibility="standard")
    rows = w.covering_rows(N, torch.cuda.get_device_properties(0).multi_processor_count, seed)
    Xo = np.empty_like(X)
    Xo[Ho.tree.perm] = X
    return rel(Y[rows], o.hmat_matvec_rows(Ho, Xo, rows))


def test_standard_2d_n262144_sampled_rows(hm):
    """512^2 grid, random fill rank 8, FP32: rows of every tile and CTA range."""
    e = sampled(hm, w.grid_points(512, 2), 64, 8, 66)
    assert e <= TOL[1], e


def test_standard_3d_n32768_sampled_rows(hm):
    """32^3 grid, leaf 64, random fill rank 4: 189 interaction-list slots per
    node, near field over 27 groups of 512 slots."""
    e = sampled(hm, w.grid_points(32, 3), 64, 4, 67)
    assert e <= TOL[1], e


def test_standard_refusals(hm):
    """Ragged leaves (no streamed geometry) are refused at build; the
    allocation-free and transposed products are refused for a standard
    handle."""
    import torch
    with pytest.raises(hm.HMatError) as ei:
        build(hm, w.uniform_points(5000, 2, 68), 2, 32, 4, METHOD_RANDOM, 68, 1)
    assert ei.value.code == hm.HMAT_EUNSUPPORTED
    H = build(hm, w.grid_points(64, 2), 2, 64, 4, METHOD_RANDOM, 69, 1)
    x = torch.zeros(4096, 1, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(hm.HMatError) as ei:
        hm.hmat_matvec_noalloc(H.h, x, y, 1, 1, 1, 0, None)
    assert ei.value.code == hm.HMAT_EUNSUPPORTED
    with pytest.raises(hm.HMatError) as ei:
        hm.hmat_matvec(H.h, x, y, 1, 1, 1, hm.HMAT_TRANSPOSE, None)
    assert ei.value.code == hm.HMAT_EUNSUPPORTED
    H.close()
