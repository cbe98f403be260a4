"""Tensor-core path at the full sizes and in the launch configuration that
bench.py times for several right-hand sides (bf16 storage):

  3D 64^3 grid (N = 262,144), leaf 64, rank 32, 32 right-hand sides --
     s r = 224 columns per node: one 128-column box and a 96-column
     remainder box per level;
  2D 1024^2 grid (N = 1,048,576), leaf 64, rank 16, 64 right-hand sides.

Random-filled blocks (the paper's benchmark matrices), so the oracle
regenerates any block exactly and computes sampled output rows one by one
(eq. (hmat-vec-add) restricted to those rows).  Error = rel-L2 over the
sampled rows and all right-hand sides against the float64 oracle on the
unrounded blocks.  Tolerances: bf16 1e-2 (factors, x and the summed t are
rounded to bf16, accumulation is float), split bf16 1e-5, e4m3 5e-2."""
import numpy as np
import pytest

import oracle as o
import workloads as w
from oracle.hmatrix import KERNEL_RANDOM, METHOD_RANDOM

pytestmark = pytest.mark.gpu

BF16_TOL = 1e-2
TOL = {2: 1e-2, 3: 1e-5, 4: 5e-2}
_ORACLE = {}


@pytest.fixture(scope="module")
def hm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_12441_gb300 import _build
    _build.build()
    from paper_2008_12441_gb300 import hmat
    return hmat


def oracle_rows(P, r, seed, X, rows):
    """FP64 oracle rows, cached per workload (shared by the storage modes)."""
    key = (P.shape, r, seed, X.shape)
    if key not in _ORACLE:
        Ho = o.build_hmatrix(P, KERNEL_RANDOM, 64, r, method=METHOD_RANDOM, seed=seed,
                             materialize=False)
        Xo = np.empty_like(X)
        Xo[Ho.tree.perm] = X
        _ORACLE[key] = o.hmat_matvec_rows(Ho, Xo, rows)
    return _ORACLE[key]


def sampled_rows_error(hm, n, d, r, k, seed, prec=2):
    """Rows at one position of every 128- and 256-slot tile and at both ends
    of every persistent CTA range (workloads.covering_rows), x and y in tree
    order as bench.py passes them; asserts the tensor-core kernels ran."""
    import torch
    P = w.grid_points(n, d)
    N = P.shape[0]
    H = hm.HMatrix(P, KERNEL_RANDOM, 64, r, 0.0, prec=prec, method=METHOD_RANDOM, seed=seed,
                   max_nrhs=k)
    X = w.gaussian_rhs(N, k, seed + 1)
    x = torch.from_numpy(X).float().cuda()
    y = H.matvec(x, flags=hm.HMAT_TREE_ORDER)
    torch.cuda.synchronize()
    assert H.check() == (0, 0)
    assert H.last_path() == hm.PATH_TENSOR, H.last_path()
    Y = y.double().cpu().numpy()
    H.close()
    rows = w.covering_rows(N, torch.cuda.get_device_properties(0).multi_processor_count, seed)
    Yo = oracle_rows(P, r, seed, X, rows)
    Yg = Y[rows]
    assert np.all(np.isfinite(Yg))
    return float(np.linalg.norm(Yg - Yo) / np.linalg.norm(Yo))


@pytest.mark.parametrize("prec", [2, 3, 4])
def test_3d_n262144_rank32_32rhs_tensor_cores(hm, prec):
    e = sampled_rows_error(hm, 64, 3, 32, 32, 23, prec=prec)
    assert e <= TOL[prec], e


@pytest.mark.parametrize("prec", [2, 3, 4])
def test_2d_n1048576_rank16_64rhs_tensor_cores(hm, prec):
    """The precision sweep's configuration: bf16 (block scales), split bf16
    (accumulation segments of four tiles keep the tensor-memory sums short
    enough for 1e-5), e4m3 (column scales, bf16 near field)."""
    e = sampled_rows_error(hm, 1024, 2, 16, 64, 24, prec=prec)
    assert e <= TOL[prec], e
