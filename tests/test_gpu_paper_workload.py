"""GPU parity on the matrices of the paper's experiments (Sec. 5.1, 5.2):
random-filled H-matrices under weak admissibility, rank 4, on n^d grids,
one right-hand side at a time (the paper averages over random input
vectors).  Leaf size 64, the one `bench.py --paper-table` times; the sizes
here are small enough for the oracle but span several streamed tiles.
Error = ||y_gpu - y_oracle|| / ||y_oracle|| against the FP64 oracle, which
regenerates the same blocks from the same seed."""
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


@pytest.mark.parametrize("d,n,prec,flags", [(2, 128, 1, 0), (2, 256, 1, 0), (2, 128, 0, 0),
                                            (3, 32, 1, 0), (3, 32, 0, 0), (2, 256, 1, 1),
                                            (3, 32, 1, 1)])
def test_paper_matrices_rank4(hm, d, n, prec, flags):
    """flags 1: vectors in tree order (on a grid, x is then copied per tile
    with one bulk copy instead of through the slot map)."""
    import torch
    P = w.grid_points(n, d)
    N = P.shape[0]
    seed = 12446
    Ho = o.build_hmatrix(P, KERNEL_RANDOM, 64, 4, method=METHOD_RANDOM, seed=seed)
    H = hm.HMatrix(P, KERNEL_RANDOM, 64, 4, 0.0, prec=prec, method=METHOD_RANDOM, seed=seed,
                   max_nrhs=1)
    assert H.info.rank_per_level[1] == 4
    perm = H.perm() if flags else np.arange(N)
    for v in range(3):
        x = w.gaussian_rhs(N, 1, 900 + v)
        xt = torch.from_numpy(np.ascontiguousarray(x[perm])).to(H.vec_dtype).cuda()
        y = H.matvec(xt, flags=flags)
        torch.cuda.synchronize()
        assert H.check() == (0, 0)
        e = rel(y.double().cpu().numpy(), o.hmat_matvec(Ho, x)[perm])
        assert e <= TOL[prec], (d, n, prec, flags, v, e)
    H.close()
