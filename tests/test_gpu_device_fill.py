"""The random fill written straight into the device layout (build_gpu, no
float64 host copy) against the host-built fill of the same seed: the same
blocks bit for bit, hence bitwise equal products through the same kernels.
(The full-size FP32 parity tests at 512^2 and 1024^2 build their random
fills this way: N >= 65536 selects it by default.)"""
import numpy as np
import pytest

import oracle as o
import workloads as w
from oracle.hmatrix import METHOD_RANDOM

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


@pytest.mark.parametrize("d,n,r,prec,lr", [(2, 256, 16, 1, 0), (3, 32, 8, 0, 0), (2, 128, 4, 1, 1)])
def test_device_fill_equals_host_fill(hm, d, n, r, prec, lr):
    import torch
    P = w.grid_points(n, d)
    N = P.shape[0]
    Hd = hm.HMatrix(P, 2, 64, r, 0.0, prec=prec, method=METHOD_RANDOM, seed=71, build_gpu=1,
                    leaf_lowrank=lr)
    Hh = hm.HMatrix(P, 2, 64, r, 0.0, prec=prec, method=METHOD_RANDOM, seed=71, keep_host=1,
                    leaf_lowrank=lr)
    for f in ("factor_entries", "dense_entries", "lowrank_blocks", "dense_blocks", "depth"):
        assert getattr(Hd.info, f) == getattr(Hh.info, f), f
    x = torch.from_numpy(w.gaussian_rhs(N, 1, 72)).to(Hd.vec_dtype).cuda()
    yd = Hd.matvec(x, flags=hm.HMAT_TREE_ORDER)
    yh = Hh.matvec(x, flags=hm.HMAT_TREE_ORDER)
    torch.cuda.synchronize()
    assert Hd.check() == (0, 0) and Hh.check() == (0, 0)
    assert torch.equal(yd, yh)
    # the device-filled handle has no host copy
    with pytest.raises(hm.HMatError):
        hm.hmat_export_dense(Hd.h, 0)
    Hd.close()
    Hh.close()
