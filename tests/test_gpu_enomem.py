"""Out-of-memory paths on the device, without exhausting the GPU: the
library's allocation-failure hook makes the k-th allocation of a build, a
workspace clone or a precision conversion fail; each call must return
HMAT_ENOMEM and leave the device's free memory where it was (everything it
had allocated is freed), and the library must work normally afterwards."""
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


def free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("prec", [1, 2])
def test_every_device_allocation_of_a_build_can_fail_cleanly(hm, prec):
    import torch
    P = w.grid_points(64, 2)
    opts = hm.hmat_default_opts(device=0, method=2, seed=7, prec=prec, keep_host=1)
    h = hm.hmat_build(P, 2, 64, 8, 0.0, opts)          # warm: driver pools settled
    hm.hmat_destroy(h)
    base = free_bytes()
    failures = 0
    try:
        for after in range(64):
            hm.hmat_inject_alloc_failure(after)
            try:
                h = hm.hmat_build(P, 2, 64, 8, 0.0, opts)
            except hm.HMatError as err:
                assert err.code == hm.HMAT_ENOMEM, err
                failures += 1
                assert free_bytes() == base, after
                continue
            hm.hmat_inject_alloc_failure(-1)
            break
    finally:
        hm.hmat_inject_alloc_failure(-1)
    assert failures >= 8                    # factors, scales, maps, workspace, staging, ...
    # the handle built after the failures is correct
    Ho = o.build_hmatrix(P, 2, 64, 8, method=2, seed=7)
    x = w.gaussian_rhs(P.shape[0], 1, 8)
    xt = torch.from_numpy(x).float().cuda()
    y = torch.empty_like(xt)
    hm.hmat_matvec(h, xt, y, 1, 1, 1, 0, None)
    torch.cuda.synchronize()
    yo = o.hmat_matvec(Ho, x)
    tol = 1e-5 if prec == 1 else 1e-2
    assert np.linalg.norm(y.double().cpu().numpy() - yo) <= tol * np.linalg.norm(yo)
    # a clone and a conversion whose first allocation fails
    base = free_bytes()
    hm.hmat_inject_alloc_failure(0)
    with pytest.raises(hm.HMatError) as ei:
        hm.hmat_clone_workspace(h)
    assert ei.value.code == hm.HMAT_ENOMEM
    hm.hmat_inject_alloc_failure(3)
    with pytest.raises(hm.HMatError) as ei:
        hm.hmat_convert(h, 3)
    assert ei.value.code == hm.HMAT_ENOMEM
    hm.hmat_inject_alloc_failure(-1)
    assert free_bytes() == base
    hm.hmat_destroy(h)
