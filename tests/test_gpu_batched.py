"""Batched products (one CUDA graph, persistent CTAs pulling tasks) against
the FP64 oracle and against the single-instance entry point."""
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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def uneven_instances(count, seed):
    """Uneven instances as in the batched workload (2D and 3D uniform random
    points, log-uniform N, rank in {8, 16, 32}, 1..16 right-hand sides), at
    sizes the oracle handles quickly; random blocks."""
    insts = w.c5_batched(count=count, seed=seed, n_lo=600, n_hi=6000)
    return insts


@pytest.mark.parametrize("prec,tol", [(1, 1e-5), (2, 1e-2), (0, 1e-12)])
def test_batched_against_oracle_and_single(hm, prec, tol):
    import torch
    insts = uneven_instances(10, 777)
    Hs, Xs, Ys, refs = [], [], [], []
    for i, inst in enumerate(insts):
        P = inst.points()
        H = hm.HMatrix(P, hm.HMAT_K_RANDOM, 64, inst.rank, 0.0, prec=prec,
                       method=hm.HMAT_RANDOM_FILL, seed=inst.seed)
        Ho = o.build_hmatrix(P, 2, 64, inst.rank, method=METHOD_RANDOM, seed=inst.seed)
        X = w.gaussian_rhs(inst.N, inst.nrhs, inst.seed + 5)
        refs.append(o.hmat_matvec(Ho, X))
        x = torch.from_numpy(X).to(H.vec_dtype).cuda()
        Hs.append(H)
        Xs.append(x)
        Ys.append(torch.full_like(x, float("nan")))
    b = hm.hmat_batch_create([H.h for H in Hs], [x.shape[1] for x in Xs])
    for rep in range(2):
        hm.hmat_batch_matvec(b, Xs, Ys)
        torch.cuda.synchronize()
        for H, x, y, ref in zip(Hs, Xs, Ys, refs):
            e = rel(y.double().cpu().numpy(), ref)
            assert e <= tol, e
            single = H.matvec(x)
            torch.cuda.synchronize()
            if prec in (0, 1) and x.shape[1] > 1:
                assert torch.equal(single, y)    # same CUDA-core kernels, same order
            else:
                # one right-hand side: the single path streams (another fixed
                # summation order); bf16: it may take the tensor cores
                assert rel(single.double().cpu().numpy(), ref) <= tol
                if prec in (0, 1):
                    close = 1e-13 if prec == 0 else 1e-6
                    assert rel(single.double().cpu().numpy(), y.double().cpu().numpy()) <= close
    hm.hmat_batch_destroy(b)
    for H in Hs:
        H.close()


def test_convert_matches_direct_build(hm):
    import torch
    P = w.grid_points(64, 2)
    H32 = hm.HMatrix(P, hm.HMAT_K_LOG2D, 32, 8, 0.0, prec=1, method=hm.HMAT_RSVD, seed=3,
                     keep_host=1)
    Hb = hm.HMatrix(P, hm.HMAT_K_LOG2D, 32, 8, 0.0, prec=2, method=hm.HMAT_RSVD, seed=3)
    hc = hm.hmat_convert(H32.h, 2)
    x = torch.from_numpy(w.gaussian_rhs(4096, 3, 9)).float().cuda()
    y1 = Hb.matvec(x)
    y2 = torch.empty_like(x)
    hm.hmat_matvec(hc, x, y2, 3, 3, 3, 0, None)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)
    hm.hmat_destroy(hc)


def test_autotuned_plan_against_oracle(hm):
    """hmat_batch_autotune times the candidate schedules (grid size x width
    classes), keeps the fastest and leaves its results in ys; the tuned plan
    then gives the same products (bitwise) and stays within the bf16
    tolerance of the FP64 oracle."""
    import torch
    insts = uneven_instances(8, 4242)
    Hs, Xs, Ys, refs = [], [], [], []
    for inst in insts:
        P = inst.points()
        H = hm.HMatrix(P, hm.HMAT_K_RANDOM, 64, inst.rank, 0.0, prec=2,
                       method=hm.HMAT_RANDOM_FILL, seed=inst.seed)
        Ho = o.build_hmatrix(P, 2, 64, inst.rank, method=METHOD_RANDOM, seed=inst.seed)
        X = w.gaussian_rhs(inst.N, inst.nrhs, inst.seed + 5)
        refs.append(o.hmat_matvec(Ho, X))
        Hs.append(H)
        Xs.append(torch.from_numpy(X).float().cuda())
        Ys.append(torch.full_like(Xs[-1], float("nan")))
    b = hm.hmat_batch_create([H.h for H in Hs], [x.shape[1] for x in Xs])
    t = hm.hmat_batch_autotune(b, Xs, Ys, reps=2)
    # six queue schedules, branch schedules of 4 and 8 branches
    assert t["candidates"] == 8
    if t["schedule"] == "queue":
        assert t["grid_div"] in (1, 2, 4) and t["coarse_widths"] in (0, 1) and t["branches"] == 0
    else:
        assert t["schedule"] == "branches" and t["branches"] in (4, 8)
    assert 0 < t["ms"] <= t["ms_default"]
    assert t["ms"] == min(t["ms_queue"], t["ms_branches"])
    for y, ref in zip(Ys, refs):
        assert rel(y.double().cpu().numpy(), ref) <= 1e-2
    Y2 = [torch.full_like(x, float("nan")) for x in Xs]
    hm.hmat_batch_matvec(b, Xs, Y2)
    torch.cuda.synchronize()
    for y, y2 in zip(Ys, Y2):
        assert torch.equal(y, y2)
    hm.hmat_batch_destroy(b)
    for H in Hs:
        H.close()


def padded_instances(hm, insts, prec, max_nrhs=16):
    """The uneven instances with leaf slots padded to 32 (2D) / 16 (3D): every
    near-field group a multiple of 128 slots, so the tensor-core kernels
    take them."""
    import torch
    Hs, Xs, Ys, refs = [], [], [], []
    for inst in insts:
        P = inst.points()
        H = hm.HMatrix(P, hm.HMAT_K_RANDOM, 64, inst.rank, 0.0, prec=prec,
                       method=hm.HMAT_RANDOM_FILL, seed=inst.seed, max_nrhs=max_nrhs,
                       leaf_slot_multiple=32 if inst.d == 2 else 16)
        assert H.info.leaf_slots % (32 if inst.d == 2 else 16) == 0
        Ho = o.build_hmatrix(P, 2, 64, inst.rank, method=METHOD_RANDOM, seed=inst.seed)
        X = w.gaussian_rhs(inst.N, inst.nrhs, inst.seed + 5)
        refs.append(o.hmat_matvec(Ho, X))
        Hs.append(H)
        Xs.append(torch.from_numpy(X).to(H.vec_dtype).cuda())
        Ys.append(torch.full_like(Xs[-1], float("nan")))
    return Hs, Xs, Ys, refs


@pytest.mark.parametrize("prec,tol", [(2, 1e-2), (3, 1e-5), (1, 1e-5)])
def test_branch_schedule_padded_instances(hm, prec, tol):
    """Branch schedule (each instance's own product on parallel graph
    branches) over padded uneven instances: bf16 and split bf16 take the
    tensor cores at 2..16 right-hand sides and the streamed project at one;
    every output against the FP64 oracle, twice, and again after the output
    buffers change (the graph is recorded again)."""
    import torch
    insts = uneven_instances(12, 9090)
    Hs, Xs, Ys, refs = padded_instances(hm, insts, prec)
    b = hm.hmat_batch_create([H.h for H in Hs], [x.shape[1] for x in Xs],
                             hm.HMAT_BATCH_BRANCHES)
    for rep in range(2):
        hm.hmat_batch_matvec(b, Xs, Ys)
        assert hm.hmat_batch_check(b) == 0
        for H, y, ref, inst in zip(Hs, Ys, refs, insts):
            e = rel(y.double().cpu().numpy(), ref)
            assert e <= tol, (inst, e)
            path = H.last_path()
            if prec in (2, 3) and inst.nrhs >= 2:
                assert path == hm.PATH_TENSOR, (inst, path)
            elif inst.nrhs == 1:
                assert path & hm.HMAT_PATH_PROJECT_STREAMED, (inst, path)
    Y2 = [torch.full_like(x, float("nan")) for x in Xs]
    hm.hmat_batch_matvec(b, Xs, Y2)
    assert hm.hmat_batch_check(b) == 0
    for y, y2 in zip(Ys, Y2):
        assert torch.equal(y, y2)
    hm.hmat_batch_destroy(b)
    for H in Hs:
        H.close()


def test_batch_refuses_repeated_handle(hm):
    import torch
    P = w.uniform_points(3000, 2, 5)
    H = hm.HMatrix(P, hm.HMAT_K_RANDOM, 64, 8, 0.0, prec=1, method=hm.HMAT_RANDOM_FILL, seed=5)
    for flags in (0, hm.HMAT_BATCH_BRANCHES):
        with pytest.raises(hm.HMatError) as ei:
            hm.hmat_batch_create([H.h, H.h], [1, 2], flags)
        assert ei.value.code == hm.HMAT_EINVAL
    with pytest.raises(hm.HMatError) as ei:
        hm.hmat_batch_create([H.h], [1], hm.HMAT_BATCH_BRANCHES | hm.HMAT_BATCH_QUEUE)
    assert ei.value.code == hm.HMAT_EINVAL
    # a workspace clone repeats the operator legally
    c = H.clone_workspace()
    b = hm.hmat_batch_create([H.h, c.h], [1, 2], hm.HMAT_BATCH_BRANCHES)
    x1 = torch.from_numpy(w.gaussian_rhs(3000, 1, 6)).float().cuda()
    x2 = torch.from_numpy(w.gaussian_rhs(3000, 2, 7)).float().cuda()
    y1, y2 = torch.empty_like(x1), torch.empty_like(x2)
    hm.hmat_batch_matvec(b, [x1, x2], [y1, y2])
    assert hm.hmat_batch_check(b) == 0
    assert rel(y1.double().cpu().numpy(), H.matvec(x1).double().cpu().numpy()) <= 1e-6
    assert rel(y2.double().cpu().numpy(), H.matvec(x2).double().cpu().numpy()) <= 1e-6
    hm.hmat_batch_destroy(b)
    c.close()
    H.close()


@pytest.mark.parametrize("bad", ["instance", "tile", "negative"])
def test_poisoned_task_table_reports_edevice(hm, bad):
    """A task naming an instance outside the plan, or a tile outside its
    instance, is skipped by the queue kernels before any access and reported:
    hmat_batch_check returns HMAT_EDEVICE, the status word is cleared, and a
    fresh plan computes the products again."""
    import torch
    insts = uneven_instances(4, 31)
    Hs, Xs, Ys, refs = [], [], [], []
    for inst in insts:
        P = inst.points()
        H = hm.HMatrix(P, hm.HMAT_K_RANDOM, 64, inst.rank, 0.0, prec=1,
                       method=hm.HMAT_RANDOM_FILL, seed=inst.seed)
        Ho = o.build_hmatrix(P, 2, 64, inst.rank, method=METHOD_RANDOM, seed=inst.seed)
        X = w.gaussian_rhs(inst.N, inst.nrhs, inst.seed + 5)
        refs.append(o.hmat_matvec(Ho, X))
        Hs.append(H)
        Xs.append(torch.from_numpy(X).float().cuda())
        Ys.append(torch.zeros_like(Xs[-1]))
    ks = [x.shape[1] for x in Xs]
    b = hm.hmat_batch_create([H.h for H in Hs], ks)
    inst, tile = {"instance": (len(Hs) + 3, 0), "tile": (0, 1 << 20), "negative": (-1, 0)}[bad]
    hm.hmat_batch_poison_task(b, 0, inst, tile)
    hm.hmat_batch_matvec(b, Xs, Ys)
    with pytest.raises(hm.HMatError) as ei:
        hm.hmat_batch_check(b)
    assert ei.value.code == hm.HMAT_EDEVICE
    assert hm.hmat_batch_check(b) == 0          # cleared
    hm.hmat_batch_destroy(b)
    b = hm.hmat_batch_create([H.h for H in Hs], ks)
    hm.hmat_batch_matvec(b, Xs, Ys)
    assert hm.hmat_batch_check(b) == 0
    for y, ref in zip(Ys, refs):
        assert rel(y.double().cpu().numpy(), ref) <= 1e-5
    with pytest.raises(hm.HMatError) as ei:
        hm.hmat_batch_poison_task(b, 1 << 30, 0, 0)
    assert ei.value.code == hm.HMAT_EINVAL
    hm.hmat_batch_destroy(b)
    bb = hm.hmat_batch_create([H.h for H in Hs], ks, hm.HMAT_BATCH_BRANCHES)
    with pytest.raises(hm.HMatError) as ei:
        hm.hmat_batch_poison_task(bb, 0, 0, 0)
    assert ei.value.code == hm.HMAT_EUNSUPPORTED
    hm.hmat_batch_destroy(bb)
    for H in Hs:
        H.close()
