#!/usr/bin/env python3
"""H-matrix-vector product benchmark (one JSON line on rank 0).

Workload (default): 2D log kernel on a 1024x1024 grid (N = 1,048,576),
quadtree with leaf 64, weak admissibility, rank 16 by randomized SVD, FP32
factors, one right-hand side.  A step is one product y = K x (project +
expand kernels) with x and the factors resident in HBM; the factor
footprint (3.5 GB) exceeds L2, so no flush is needed between steps.

  value  = algorithmic bytes (factor + dense entries + x + y) / step time, GB/s
  e2e    = the same through hmat_matvec_host (pinned host x, y; copies timed)
  roofline: the dominant kernel's algorithmic bytes per launch / its mean
            CUDA-event duration, against the measured HBM copy bandwidth
  accuracy: rel-L2 against the FP64 oracle on rows of every tile and every
            persistent CTA range; for a kernel-compressed workload on its
            random-filled twin (same grid, tree, rank, storage and kernels),
            whose blocks the oracle regenerates itself
  mixed_vs_plain: the same operator in split bf16 and bf16 storage with 64
            right-hand sides on the tensor cores, RHS-matvecs/s and error,
            beside the plain FP32 one-right-hand-side product
  cpu_baseline: the FP64 oracle (numpy) on the same structure, 1 thread and
            all host cores

--impl reference times the oracle itself as the reference arm.
Multi-GPU: replicas only (each rank runs its own copy; no collective on
the data path); value = bytes of all ranks / max step time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import re
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as w  # noqa: E402

METRIC = "H-matvec GB/s (% of HBM peak) & RHS-matvecs/s, mixed vs FP32 plain at rel err"
FALLBACK_HBM = 6800.0
L2_BYTES = 129e6


def workload_table():
    return {
        "2d-log-n262144-rsvd-r16": dict(d=2, grid=512, kernel=0, rank=16, nrhs=1, prec=1,
                                        method=1, seed=12442),
        "2d-random-n262144-r16": dict(d=2, grid=512, kernel=2, rank=16, nrhs=1, prec=1,
                                      method=2, seed=12442),
        "3d-inv4pir-n262144-r32-k32": dict(d=3, grid=64, kernel=1, rank=32, nrhs=32, prec=1,
                                           method=1, seed=12443),
        "2d-random-n262144-r16-k64": dict(d=2, grid=512, kernel=2, rank=16, nrhs=64, prec=2,
                                          method=2, seed=12442),
        "2d-log-n1048576-r16-k64": dict(d=2, grid=1024, kernel=0, rank=16, nrhs=64, prec=1,
                                        method=1, seed=12444),
        "2d-log-n1048576-r16": dict(d=2, grid=1024, kernel=0, rank=16, nrhs=1, prec=1,
                                    method=1, seed=12444),
        "2d-log-n4096-tsvd-r8-fp64": dict(d=2, grid=64, kernel=0, rank=8, nrhs=1, prec=0,
                                          method=0, seed=12441),
        # standard admissibility (interaction lists, near field over the
        # touching groups), the paper's random blocks
        "2d-random-n262144-r8-standard": dict(d=2, grid=512, kernel=2, rank=8, nrhs=1, prec=1,
                                              method=2, seed=12447, adm=1),
        "2d-random-n1048576-r4-standard": dict(d=2, grid=1024, kernel=2, rank=4, nrhs=1, prec=1,
                                               method=2, seed=12448, adm=1),
    }


ADM_NAMES = {0: "weak", 1: "standard"}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


def code_text(src):
    """C/C++ source without its comments and blank or trailing space: what
    the compiler sees of it (the sources hold no string literal with a
    comment marker)."""
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    lines = (ln.rstrip() for ln in src.splitlines())
    return "\n".join(ln for ln in lines if ln)


# sources of the kernels a recorded traffic figure depends on: the kernel
# file of the path and the headers every kernel includes
KERNEL_SOURCES = {
    "streamed": ["stream.cu", "hm_elem.cuh", "hm_device.h", "hm_once.h"],
    "tensor": ["tc_matvec.cu", "hm_device.h", "hm_once.h"],
}


def kernel_source_hash(files=None):
    """Hash of the code of `files` in csrc (all sources if None; comments and
    layout excluded), stored beside each recorded traffic figure: a figure
    whose kernels' code has changed since it was measured is not reported."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2008_12441_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".h", ".cpp")) and (files is None or f in files):
            h.update(f.encode())
            h.update(code_text(open(os.path.join(csrc, f)).read()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(workload, kernel_name):
    """DRAM bytes per launch (read + write) from a committed ncu launch list
    (profiles/traffic.json, keyed "workload:precision" and by the bench's
    kernel label), if the sources of those kernels are unchanged since it
    was taken (else None).  The label "project_kernel" covers every kernel
    launched for Steps 1-4, "expand_kernel" those for Step 5."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        e = d[workload][kernel_name]
        files = KERNEL_SOURCES.get(e.get("path"))
        if e.get("source_hash") != kernel_source_hash(files):
            return None
        return float(e["dram_bytes_per_launch"])
    except Exception:
        return None


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"],
                    "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# bytes per stored entry: (low-rank factors, dense blocks, vectors)
ENTRY_BYTES = {0: (8, 8, 8), 1: (4, 4, 4), 2: (2, 2, 4), 3: (4, 4, 4), 4: (1, 2, 4)}


def algorithmic_bytes(info, k, prec):
    """Per step: stored factor + dense entries (real, unpadded) read once in
    their storage format, x read once, y written once (scales not counted)."""
    fb, db, vb = ENTRY_BYTES[prec]
    fac = info.factor_entries * fb
    den = info.dense_entries * db
    vec = info.N * k * vb
    proj = fac // 2 + vec
    expd = fac // 2 + den + 2 * vec
    return fac + den + 2 * vec, proj, expd


# ------------------------------------------------------------ oracle arm
def oracle_child(args):
    """Runs in a fresh single-threaded process: the FP64 oracle on the same
    H-matrix structure, block contents seeded standard normals."""
    import oracle as o
    cfg = workload_table()[args.workload]
    P = w.grid_points(cfg["grid"], cfg["d"])
    N = P.shape[0]
    t0 = time.perf_counter()
    kern = cfg["kernel"] if cfg["method"] != 2 else 2
    H = o.build_hmatrix(P, 2, 64, cfg["rank"], method=2, seed=cfg["seed"], materialize=False,
                        admissibility=ADM_NAMES[cfg.get("adm", 0)])
    rng = np.random.default_rng(cfg["seed"])
    for b in H.blocks:
        if b.kind == "dense":
            b.D = rng.standard_normal((b.t.size, b.s.size))
        else:
            rb = min(cfg["rank"], b.t.size, b.s.size)
            b.U = rng.standard_normal((b.t.size, rb))
            b.V = rng.standard_normal((b.s.size, rb))
    setup = time.perf_counter() - t0
    fac, den = o.entry_counts(H)
    k = cfg["nrhs"]
    X = w.gaussian_rhs(N, k, cfg["seed"] + 1)
    for _ in range(args.warmup):
        o.hmat_matvec(H, X)
    ts = []
    for _ in range(args.steps):
        t = time.perf_counter()
        o.hmat_matvec(H, X)
        ts.append(time.perf_counter() - t)
    elem = 8 if cfg["prec"] == 0 else 4
    alg = (fac + den) * elem + 2 * N * k * elem
    sec = float(np.mean(ts))
    print(json.dumps({"sec_per_step": sec, "gbs": alg / sec / 1e9, "steps": len(ts),
                      "setup_s": setup, "alg_bytes": alg, "kernel_cfg": kern,
                      "rhs_per_s": k / sec}))


def run_oracle(workload, steps, warmup, threads=1):
    """The oracle's product timed in a child process whose BLAS uses
    `threads` threads (the oracle's loop itself is sequential)."""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = str(threads)
    cmd = [sys.executable, os.path.abspath(__file__), "--_oracle_child", "--workload", workload,
           "--steps", str(steps), "--warmup", str(warmup)]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env,
                       cwd=ROOT)
    if r.returncode:
        raise RuntimeError("oracle child failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_sample_text(workload, threads=1):
    return (f"full product on the {workload} tree structure (all low-rank and dense "
            f"blocks), seeded standard-normal block contents, float64 numpy, "
            f"{threads} BLAS thread{'s' if threads > 1 else ''}")


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ------------------------------------------------ accuracy and mixed storage
TOL = {0: 1e-12, 1: 1e-5, 2: 1e-2, 3: 1e-5, 4: 5e-2}


def time_products(hm, h, X, Y, k, flags, stream, steps, warmup):
    """Mean ms of `steps` products y = K x on device-resident X (CUDA events),
    and the kernel families they took."""
    import torch
    for _ in range(warmup):
        hm.hmat_matvec(h, X, Y, k, k, k, flags, stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        hm.hmat_matvec(h, X, Y, k, k, k, flags, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    status = hm.hmat_check(h)[1]
    return e0.elapsed_time(e1) / steps, hm.hmat_last_path(h), status


def oracle_rows(cfg, P, X, rows):
    """FP64 oracle rows (tree order) of the random-filled H-matrix of this
    grid, rank and seed for tree-order right-hand sides X."""
    import oracle as o
    Ho = o.build_hmatrix(P, 2, 64, cfg["rank"], method=2, seed=cfg["seed"], materialize=False,
                         admissibility=ADM_NAMES[cfg.get("adm", 0)])
    Xo = np.empty_like(X)
    Xo[Ho.tree.perm] = X
    return o.hmat_matvec_rows(Ho, Xo, rows)


def rel_rows(Yg, Yo):
    e = float(np.linalg.norm(Yg - Yo) / np.linalg.norm(Yo))
    worst = float(np.max(np.linalg.norm(Yg - Yo, axis=1) /
                         np.maximum(np.linalg.norm(Yo, axis=1), 1e-300)))
    return e, worst


def storage_runs(hm, cfg, P, H, modes, flags, stream, steps, warmup, device):
    """For each (storage, right-hand sides) in `modes`: the workload's operator
    H in that storage (hmat_convert; H itself for its own storage) timed with
    that many right-hand sides, and the error of the same storage and kernels
    on the random-filled twin of the workload (built here unless the
    workload is itself random-filled) against the FP64 oracle on rows of
    every tile and persistent CTA range.  Returns ({"prec/kK": dict}, info)."""
    import torch
    N = P.shape[0]
    kmax = max(k for _, k in modes)
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    rows = w.covering_rows(N, sms, cfg["seed"])
    Xh = w.gaussian_rhs(N, kmax, cfg["seed"] + 7)        # tree order
    t0 = time.perf_counter()
    Yo_all = oracle_rows(cfg, P, Xh, rows)
    oracle_s = time.perf_counter() - t0
    twin = H.h if cfg["method"] == 2 else hm.hmat_build(
        P, 2, 64, cfg["rank"], 0.0, hm.hmat_default_opts(
            prec=cfg["prec"], method=2, seed=cfg["seed"], device=device, max_nrhs=kmax,
            keep_host=1, admissibility=cfg.get("adm", 0)))
    out = {}
    try:
        for prec, k in modes:
            X = torch.from_numpy(np.ascontiguousarray(Xh[:, :k])).float().cuda()
            Y = torch.empty_like(X)
            hp = H.h if prec == cfg["prec"] else hm.hmat_convert(H.h, prec)
            tp = twin if prec == cfg["prec"] else hm.hmat_convert(twin, prec)
            try:
                ms, path, status = time_products(hm, hp, X, Y, k, flags, stream, steps, warmup)
                hm.hmat_matvec(tp, X, Y, k, k, k, flags, stream)
                torch.cuda.synchronize()
                tstatus = hm.hmat_check(tp)[1]
                tpath = hm.hmat_last_path(tp)
                e, worst = rel_rows(Y.double().cpu().numpy()[rows], Yo_all[:, :k])
                alg = algorithmic_bytes(H.info, k, prec)[0]
                gbs = alg / (ms * 1e-3) / 1e9
                out[f"{w.PREC_NAMES[prec]}/k{k}"] = {
                    "storage": w.PREC_NAMES[prec], "nrhs": k, "ms_per_product": ms, "GB/s": gbs,
                    "rhs_matvecs_per_s": k / (ms * 1e-3), "rel_err": e,
                    "max_row_rel_err": worst, "tol": TOL[prec], "within_tol": bool(e <= TOL[prec]),
                    "kernel_path": path, "twin_kernel_path": tpath,
                    "status_words": [status, tstatus], "alg_bytes": int(alg)}
            finally:
                if hp != H.h:
                    hm.hmat_destroy(hp)
                if tp != twin:
                    hm.hmat_destroy(tp)
    finally:
        if twin != H.h:
            hm.hmat_destroy(twin)
    return out, {"rows": int(rows.size), "oracle_s": oracle_s,
                 "operator": "the workload itself" if cfg["method"] == 2 else
                 "random-filled twin: same grid, tree, leaf, rank, storage and kernels "
                 "(the oracle regenerates its blocks from the seed)",
                 "rows_cover": "one row in every 256- and 128-slot tile and both ends of "
                               "every persistent CTA range"}


# ------------------------------------------------------------ batched arm
def run_batched(args):
    """256 uneven instances (2D log / 3D 1/r kernels on uniform random
    points, log-uniform N in [4096, 65536], rank in {8,16,32}, 1..16 RHS).
    Mixed-precision batched products (bf16 and split bf16 factors, leaf
    slots padded to 32 in 2D / 16 in 3D so that the uneven trees take the
    tensor-core kernels; schedule chosen by hmat_batch_autotune) against one
    plain FP32 hmat_matvec per instance in sequence (unpadded handles).
    Errors are taken against the FP32 products of the same (padded)
    operators, themselves within 1e-5 of the FP64 oracle in the parity
    tests."""
    import torch
    from paper_2008_12441_gb300 import _build
    from paper_2008_12441_gb300 import hmat as hm
    _build.build()
    torch.cuda.set_device(0)
    insts = w.c5_batched(count=args.count)
    t0 = time.perf_counter()
    H32, Hsame, X, Y32 = [], [], [], []
    mixed = {"bf16": (hm.HMAT_BF16, []), "bf16x2": (hm.HMAT_BF16X2, [])}
    alg = {"fp32": 0, "bf16": 0, "bf16x2": 0}
    stored = {"bf16": 0, "bf16x2": 0}
    ksum = 0
    for inst in insts:
        P = inst.points()
        kw = dict(prec=1, method=inst.method, seed=inst.seed, oversample=inst.oversample,
                  build_gpu=1, max_nrhs=16)
        h32 = hm.HMatrix(P, inst.kernel, inst.leaf_size, inst.rank, 0.0, **kw)
        hp = hm.HMatrix(P, inst.kernel, inst.leaf_size, inst.rank, 0.0, keep_host=1,
                        leaf_slot_multiple=32 if inst.d == 2 else 16, **kw)
        for name, (prec, lst) in mixed.items():
            h = hm.hmat_convert(hp.h, prec)
            lst.append(h)
            stored[name] += hm.hmat_info(h).device_bytes + 2 * inst.N * inst.nrhs * 4
        # the same operator in FP32 storage: the reference of the errors
        Hsame.append(hm.hmat_convert(hp.h, hm.HMAT_FP32))
        hp.close()
        info = h32.info
        alg["fp32"] += algorithmic_bytes(info, inst.nrhs, 1)[0]
        alg["bf16"] += algorithmic_bytes(info, inst.nrhs, 2)[0]
        alg["bf16x2"] += algorithmic_bytes(info, inst.nrhs, 3)[0]
        ksum += inst.nrhs
        x = torch.from_numpy(inst.rhs()).float().cuda()
        H32.append(h32)
        X.append(x)
        Y32.append(torch.empty_like(x))
    build_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    ks = [x.shape[1] for x in X]
    plans, tunings, Ym = {}, {}, {}
    for name, (prec, hs) in mixed.items():
        Ym[name] = [torch.empty_like(x) for x in X]
        plans[name] = hm.hmat_batch_create(hs, ks, hm.HMAT_BATCH_BRANCHES)
        tunings[name] = hm.hmat_batch_autotune(plans[name], X, Ym[name], stream, reps=3)

    def seq():
        for h, x, y in zip(H32, X, Y32):
            hm.hmat_matvec(h.h, x, y, x.shape[1], x.shape[1], x.shape[1], 0, stream)

    def runner(name):
        return lambda: hm.hmat_batch_matvec(plans[name], X, Ym[name], stream)

    res = {}
    arms = [("sequential_fp32", seq)] + [(f"batched_{n}", runner(n)) for n in mixed]
    for name, fn in arms:
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        res[name] = e0.elapsed_time(e1) / args.steps
    for name in mixed:
        hm.hmat_batch_check(plans[name], stream)
    # FP32 products of the padded operators the mixed plans apply
    Ysame = []
    for h, x in zip(Hsame, X):
        y = torch.empty_like(x)
        hm.hmat_matvec(h, x, y, x.shape[1], x.shape[1], x.shape[1], 0, stream)
        Ysame.append(y)
    torch.cuda.synchronize()
    cross = [float(torch.linalg.norm(a.double() - b.double()) / torch.linalg.norm(b.double()))
             for a, b in zip(Ysame, Y32)]
    peak, _ = measured_peaks()
    ts = res["sequential_fp32"] * 1e-3
    arms_out = {}
    for name in mixed:
        tb = res[f"batched_{name}"] * 1e-3
        errs = [float(torch.linalg.norm(yb.double() - y.double()) / torch.linalg.norm(y.double()))
                for yb, y in zip(Ym[name], Ysame)]
        arms_out[name] = {
            "ms_per_step": res[f"batched_{name}"], "GB/s": alg[name] / tb / 1e9,
            "hbm_frac_of_measured": alg[name] / tb / 1e9 / peak,
            "stored_GB/s": stored[name] / tb / 1e9,
            "rhs_matvecs_per_s": ksum / tb, "speedup_rhs_matvecs_vs_fp32": ts / tb,
            "rel_err_vs_fp32_same_operator": {"max": max(errs), "median": float(np.median(errs))},
            "tol": 1e-5 if name == "bf16x2" else 1e-2,
            "instances_within_tol": int(sum(e <= (1e-5 if name == "bf16x2" else 1e-2) for e in errs)),
            "alg_bytes": int(alg[name]), "stored_bytes": int(stored[name]),
            "autotune": tunings[name]}
    head = arms_out["bf16x2"]
    line = {"metric": METRIC, "workload": f"batched-{args.count}-uneven", "unit": "GB/s",
            "value": head["GB/s"], "hbm_frac_of_measured": head["hbm_frac_of_measured"],
            "ms_per_step": head["ms_per_step"], "rhs_matvecs_per_s": head["rhs_matvecs_per_s"],
            "headline": "split bf16 (hi + lo) factors, the FP32 tolerance 1e-5",
            "mixed": arms_out,
            "sequential_fp32": {"ms_per_step": res["sequential_fp32"], "GB/s": alg["fp32"] / ts / 1e9,
                                "rhs_matvecs_per_s": ksum / ts, "launches": "one product per instance"},
            "padded_vs_unpadded_fp32_rel_diff": {"max": max(cross), "median": float(np.median(cross)),
                                                 "note": "the same kernel compressed on the padded and on the "
                                                         "unpadded tree; differences from summation order only"},
            "instances": len(insts), "sum_N": int(sum(i.N for i in insts)), "sum_k": ksum,
            "alg_bytes_fp32": int(alg["fp32"]), "build_s": build_s,
            "leaf_slot_multiple": {"2d": 32, "3d": 16},
            "steps": args.steps, "warmup": args.warmup, "data": "synthetic"}
    print(json.dumps(line))
    for name, (prec, hs) in mixed.items():
        hm.hmat_batch_destroy(plans[name])
        for h in hs:
            hm.hmat_destroy(h)
    for h in Hsame:
        hm.hmat_destroy(h)
    for h in H32:
        h.close()


# ------------------------------------------------------- paper's matrices
# The paper's times per matvec, rank 4, weak admissibility (tables of the 2D
# and 3D experiments on Stampede2): (processes, seconds) at the fewest
# processes listed and at the best time.
PAPER_TIMES = {
    (2, 512): (32, 3.58e-03, 128, 3.08e-03),
    (2, 1024): (32, 1.17e-02, 512, 3.40e-03),
    (2, 2048): (32, 5.03e-02, 2048, 3.51e-03),
    (2, 4096): (32, 2.30e-01, 2048, 6.36e-03),
    (2, 8192): (256, 1.56e-01, 16384, 4.12e-03),
    (3, 64): (32, 3.27e-03, 32, 3.27e-03),
    (3, 128): (32, 1.70e-02, 1024, 4.70e-03),
    (3, 256): (32, 1.65e-01, 4096, 4.75e-03),
}


def paper_table_workloads():
    """The matrices of the paper's 2D and 3D experiments (Sec. 5.1, 5.2 and
    their tables): random-filled H-matrices under weak admissibility, ranks
    4 and 8 (the paper tabulates rank 4 and plots rank 8), on n x n and
    n x n x n grids, times averaged over 128 random input vectors.  The paper
    states no leaf size; these use 64.  The blocks are written straight into
    device memory (no host copy), so the grids go as far as one GPU's memory:
    8192^2 (67M points) and 256^3 (16.8M points); the paper goes up to
    65536^2 and 1024^3 on thousands of processes."""
    grids = [(2, 512), (2, 1024), (2, 2048), (2, 4096), (2, 8192), (3, 64), (3, 128), (3, 256)]
    return [(d, n, r) for r in (4, 8) for d, n in grids]


def run_paper_table(args):
    """One JSON line per paper matrix: FP32 storage, one right-hand side,
    128 products timed back to back with CUDA events over 8 distinct seeded
    Gaussian x (made on the host, device-resident while timed; the time does
    not depend on the values); the mean per product is the paper's "time
    per matvec".  `args.paper_table` selects matrices ("2:512,3:64" for
    both ranks, "2:512:8" for one), or "all".  Rank-4 lines carry the
    paper's time at its fewest processes and its best time (tables of the
    2D and 3D experiments, weak admissibility)."""
    import torch
    from paper_2008_12441_gb300 import _build
    from paper_2008_12441_gb300 import hmat as hm

    torch.cuda.set_device(0)
    _build.build()
    peak, peak_kind = measured_peaks()
    stream = torch.cuda.current_stream()
    nvec, ndistinct = 128, 8
    todo = paper_table_workloads()
    if args.paper_table != "all":
        want = [tuple(int(v) for v in item.split(":")) for item in args.paper_table.split(",")]
        todo = [(d, n, r) for d, n, r in todo
                if (d, n) in [x[:2] for x in want if len(x) == 2] or (d, n, r) in want]
    for d, n, rank in todo:
        N = n ** d
        P = w.grid_points(n, d)
        t0 = time.perf_counter()
        H = hm.HMatrix(P, 2, 64, rank, 0.0, prec=1, method=2, seed=12446, device=0, max_nrhs=1)
        build_s = time.perf_counter() - t0
        info = H.info
        X = torch.from_numpy(np.stack([w.gaussian_rhs(N, 1, 12446 + n + i)
                                       for i in range(ndistinct)])).float().cuda()
        Y = torch.empty(N, 1, device="cuda")
        flags = hm.HMAT_TREE_ORDER
        for i in range(max(args.warmup, 3)):
            hm.hmat_matvec(H.h, X[i % ndistinct], Y, 1, 1, 1, flags, stream)
        torch.cuda.synchronize()
        warm_status = hm.hmat_check(H.h)[1]
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for i in range(nvec):
            hm.hmat_matvec(H.h, X[i % ndistinct], Y, 1, 1, 1, flags, stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / nvec
        alg, _, _ = algorithmic_bytes(info, 1, 1)
        gbs = alg / (ms * 1e-3) / 1e9
        paper = PAPER_TIMES.get((d, n)) if rank == 4 else None
        print(json.dumps({
            "impl": "ours", "mode": "paper-table",
            "workload": f"{d}d-random-n{n}^{d}-r{rank}", "N": N, "d": d, "rank": rank,
            "leaf_size": 64, "depth": info.depth, "precision": "fp32", "nrhs": 1,
            "products": nvec, "distinct_vectors": ndistinct, "ms_per_product": ms, "GB/s": gbs,
            "frac_of_" + peak_kind: gbs / peak, "alg_bytes": int(alg),
            "device_bytes": int(info.device_bytes), "build_s": build_s,
            "fill": "device" if N >= 65536 else "host",
            "paper_s_per_matvec": None if paper is None else
            {"fewest_processes": paper[0], "s": paper[1], "best_processes": paper[2], "best_s": paper[3]},
            "status_word": {"warmup": warm_status, "timed": hm.hmat_check(H.h)[1]}}), flush=True)
        H.close()
        del X, Y
        torch.cuda.empty_cache()


# ------------------------------------------------------- precision sweep
def run_precision_sweep(args):
    """The 1024^2 log-kernel operator (rank 16, randomized SVD) with 64
    right-hand sides in the four storage modes -- FP32 (CUDA cores), bf16
    with block scales, split bf16, e4m3 with column scales (bf16, split and
    e4m3 on the tensor cores) -- one JSON line: time, GB/s and fraction of
    the measured HBM bandwidth, RHS-matvecs/s, and rel-L2 against the FP64
    oracle on the random-filled twin (rows of every tile and CTA range)."""
    import torch
    from paper_2008_12441_gb300 import _build
    from paper_2008_12441_gb300 import hmat as hm
    _build.build()
    torch.cuda.set_device(0)
    name = "2d-log-n1048576-r16-k64"
    cfg = workload_table()[name]
    P = w.grid_points(cfg["grid"], cfg["d"])
    t0 = time.perf_counter()
    H = hm.HMatrix(P, cfg["kernel"], 64, cfg["rank"], 0.0, prec=1, method=cfg["method"],
                   seed=cfg["seed"], device=0, max_nrhs=64, keep_host=1)
    build_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    runs, ainfo = storage_runs(hm, cfg, P, H, [(1, 64), (2, 64), (3, 64), (4, 64)],
                               hm.HMAT_TREE_ORDER, stream, min(args.steps, 20), args.warmup, 0)
    peak, peak_kind = measured_peaks()
    for r in runs.values():
        r["frac_of_" + peak_kind] = r["GB/s"] / peak
    print(json.dumps({"impl": "ours", "mode": "precision-sweep", "metric": METRIC,
                      "workload": name, "N": int(P.shape[0]), "rank": cfg["rank"], "nrhs": 64,
                      "modes": runs, "accuracy": ainfo, "build_s": build_s,
                      "data": "synthetic"}))
    H.close()


# ---------------------------------------------------------------- GPU arm
def max_over_ranks(value, ws, device):
    """Max of a per-rank float over the replicas (the slowest rank's time);
    the value itself with one rank.  `device`: where the collective's
    tensor lives ("cuda" with NCCL, "cpu" with gloo)."""
    if ws == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(bytes_per_rank, ws, sec_per_step):
    """Whole-job GB/s of ws independent replicas: the bytes of all ranks
    over the slowest rank's step time."""
    return bytes_per_rank * ws / sec_per_step / 1e9


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="2d-log-n1048576-r16",
                    choices=sorted(workload_table()))
    ap.add_argument("--prec", default=None, choices=sorted(w.PREC_NAMES.values()),
                    help="override the workload's storage precision")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the oracle rows and the mixed-precision comparison")
    ap.add_argument("--batched", action="store_true",
                    help="uneven instances in one batched graph vs sequential FP32 launches")
    ap.add_argument("--count", type=int, default=256)
    ap.add_argument("--paper-table", default=None, metavar="SEL",
                    help="the paper's random-filled rank-4 matrices, one line each: "
                         "'all' or d:n items, e.g. 2:512,3:64")
    ap.add_argument("--precision-sweep", action="store_true",
                    help="1024^2 operator, 64 right-hand sides, four storage modes with errors")
    ap.add_argument("--_oracle_child", action="store_true")
    args = ap.parse_args()
    if args._oracle_child:
        oracle_child(args)
        return
    args.warmup = max(args.warmup, 3)
    if args.paper_table is not None:
        run_paper_table(args)
        return
    if args.batched:
        run_batched(args)
        return
    if args.precision_sweep:
        run_precision_sweep(args)
        return
    ws, rank, local = dist_env()
    cfg = dict(workload_table()[args.workload])
    if args.prec is not None:
        cfg["prec"] = {v: k for k, v in w.PREC_NAMES.items()}[args.prec]
    N = cfg["grid"] ** cfg["d"]
    k = cfg["nrhs"]
    prec_name = w.PREC_NAMES[cfg["prec"]]
    config = {"workload": args.workload, "N": N, "d": cfg["d"], "leaf_size": 64,
              "rank": cfg["rank"], "nrhs": k, "precision": prec_name,
              "fill": "random" if cfg["method"] == 2 else ("rsvd" if cfg["method"] == 1 else "tsvd"),
              "admissibility": ADM_NAMES[cfg.get("adm", 0)], "vector_order": "tree",
              "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas{ws}"}

    if args.impl == "reference":
        if rank != 0:
            return
        ref = run_oracle(args.workload, args.steps, args.warmup)
        cores = 1
        line = {"impl": "reference", "metric": METRIC, "value": ref["gbs"], "unit": "GB/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ref["sec_per_step"] * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": config, "rhs_matvecs_per_s": ref["rhs_per_s"],
                "cpu_baseline": {"value": ref["gbs"], "unit": "GB/s", "cores": cores,
                                 "kind": "oracle", "sample": oracle_sample_text(args.workload)},
                "e2e": {"value": ref["gbs"], "unit": "GB/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    from paper_2008_12441_gb300 import _build
    from paper_2008_12441_gb300 import hmat as hm

    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0 or ws == 1:
        _build.build()
    if ws > 1:
        dist.barrier()
    P = w.grid_points(cfg["grid"], cfg["d"])
    # the mixed-storage comparison converts this operator (host copy kept)
    # and runs it with 64 right-hand sides
    # (tensor cores: weak admissibility only)
    mixed = (rank == 0 and ws == 1 and not args.no_accuracy and k == 1 and cfg["prec"] == 1 and
             cfg.get("adm", 0) == 0)
    t0 = time.perf_counter()
    H = hm.HMatrix(P, cfg["kernel"], 64, cfg["rank"], 0.0, prec=cfg["prec"], method=cfg["method"],
                   seed=cfg["seed"], device=local, max_nrhs=64 if mixed else max(k, 1),
                   keep_host=1 if mixed else 0, admissibility=cfg.get("adm", 0))
    build_s = time.perf_counter() - t0
    info = H.info
    elem = 8 if cfg["prec"] == 0 else 4
    vdt = torch.float64 if cfg["prec"] == 0 else torch.float32
    X = torch.from_numpy(w.gaussian_rhs(N, k, cfg["seed"] + 1)).to(vdt).cuda()
    Y = torch.empty_like(X)
    stream = torch.cuda.current_stream()
    flags = hm.HMAT_TREE_ORDER

    def step():
        hm.hmat_matvec(H.h, X, Y, k, k, k, flags, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    n0 = hm.hmat_launch_count()
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    gpu_launches = hm.hmat_launch_count() - n0
    kernel_path = hm.hmat_last_path(H.h)
    if ws > 1:
        dist.barrier()
    ms_total = ev0.elapsed_time(ev1)
    # device status word (a bounded wait that gave up records its site code)
    status_words = {"timed": hm.hmat_check(H.h)[1]}
    # the same steps again with an event pair around each kernel launch
    # (per-kernel durations for the roofline; the events keep consecutive
    # kernels from overlapping, so the step time above is taken without them)
    hm.hmat_profile(H.h, 1)
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    launches, kms = hm.hmat_profile_read(H.h)
    hm.hmat_profile(H.h, 0)
    status_words["profiled"] = hm.hmat_check(H.h)[1]
    clocks = sampler.stop()
    ms_step = max_over_ranks(ms_total / args.steps, ws, "cuda")
    alg, proj_b, exp_b = algorithmic_bytes(info, k, cfg["prec"])
    value = replica_throughput(alg, ws, ms_step * 1e-3)
    peak, peak_kind = measured_peaks()
    # dominant kernel
    names = ["project_kernel", "expand_kernel"]
    avg = [kms[i] / launches[i] if launches[i] else 0.0 for i in range(2)]
    dom = 1 if avg[1] >= avg[0] else 0
    dom_bytes = exp_b if dom == 1 else proj_b
    achieved = dom_bytes / (avg[dom] * 1e-3) / 1e9 if avg[dom] > 0 else None
    traffic = recorded_traffic(f"{args.workload}:{prec_name}", names[dom])
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "kernel": names[dom], "peak_kind": peak_kind + " (copy bandwidth, burst)",
                "alg_bytes_per_launch": dom_bytes,
                "kernels": {names[i]: {"launches": launches[i], "mean_ms": avg[i],
                                       "share": kms[i] / max(sum(kms), 1e-12)} for i in range(2)}}

    # end to end through the host-buffer entry point (pinned memory)
    Xh = torch.from_numpy(w.gaussian_rhs(N, k, cfg["seed"] + 1)).to(vdt).pin_memory()
    Yh = torch.empty_like(Xh).pin_memory()
    xa, ya = Xh.numpy(), Yh.numpy()
    def host_step():
        try:
            hm.hmat_matvec_host(H.h, xa, ya, k, k, k, flags, stream)
        except hm.HMatError as err:
            if err.code != hm.HMAT_ETIMEOUT:
                raise
            import re
            m = re.search(r"status word (-?\d+)", str(err))
            status_words["e2e"] = int(m.group(1)) if m else -6

    for _ in range(3):
        host_step()
    e2e_steps = max(3, min(args.steps, 50))
    t = time.perf_counter()
    for _ in range(e2e_steps):
        host_step()
    e2e_sec = max_over_ranks((time.perf_counter() - t) / e2e_steps, ws, "cuda")
    e2e = {"value": replica_throughput(alg, ws, e2e_sec), "unit": "GB/s",
           "h2d_bytes_per_step": int(N * k * elem), "d2h_bytes_per_step": int(N * k * elem),
           "ms_per_step": e2e_sec * 1e3}

    # accuracy against the FP64 oracle (rows of every tile and CTA range) and,
    # for the plain FP32 one-right-hand-side workload, the same operator in
    # split bf16 and bf16 storage with 64 right-hand sides on the tensor cores
    accuracy = None
    mixed_line = None
    if rank == 0 and ws == 1 and not args.no_accuracy:
        modes = [(cfg["prec"], k)] + ([(3, 64), (2, 64)] if mixed else [])
        runs, ainfo = storage_runs(hm, cfg, P, H, modes, flags, stream, min(args.steps, 50),
                                   args.warmup, local)
        plain = runs[f"{prec_name}/k{k}"]
        accuracy = dict(ainfo, rel_err=plain["rel_err"], max_row_rel_err=plain["max_row_rel_err"],
                        tol=plain["tol"], within_tol=plain["within_tol"],
                        kernel_path=plain["twin_kernel_path"], status_word=plain["status_words"][1])
        if mixed:
            mixed_line = {"plain": {"storage": prec_name, "nrhs": k,
                                    "rhs_matvecs_per_s": k / (ms_step * 1e-3),
                                    "GB/s": value, "rel_err": plain["rel_err"]}}
            for key, r in runs.items():
                if r["storage"] != prec_name:
                    mixed_line[key] = dict(r, hbm_frac_of_measured=r["GB/s"] / measured_peaks()[0],
                                           rhs_matvecs_vs_plain=r["rhs_matvecs_per_s"] /
                                           (k / (ms_step * 1e-3)))

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = {}
        for threads in sorted({1, host_cores()}):
            try:
                ref = run_oracle(args.workload, 3, 1, threads)
                c = {"value": ref["gbs"], "unit": "GB/s", "cores": threads, "kind": "oracle",
                     "sample": oracle_sample_text(args.workload, threads) + ", 3 steps",
                     "rhs_matvecs_per_s": ref["rhs_per_s"]}
            except Exception as exc:  # reported, not fatal
                c = {"value": None, "unit": "GB/s", "cores": threads, "kind": "oracle",
                     "sample": f"failed: {exc}"[:300]}
            if threads == 1:
                cpu.update(c)
            else:
                cpu["all_cores"] = c

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {0: "f64", 1: "f32", 2: "bf16", 3: "bf16x2", 4: "e4m3"}[cfg["prec"]],
                "data": "synthetic",
                "config": config, "hbm_frac_of_measured": value / ws / peak,
                "rhs_matvecs_per_s": k * ws / (ms_step * 1e-3),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(gpu_launches), "kernel_path": kernel_path,
                "clocks": clocks, "status_words": status_words,
                "accuracy": accuracy, "mixed_vs_plain": mixed_line, "build_s": build_s,
                "device_bytes": int(info.device_bytes), "alg_bytes_per_step": int(alg)}
        print(json.dumps(line))
    H.close()
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
