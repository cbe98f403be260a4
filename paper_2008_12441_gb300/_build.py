"""Builds the C-ABI shared library libhmat_gb300.so in-tree (sm_103a).

Host C++ sources go through g++, CUDA sources through nvcc with
``-gencode arch=compute_103a,code=sm_103a``; translation units compile in
parallel and link with nvcc.  Objects land in ``_lib/obj``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIBDIR = os.path.join(PKG, "_lib")
LIBNAME = "libhmat_gb300.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def cuda_home() -> str:
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.isdir(cand):
            return cand
    nv = shutil.which("nvcc")
    if nv:
        return os.path.dirname(os.path.dirname(nv))
    raise RuntimeError("CUDA toolkit not found (nvcc)")


def sources():
    cu = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    cpp = sorted(f for f in os.listdir(CSRC) if f.endswith(".cpp"))
    return cu, cpp


def lib_path() -> str:
    return os.path.join(LIBDIR, LIBNAME)


def _stale(out: str, deps: list[str]) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False) -> str:
    home = cuda_home()
    nvcc = os.path.join(home, "bin", "nvcc")
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC,
           "-I", os.path.join(home, "include")]
    objdir = os.path.join(LIBDIR, "obj")
    os.makedirs(objdir, exist_ok=True)
    cu, cpp = sources()
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(ROOT, "include", "hmat.h"))
    jobs = []
    objs = []
    for f in cu:
        src = os.path.join(CSRC, f)
        obj = os.path.join(objdir, f + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + headers):
            cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
                   "-Xcompiler", "-fPIC,-O3", *inc, "-c", src, "-o", obj]
            jobs.append(cmd)
    for f in cpp:
        src = os.path.join(CSRC, f)
        obj = os.path.join(objdir, f + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + headers):
            cmd = ["g++", "-O3", "-fPIC", "-std=c++17", "-pthread", "-Wall",
                   "-Wno-unused-function", *inc, "-c", src, "-o", obj]
            jobs.append(cmd)
    procs = [(cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT))
             for cmd in jobs]
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode:
            sys.stderr.write(" ".join(cmd) + "\n" + out.decode(errors="replace"))
        if p.returncode:
            failed.append(cmd[-1])
    if failed:
        raise RuntimeError("compilation failed: " + ", ".join(failed))
    out = lib_path()
    if force or jobs or _stale(out, objs):
        cmd = [nvcc, *ARCH, "-shared", "-o", out, *objs, "-lcudart", "-lpthread"]
        r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        if verbose or r.returncode:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout.decode(errors="replace"))
        if r.returncode:
            raise RuntimeError("link failed")
    return out


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
