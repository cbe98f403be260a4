"""Python binding of the C ABI in include/hmat.h (ctypes).

Argument marshalling only: every step of the product runs in the CUDA
kernels of libhmat_gb300.so.  Functions carry the C names; ``HMatrix`` is
a small owner object around a handle.  torch is used for device tensors
and streams only.  If the shared library is missing, importing this module
raises: there is no host fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

HMAT_OK, HMAT_EINVAL, HMAT_ENOMEM, HMAT_ECUDA = 0, -1, -2, -3
HMAT_EUNSUPPORTED, HMAT_EDEVICE, HMAT_ETIMEOUT = -4, -5, -6
HMAT_K_LOG2D, HMAT_K_INV4PIR_3D, HMAT_K_RANDOM = 0, 1, 2
HMAT_TSVD, HMAT_RSVD, HMAT_RANDOM_FILL = 0, 1, 2
HMAT_FP64, HMAT_FP32, HMAT_BF16, HMAT_BF16X2, HMAT_FP8E4M3 = 0, 1, 2, 3, 4
HMAT_ADM_WEAK, HMAT_ADM_STANDARD = 0, 1
HMAT_TREE_ORDER = 1
HMAT_TRANSPOSE = 2
HMAT_BATCH_QUEUE = 0x100
HMAT_BATCH_BRANCHES = 0x200
HMAT_PATH_PROJECT_STREAMED, HMAT_PATH_EXPAND_STREAMED = 1, 2
HMAT_PATH_PROJECT_TENSOR, HMAT_PATH_EXPAND_TENSOR = 4, 8
HMAT_PATH_PROJECT_CACHED, HMAT_PATH_EXPAND_CACHED = 16, 32
PATH_STREAMED = HMAT_PATH_PROJECT_STREAMED | HMAT_PATH_EXPAND_STREAMED
PATH_TENSOR = HMAT_PATH_PROJECT_TENSOR | HMAT_PATH_EXPAND_TENSOR
PATH_CACHED = HMAT_PATH_PROJECT_CACHED | HMAT_PATH_EXPAND_CACHED

STATUS_NAMES = {0: "HMAT_OK", -1: "HMAT_EINVAL", -2: "HMAT_ENOMEM", -3: "HMAT_ECUDA",
                -4: "HMAT_EUNSUPPORTED", -5: "HMAT_EDEVICE", -6: "HMAT_ETIMEOUT"}

# Every entry point declared in include/hmat.h.
EXPORTED = ("hmat_default_opts", "hmat_build", "hmat_matvec", "hmat_matvec_host",
            "hmat_destroy", "hmat_info", "hmat_get_perm", "hmat_export_block",
            "hmat_export_dense", "hmat_last_error", "hmat_profile", "hmat_profile_read",
            "hmat_matvec_noalloc", "hmat_convert", "hmat_batch_create", "hmat_batch_matvec",
            "hmat_batch_destroy", "hmat_check", "hmat_selftest_timeout", "hmat_launch_count",
            "hmat_batch_autotune", "hmat_save", "hmat_load", "hmat_gemv",
            "hmat_clone_workspace", "hmat_last_path", "hmat_prepare_transpose",
            "hmat_inject_alloc_failure", "hmat_batch_check", "hmat_batch_poison_task")


class hmat_opts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("method", ctypes.c_int),
                ("leaf_lowrank", ctypes.c_int), ("oversample", ctypes.c_int),
                ("power_iters", ctypes.c_int), ("device", ctypes.c_int),
                ("max_nrhs", ctypes.c_int), ("threads", ctypes.c_int),
                ("keep_host", ctypes.c_int), ("build_gpu", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("admissibility", ctypes.c_int),
                ("leaf_slot_multiple", ctypes.c_int)]


class hmat_batch_tuning(ctypes.Structure):
    _fields_ = [("grid_div", ctypes.c_int), ("coarse_widths", ctypes.c_int),
                ("candidates", ctypes.c_int), ("ms", ctypes.c_double),
                ("ms_default", ctypes.c_double), ("schedule", ctypes.c_int),
                ("branches", ctypes.c_int), ("ms_queue", ctypes.c_double),
                ("ms_branches", ctypes.c_double)]


class hmat_info_t(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("d", ctypes.c_int), ("depth", ctypes.c_int),
                ("lowrank_levels", ctypes.c_int), ("leaf_slots", ctypes.c_int),
                ("prec", ctypes.c_int), ("padded_N", ctypes.c_int64),
                ("lowrank_blocks", ctypes.c_int64), ("dense_blocks", ctypes.c_int64),
                ("factor_entries", ctypes.c_int64), ("dense_entries", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64),
                ("rank_per_level", ctypes.c_int * 32), ("admissibility", ctypes.c_int),
                ("partners", ctypes.c_int), ("near_groups", ctypes.c_int)]


class HMatError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_LIB = None


def library(path: str | None = None) -> ctypes.CDLL:
    """Load libhmat_gb300.so (built by __graft_entry__.build()); raise if absent."""
    global _LIB
    if _LIB is not None:
        return _LIB
    p = path or _build.lib_path()
    if not os.path.exists(p):
        raise ImportError(f"{p} is missing: run __graft_entry__.build() first")
    lib = ctypes.CDLL(p)
    vp, i64, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    lib.hmat_default_opts.argtypes = [ctypes.POINTER(hmat_opts)]
    lib.hmat_default_opts.restype = None
    lib.hmat_build.argtypes = [ctypes.POINTER(ctypes.c_double), i64, c_int, c_int, c_int, c_int,
                               ctypes.c_double, ctypes.POINTER(hmat_opts), ctypes.POINTER(vp)]
    lib.hmat_matvec.argtypes = [vp, vp, vp, c_int, i64, i64, c_int, vp]
    lib.hmat_matvec_host.argtypes = [vp, vp, vp, c_int, i64, i64, c_int, vp]
    lib.hmat_matvec_noalloc.argtypes = [vp, vp, vp, c_int, i64, i64, c_int, vp]
    lib.hmat_gemv.argtypes = [vp, ctypes.c_double, vp, ctypes.c_double, vp, c_int, i64, i64,
                              c_int, vp]
    lib.hmat_clone_workspace.argtypes = [vp, ctypes.POINTER(vp)]
    lib.hmat_destroy.argtypes = [vp]
    lib.hmat_info.argtypes = [vp, ctypes.POINTER(hmat_info_t)]
    lib.hmat_get_perm.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
    lib.hmat_export_block.argtypes = [vp, c_int, i64, i64, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)]
    lib.hmat_export_dense.argtypes = [vp, i64, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(i64)]
    lib.hmat_convert.argtypes = [vp, c_int, ctypes.POINTER(vp)]
    lib.hmat_batch_create.argtypes = [ctypes.POINTER(vp), c_int, ctypes.POINTER(c_int), c_int,
                                      ctypes.POINTER(vp)]
    lib.hmat_batch_matvec.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
    lib.hmat_batch_destroy.argtypes = [vp]
    lib.hmat_batch_check.argtypes = [vp, vp, ctypes.POINTER(c_int)]
    lib.hmat_batch_poison_task.argtypes = [vp, c_int, c_int, c_int]
    lib.hmat_batch_autotune.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp, c_int,
                                        ctypes.POINTER(hmat_batch_tuning)]
    lib.hmat_profile.argtypes = [vp, c_int]
    lib.hmat_profile_read.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_double)]
    lib.hmat_check.argtypes = [vp, vp, ctypes.POINTER(c_int)]
    lib.hmat_selftest_timeout.argtypes = [vp, c_int, vp, ctypes.POINTER(c_int)]
    lib.hmat_launch_count.argtypes = []
    lib.hmat_last_path.argtypes = [vp]
    lib.hmat_prepare_transpose.argtypes = [vp]
    lib.hmat_inject_alloc_failure.argtypes = [i64]
    lib.hmat_save.argtypes = [vp, ctypes.c_char_p]
    lib.hmat_load.argtypes = [ctypes.c_char_p, ctypes.POINTER(hmat_opts), ctypes.POINTER(vp)]
    lib.hmat_last_error.restype = ctypes.c_char_p
    for name in EXPORTED:
        if name not in ("hmat_default_opts", "hmat_last_error", "hmat_launch_count",
                        "hmat_inject_alloc_failure"):
            getattr(lib, name).restype = c_int
    lib.hmat_launch_count.restype = i64
    lib.hmat_inject_alloc_failure.restype = i64
    _LIB = lib
    return lib


def hmat_last_error() -> str:
    return library().hmat_last_error().decode()


def _check(rc: int):
    if rc != HMAT_OK:
        raise HMatError(rc, hmat_last_error())


def hmat_default_opts(**kw) -> hmat_opts:
    o = hmat_opts()
    library().hmat_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if v is not None:
            setattr(o, k, v)
    return o


def hmat_build(points: np.ndarray, kernel: int, leaf_size: int, rank: int, tol: float = 0.0,
               opts: hmat_opts | None = None) -> int:
    """Returns the raw handle (int) of a new H-matrix; see include/hmat.h."""
    P = np.ascontiguousarray(points, dtype=np.float64)
    if P.ndim != 2:
        raise ValueError("points must be N x d")
    h = ctypes.c_void_p()
    _check(library().hmat_build(P.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), P.shape[0],
                                P.shape[1], kernel, leaf_size, rank, tol,
                                ctypes.byref(opts) if opts is not None else None,
                                ctypes.byref(h)))
    return h.value


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def hmat_matvec(h: int, x, y, nrhs: int, ldx: int, ldy: int, flags: int = 0, stream=None):
    """x, y: device pointers (int) or torch CUDA tensors."""
    xp = x if isinstance(x, int) else x.data_ptr()
    yp = y if isinstance(y, int) else y.data_ptr()
    _check(library().hmat_matvec(h, xp, yp, nrhs, ldx, ldy, flags, _stream_ptr(stream)))


def hmat_gemv(h: int, alpha: float, x, beta: float, y, nrhs: int, ldx: int, ldy: int,
              flags: int = 0, stream=None):
    """y = alpha K x + beta y; x, y: device pointers (int) or torch CUDA tensors."""
    xp = x if isinstance(x, int) else x.data_ptr()
    yp = y if isinstance(y, int) else y.data_ptr()
    _check(library().hmat_gemv(h, float(alpha), xp, float(beta), yp, nrhs, ldx, ldy, flags,
                               _stream_ptr(stream)))


def hmat_clone_workspace(h: int) -> int:
    """A handle on the same device factors with its own workspace."""
    out = ctypes.c_void_p()
    _check(library().hmat_clone_workspace(h, ctypes.byref(out)))
    return out.value


def hmat_matvec_noalloc(h: int, x, y, nrhs: int, ldx: int, ldy: int, flags: int = 0,
                        stream=None):
    """As hmat_matvec, without any device allocation: partial sums go to the
    library's static 8 MiB device array (see include/hmat.h)."""
    xp = x if isinstance(x, int) else x.data_ptr()
    yp = y if isinstance(y, int) else y.data_ptr()
    _check(library().hmat_matvec_noalloc(h, xp, yp, nrhs, ldx, ldy, flags, _stream_ptr(stream)))


def hmat_matvec_host(h: int, x: np.ndarray, y: np.ndarray, nrhs: int, ldx: int, ldy: int,
                     flags: int = 0, stream=None):
    """x, y: host arrays (numpy, or pinned torch CPU tensors via .numpy())."""
    _check(library().hmat_matvec_host(h, x.ctypes.data, y.ctypes.data, nrhs, ldx, ldy, flags,
                                      _stream_ptr(stream)))


def hmat_convert(h: int, prec: int) -> int:
    out = ctypes.c_void_p()
    _check(library().hmat_convert(h, prec, ctypes.byref(out)))
    return out.value


def hmat_batch_create(handles, nrhs, flags: int = 0) -> int:
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*handles)
    ks = (ctypes.c_int * n)(*nrhs)
    out = ctypes.c_void_p()
    _check(library().hmat_batch_create(hs, n, ks, flags, ctypes.byref(out)))
    return out.value


def hmat_batch_matvec(b: int, xs, ys, stream=None):
    """xs, ys: sequences of device pointers (int) or CUDA tensors."""
    n = len(xs)
    xp = (ctypes.c_void_p * n)(*[x if isinstance(x, int) else x.data_ptr() for x in xs])
    yp = (ctypes.c_void_p * n)(*[y if isinstance(y, int) else y.data_ptr() for y in ys])
    _check(library().hmat_batch_matvec(b, xp, yp, _stream_ptr(stream)))


def hmat_batch_autotune(b: int, xs, ys, stream=None, reps: int = 5) -> dict:
    """Times the candidate schedules on xs / ys, keeps the fastest (ys hold
    its results, the stream is synchronised); returns the chosen schedule."""
    n = len(xs)
    xp = (ctypes.c_void_p * n)(*[x if isinstance(x, int) else x.data_ptr() for x in xs])
    yp = (ctypes.c_void_p * n)(*[y if isinstance(y, int) else y.data_ptr() for y in ys])
    t = hmat_batch_tuning()
    _check(library().hmat_batch_autotune(b, xp, yp, _stream_ptr(stream), int(reps), ctypes.byref(t)))
    return {"schedule": {HMAT_BATCH_QUEUE: "queue", HMAT_BATCH_BRANCHES: "branches"}.get(t.schedule,
                                                                                          t.schedule),
            "branches": t.branches, "grid_div": t.grid_div, "coarse_widths": t.coarse_widths,
            "candidates": t.candidates, "ms": t.ms, "ms_default": t.ms_default,
            "ms_queue": t.ms_queue, "ms_branches": t.ms_branches}


def hmat_batch_check(b: int, stream=None) -> int:
    """Synchronises the stream, returns and clears the plan's first nonzero
    status word (raises HMatError on HMAT_EDEVICE / HMAT_ETIMEOUT)."""
    code = ctypes.c_int(0)
    rc = library().hmat_batch_check(b, _stream_ptr(stream), ctypes.byref(code))
    if rc != HMAT_OK:
        raise HMatError(rc, hmat_last_error())
    return code.value


def hmat_batch_poison_task(b: int, task: int, inst: int, tile: int):
    _check(library().hmat_batch_poison_task(b, task, inst, tile))


def hmat_batch_destroy(b: int):
    _check(library().hmat_batch_destroy(b))


def hmat_destroy(h: int):
    _check(library().hmat_destroy(h))


def hmat_profile(h: int, enable: int):
    _check(library().hmat_profile(h, enable))


def hmat_profile_read(h: int):
    """Returns ([launches_project, launches_expand], [ms_project, ms_expand])."""
    n = (ctypes.c_int64 * 2)()
    ms = (ctypes.c_double * 2)()
    _check(library().hmat_profile_read(h, n, ms))
    return [n[0], n[1]], [ms[0], ms[1]]


def hmat_save(h: int, path: str):
    _check(library().hmat_save(h, os.fsencode(path)))


def hmat_load(path: str, opts: "hmat_opts | None" = None) -> int:
    """Handle read from a file of hmat_save (opts None: the saved options)."""
    out = ctypes.c_void_p()
    _check(library().hmat_load(os.fsencode(path), ctypes.byref(opts) if opts is not None else None,
                               ctypes.byref(out)))
    return out.value


def hmat_launch_count() -> int:
    """Kernel launches issued by the library so far in this process."""
    return int(library().hmat_launch_count())


def hmat_inject_alloc_failure(after: int) -> int:
    """Test hook: the (after + 1)-th allocation from now on fails (negative: off)."""
    return int(library().hmat_inject_alloc_failure(int(after)))


def hmat_prepare_transpose(h: int):
    """Device state of y = K^T x (allocates, synchronises; idempotent)."""
    _check(library().hmat_prepare_transpose(h))


def hmat_last_path(h: int) -> int:
    """HMAT_PATH_* bits of the kernels the handle's last product launched."""
    rc = library().hmat_last_path(h)
    if rc < 0:
        _check(rc)
    return rc


def hmat_check(h: int, stream=None):
    """Synchronises the stream and returns (status, word): status is 0 or
    HMAT_ETIMEOUT (-6) when a bounded device-side wait gave up; the word is
    cleared.  Other errors raise."""
    code = ctypes.c_int(0)
    rc = library().hmat_check(h, _stream_ptr(stream), ctypes.byref(code))
    if rc not in (0, -6):
        _check(rc)
    return rc, code.value


def hmat_selftest_timeout(h: int, limit_us: int = 5000, stream=None):
    """Runs the device error-path self-test; returns (status, word)."""
    code = ctypes.c_int(0)
    rc = library().hmat_selftest_timeout(h, int(limit_us), _stream_ptr(stream), ctypes.byref(code))
    if rc not in (0, -6):
        _check(rc)
    return rc, code.value


def hmat_info(h: int) -> hmat_info_t:
    inf = hmat_info_t()
    _check(library().hmat_info(h, ctypes.byref(inf)))
    return inf


def hmat_get_perm(h: int, N: int) -> np.ndarray:
    perm = np.empty(N, dtype=np.int64)
    _check(library().hmat_get_perm(h, perm.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return perm


def hmat_export_block(h: int, level: int, t: int, s: int, r: int):
    sizes = (ctypes.c_int64 * 2)()
    _check(library().hmat_export_block(h, level, t, s, None, None, sizes))
    nt, ns = sizes[0], sizes[1]
    U = np.zeros((nt, r))
    V = np.zeros((ns, r))
    dp = ctypes.POINTER(ctypes.c_double)
    _check(library().hmat_export_block(h, level, t, s, U.ctypes.data_as(dp),
                                       V.ctypes.data_as(dp), sizes))
    return U, V


def hmat_export_dense(h: int, g: int) -> np.ndarray:
    n = ctypes.c_int64()
    _check(library().hmat_export_dense(h, g, None, ctypes.byref(n)))
    D = np.zeros((n.value, n.value))
    _check(library().hmat_export_dense(h, g, D.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       ctypes.byref(n)))
    return D


class HMatrix:
    """Owner of one handle: build on construction, destroy on close()/GC."""

    def __init__(self, points, kernel, leaf_size, rank, tol=0.0, **opt_kw):
        self.opts = hmat_default_opts(**opt_kw)
        self.h = hmat_build(points, kernel, leaf_size, rank, tol, self.opts)
        self.info = hmat_info(self.h)
        self.N = self.info.N

    @property
    def vec_dtype(self):
        import torch
        return torch.float64 if self.opts.prec == HMAT_FP64 else torch.float32

    def matvec(self, x, y=None, flags: int = 0, stream=None):
        """y = K x for a CUDA tensor x of shape (N,) or (N, k)."""
        import torch
        if x.dtype != self.vec_dtype or not x.is_cuda:
            raise TypeError(f"x must be a CUDA {self.vec_dtype} tensor")
        X = x.reshape(self.N, -1)
        if X.stride(1) != 1:
            raise ValueError("x must be row-major (unit stride across right-hand sides)")
        k = X.shape[1]
        if y is None:
            y = torch.empty_like(x)
        Y = y.reshape(self.N, -1)
        hmat_matvec(self.h, X, Y, k, X.stride(0), Y.stride(0), flags, stream)
        return y

    def gemv(self, alpha, x, beta, y, flags: int = 0, stream=None):
        """y = alpha K x + beta y in place, CUDA tensors x, y of shape (N,) or (N, k)."""
        for v in (x, y):
            if v.dtype != self.vec_dtype or not v.is_cuda:
                raise TypeError(f"x and y must be CUDA {self.vec_dtype} tensors")
        X = x.reshape(self.N, -1)
        Y = y.reshape(self.N, -1)
        if X.stride(1) != 1 or Y.stride(1) != 1 or X.shape != Y.shape:
            raise ValueError("x and y must be row-major N x k of the same shape")
        hmat_gemv(self.h, alpha, X, beta, Y, X.shape[1], X.stride(0), Y.stride(0), flags, stream)
        return y

    def clone_workspace(self) -> "HMatrix":
        """A second owner on the same device factors with its own workspace
        (for products on another stream at the same time).  It keeps this
        owner alive; close it first."""
        c = HMatrix.__new__(HMatrix)
        c.opts = self.opts
        c.h = hmat_clone_workspace(self.h)
        c.info = hmat_info(c.h)
        c.N = self.N
        c._base = self
        return c

    def check(self, stream=None):
        """(status, word) of the device status word (see hmat_check)."""
        return hmat_check(self.h, stream)

    def last_path(self) -> int:
        """HMAT_PATH_* bits of the kernels the last product launched."""
        return hmat_last_path(self.h)

    def perm(self) -> np.ndarray:
        return hmat_get_perm(self.h, self.N)

    def close(self):
        if getattr(self, "h", None):
            hmat_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
