"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only *draws* inputs: point sets, right-hand sides and the
workload table.  It holds none of the H-matrix arithmetic (no tree, no
blocks, no compression, no product), so the CPU oracle and the CUDA path can
both consume its arrays without sharing any code of the method.

Point sets follow the paper's numerical experiments (Section 5): an ideal
d-dimensional domain [0,1]^d discretised by n points per dimension
(Sections 5.1 and 5.2), plus uniform random points for the batched
workload of uneven instances.  The paper fills its H-matrices with random
numbers; those numbers are drawn by a counter-based generator that each
side implements on its own, keyed by the block, so they are not produced
here.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Kernel identifiers (same numbering as the C-ABI's hmat_kernel enum).
KERNEL_LOG2D = 0        # K(x,y) = -log|x-y|, K(x,x) = 1
KERNEL_INV4PIR3D = 1    # K(x,y) = 1/(4 pi |x-y|), K(x,x) = 1
KERNEL_RANDOM = 2       # blocks filled with counter-based random numbers

# Compression methods (same numbering as the C-ABI).
METHOD_TSVD = 0
METHOD_RSVD = 1
METHOD_RANDOM = 2

# Storage precisions (same numbering as the C-ABI's hmat_prec enum).
PREC_FP64 = 0
PREC_FP32 = 1
PREC_BF16 = 2
PREC_BF16X2 = 3
PREC_FP8E4M3 = 4
PREC_NAMES = {PREC_FP64: "fp64", PREC_FP32: "fp32", PREC_BF16: "bf16",
              PREC_BF16X2: "bf16x2", PREC_FP8E4M3: "fp8e4m3"}


def grid_points(n: int, d: int) -> np.ndarray:
    """Cell centres (i + 1/2)/n of a uniform n^d grid on [0,1]^d.

    Original point index = i_0 + n*i_1 (+ n^2*i_2): x varies fastest.
    Returns an (n^d, d) float64 array.
    """
    if n <= 0 or d not in (2, 3):
        raise ValueError("grid_points: n > 0 and d in {2, 3}")
    c = (np.arange(n, dtype=np.float64) + 0.5) / n
    axes = np.meshgrid(*([c] * d), indexing="ij")   # axes[a][i_0, i_1, ...]
    # flatten with i_0 fastest
    cols = [ax.transpose(tuple(range(d))[::-1]).reshape(-1) for ax in axes]
    return np.ascontiguousarray(np.stack(cols, axis=1))


def uniform_points(N: int, d: int, seed: int) -> np.ndarray:
    """N points drawn uniformly in [0,1]^d (numpy PCG64 stream `seed`)."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.random((N, d), dtype=np.float64))


def gaussian_rhs(N: int, k: int, seed: int) -> np.ndarray:
    """N x k right-hand sides with i.i.d. N(0,1) entries, row-major."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.standard_normal((N, k), dtype=np.float64))


@dataclass
class Instance:
    """One H-matrix problem: points, kernel, tree and compression choice."""
    name: str
    d: int
    N: int
    kernel: int
    leaf_size: int
    rank: int
    method: int
    nrhs: int
    seed: int
    oversample: int = 8
    power_iters: int = 1
    leaf_lowrank: int = 0
    grid_n: int = 0              # > 0: uniform grid with grid_n points per dim
    precisions: tuple = (PREC_FP32,)

    def points(self) -> np.ndarray:
        if self.grid_n > 0:
            return grid_points(self.grid_n, self.d)
        return uniform_points(self.N, self.d, self.seed)

    def rhs(self, k: int | None = None, salt: int = 0) -> np.ndarray:
        return gaussian_rhs(self.N, self.nrhs if k is None else k,
                            self.seed * 1000 + 17 + salt)


def c1_small() -> Instance:
    """2D log kernel, 64x64 grid, leaf 64, truncated SVD rank 8, FP64, 1 RHS."""
    return Instance("2d-log-n4096-tsvd-r8", 2, 4096, KERNEL_LOG2D, 64, 8,
                    METHOD_TSVD, 1, 12441, grid_n=64, precisions=(PREC_FP64,))


def c2_fp32_gemv() -> Instance:
    """2D log kernel, 512x512 grid, leaf 64, randomized SVD rank 16 (p=8), FP32, 1 RHS."""
    return Instance("2d-log-n262144-rsvd-r16", 2, 262144, KERNEL_LOG2D, 64, 16,
                    METHOD_RSVD, 1, 12442, grid_n=512, precisions=(PREC_FP32,))


def c3_3d_multi() -> Instance:
    """3D 1/(4 pi r) kernel, 64^3 grid, leaf 64, rank 32, 32 RHS, FP32 vs BF16."""
    return Instance("3d-inv4pir-n262144-r32-k32", 3, 262144, KERNEL_INV4PIR3D, 64, 32,
                    METHOD_RSVD, 32, 12443, grid_n=64,
                    precisions=(PREC_FP32, PREC_BF16))


def c4_precision_sweep() -> Instance:
    """2D log kernel, 1024x1024 grid, leaf 64, rank 16, 64 RHS, four storage modes."""
    return Instance("2d-log-n1048576-r16-k64", 2, 1048576, KERNEL_LOG2D, 64, 16,
                    METHOD_RSVD, 64, 12444, grid_n=1024,
                    precisions=(PREC_FP32, PREC_BF16, PREC_BF16X2, PREC_FP8E4M3))


def c5_batched(count: int = 256, seed: int = 12445,
               n_lo: int = 4096, n_hi: int = 65536) -> list[Instance]:
    """Uneven instances: half 2D log, half 3D 1/r kernel, uniform random points.

    N is log-uniform on [n_lo, n_hi], rank uniform on {8,16,32}, RHS count
    uniform on {1..16}; leaf 64; randomized SVD with oversampling 8.
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        d = 2 if i < count // 2 else 3
        N = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        r = int(rng.choice([8, 16, 32]))
        k = int(rng.integers(1, 17))
        kern = KERNEL_LOG2D if d == 2 else KERNEL_INV4PIR3D
        out.append(Instance(f"batch{i}-d{d}-n{N}-r{r}-k{k}", d, N, kern, 64, r,
                            METHOD_RSVD, k, seed * 1000 + i,
                            precisions=(PREC_BF16,)))
    return out


def random_fill(name: str, d: int, grid_n: int, rank: int, nrhs: int, seed: int,
                leaf_size: int = 64) -> Instance:
    """The paper's own benchmark workload: random dense and low-rank blocks
    on an ideal grid (Sections 5.1, 5.2), random input vectors."""
    return Instance(name, d, grid_n ** d, KERNEL_RANDOM, leaf_size, rank,
                    METHOD_RANDOM, nrhs, seed, grid_n=grid_n)


def covering_rows(N: int, sms: int, seed: int, tiles=(256, 128)) -> np.ndarray:
    """Output positions (tree order, no padding) to compare one by one at a
    full size: for every tile size T in `tiles`, one position drawn
    uniformly inside every run of T consecutive positions, plus the first
    and last position of every contiguous range of ceil((N / T) / sms)
    tiles -- the ranges that persistent kernels with one CTA per SM walk.
    Sorted, without repeats."""
    rng = np.random.default_rng(seed)
    out = []
    for T in tiles:
        ntile = -(-N // T)
        starts = np.arange(ntile, dtype=np.int64) * T
        span = np.minimum(T, N - starts)
        out.append(starts + rng.integers(0, span))
        R = -(-ntile // max(sms, 1))
        r0 = np.arange(0, ntile, R, dtype=np.int64) * T
        r1 = np.minimum(r0 + R * T, N) - 1
        out.extend([r0, r1])
    return np.unique(np.concatenate(out))
