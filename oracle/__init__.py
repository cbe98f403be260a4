"""FP64 CPU oracle for the H-matrix-vector product (test infrastructure only).

This package is the plain, slow, obviously correct statement of what the
GPU path computes.  It is *test infrastructure*: only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it.  The product library never calls it, and it shares no code with
the product (it builds its own domain tree, its own block list, its own
block contents and its own product).

Modules
-------
philox   Philox4x32-10 counter-based generator (Salmon et al., SC'11),
         written from its published definition; used to fill random blocks
         and to draw randomized-SVD test matrices.
tree     Domain tree (Section 2, Definition "Domain tree"): recursive 2^d
         partition of the point set.
hmatrix  Block structure of Definition "H-matrix" (Section 2, def:hmat)
         under the weak admissibility condition, and the contents of each
         block (kernel evaluation, truncated / randomized SVD, random fill).
matvec   The product y = K x by eq. (hmat-vec-add) of Section 2, a dense
         assembly of the same blocks (brute force), and exact entry / flop
         counts.

Everything is float64.  Pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` (worked example, closed-form counts, brute
force, full-rank exactness, Eckart-Young, linearity, permutation
equivariance, Philox known answers).
"""
from .philox import philox4x32_10, block_uniform
from .tree import DomainTree, build_tree
from .hmatrix import (HMatrix, Block, build_hmatrix, kernel_eval,
                      dense_kernel_matrix)
from .matvec import (hmat_matvec, hmat_matvec_rows, hmat_matvec_transpose,
                     hmat_matvec_transpose_rows, assemble_dense, entry_counts, flop_count)

__all__ = ["philox4x32_10", "block_uniform", "DomainTree", "build_tree",
           "HMatrix", "Block", "build_hmatrix", "kernel_eval",
           "dense_kernel_matrix", "hmat_matvec", "hmat_matvec_rows",
           "hmat_matvec_transpose", "hmat_matvec_transpose_rows",
           "assemble_dense", "entry_counts", "flop_count"]
