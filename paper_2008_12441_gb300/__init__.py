"""Single-GPU (GB300, sm_103a) H-matrix-vector product under weak admissibility.

Li, Poulson, Ying, "Distributed-memory H-matrix Algebra I: Data
distribution and matrix-vector multiplication": the product y = K x of
Section 2 (eq. (hmat-vec-add)), computed by the steps of Section 4.1
collapsed onto one device.  The compute path is the C-ABI library
libhmat_gb300.so (include/hmat.h); ``hmat`` is its Python binding.
"""
from .hmat import (HMatrix, HMatError, hmat_build, hmat_default_opts, hmat_destroy,  # noqa: F401
                   hmat_export_block, hmat_export_dense, hmat_get_perm, hmat_info,
                   hmat_last_error, hmat_matvec, hmat_matvec_host, hmat_matvec_noalloc,
                   hmat_profile,
                   hmat_profile_read, hmat_convert, hmat_batch_create, hmat_batch_matvec,
                   hmat_batch_destroy, library)
