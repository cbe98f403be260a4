/*
 * hmat.h -- C ABI of the single-GPU (GB300, sm_103a) H-matrix-vector product.
 *
 * Problem (Li, Poulson, Ying, "Distributed-memory H-matrix Algebra I",
 * Section 2): the Nystrom discretisation of u(t) = int K(t,s) f(s) ds on a
 * point set in [0,1]^d (eq. (intop)) gives a dense N x N matrix that is
 * approximated by an H-matrix (Definition "H-matrix", def:hmat) built on a
 * domain tree (Definition "Domain tree") under the weak admissibility
 * condition (Definition "Weak admissibility condition").  The product
 * y = K x is the sum, over every dense block D and every low-rank block
 * U V^T, of D x_{w_s} or U (V^T x_{w_s}) into y_{w_t} (eq. (hmat-vec-add)).
 * On the GPU it runs as the paper's Section 4.1 steps collapsed onto one
 * device: Step 1 (source-side V^T x, eq. (prod-vx)), Step 2 (the reduction
 * of partial sums, here a fixed-order on-device sum), Steps 3-4 (transfer
 * and broadcast, here pure indexing into the partial-sum buffer) and Step 5
 * (target-side U z and D x, eqs. (prod-yuz), (prod-ydz)).
 *
 * Conventions for every entry point:
 *   - Return value: HMAT_OK (0) or a negative hmat_status; the message of
 *     the last error of the calling thread is in hmat_last_error().
 *   - Host pointers are only read during the call unless stated.
 *   - Device pointers refer to memory on the handle's device.
 *   - Vectors are row-major N x nrhs with a leading dimension (elements
 *     between consecutive points) >= nrhs; element type double in the
 *     HMAT_FP64 mode, float in every other mode.
 *   - Streams are cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Device work is stream-ordered and asynchronous unless stated.
 */
#ifndef HMAT_H
#define HMAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hmat_s* hmat_t;   /* opaque; owns host tree data and device buffers */

typedef enum {
    HMAT_OK = 0,
    HMAT_EINVAL = -1,        /* bad argument (null, negative size, bad enum, ...) */
    HMAT_ENOMEM = -2,        /* host or device allocation failed */
    HMAT_ECUDA = -3,         /* a CUDA runtime call failed */
    HMAT_EUNSUPPORTED = -4,  /* valid request the library does not serve */
    HMAT_EDEVICE = -5,       /* a kernel reported an error through its status word */
    HMAT_ETIMEOUT = -6       /* a bounded device-side wait gave up */
} hmat_status;

typedef enum {
    HMAT_K_LOG2D = 0,        /* K(x,y) = -log|x-y|, K(x,x) = 1, d = 2 */
    HMAT_K_INV4PIR_3D = 1,   /* K(x,y) = 1/(4 pi |x-y|), K(x,x) = 1, d = 3 */
    HMAT_K_RANDOM = 2        /* random blocks (the paper's benchmark matrices, Section 5.1) */
} hmat_kernel;

typedef enum {
    HMAT_TSVD = 0,           /* truncated SVD of each admissible block */
    HMAT_RSVD = 1,           /* randomized SVD (range finder, oversampling p, q power iterations) */
    HMAT_RANDOM_FILL = 2     /* counter-based random U, V, D (requires HMAT_K_RANDOM) */
} hmat_method;

typedef enum {
    HMAT_ADM_WEAK = 0,       /* Definition "Weak admissibility condition": distinct nodes of a level */
    HMAT_ADM_STANDARD = 1    /* Definition "Standard admissibility condition", eq. (standard-ad-cond),
                                rho = sqrt(d), on the nodes' boxes of the ideal domain: boxes that do
                                not touch */
} hmat_admissibility;

typedef enum {
    HMAT_FP64 = 0,           /* factors, vectors and accumulation in double */
    HMAT_FP32 = 1,           /* float factors, float accumulation */
    HMAT_BF16 = 2,           /* bf16 factors with a power-of-two scale per block, float accumulation */
    HMAT_BF16X2 = 3,         /* split factors hi + lo (two bf16), float accumulation */
    HMAT_FP8E4M3 = 4         /* e4m3 low-rank factors with a float scale per column; bf16 dense blocks */
} hmat_prec;

/* Flags of hmat_matvec. */
#define HMAT_TREE_ORDER 1    /* x and y are in tree order (hmat_get_perm) instead of original order */
#define HMAT_TRANSPOSE 2     /* y = K^T x instead of K x (see hmat_prepare_transpose) */

/* Kernel families of a product (bits of hmat_last_path). */
#define HMAT_PATH_PROJECT_STREAMED 1   /* Steps 1-2: persistent TMA-ring kernel, one right-hand side */
#define HMAT_PATH_EXPAND_STREAMED 2    /* Steps 3-5: persistent TMA-ring kernel, one right-hand side */
#define HMAT_PATH_PROJECT_TENSOR 4     /* Steps 1-2: tcgen05 kernels (bf16 family, 2..64 right-hand sides) */
#define HMAT_PATH_EXPAND_TENSOR 8      /* Steps 3-5: tcgen05 kernels */
#define HMAT_PATH_PROJECT_CACHED 16    /* Steps 1-2: CUDA-core kernel, one tile per CTA */
#define HMAT_PATH_EXPAND_CACHED 32     /* Steps 3-5: CUDA-core kernel, one tile per CTA */

typedef struct {
    int prec;            /* hmat_prec of the device factors (default HMAT_FP32) */
    int method;          /* hmat_method (default HMAT_RSVD) */
    int leaf_lowrank;    /* 0: sibling leaves are dense (Definition def:hmat checks leafness
                            first); 1: sibling leaves are low-rank too (default 0) */
    int oversample;      /* randomized SVD oversampling p (default 8) */
    int power_iters;     /* randomized SVD power iterations q (default 1) */
    int device;          /* CUDA device ordinal (default 0); -1 builds on the host only
                            (no upload; hmat_matvec returns HMAT_EUNSUPPORTED) */
    int max_nrhs;        /* right-hand sides per pass; sizes the workspace (default 64) */
    int threads;         /* host threads used by hmat_build, 0 = all cores (default 0) */
    int keep_host;       /* 1: keep the float64 master factors on the host after the upload
                            (needed by hmat_export_block / hmat_export_dense; default 0;
                            always kept when device = -1) */
    int build_gpu;       /* build steps on the GPU: the randomized SVD products K_b M (float
                            evaluation, double chunk sums), and the random fill written straight
                            into the device layout (bit-identical to the host fill; unpadded
                            trees, weak admissibility, FP32/FP64 storage, keep_host = 0; no
                            host copy exists then): 1 yes, 0 no, -1 auto = yes when
                            N >= 65536 and device >= 0 (default -1) */
    uint64_t seed;       /* seed of the counter-based generator (sketches, random fill) */
    int admissibility;   /* hmat_admissibility (default HMAT_ADM_WEAK).  Standard: low-rank
                            blocks between the non-touching children of touching parents
                            (interaction lists of 27 nodes in 2D, 189 in 3D, on levels
                            2..L-1), dense blocks between all leaves under touching parents
                            (leafness checked first, as for weak); needs leaf_lowrank = 0 and
                            the streamed kernels' geometry (near-field groups and level nodes
                            of whole 256-slot tiles); products run one right-hand side per
                            pass on those kernels; not available: the tensor-core, batched,
                            allocation-free and transposed products */
    int leaf_slot_multiple; /* 0 (default): every leaf is padded to the smallest multiple of the
                            storage's own alignment (8 slots, 16 in e4m3) that holds the largest
                            leaf.  q > 0, a multiple of 8 up to 256: a multiple of q (and of that
                            alignment) instead.  q = 32 in 2D or 16 in 3D makes every near-field
                            group (2^d leaves) a multiple of 128 slots, so that trees of uneven
                            leaves (random points) take the tensor-core kernels (2..64
                            right-hand sides, bf16 family) and the streamed project at the cost
                            of the zero slots' bytes */
} hmat_opts;

typedef struct {
    int64_t N;           /* points */
    int d;               /* dimension, 2 or 3 */
    int depth;           /* L: leaves at level L of the domain tree */
    int lowrank_levels;  /* levels 1..lowrank_levels hold low-rank sibling blocks */
    int leaf_slots;      /* points per padded leaf (>= largest leaf) */
    int prec;            /* hmat_prec */
    int64_t padded_N;    /* leaf_slots * 2^(d*depth) */
    int64_t lowrank_blocks;
    int64_t dense_blocks;      /* dense blocks of Definition def:hmat (leaf pairs) */
    int64_t factor_entries;    /* sum over low-rank blocks of (|w_t| + |w_s|) r_b */
    int64_t dense_entries;     /* sum over dense blocks of |w_t| |w_s| */
    int64_t device_bytes;      /* factor + dense + scale bytes stored on the device */
    int64_t workspace_bytes;   /* partial-sum buffer and staging */
    int rank_per_level[32];    /* padded rank r_l of level l (index l) */
    int admissibility;         /* hmat_admissibility */
    int partners;              /* low-rank partners per node and level: 2^d - 1 siblings (weak), or
                                  6^d - 3^d interaction-list slots (standard; zero factor columns
                                  where a slot lies outside the domain) */
    int near_groups;           /* source groups of a near-field group: 1 (weak), 3^d (standard) */
} hmat_info_t;

/* Default options (see the field comments). */
void hmat_default_opts(hmat_opts* opts);

/*
 * hmat_build -- build the H-matrix of `kernel` on `points` and upload it.
 *   points     host, N x d row-major double, copied.
 *   N          >= 1.
 *   d          2 or 3 (HMAT_K_LOG2D needs 2, HMAT_K_INV4PIR_3D needs 3).
 *   leaf_size  >= 1: the tree depth L is the smallest with ceil(N/2^(dL)) <= leaf_size
 *              (Definition "Domain tree", 2^d partition of an ideal domain).
 *   rank       > 0: fixed rank r per admissible block, clamped to the block size;
 *              <= 0: rank chosen per block by the relative tolerance `tol`.
 *   opts       NULL for defaults.
 *   out        receives the handle; untouched on error.
 * Blocks follow Definition def:hmat with weak admissibility; construction
 * itself is outside the paper (end of Section 2).  Runs on the host (all
 * cores unless opts->threads) and uploads with synchronous copies.
 * Errors: HMAT_EINVAL, HMAT_ENOMEM, HMAT_ECUDA.
 */
int hmat_build(const double* points, int64_t N, int d, int kernel, int leaf_size,
               int rank, double tol, const hmat_opts* opts, hmat_t* out);

/*
 * hmat_matvec -- y = K x for nrhs right-hand sides (eq. (hmat-vec-add)).
 *   x      device, N x nrhs, leading dimension ldx >= nrhs; not modified.
 *   y      device, N x nrhs, leading dimension ldy >= nrhs; overwritten.
 *   nrhs   >= 1; more than opts.max_nrhs is processed in passes.
 *   flags  OR of HMAT_TREE_ORDER and HMAT_TRANSPOSE (y = K^T x: every
 *          block applied transposed, from its target rows to its source
 *          columns; the first such product on a handle runs
 *          hmat_prepare_transpose, which allocates and synchronises).
 *   stream cudaStream_t or NULL.
 * Per pass of right-hand sides it launches the project side (Steps 1-2:
 * V^T x of every source node and the tree reduction of the partial sums)
 * and then the expand side (Steps 3-5: routing of the sums to their
 * targets, U z and the dense near field), as one to five kernels depending
 * on the path (hmat_last_path says which), and returns without
 * synchronising.  x and y must not overlap.  The
 * handle's partial-sum workspace is shared by all calls on the handle, so
 * calls on one handle must be ordered: the handle records an event after
 * each product, and a product on another stream while that event is still
 * pending is refused (HMAT_EUNSUPPORTED; nothing is launched).  For
 * concurrent products give each stream its own hmat_clone_workspace.  The
 * check is skipped while `stream` is being captured into a graph.
 * Errors: HMAT_EINVAL (null, nrhs < 1, ld < nrhs), HMAT_EUNSUPPORTED (the
 * previous product on another stream is in flight), HMAT_ECUDA (launch).
 */
int hmat_matvec(hmat_t h, const void* x, void* y, int nrhs, int64_t ldx,
                int64_t ldy, int flags, void* stream);

/*
 * hmat_prepare_transpose -- device state of the transposed product y = K^T x
 * (the transposed and symmetric products of the H-matrix algebra the paper
 * points to after Sec. 3.2).  Under weak admissibility block (j, i) of K^T is
 * V_ij U_ij^T, and the sibling slot of i at j has the formula of the slot of
 * j at i, so K^T runs the same kernels with the U and V arrays (and their
 * scales) swapped; the dense near-field blocks need D^T: a transposed device
 * copy (the dense bytes again) unless every near-field block is symmetric
 * (a symmetric kernel), in which case D serves both products.  Allocates
 * that copy and the tensor maps over the swapped arrays, synchronises the
 * device, and is idempotent; workspace clones share it with their original.
 * Call it before capturing HMAT_TRANSPOSE products into a graph and before
 * hmat_matvec_noalloc with HMAT_TRANSPOSE.
 * Errors: HMAT_EINVAL (null), HMAT_EUNSUPPORTED (host-only handle),
 * HMAT_ENOMEM, HMAT_ECUDA.
 */
int hmat_prepare_transpose(hmat_t h);

/*
 * hmat_gemv -- y = alpha K x + beta y, the level-2 BLAS form of the product
 * (the remark closing the algorithm of Sec. 4.1).
 *   alpha, beta  finite scalars, applied in the vectors' precision (float,
 *                or double in the FP64 mode).
 *   x, y, nrhs, ldx, ldy, flags, stream  as hmat_matvec; y is read and
 *                overwritten, and not read at all when beta == 0 (it may
 *                then hold anything, NaN included).
 * K x of up to opts.max_nrhs columns at a time goes to the handle's device
 * staging (hmat_matvec_host uses the same buffer), then one elementwise
 * kernel forms alpha (K x) + beta y.  Asynchronous, ordered as hmat_matvec.
 * Errors: as hmat_matvec; HMAT_EINVAL also for a non-finite alpha or beta.
 */
int hmat_gemv(hmat_t h, double alpha, const void* x, double beta, void* y, int nrhs,
              int64_t ldx, int64_t ldy, int flags, void* stream);

/*
 * hmat_clone_workspace -- a second handle on the same H-matrix with its own
 * workspace, for products on several streams at once.  The clone borrows
 * the source's device factors, dense blocks, scales, slot maps and tensor
 * maps (no copy) and allocates its own partial sums, arrival counters,
 * status word, prepared tensor-core operands and host-entry staging
 * (hmat_info's workspace_bytes).  Cloning a clone borrows from the same
 * original.  Host-copy functions (hmat_save, hmat_convert, hmat_export_*)
 * on a clone read the original's host copy.  Destroy every clone before
 * the original: hmat_destroy of a handle with live clones returns
 * HMAT_EINVAL and frees nothing.
 * Errors: HMAT_EINVAL (null), HMAT_EUNSUPPORTED (built on the host only),
 * HMAT_ENOMEM / HMAT_ECUDA (allocation).
 */
int hmat_clone_workspace(hmat_t src, hmat_t* out);

/*
 * hmat_matvec_host -- as hmat_matvec, with x and y in HOST memory.  Copies x
 * to a device staging buffer, runs the product, copies y back and
 * synchronises the stream before returning.  Pinned host memory gives
 * asynchronous copies; pageable memory works but is slower.
 * Errors: as hmat_matvec; HMAT_EUNSUPPORTED if nrhs > opts.max_nrhs.
 */
int hmat_matvec_host(hmat_t h, const void* x_host, void* y_host, int nrhs,
                     int64_t ldx, int64_t ldy, int flags, void* stream);

/*
 * hmat_matvec_noalloc -- y = K x exactly as hmat_matvec, for callers that must
 * not have device memory allocated on their behalf when they run the
 * product: a runtime whose device memory is handed out only by its own
 * pre-reserved pool, or a latency-critical loop that cannot afford the
 * implicit device synchronisation of cudaMalloc / cudaFree.  (hmat_matvec
 * does not allocate either, but it writes its partial sums into a workspace
 * that hmat_build allocated for the handle; this entry point leaves that
 * workspace alone.)  The paper has no counterpart: it is an interface
 * choice of this library.
 *   Arguments, layouts and errors as hmat_matvec.
 * Scratch: the partial sums live in one static device array of 8 MiB
 * compiled into the library; every GPU that loads the library holds it until
 * the process exits.  The array is shared by every call on every handle of a
 * device and keeps the last call's contents (every entry a call reads is
 * written by the same call first, so nothing needs clearing).  Calls whose
 * kernels overlap on the GPU (different streams, or different host threads
 * without ordering) race on the array and give wrong results: order them.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it; make that first call before any
 * stream capture.  No cudaMalloc, cudaFree or allocating library routine is
 * called.  Right-hand sides run in passes sized to the array.
 * Errors: as hmat_matvec; HMAT_EUNSUPPORTED if one right-hand side needs more
 * partial-sum storage than the array holds (the message gives both sizes),
 * or for HMAT_TRANSPOSE before hmat_prepare_transpose (which allocates);
 * HMAT_ECUDA if the address lookup fails.
 */
int hmat_matvec_noalloc(hmat_t h, const void* x, void* y, int nrhs, int64_t ldx,
                        int64_t ldy, int flags, void* stream);

/*
 * hmat_convert -- a new handle holding the same H-matrix in another storage
 * precision (same tree, blocks and float64 master; re-rounded and uploaded).
 * The source must keep its host copy (opts.keep_host = 1).  e4m3 needs leaf
 * slots that are a multiple of 16 (a tree built for another precision may
 * not have them: HMAT_EUNSUPPORTED).  Construction of the storage formats is
 * this library's choice; the paper stores factors in one precision.
 */
int hmat_convert(hmat_t src, int prec, hmat_t* out);

/*
 * Batched products of many H-matrices (different N, rank, depth, right-hand
 * side count; same device and precision) in one CUDA graph, in one of two
 * schedules:
 *   HMAT_BATCH_QUEUE: a persistent project launch and a persistent expand
 *     launch per right-hand-side width class (CUDA-core kernels), whose CTAs
 *     pull (instance, tile) tasks, largest first, from an atomic queue
 *     counter; x and y pointers are read from a device table, so the graph
 *     serves any buffers.
 *   HMAT_BATCH_BRANCHES: each instance's own product (the kernels
 *     hmat_matvec would launch for it: tensor cores, streamed or CUDA-core)
 *     on one of `branches` parallel branches of the graph, instances dealt
 *     to the branches largest first (by bytes) onto the least loaded one.
 *     The graph holds the x and y pointers: the first hmat_batch_matvec,
 *     and any later call with other pointers, records it again (host time
 *     that grows with the number of kernels recorded; the executable graph
 *     is updated in place when the topology allows).
 * Outputs stay atomic-free.  The paper's benchmarks run one H-matrix at a
 * time; this is the single-GPU counterpart of running many independent
 * problems.
 *
 * hmat_batch_create -- plan for handles hs[0..count) with nrhs[i] right-hand
 *   sides each (one pass per instance: nrhs[i] <= 64, 32 in FP64).
 *   flags: 0 or HMAT_TREE_ORDER, OR one schedule: HMAT_BATCH_QUEUE
 *   (the default when no schedule bit is given) or
 *   HMAT_BATCH_BRANCHES (8 branches; hmat_batch_autotune tries others).
 *   The handles must be distinct (a handle's workspace serves one product
 *   at a time: pass hmat_clone_workspace handles to repeat an operator) and
 *   outlive the plan, and a plan's products must not overlap other products
 *   on the same handles (the cross-stream check of hmat_matvec does not see
 *   plan launches, so order them).
 *   Errors: HMAT_EINVAL (including a repeated handle), HMAT_EUNSUPPORTED
 *   (mixed devices / precisions, too many right-hand sides), HMAT_ECUDA
 *   (including a failed graph capture).
 * hmat_batch_matvec -- y_i = K_i x_i for every instance: xs[i], ys[i] device
 *   pointers, row-major N_i x nrhs[i] (leading dimension nrhs[i]).  Queue
 *   schedule: uploads the pointer table (asynchronously, pinned) and
 *   launches the graph on `stream`.  Branch schedule: records the graph
 *   again if the pointers changed, then launches it on `stream`.  Returns
 *   without synchronising.
 * hmat_batch_check -- synchronises `stream` and reads the status words of
 *   the plan (a queue kernel that met a task outside the plan's instances or
 *   their tiles skips it and sets the word) and of every instance's handle
 *   (bounded waits); the words are cleared, and after a refused task so are
 *   the instances' arrival counters (a skipped tile leaves its nodes'
 *   counts short), so that later products start clean.
 *   code  host int (may be NULL): the first nonzero word, else 0.
 *   Errors: HMAT_EINVAL, HMAT_ECUDA, HMAT_EDEVICE (a task was refused),
 *   HMAT_ETIMEOUT (an instance's wait gave up).
 * hmat_batch_destroy -- free the plan (NULL is OK).
 */
#define HMAT_BATCH_QUEUE 0x100
#define HMAT_BATCH_BRANCHES 0x200
typedef struct hmat_batch_s* hmat_batch_t;
int hmat_batch_create(const hmat_t* hs, int count, const int* nrhs, int flags,
                      hmat_batch_t* out);
int hmat_batch_matvec(hmat_batch_t b, const void* const* xs, void* const* ys, void* stream);
int hmat_batch_check(hmat_batch_t b, void* stream, int* code);
int hmat_batch_destroy(hmat_batch_t b);

/*
 * hmat_batch_poison_task -- test hook for the queue schedule's task check:
 * overwrites task `task` of the plan's device task table (in launch order)
 * with instance index `inst` and tile `tile`, which the kernels check
 * against the plan before any access.  An entry outside the plan makes the
 * next hmat_batch_matvec skip that task and set the plan's status word
 * (hmat_batch_check then returns HMAT_EDEVICE); the other tasks still run.
 * Rebuild the plan afterwards.  Not for production use.
 * Errors: HMAT_EINVAL (null plan, task out of range), HMAT_EUNSUPPORTED
 * (branch schedule), HMAT_ECUDA.
 */
int hmat_batch_poison_task(hmat_batch_t b, int task, int inst, int tile);

/*
 * hmat_batch_autotune -- choose the plan's schedule by measurement.  Tries
 * the queue schedule with every combination of (a) the persistent grid of
 * each launch: all CTAs the SMs hold, half, a quarter; and (b) the
 * right-hand-side width classes: each instance's own compiled width, or
 * widths rounded up to 1, 4, 16, 64 (fewer launches, more idle lanes); and
 * the branch schedule with 4, 8, 16 and 32 branches.  Each candidate plan
 * runs once to warm up and then `reps` times on `stream` with the caller's
 * xs / ys (as hmat_batch_matvec), timed with CUDA events; the plan is
 * rebuilt (graph included) with the fastest and run once more, so ys hold
 * its results on return (the stream is synchronised).
 *   out  host struct (may be NULL): the chosen schedule and times.
 * Errors: HMAT_EINVAL (null plan or vectors, reps < 1), HMAT_ECUDA.
 */
typedef struct {
    int grid_div;        /* queue: persistent CTAs = resident CTAs per SM x SMs / grid_div */
    int coarse_widths;   /* queue: 1 = widths rounded up to 1, 4, 16, 64 */
    int candidates;      /* schedules timed */
    double ms;           /* mean time per batched product of the chosen schedule */
    double ms_default;   /* the same for hmat_batch_create's schedule */
    int schedule;        /* HMAT_BATCH_QUEUE or HMAT_BATCH_BRANCHES */
    int branches;        /* branch schedule: parallel branches (0 for the queue) */
    double ms_queue;     /* the fastest queue schedule */
    double ms_branches;  /* the fastest branch schedule */
} hmat_batch_tuning;
int hmat_batch_autotune(hmat_batch_t b, const void* const* xs, void* const* ys, void* stream, int reps,
                        hmat_batch_tuning* out);

/*
 * hmat_save -- write the handle to `path`: the options, the tree and the
 * geometry, and the float64 master factors (a little-endian binary file of
 * this library's own format).  Needs the host copy (built with keep_host,
 * or on the host only).
 * Errors: HMAT_EINVAL (null, the file cannot be written), HMAT_EUNSUPPORTED
 * (no host copy).
 *
 * hmat_load -- read a file written by hmat_save and build the handle from it
 * (no recompression; the device layout and storage rounding are redone).
 *   opts  NULL: the saved options; else the caller's device, precision,
 *         keep_host, max_nrhs, threads (the structure options of the file are
 *         kept: method, leaf_lowrank, oversample, power_iters, seed).
 * Errors: HMAT_EINVAL (null, unreadable, truncated or foreign file),
 * HMAT_EUNSUPPORTED (the leaf slots do not suit the precision), HMAT_ENOMEM,
 * HMAT_ECUDA.
 */
int hmat_save(hmat_t h, const char* path);
int hmat_load(const char* path, const hmat_opts* opts, hmat_t* out);

/* hmat_destroy -- free every host and device resource of the handle (NULL is OK);
 * a workspace clone frees only its own workspace.  Synchronises the handle's
 * device first.  Errors: HMAT_EINVAL while clones of the handle are alive
 * (nothing is freed). */
int hmat_destroy(hmat_t h);

/*
 * hmat_profile -- enable (1) or disable (0) per-kernel timing of later
 * hmat_matvec calls on this handle: every kernel launch is bracketed by a
 * pair of CUDA events recorded on the launch stream.  Either call resets
 * the accumulated totals.
 */
int hmat_profile(hmat_t h, int enable);

/*
 * hmat_profile_read -- waits for the recorded events and returns, per kernel
 * (index 0 = project, Step 1; index 1 = expand, Steps 2-5), the number of
 * launches and the summed device time in milliseconds since hmat_profile(h, 1).
 *   launches  host int64[2];  ms  host double[2].
 */
int hmat_profile_read(hmat_t h, int64_t* launches, double* ms);

/* hmat_info -- sizes and counts of the handle (host struct filled in). */
int hmat_info(hmat_t h, hmat_info_t* out);

/* hmat_get_perm -- perm[i] = original index of the point at tree position i
 * (host array of N int64). */
int hmat_get_perm(hmat_t h, int64_t* perm);

/*
 * hmat_export_block -- float64 master factors of the low-rank block with
 * target node t and source node s of `level` (distinct siblings; under
 * standard admissibility s in the interaction list of t)
 * (1 <= level <= lowrank_levels; nodes numbered in tree order within the level).
 *   U  host, |w_t| x r_l row-major (rows in tree order of the node's points);
 *   V  host, |w_s| x r_l row-major; r_l = rank_per_level[level] (zero-padded columns).
 *   sizes  host int64[2] receiving |w_t|, |w_s| (may be NULL).
 * Pass U = V = NULL to query sizes only.  Needs a host copy (keep_host or device = -1).
 */
int hmat_export_block(hmat_t h, int level, int64_t t, int64_t s, double* U, double* V,
                      int64_t* sizes);

/*
 * hmat_export_dense -- float64 dense near-field block of group g (the nodes of
 * level lowrank_levels) with itself, |g| x |g| row-major in tree order; NULL D
 * queries |g| into *size.  In the default structure this is the union of the
 * dense blocks between the group's sibling leaves (Definition def:hmat,
 * condition 1); under standard admissibility the near field also couples g
 * with its touching groups, whose blocks this does not export.
 */
int hmat_export_dense(hmat_t h, int64_t g, double* D, int64_t* size);

/*
 * hmat_check -- synchronises `stream` (cudaStream_t or NULL) and reads the
 * handle's device status word, which a kernel sets when one of its bounded
 * waits (every mbarrier wait of the streamed and tensor-core kernels is
 * limited to about two seconds) gave up instead of hanging; the word is
 * cleared.  The products launched since the last check are then not
 * trustworthy.  hmat_matvec_host performs this check itself.
 *   code  host int (may be NULL): the status word (0 = no wait gave up).
 * Errors: HMAT_EINVAL (null handle), HMAT_ECUDA, HMAT_ETIMEOUT (word nonzero).
 */
int hmat_check(hmat_t h, void* stream, int* code);

/*
 * hmat_selftest_timeout -- exercises the device error path on the handle's
 * device: launches one CTA whose single bounded wait (limit_us microseconds)
 * waits for an mbarrier phase that nothing completes, so the wait gives up,
 * sets the handle's status word and the kernel returns; then runs
 * hmat_check.  Expected result: HMAT_ETIMEOUT with *code = 1.  No other
 * state of the handle is touched.
 * Errors: HMAT_EINVAL (null handle, limit_us outside [1, 1000000]),
 * HMAT_EUNSUPPORTED (host-only handle), HMAT_ECUDA.
 */
int hmat_selftest_timeout(hmat_t h, int limit_us, void* stream, int* code);

/*
 * hmat_launch_count -- number of kernel launches the library has issued in
 * this process (all handles and devices; launches recorded into a CUDA graph
 * count once, when recorded).  Differences around a call give the kernels
 * per call.
 */
int64_t hmat_launch_count(void);

/*
 * hmat_last_path -- the kernel families the handle's last product (hmat_matvec,
 * hmat_gemv, hmat_matvec_host, hmat_matvec_noalloc) launched: an OR of the
 * HMAT_PATH_* bits (0 before the first product).  The choice is made per
 * call from the geometry, the storage precision and the right-hand-side
 * count; tests use it to assert which kernels ran.
 * Errors: HMAT_EINVAL (null handle).
 */
int hmat_last_path(hmat_t h);

/*
 * hmat_inject_alloc_failure -- test hook for the out-of-memory paths: the
 * library's (after + 1)-th allocation from now on (device buffers, pinned
 * host words and the float64 host master arrays, counted process-wide) fails
 * as if memory were exhausted, so that the call making it returns
 * HMAT_ENOMEM after freeing what it had allocated; after < 0 switches the
 * injection off.  Returns the previous setting.  Not for production use.
 */
int64_t hmat_inject_alloc_failure(int64_t after);

/* hmat_last_error -- message of the calling thread's last error ("" if none). */
const char* hmat_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HMAT_H */
