// Device-side parameter blocks and launcher declarations shared by the
// CUDA translation units and the C-ABI glue.
#pragma once
#include <cstddef>
#include <cstdint>

namespace hm {

constexpr int kMaxLevels = 24;

struct DevLevel {
    int r;            // padded rank r_l
    int nsub;         // project tiles per node (> 1: partial sums + last-CTA reduction)
    int64_t n;        // slots per node n_l
    int64_t fac_off;  // entry offset of the level in U / V
    int64_t fin_off;  // offset of the node sums [node][s*r_l] (units of one rhs)
    int64_t part_off; // offset of the per-tile partial sums [tile][s*r_l] (units of one rhs)
    int64_t cnt_off;  // offset of the per-node arrival counters (ints)
    int64_t sc_off;   // offset of the level's scales (bf16: per block, fp8: per column)
    int64_t tt_off;   // element offset of the level in the prepared t operands (tensor cores)
    int tma_rb;       // rows of one V box of the streamed project (0: no map)
    int tma_rb_u;     // rows of one U box of the streamed expand (0: no map)
};

// Storage codes (device factor element types).
enum StoreKind { ST_F64 = 0, ST_F32 = 1, ST_BF16 = 2, ST_BF16X2 = 3, ST_FP8 = 4 };

struct MatvecArgs {
    // geometry (s: partners per node -- siblings under weak admissibility,
    // interaction-list slots under standard)
    int d, s, nf, store;
    int adm;              // 0 weak, 1 standard admissibility
    int nnb;              // near-field source groups per group (1, or 3^d)
    const int* stencil;   // standard: per parity class and slot, packed offsets and reverse slot
    int64_t Np, G, tile_p, tile_e;
    DevLevel lv[kMaxLevels + 1];
    // factors (element type given by the storage kind; the dense blocks are
    // bf16 in the fp8 mode)
    const void* U;
    const void* V;
    const void* D;
    const void* U_lo;     // split storage: low parts
    const void* V_lo;
    const void* D_lo;
    const float* scU;     // scales (bf16: per block, fp8: per column)
    const float* scV;
    const float* scD;     // per near-field group (bf16 and fp8 modes)
    // vectors
    const void* x;
    void* y;
    int64_t ldx, ldy;
    const int64_t* map;   // slot -> vector row (or -1); nullptr = identity
    int k;                // right-hand sides in this pass
    int kc;               // rhs stride of the partial-sum buffer
    void* T;              // node sums + partials (float, or double in the FP64 mode)
    int* cnt;             // arrival counters (zero between calls)
    int* status;          // device status word: nonzero after a bounded wait gave up
    // tensor-core path: bf16 B operands prepared in global memory
    void* xprep;          // x tiles (64 rows x tile_p slots per project tile)
    void* xprep_lo;
    void* ttprep;         // summed t per target node (64 rows x sr_pad per node)
    void* ttprep_lo;
    int tc_range;         // tiles per CTA of the persistent tensor-core project (0: one)
    int tc_seg;           // tiles per accumulation segment of that kernel (flush at least this often)
    // tensor maps (device array of kTensorMapBytes-byte descriptors, 64-byte
    // aligned), [kind][level]: kind 0 / 1 = V / V_lo over the rows of V^l
    // (row = node * s r_l + column, n_l slots), box tile_p x lv[l].tma_rb;
    // kind 2 / 3 = U / U_lo likewise with box kExpandStreamTile x
    // lv[l].tma_rb_u, and at level 0 the dense blocks D / D_lo over rows
    // g * G + b (G slots), box kExpandStreamTile x tma_rb_d.
    // kinds 4 / 5 = V / V_lo with the 128-byte swizzle, box 64 slots x 128
    // columns, and kinds 6 / 7 likewise with box 64 x (s r_l mod 128): the
    // A operands of the tensor-core project kernel (K-major); kinds 8-11 the
    // same for U (level 0: D) with boxes of tc_expand_kb columns: the A
    // operands of the tensor-core expand kernel (MN-major).
    const void* tmaps;    // V maps (nullptr: no streamed project)
    const void* tmaps_u;  // same array when the U and D maps exist (nullptr: no streamed expand)
    const void* tmaps_tc; // same array when the swizzled V maps exist (nullptr: none)
    int tma_rb_d;
    int pdl;              // streamed kernels: launch Step 2 and the expand as programmatic dependents
};

constexpr int kTensorMapBytes = 128;
constexpr int kTensorMapKinds = 16;
constexpr int kMapU8 = 14;       // e4m3 U^l, no swizzle, box 64 slots x 64 columns
constexpr int kMapU8Rem = 15;    // e4m3 U^l, box 64 x (s r_l mod 64, rounded up to 16)
constexpr int kMapV8 = 12;       // e4m3 V^l, no swizzle, box 64 slots x 128 columns
constexpr int kMapV8Rem = 13;    // e4m3 V^l, box 64 x (s r_l mod 128)
constexpr int kMapVSw = 4;       // + part: box 64 x 128
constexpr int kMapVSwRem = 6;    // + part: box 64 x (s r_l mod 128)
constexpr int kMapUSw = 8;       // + part: U^l (level 0: D), box 64 slots x tc_expand_kb columns
constexpr int kMapUSwRem = 10;   // + part: U^l, box 64 x (s r_l mod kb, rounded up to 16)
// K columns per stage of the tensor-core expand
inline int tc_expand_kb(int /*store*/) { return 64; }
constexpr int kExpandStreamTile = 256;   // slots per tile of the streamed expand
// Encode a 2-D tensor map over `rows` rows of `row_len` elements of `esize`
// bytes (row pitch row_len * esize) starting at `base`, box box_x x box_y,
// no interleave, optional 128-byte swizzle, into the kTensorMapBytes bytes
// at `map`.  Returns 0, or nonzero if the driver refused it or could not be
// reached.
int encode_rows_map(void* map, const void* base, int esize, uint64_t row_len, uint64_t rows,
                    uint32_t box_x, uint32_t box_y, bool swizzle128);

// Streamed project: stage capacity (rows) for tile_p slots of `esize`-byte
// elements in `parts` arrays (24 KB and 32 rows at most per stage), and the
// box rows of a level with sr = s r_l columns (the largest divisor of sr
// within the capacity, so that a stage holds whole boxes of one node).
inline int stream_stage_rows(int64_t tile, int esize, int parts) {
    const int64_t r = (int64_t)(24 * 1024) / (tile * esize * parts);
    return r < 1 ? 1 : r > 32 ? 32 : (int)r;
}
// Streamed expand: box rows for `cols` columns of kExpandStreamTile slots of
// `esize`-byte elements in `parts` arrays (16 KB per stage).
inline int expand_box_rows(int cols, int esize, int parts) {
    int cap = (16 * 1024) / (kExpandStreamTile * esize * parts);
    cap = cap < 1 ? 1 : cap > 64 ? 64 : cap;
    for (int b = cols < cap ? cols : cap; b > 1; --b)
        if (cols % b == 0) return b;
    return 1;
}
inline int stream_box_rows(int sr, int cap) {
    for (int b = sr < cap ? sr : cap; b > 1; --b)
        if (sr % b == 0) return b;
    return 1;
}

// Kernel families a product can take (the bits of hmat_last_path).
constexpr unsigned kPathProjectStreamed = 1u;
constexpr unsigned kPathExpandStreamed = 2u;
constexpr unsigned kPathProjectTensor = 4u;
constexpr unsigned kPathExpandTensor = 8u;
constexpr unsigned kPathProjectCached = 16u;
constexpr unsigned kPathExpandCached = 32u;
// Launch kernel `which` (0 = project: Steps 1-2; 1 = expand: Steps 3-5) for
// one pass of a.k <= a.kc right-hand sides; ORs the family it took into
// *path (may be null).  Returns a cudaError_t value.
int launch_kernel(int which, const MatvecArgs& a, void* stream, unsigned* path);
// Maximum right-hand sides per pass supported by the kernels of a storage kind.
int max_pass_rhs(int store_kind);
// Compiled RHS width for a pass of k right-hand sides: the smallest width
// >= k whose shared-memory staging fits, else the widest that fits (0: none).
int pass_width(const MatvecArgs& a, int k);
// Slot alignment (elements) the storage kind needs for 16-byte vector loads.
int slot_align(int store_kind);

// Persistent single-right-hand-side project kernel (stream.cu): bulk
// copies of the factor rows through a shared-memory ring; needs a.k == 1,
// a.kc == 1, a status word and a tile structure within its tables.
// Returns a cudaError_t value, or kStreamNotEligible (nothing launched).
constexpr int kStreamNotEligible = -1;
int stream_project(const MatvecArgs& a, void* stream);
// Process-wide count of kernel launches issued by the library (every
// launch site adds its launches; captured launches count when captured).
void count_launches(int n);
int64_t launch_count();
// Persistent single-right-hand-side expand kernel (stream.cu), same
// conventions: needs a.tmaps_u, G a multiple of kExpandStreamTile.
int stream_expand(const MatvecArgs& a, void* stream);
// Launch a kernel whose one bounded wait (limit_ns) cannot complete: it sets
// *status (device) to 1 and returns.  Returns a cudaError_t value.
int wait_selftest(int* status, uint64_t limit_ns, void* stream);
// GEMV epilogue (gemv.cu): y[i ldy + c] = alpha t[i ldt + c] + beta y[i ldy + c]
// for i < n, c < k, in double (f64) or float; y is not read when beta == 0.
// Returns a cudaError_t value.
int axpby(bool f64, int64_t n, int k, double alpha, const void* t, int64_t ldt, double beta, void* y,
          int64_t ldy, void* stream);

// Device random fill (fill.cu), float or double: one level of U (kind 0) or
// V (kind 1), nodes x (s r columns) x n slots, entries scale * Philox value
// of block (target, source) at (row, column); the dense near-field groups,
// groups x G x G stored column-major per group (leaf pairs of m slots, or
// the diagonal block).  Return a cudaError_t value (asynchronous on the
// legacy stream).
int fill_random_factor(void* dst, bool f64, int kind, uint64_t seed, int level, int64_t nodes, int64_t n, int s,
                       int r, double scale);
int fill_random_dense(void* dst, bool f64, uint64_t seed, int lev, int64_t groups, int64_t G, int64_t m, int nc,
                      int leaf_pairs, double scale);

// Transposed copy of the dense near-field blocks (transpose.cu): for each of
// `groups` row-major G x G blocks of `esize`-byte elements (2, 4 or 8),
// dst = src^T.  Returns a cudaError_t value.
int transpose_groups(const void* src, void* dst, int esize, int64_t groups, int64_t G, void* stream);

// Tensor-core path (tc_matvec.cu): bf16-family storage, tiles aligned with
// the near-field groups and the low-rank nodes.  a.k <= 64.
bool tc_eligible(const MatvecArgs& a);
int tc_launch(int which, const MatvecArgs& a, int* status, void* stream);

// ---- batched launches (many H-matrices, persistent CTAs pulling tasks)
struct BatchTask {
    int inst;   // instance (index into the argument array)
    int tile;   // tile of that instance
};
struct BatchLaunch {
    const MatvecArgs* args;     // device array, one per instance
    const int* units;           // device: project units per instance
    const void* const* xs;      // device: x of every instance for this call
    void* const* ys;            // device: y of every instance
    const BatchTask* tasks;     // device, largest first
    int ntasks;
    int* queue;                 // device counter, zero before the launch
    size_t smem;                // dynamic shared memory (max over the instances)
    int grid_div;               // persistent CTAs = (resident CTAs per SM x SMs) / grid_div
    int count;                  // instances of the plan (tasks are checked against it)
    int* status;                // device: the plan's status word (refused tasks)
};
// Per-instance setup of kernel `which` (0 project, 1 expand) at width a.kc:
// tile count (`units`: project units per tile, or expand tiles) and the
// dynamic shared memory; sets a.tile_e for the expand kernel.
int batch_setup(MatvecArgs& a, int which, int* units, size_t* smem);
// One persistent launch of kernel `which` over the tasks (all instances of
// one storage kind and width kc); with dry != 0 only the kernel attributes
// are set (do this before a stream capture).  Returns a cudaError_t value.
int batch_launch(int which, int store, int kc, const BatchLaunch& b, void* stream, int dry);

// Size of the static partial-sum array used by hmat_matvec_noalloc (8 MiB).
constexpr size_t kStaticScratchBytes = (size_t)8 << 20;
// Device address of that array on `device` (which must be current); the
// first call per device looks it up with cudaGetSymbolAddress.  Returns a
// cudaError_t value.
int static_scratch_address(int device, void** ptr);

// Host-side quantisation (quantize.cu), round to nearest even:
// dst = bf16(src * scale_inv), hi + lo = bf16 split of src, dst = e4m3(src * scale_inv)
// (saturating to +-448).
void to_bf16(const double* src, uint16_t* dst, size_t n, double scale_inv);
void to_bf16_split(const double* src, uint16_t* hi, uint16_t* lo, size_t n);
void to_fp8e4m3(const double* src, uint8_t* dst, size_t n, double scale_inv);

}  // namespace hm
