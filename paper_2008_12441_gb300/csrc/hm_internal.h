// Internal declarations of the H-matrix library (host side).
#pragma once

#include <atomic>
#include <cstdint>
#include <cstring>
#include <functional>
#include <string>
#include <thread>
#include <vector>

#include "hmat.h"

namespace hm {

// ------------------------------------------------------------------ errors
void set_error(const char* fmt, ...);
struct Error {
    int code;
    std::string msg;
};

// Allocation-failure injection (hmat_inject_alloc_failure): true when this
// allocation is the one to fail (counts the allocation either way).
bool injected_alloc_failure();

// ------------------------------------------------------------- threading
// Runs fn(i) for i in [0, n) on `threads` host threads (dynamic schedule).
void parallel_for(int64_t n, int threads, const std::function<void(int64_t)>& fn);
int default_threads();

// ------------------------------------------------------------------- tree
// Domain tree by recursive 2^d partition (x, then y, then z halving of the
// node's points; ties broken by original index), leaves at depth L.
struct Tree {
    int d = 0, L = 0, leaf_size = 0;
    int64_t N = 0;
    std::vector<int64_t> perm;                 // tree position -> original index
    std::vector<std::vector<int64_t>> beg;     // [level][node] tree-order begin
    std::vector<std::vector<int64_t>> cnt;     // [level][node] number of points
    int m_pad = 0;                             // slots per padded leaf
    int64_t Np = 0;                            // m_pad * 2^(d L)
    std::vector<int64_t> slot;                 // tree position -> padded slot
    std::vector<int64_t> slot_src;             // padded slot -> original index or -1
};
int tree_depth(int64_t N, int d, int leaf_size);

// ------------------------------------------------- standard admissibility
// Coordinates of node i of level l on the ideal-domain boxes: bit b of
// coordinate a is bit d b + a of i (child id c = b_0 + 2 b_1 + 4 b_2 at
// every level, children stored in id order).
void node_coords(int64_t i, int d, int l, int* c);
int64_t node_index(const int* c, int d, int l);
// Standard admissibility (Definition "Standard admissibility condition",
// eq. (standard-ad-cond), rho = sqrt(d)) between two boxes of one level
// holds iff they do not touch.  The low-rank blocks of a level-l node i are
// the nodes j whose parent touches (or is) i's parent and that do not touch
// i: offsets delta = c_j - c_i with delta_a in [-2 - p_a, 3 - p_a]
// (p_a = c_i,a mod 2), not all |delta_a| <= 1 -- 6^d - 3^d slots (27 in 2D,
// 189 in 3D) in increasing (delta_{d-1}, ..., delta_0) order.  Per parity
// class p (bit a = p_a) and slot q: the offset and the slot of -delta in
// the class of the node at that offset.
struct Stencil {
    int d = 0, nslot = 0, nnb = 0;        // nnb: touching boxes 3^d (near field)
    std::vector<int> off;                  // [(class * nslot + q) * 3 + a]
    std::vector<int> rev;                  // [class * nslot + q]
    // device table: (off_a + 4) << 4a for a < 3, | rev << 12
    std::vector<int> packed;
};
void build_stencil(int d, Stencil& st);
// Slot of offset delta (c_j - c_i) in the class of c_i, or -1.
int stencil_slot(const Stencil& st, const int* ci, const int* delta);
// slot_multiple: the padded leaf size is a multiple of this (8 or 16).
void build_tree(const double* points, int64_t N, int d, int leaf_size, int threads,
                int slot_multiple, Tree& t);

// ---------------------------------------------------------------- layout
// Device layout (element offsets are in "entries"; the byte size depends on
// the storage precision).  Level l = 1..nf holds low-rank blocks between
// siblings.  For node j of level l (n_l slots), its factors are s*r_l
// columns of n_l slots: column (q*r_l + c) of V_j is column c of the V
// factor of the block with target = the q-th other sibling of j; column
// (q*r_l + c) of U_i is column c of the U factor of the block with source =
// the q-th other sibling of i.  Near-field group g (node of level nf, G
// slots) stores D_g transposed: entry (b, p) at g*G*G + b*G + p.
struct LevelGeom {
    int level = 0;
    int r = 0;              // padded rank r_l
    int64_t n = 0;          // slots per node n_l
    int64_t nodes = 0;      // 2^(d l)
    int nsub = 1;           // project tiles per node (n_l / tile when n_l > tile)
    int64_t fac_off = 0;    // entry offset of level l in the U (and V) arrays
    int64_t fin_off = 0;    // node sums [node][s r_l] (units of one rhs)
    int64_t part_off = 0;   // per-tile partials [tile][s r_l] when nsub > 1
    int64_t cnt_off = 0;    // arrival counters (ints) when nsub > 1
};

struct Geometry {
    int d = 0, s = 0, L = 0, nf = 0, m_pad = 0;
    int adm = 0;                     // 0 weak, 1 standard admissibility
    int nnb = 1;                     // near-field source groups per group (1, or 3^d)
    int64_t Np = 0, G = 0, groups = 0;
    int64_t tile_p = 0;              // project tile (slots)
    int64_t fac_entries = 0;         // entries of U (== of V) over all levels
    int64_t dense_entries = 0;       // groups * G * G
    int64_t t_per_rhs = 0;           // node sums + partials per right-hand side
    int64_t counters = 0;            // arrival counters (ints)
    std::vector<LevelGeom> lv;       // lv[l] for l = 1..nf (lv[0] unused)
};

// Host master copy of every block, float64, in the device layout.
struct Master {
    std::vector<double> U, V, D;
    int64_t factor_entries = 0;      // real (unpadded) entries
    int64_t dense_entries = 0;
    int64_t lowrank_blocks = 0, dense_blocks = 0;
};

// GPU helper of the builder (build_gpu.cu): Y = K(rows, cols) M for many
// kernel blocks at once; M is ncols x ell row-major (float), Y is nrows x
// ell row-major (double).  Rows and columns are tree-position ranges.
struct SketchTask {
    int64_t row0, nrows, col0, ncols, m_off, y_off;
};
struct GpuSketch;
int gpu_sketch_init(GpuSketch** out, int device, const double* pts_tree, const int64_t* orig,
                    int64_t N, int d, int kernel);
int gpu_sketch_apply(GpuSketch* s, const std::vector<SketchTask>& tasks, int ell,
                     const std::vector<float>& M, std::vector<double>& Y);
void gpu_sketch_free(GpuSketch* s);

struct BuildParams {
    int kernel = 0, rank = 0, method = 0, oversample = 8, power_iters = 1;
    int adm = 0;                // 0 weak, 1 standard admissibility
    int leaf_lowrank = 0, threads = 0;
    double tol = 0.0;
    uint64_t seed = 0;
    GpuSketch* gpu = nullptr;   // non-null: randomized SVD products on the GPU
};

// Fills geometry + master from the tree and the points (tree order).
int compress_all(const Tree& t, const double* pts_tree, const BuildParams& bp,
                 Geometry& g, Master& m);
// Partial-sum workspace offsets of the levels (fin_off, part_off, cnt_off,
// counters, t_per_rhs) from their ranks, node sizes and tile counts.
void layout_workspace(Geometry& g);
// The random fill generated on the device (fill.cu): possible for unpadded
// trees (every leaf full) under weak admissibility.  random_fill_layout
// sets the geometry and the entry / block counts of `m` without its arrays.
bool random_fill_on_device_ok(const Tree& t, const BuildParams& bp);
int random_fill_layout(const Tree& t, const BuildParams& bp, Geometry& g, Master& m);

// Philox4x32-10 entry of a random block (see philox_hm.h for the layout).
double block_uniform(uint64_t seed, int kind, int level, uint32_t t, uint32_t s,
                     uint32_t row, uint32_t col);

}  // namespace hm
