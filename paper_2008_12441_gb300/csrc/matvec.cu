// CUDA-core kernels of the single-GPU H-matrix-vector product.
//
// The paper's distributed algorithm (Section 4.1) runs five steps; on one
// GPU they become two kernels over a padded, level-major layout:
//
//   project (Steps 1-2): for every low-rank level l and every source node j,
//     the s sibling products V_ij^T x_j at once (eq. (prod-vx)), as s*r_l
//     dot products over the node's slots.  One CTA owns a tile of slots
//     across ALL levels (x is read once).  Nodes longer than the tile leave
//     one partial sum per tile; the last CTA to finish a node (arrival
//     counter) adds that node's partials in tile order -- Step 2's tree
//     reduction, without atomics on data and with a fixed order.
//   expand (Steps 3-5): every CTA gathers, for each target node of its tile,
//     the sums t_{i<-j} of its sibling sources (Steps 3-4 are the index
//     transpose "slot of i at source j": no data moves), then streams its
//     rows of the dense near-field block and of every level's U factor
//     (eqs. (prod-yuz), (prod-ydz)).  The columns of one row are split
//     across several threads for memory-level parallelism and recombined
//     in shared memory in a fixed order; each y element is stored once.
//
// Storage kinds: float64, float32, bf16 with a power-of-two scale per block,
// split bf16 (hi + lo), e4m3 with a float scale per column (dense blocks in
// bf16).  Scales are applied to the short vectors (partial sums, staged x),
// never inside the streaming loops.  Accumulation is in float (double in
// the float64 mode).  Results are bitwise reproducible.
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "hm_device.h"
#include "hm_once.h"
#include "hm_elem.cuh"

namespace hm {
namespace {

// ------------------------------------------------------------------ project
// grid: Np / tile_p CTAs, 256 threads.  smem: tile_p * KC values of x, then
// one descriptor per unit.  A unit is R consecutive columns of one segment
// (a node, or the tile's part of a node) of one level: the R rows share
// their x values, which each lane loads once per step from shared memory.
struct UnitDesc {
    int64_t voff;   // first element of the first row in V (rows are n_l apart)
    int64_t dst;    // destination of the first row (rows are kc apart)
    int64_t node;   // node of the segment
    int64_t n;      // n_l: distance between consecutive rows in V
    int xoff;       // first staged x value of the segment
    int seg;        // row length (slots)
    int col0;       // first column
    int nrow;       // rows in the unit (<= R)
    int level;
    int pad_[3];
};

// x values a lane needs for one 16-byte vector of the factor: VEC * KC
// consecutive values, loaded as 16-byte words.
template <typename A, int N>
__device__ __forceinline__ void lds_vec(const A* p, A (&o)[N]) {
    constexpr int B = N * (int)sizeof(A);
    if constexpr (B % 16 == 0) {
#pragma unroll
        for (int q = 0; q < B / 16; ++q) {
            union { float4 v; A e[16 / sizeof(A)]; } u;
            u.v = reinterpret_cast<const float4*>(p)[q];
#pragma unroll
            for (int t = 0; t < (int)(16 / sizeof(A)); ++t) o[q * (16 / sizeof(A)) + t] = u.e[t];
        }
    } else {
#pragma unroll
        for (int t = 0; t < N; ++t) o[t] = p[t];
    }
}

template <typename A>
struct ProjShared {
    int last[kMaxLevels + 1];
    int units[kMaxLevels + 2];   // first unit of each level
    A red[256];
};

// One project tile `ptile` of one H-matrix (x, y of this call passed apart
// from the argument block so that batched launches can share it).
template <int ST, int KC, int R>
__device__ __forceinline__ void project_tile(const MatvecArgs& a, const void* xptr,
                                             int64_t ptile, int total_units,
                                             unsigned char* smem_raw,
                                             ProjShared<typename Tr<ST>::A>& sh) {
    using A = typename Tr<ST>::A;
    constexpr int VEC = Tr<ST>::VEC;
    int* s_last = sh.last;
    int* s_units = sh.units;
    A* s_red = sh.red;
    const int tile = (int)a.tile_p;
    A* xs = reinterpret_cast<A*>(smem_raw);
    UnitDesc* desc =
        reinterpret_cast<UnitDesc*>(smem_raw + (((size_t)tile * KC * sizeof(A) + 15) / 16) * 16);
    const int64_t p0 = ptile * tile;
    const A* __restrict__ x = static_cast<const A*>(xptr);

    for (int e = threadIdx.x; e < tile * KC; e += blockDim.x) {
        const int pl = e / KC;
        const int c = e - pl * KC;
        const int64_t src = a.map ? a.map[p0 + pl] : p0 + pl;
        xs[e] = (src >= 0 && c < a.k) ? x[src * a.ldx + c] : A(0);
    }
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int l = 1; l <= a.nf; ++l) {
            s_units[l] = acc;
            const int seg = a.lv[l].n < tile ? (int)a.lv[l].n : tile;
            const int sr = a.s * a.lv[l].r;
            acc += (tile / seg) * ((sr + R - 1) / R);
        }
        s_units[a.nf + 1] = acc;
    }
    __syncthreads();
    for (int u = threadIdx.x; u < total_units; u += blockDim.x) {
        int l = 1;
        while (s_units[l + 1] <= u) ++l;
        const DevLevel& L = a.lv[l];
        const int sr = a.s * L.r;
        const int ub = (sr + R - 1) / R;          // units per segment
        const int lu = u - s_units[l];
        const bool small = L.n < tile;             // several whole nodes per tile
        const int seg = small ? (int)L.n : tile;
        const int sg = lu / ub, cb = lu - sg * ub;
        const int64_t node = small ? p0 / L.n + sg : p0 / L.n;
        const int64_t inoff = small ? 0 : p0 - node * L.n;
        UnitDesc d;
        d.col0 = cb * R;
        d.nrow = sr - d.col0 < R ? sr - d.col0 : R;
        d.voff = L.fac_off + (node * sr + d.col0) * L.n + inoff;
        d.dst = L.nsub > 1 ? (L.part_off + ptile * sr + d.col0) * a.kc
                           : (L.fin_off + node * sr + d.col0) * a.kc;
        d.node = node;
        d.n = L.n;
        d.xoff = sg * seg * KC;
        d.seg = seg;
        d.level = l;
        desc[u] = d;
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = blockDim.x >> 5;
    A* __restrict__ T = static_cast<A*>(a.T);
    const uint4* __restrict__ V = static_cast<const uint4*>(a.V);
    const uint4* __restrict__ Vlo = static_cast<const uint4*>(a.V_lo);
    for (int u = warp; u < total_units; u += nw) {
        const UnitDesc d = desc[u];
        A acc[R][KC];
#pragma unroll
        for (int rr = 0; rr < R; ++rr)
#pragma unroll
            for (int c = 0; c < KC; ++c) acc[rr][c] = A(0);
        // each lane takes two vectors per step (i and i + 32 VEC) so that both
        // of them are in flight together
        const int64_t rs = d.n / VEC;
        for (int i = lane * VEC; i < d.seg; i += 64 * VEC) {
            const int i2 = i + 32 * VEC;
            const bool two = i2 < d.seg;
            uint4 hi[R][2], lo[R][2];
            const int64_t base = (d.voff + i) / VEC;
#pragma unroll
            for (int rr = 0; rr < R; ++rr) {
                if (rr < d.nrow) {
                    hi[rr][0] = __ldg(V + base + rr * rs);
                    if (two) hi[rr][1] = __ldg(V + base + 32 + rr * rs);
                    if constexpr (ST == ST_BF16X2) {
                        lo[rr][0] = __ldg(Vlo + base + rr * rs);
                        if (two) lo[rr][1] = __ldg(Vlo + base + 32 + rr * rs);
                    }
                }
            }
            if constexpr (KC == 1) {
                A xv[VEC * KC];
                lds_vec<A, VEC * KC>(xs + d.xoff + i * KC, xv);
#pragma unroll
                for (int rr = 0; rr < R; ++rr)
                    if (rr < d.nrow) DotStep<ST, KC, 0>::go(hi[rr][0], lo[rr][0], xv, acc[rr]);
                if (two) {
                    lds_vec<A, VEC * KC>(xs + d.xoff + i2 * KC, xv);
#pragma unroll
                    for (int rr = 0; rr < R; ++rr)
                        if (rr < d.nrow) DotStep<ST, KC, 0>::go(hi[rr][1], lo[rr][1], xv, acc[rr]);
                }
            } else {
                // several right-hand sides: the KC x values of one slot at a
                // time, shared by the R rows (per accumulator the same order
                // as one vector after the other, element by element)
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    if (j == 1 && !two) break;
                    const int ij = j == 0 ? i : i2;
#pragma unroll
                    for (int e = 0; e < VEC; ++e) {
                        A xe[KC];
                        lds_vec<A, KC>(xs + d.xoff + (ij + e) * KC, xe);
#pragma unroll
                        for (int rr = 0; rr < R; ++rr) {
                            if (rr >= d.nrow) continue;
                            A v = elem_at<ST>(hi[rr][j], e);
                            if constexpr (ST == ST_BF16X2) v += elem_at<ST>(lo[rr][j], e);
#pragma unroll
                            for (int c = 0; c < KC; ++c) acc[rr][c] += v * xe[c];
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int rr = 0; rr < R; ++rr)
#pragma unroll
                for (int c = 0; c < KC; ++c)
                    acc[rr][c] += __shfl_xor_sync(0xffffffffu, acc[rr][c], off);
        const DevLevel& L = a.lv[d.level];
#pragma unroll
        for (int rr = 0; rr < R; ++rr) {
            if (rr >= d.nrow) continue;
            const A sc = (A)factor_scale<ST>(a.scV, L, a.s, d.node, d.col0 + rr);
#pragma unroll
            for (int c = 0; c < KC; ++c)
                if ((c & 31) == lane && c < a.k) T[d.dst + (int64_t)rr * a.kc + c] = acc[rr][c] * sc;
        }
    }

    // Step 2: the last CTA of every node longer than the tile adds the
    // node's partial sums in a fixed order (per item: tiles u = f mod F in
    // increasing order, four interleaved accumulators, then f = 0..F-1).
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int l = 1; l <= a.nf; ++l) {
            const DevLevel& L = a.lv[l];
            s_last[l] = 0;
            if (L.nsub <= 1 || L.r == 0) continue;
            const int64_t node = p0 / L.n;
            const int prev = atomicAdd(a.cnt + L.cnt_off + node, 1);
            s_last[l] = prev == L.nsub - 1;
        }
        __threadfence();
    }
    __syncthreads();
    for (int l = 1; l <= a.nf; ++l) {
        if (!s_last[l]) continue;
        const DevLevel L = a.lv[l];
        const int64_t node = p0 / L.n;
        node_step2<A>(a, L, node, (int)threadIdx.x, s_red, [] { __syncthreads(); });
        if (threadIdx.x == 0) a.cnt[L.cnt_off + node] = 0;
    }
}

template <int ST, int KC, int R>
__global__ void __launch_bounds__(256) project_kernel(const MatvecArgs a, int total_units) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ ProjShared<typename Tr<ST>::A> sh;
    project_tile<ST, KC, R>(a, a.x, (int64_t)blockIdx.x, total_units, smem_raw, sh);
}

// Persistent project over many H-matrices: CTAs pull (instance, tile) tasks,
// largest first, from an atomic queue counter.  A task naming an instance
// outside the plan or a tile outside its instance is skipped before any
// access and reported in the plan's status word (0x401 project, 0x402
// expand); every thread of the CTA reads the same task, so the decision is
// uniform.

__device__ __forceinline__ bool task_ok(const BatchTask& bt, const MatvecArgs* args, int count, int which) {
    if (bt.inst < 0 || bt.inst >= count || bt.tile < 0) return false;
    const MatvecArgs& a = args[bt.inst];
    const int64_t tile = which == 0 ? a.tile_p : a.tile_e;
    return tile > 0 && (int64_t)bt.tile < a.Np / tile;
}

template <int ST, int KC, int R>
__global__ void __launch_bounds__(256)
    project_batched(const MatvecArgs* __restrict__ args, const int* __restrict__ units,
                    const void* const* __restrict__ xs, const BatchTask* __restrict__ tasks,
                    int ntasks, int* queue, int count, int* status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ ProjShared<typename Tr<ST>::A> sh;
    __shared__ int s_task;
    for (;;) {
        if (threadIdx.x == 0) s_task = atomicAdd(queue, 1);
        __syncthreads();
        const int t = s_task;
        if (t >= ntasks) break;
        const BatchTask bt = tasks[t];
        if (!task_ok(bt, args, count, 0)) {
            if (threadIdx.x == 0) atomicCAS(status, 0, 0x401);
            __syncthreads();
            continue;
        }
        project_tile<ST, KC, R>(args[bt.inst], xs[bt.inst], bt.tile, units[bt.inst], smem_raw, sh);
        __syncthreads();
    }
}

// ------------------------------------------------------------------- expand
// grid: Np / tile_e CTAs; (tile_e / PT) slot groups x SPLIT column ranges of
// threads.  smem: x of the near-field group(s) covering the tile (times the
// group's dense-block scale), per level the sums t_{i<-j} of the tile's
// target nodes (times the U scales) [node][s*r_l][KC], and SPLIT-1 partial
// outputs for the fixed-order recombination.
struct ExpShared {
    int ttoff[kMaxLevels + 1];
    int i0[kMaxLevels + 1];     // first target node of the tile per level
};

template <int ST, int KC, int PT, int SPLIT>
__device__ __forceinline__ void expand_tile_body(const MatvecArgs& a, const void* xptr, void* yptr,
                                                 int64_t etile, unsigned char* smem_raw,
                                                 ExpShared& sh) {
    using A = typename Tr<ST>::A;
    constexpr int DST = DenseKind<ST>::value;
    int* s_ttoff = sh.ttoff;
    int* s_i0 = sh.i0;
    const int TE = (int)a.tile_e;
    const int64_t e0 = etile * TE;
    const int G = (int)a.G;
    const int64_t g0 = e0 / G;                   // first near-field group of the tile
    const int GX = TE > G ? TE : G;
    const int nc = a.s + 1;
    const A* __restrict__ x = static_cast<const A*>(xptr);
    const A* __restrict__ T = static_cast<const A*>(a.T);
    A* xg = reinterpret_cast<A*>(smem_raw);
    A* ttb = xg + GX * KC;

    if (threadIdx.x == 0) {
        int off = 0;
        for (int l = 1; l <= a.nf; ++l) {
            const int64_t n = a.lv[l].n;
            const int nodes_t = TE >= n ? (int)(TE / n) : 1;
            s_ttoff[l] = off;
            s_i0[l] = (int)(e0 / n);
            off += nodes_t * a.s * a.lv[l].r * KC;
        }
        s_ttoff[0] = off;                          // total
    }
    for (int e = threadIdx.x; e < GX * KC; e += blockDim.x) {
        const int b = e / KC;
        const int c = e - b * KC;
        const int64_t slot = g0 * G + b;
        const int64_t src = a.map ? a.map[slot] : slot;
        A v = (src >= 0 && c < a.k) ? x[src * a.ldx + c] : A(0);
        if constexpr (DST == ST_BF16) v *= a.scD[g0 + b / G];
        xg[e] = v;
    }
    __syncthreads();
    // Steps 3-4: target node i of the tile reads, for its q-th other sibling
    // j, the sums of source j at j's slot for i.
    for (int l = 1; l <= a.nf; ++l) {
        const DevLevel& L = a.lv[l];
        const int r = L.r;
        const int sr = a.s * r;
        const int nodes_t = TE >= L.n ? (int)(TE / L.n) : 1;
        const int i0 = s_i0[l];
        A* ttl = ttb + s_ttoff[l];
        const int total = nodes_t * sr * KC;
        for (int e = threadIdx.x; e < total; e += blockDim.x) {
            const int c = e % KC;
            const int rest = e / KC;
            const int il = rest / sr;
            const int col = rest - il * sr;
            const int i = i0 + il;
            const int ci = i & (nc - 1);
            const int qp = col / r, cr = col - qp * r;
            const int cj = qp < ci ? qp : qp + 1;
            const int j = i - ci + cj;
            const int qv = ci < cj ? ci : ci - 1;
            A v = A(0);
            if (c < a.k) {
                v = T[(L.fin_off + (int64_t)j * sr + qv * r + cr) * a.kc + c];
                v *= (A)factor_scale<ST>(a.scU, L, a.s, i, col);
            }
            ttl[e] = v;
        }
    }
    A* red = ttb + s_ttoff[0];   // [SPLIT-1][TE/PT][PT][KC]
    __syncthreads();

    const int groups = TE / PT;
    const bool active = (int)threadIdx.x < groups * SPLIT;   // batched launches may be wider
    const int g = threadIdx.x % groups;
    const int sp = active ? (int)threadIdx.x / groups : 0;
    const int lt = g * PT;                    // slot of this thread within the tile
    int ktot = G;
    for (int l = 1; l <= a.nf; ++l) ktot += a.s * a.lv[l].r;
    const int k0 = active ? (int)((int64_t)ktot * sp / SPLIT) : 0;
    const int k1 = active ? (int)((int64_t)ktot * (sp + 1) / SPLIT) : 0;

    A acc[PT][KC];
#pragma unroll
    for (int v = 0; v < PT; ++v)
#pragma unroll
        for (int c = 0; c < KC; ++c) acc[v][c] = A(0);

    // Step 5, dense near-field block: y_p += sum_b D[p][b] x_b (eq. (prod-ydz))
    {
        const int gl = TE > G ? lt / G : 0;                     // group within the tile
        const int pin = TE > G ? lt - gl * G : (int)(e0 - g0 * G) + lt;   // row in the group
        const int64_t dbase = (g0 + gl) * (int64_t)G * G + pin;
        const A* xgg = xg + gl * G * KC;
        const int b1 = k1 < G ? k1 : G;
#pragma unroll 4
        for (int b = k0; b < b1; ++b) {
            A dv[PT];
            load_dec<DST, PT>(a.D, a.D_lo, dbase + (int64_t)b * G, dv);
#pragma unroll
            for (int v = 0; v < PT; ++v)
#pragma unroll
                for (int c = 0; c < KC; ++c) acc[v][c] += dv[v] * xgg[b * KC + c];
        }
    }
    // Step 5, low-rank blocks, finest level first: y_p += U_p t (eq. (prod-yuz))
    {
        int off = G;
        for (int l = a.nf; l >= 1; --l) {
            const DevLevel& L = a.lv[l];
            const int sr = a.s * L.r;
            const int lo = k0 - off > 0 ? k0 - off : 0;
            const int hi = k1 - off < sr ? k1 - off : sr;
            off += sr;
            if (lo >= hi) continue;
            const bool many = TE > L.n;
            const int il = many ? lt / (int)L.n : 0;
            const int64_t i = s_i0[l] + il;
            const int64_t inoff = many ? lt - il * L.n : e0 - i * L.n + lt;
            const int64_t ubase = L.fac_off + i * sr * L.n + inoff;
            const A* tl = ttb + s_ttoff[l] + il * sr * KC;
#pragma unroll 4
            for (int col = lo; col < hi; ++col) {
                A uv[PT];
                load_dec<ST, PT>(a.U, a.U_lo, ubase + (int64_t)col * L.n, uv);
#pragma unroll
                for (int v = 0; v < PT; ++v)
#pragma unroll
                    for (int c = 0; c < KC; ++c) acc[v][c] += uv[v] * tl[col * KC + c];
            }
        }
    }
    if constexpr (SPLIT > 1) {
        if (active && sp > 0) {
            A* rd = red + ((sp - 1) * groups + g) * PT * KC;
#pragma unroll
            for (int v = 0; v < PT; ++v)
#pragma unroll
                for (int c = 0; c < KC; ++c) rd[v * KC + c] = acc[v][c];
        }
        __syncthreads();
        if (!active || sp > 0) return;
#pragma unroll
        for (int s2 = 0; s2 < SPLIT - 1; ++s2) {
            const A* rd = red + (s2 * groups + g) * PT * KC;
#pragma unroll
            for (int v = 0; v < PT; ++v)
#pragma unroll
                for (int c = 0; c < KC; ++c) acc[v][c] += rd[v * KC + c];
        }
    }
    if (!active) return;
    A* __restrict__ y = static_cast<A*>(yptr);
#pragma unroll
    for (int v = 0; v < PT; ++v) {
        const int64_t slot = e0 + lt + v;
        const int64_t dst = a.map ? a.map[slot] : slot;
        if (dst < 0) continue;
#pragma unroll
        for (int c = 0; c < KC; ++c)
            if (c < a.k) y[dst * a.ldy + c] = acc[v][c];
    }
}

template <int ST, int KC, int PT, int SPLIT>
__global__ void __launch_bounds__(512) expand_kernel(const MatvecArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ ExpShared sh;
    expand_tile_body<ST, KC, PT, SPLIT>(a, a.x, a.y, (int64_t)blockIdx.x, smem_raw, sh);
}

template <int ST, int KC, int PT, int SPLIT>
__global__ void __launch_bounds__(256)
    expand_batched(const MatvecArgs* __restrict__ args, const void* const* __restrict__ xs,
                   void* const* __restrict__ ys, const BatchTask* __restrict__ tasks, int ntasks,
                   int* queue, int count, int* status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ ExpShared sh;
    __shared__ int s_task;
    for (;;) {
        if (threadIdx.x == 0) s_task = atomicAdd(queue, 1);
        __syncthreads();
        const int t = s_task;
        if (t >= ntasks) break;
        const BatchTask bt = tasks[t];
        if (!task_ok(bt, args, count, 1)) {
            if (threadIdx.x == 0) atomicCAS(status, 0, 0x402);
            __syncthreads();
            continue;
        }
        expand_tile_body<ST, KC, PT, SPLIT>(args[bt.inst], xs[bt.inst], ys[bt.inst], bt.tile,
                                            smem_raw, sh);
        __syncthreads();
    }
}

// ----------------------------------------------------------------- launchers
constexpr size_t kSmemCap = 227 * 1024;

template <int ST, int KC>
struct Cfg {
    using A = typename Tr<ST>::A;
    static constexpr int VEC = Tr<ST>::VEC;
    // project rows in flight per warp (several right-hand sides: the rows
    // share each slot's x values)
    static constexpr int R = KC == 1 ? 8 : KC <= 8 ? 4 : KC <= 16 ? 2 : 1;
    // expand slots per thread (one vector load each) and column split
    // (about 64 accumulator registers: PT x KC values)
    static constexpr int ACC = 64 * 4 / (int)sizeof(A);
    static constexpr int PT0 = ACC / KC < 1 ? 1 : ACC / KC;
    static constexpr int PT = PT0 < VEC ? PT0 : VEC;
    static constexpr int SPLIT = KC == 1 ? 8 : KC <= 4 ? 4 : KC <= 8 ? 2 : 1;
};

// Expand tile: a power-of-two multiple or divisor of the project tile (so a
// multiple of the leaf slots and a divisor or multiple of the group size)
// with about kExpandThreads threads: small tiles keep the tail short.
constexpr int kExpandThreads = 256;
int64_t expand_tile(const MatvecArgs& a, int PT, int SPLIT) {
    int64_t te = a.tile_p;
    while ((te / PT) * SPLIT > kExpandThreads && te % 2 == 0 && (te / 2) % PT == 0) te /= 2;
    while ((te * 2 / PT) * SPLIT <= kExpandThreads && te * 2 <= a.Np && a.Np % (te * 2) == 0)
        te *= 2;
    return te;
}

template <int ST>
int64_t expand_smem_bytes(const MatvecArgs& a, int KC, int64_t TE, int SPLIT) {
    using A = typename Tr<ST>::A;
    int64_t vals = (TE > a.G ? TE : a.G) * KC;
    for (int l = 1; l <= a.nf; ++l) {
        const int64_t nodes_t = TE >= a.lv[l].n ? TE / a.lv[l].n : 1;
        vals += nodes_t * (int64_t)a.s * a.lv[l].r * KC;
    }
    vals += (int64_t)(SPLIT - 1) * TE * KC;
    return vals * (int64_t)sizeof(A);   // plus static shared memory (< 1 KB)
}

// units (level, segment, block of R columns) of one project tile
int project_units(const MatvecArgs& a, int R) {
    int64_t units = 0;
    for (int l = 1; l <= a.nf; ++l) {
        const int64_t seg = a.lv[l].n < a.tile_p ? a.lv[l].n : a.tile_p;
        const int64_t sr = (int64_t)a.s * a.lv[l].r;
        units += (a.tile_p / seg) * ((sr + R - 1) / R);
    }
    return (int)units;
}

template <int ST>
size_t project_smem_bytes(const MatvecArgs& a, int KC, int R) {
    using A = typename Tr<ST>::A;
    return ((size_t)a.tile_p * KC * sizeof(A) + 15) / 16 * 16 +
           (size_t)project_units(a, R) * sizeof(UnitDesc);
}

template <int ST, int KC>
bool fits(const MatvecArgs& a) {
    using C = Cfg<ST, KC>;
    const int64_t te = expand_tile(a, C::PT, C::SPLIT);
    return project_smem_bytes<ST>(a, KC, C::R) + 4096 <= kSmemCap &&
           (size_t)expand_smem_bytes<ST>(a, KC, te, C::SPLIT) + 1024 <= kSmemCap &&
           te % C::PT == 0 && (te / C::PT) * C::SPLIT <= 512 && te >= C::PT;
}

// Allows a kernel the shared memory cap minus its static shared memory.
template <typename K>
cudaError_t allow_dynamic_smem(K kernel) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(kSmemCap - fa.sharedSizeBytes));
}

template <int ST, int KC>
cudaError_t run_kernel(int which, const MatvecArgs& a0, cudaStream_t st, unsigned* path) {
    using C = Cfg<ST, KC>;
    static DeviceFlags attr;
    {
        const cudaError_t e = attr.once([] {
            cudaError_t r = allow_dynamic_smem(project_kernel<ST, KC, C::R>);
            if (r == cudaSuccess) r = allow_dynamic_smem(expand_kernel<ST, KC, C::PT, C::SPLIT>);
            return r;
        });
        if (e != cudaSuccess) return e;
    }
    if (which == 0) {
        if (a0.nf == 0) return cudaSuccess;
        // one right-hand side: the streamed persistent kernel
        if (KC == 1 && a0.status) {
            const int rc = stream_project(a0, st);
            if (rc != kStreamNotEligible) {
                *path |= kPathProjectStreamed;
                return (cudaError_t)rc;
            }
        }
        *path |= kPathProjectCached;
        const int units = project_units(a0, C::R);
        const size_t psmem = project_smem_bytes<ST>(a0, KC, C::R);
        const unsigned grid = (unsigned)(a0.Np / a0.tile_p);
        project_kernel<ST, KC, C::R><<<grid, 256, psmem, st>>>(a0, units);
        count_launches(1);
        return cudaGetLastError();
    }
    // one right-hand side: the streamed persistent kernel
    if (KC == 1 && a0.status) {
        const int rc = stream_expand(a0, st);
        if (rc != kStreamNotEligible) {
            *path |= kPathExpandStreamed;
            return (cudaError_t)rc;
        }
    }
    *path |= kPathExpandCached;
    MatvecArgs a = a0;
    a.tile_e = expand_tile(a0, C::PT, C::SPLIT);
    const size_t esmem = (size_t)expand_smem_bytes<ST>(a, KC, a.tile_e, C::SPLIT);
    const unsigned egrid = (unsigned)(a.Np / a.tile_e);
    const unsigned eblock = (unsigned)((a.tile_e / C::PT) * C::SPLIT);
    expand_kernel<ST, KC, C::PT, C::SPLIT><<<egrid, eblock, esmem, st>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

template <int ST>
int launch_st(int which, const MatvecArgs& a, cudaStream_t st, unsigned* path) {
    switch (a.kc) {
        case 1: return run_kernel<ST, 1>(which, a, st, path);
        case 2: return run_kernel<ST, 2>(which, a, st, path);
        case 4: return run_kernel<ST, 4>(which, a, st, path);
        case 8: return run_kernel<ST, 8>(which, a, st, path);
        case 16: return run_kernel<ST, 16>(which, a, st, path);
        case 32: return run_kernel<ST, 32>(which, a, st, path);
        case 64:
            if constexpr (ST != ST_F64) return run_kernel<ST, 64>(which, a, st, path);
            break;
    }
    return (int)cudaErrorInvalidValue;
}

template <int ST>
int width_st(const MatvecArgs& a, int k) {
    constexpr int maxw = ST == ST_F64 ? 32 : 64;
    bool ok[7] = {fits<ST, 1>(a), fits<ST, 2>(a), fits<ST, 4>(a), fits<ST, 8>(a),
                  fits<ST, 16>(a), fits<ST, 32>(a), false};
    if constexpr (maxw == 64) ok[6] = fits<ST, 64>(a);
    int best = 0;
    for (int i = 0, w = 1; i < 7 && w <= maxw; ++i, w *= 2) {
        if (!ok[i]) break;
        best = w;
        if (w >= k) break;
    }
    return best;
}

}  // namespace

int max_pass_rhs(int store_kind) { return store_kind == ST_F64 ? 32 : 64; }

int slot_align(int store_kind) { return store_kind == ST_FP8 ? 16 : 8; }

int pass_width(const MatvecArgs& a, int k) {
    switch (a.store) {
        case ST_F64: return width_st<ST_F64>(a, k);
        case ST_F32: return width_st<ST_F32>(a, k);
        case ST_BF16: return width_st<ST_BF16>(a, k);
        case ST_BF16X2: return width_st<ST_BF16X2>(a, k);
        case ST_FP8: return width_st<ST_FP8>(a, k);
    }
    return 0;
}

int launch_kernel(int which, const MatvecArgs& a, void* stream, unsigned* path) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned dummy = 0;
    if (!path) path = &dummy;
    // several right-hand sides in a bf16-family storage: tensor cores
    if (a.k >= 2 && a.status && tc_eligible(a)) {
        *path |= which == 0 ? kPathProjectTensor : kPathExpandTensor;
        return tc_launch(which, a, a.status, stream);
    }
    switch (a.store) {
        case ST_F64: return launch_st<ST_F64>(which, a, st, path);
        case ST_F32: return launch_st<ST_F32>(which, a, st, path);
        case ST_BF16: return launch_st<ST_BF16>(which, a, st, path);
        case ST_BF16X2: return launch_st<ST_BF16X2>(which, a, st, path);
        case ST_FP8: return launch_st<ST_FP8>(which, a, st, path);
    }
    return (int)cudaErrorNotSupported;
}

// ------------------------------------------------------------ batched
namespace {

template <int ST, int KC>
int batch_setup_st(MatvecArgs& a, int which, int* units, size_t* smem) {
    using C = Cfg<ST, KC>;
    if (which == 0) {
        *units = project_units(a, C::R);
        *smem = project_smem_bytes<ST>(a, KC, C::R);
    } else {
        a.tile_e = expand_tile(a, C::PT, C::SPLIT);
        *units = (int)(a.Np / a.tile_e);
        *smem = (size_t)expand_smem_bytes<ST>(a, KC, a.tile_e, C::SPLIT);
    }
    return 0;
}

template <int ST, int KC>
int batch_launch_st(int which, const BatchLaunch& b, cudaStream_t st, bool dry) {
    using C = Cfg<ST, KC>;
    static DeviceFlags attr;
    {
        const cudaError_t e = attr.once([] {
            cudaError_t r = allow_dynamic_smem(project_batched<ST, KC, C::R>);
            if (r == cudaSuccess) r = allow_dynamic_smem(expand_batched<ST, KC, C::PT, C::SPLIT>);
            return r;
        });
        if (e != cudaSuccess) return (int)e;
    }
    int per_sm = 0, sms = 0, dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) {
        if (which == 0)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, project_batched<ST, KC, C::R>,
                                                              256, b.smem);
        else
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &per_sm, expand_batched<ST, KC, C::PT, C::SPLIT>, 256, b.smem);
    }
    if (e != cudaSuccess) return (int)e;
    if (per_sm < 1) return (int)cudaErrorInvalidConfiguration;
    if (dry) return 0;
    int grid = per_sm * sms / (b.grid_div > 1 ? b.grid_div : 1);
    if (grid < 1) grid = 1;
    if (grid > b.ntasks) grid = b.ntasks;
    if (grid < 1) return 0;
    if (which == 0)
        project_batched<ST, KC, C::R><<<grid, 256, b.smem, st>>>(b.args, b.units, b.xs, b.tasks,
                                                                 b.ntasks, b.queue, b.count, b.status);
    else
        expand_batched<ST, KC, C::PT, C::SPLIT><<<grid, 256, b.smem, st>>>(b.args, b.xs, b.ys,
                                                                           b.tasks, b.ntasks,
                                                                           b.queue, b.count, b.status);
    count_launches(1);
    return (int)cudaGetLastError();
}

template <int ST>
int batch_setup_dispatch(MatvecArgs& a, int which, int* units, size_t* smem) {
    switch (a.kc) {
        case 1: return batch_setup_st<ST, 1>(a, which, units, smem);
        case 2: return batch_setup_st<ST, 2>(a, which, units, smem);
        case 4: return batch_setup_st<ST, 4>(a, which, units, smem);
        case 8: return batch_setup_st<ST, 8>(a, which, units, smem);
        case 16: return batch_setup_st<ST, 16>(a, which, units, smem);
        case 32: return batch_setup_st<ST, 32>(a, which, units, smem);
        case 64:
            if constexpr (ST != ST_F64) return batch_setup_st<ST, 64>(a, which, units, smem);
            break;
    }
    return (int)cudaErrorInvalidValue;
}

template <int ST>
int batch_launch_dispatch(int which, int kc, const BatchLaunch& b, cudaStream_t st, bool dry) {
    switch (kc) {
        case 1: return batch_launch_st<ST, 1>(which, b, st, dry);
        case 2: return batch_launch_st<ST, 2>(which, b, st, dry);
        case 4: return batch_launch_st<ST, 4>(which, b, st, dry);
        case 8: return batch_launch_st<ST, 8>(which, b, st, dry);
        case 16: return batch_launch_st<ST, 16>(which, b, st, dry);
        case 32: return batch_launch_st<ST, 32>(which, b, st, dry);
        case 64:
            if constexpr (ST != ST_F64) return batch_launch_st<ST, 64>(which, b, st, dry);
            break;
    }
    return (int)cudaErrorInvalidValue;
}

}  // namespace

int batch_setup(MatvecArgs& a, int which, int* units, size_t* smem) {
    switch (a.store) {
        case ST_F64: return batch_setup_dispatch<ST_F64>(a, which, units, smem);
        case ST_F32: return batch_setup_dispatch<ST_F32>(a, which, units, smem);
        case ST_BF16: return batch_setup_dispatch<ST_BF16>(a, which, units, smem);
        case ST_BF16X2: return batch_setup_dispatch<ST_BF16X2>(a, which, units, smem);
        case ST_FP8: return batch_setup_dispatch<ST_FP8>(a, which, units, smem);
    }
    return (int)cudaErrorNotSupported;
}

int batch_launch(int which, int store, int kc, const BatchLaunch& b, void* stream, int dry) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (store) {
        case ST_F64: return batch_launch_dispatch<ST_F64>(which, kc, b, st, dry != 0);
        case ST_F32: return batch_launch_dispatch<ST_F32>(which, kc, b, st, dry != 0);
        case ST_BF16: return batch_launch_dispatch<ST_BF16>(which, kc, b, st, dry != 0);
        case ST_BF16X2: return batch_launch_dispatch<ST_BF16X2>(which, kc, b, st, dry != 0);
        case ST_FP8: return batch_launch_dispatch<ST_FP8>(which, kc, b, st, dry != 0);
    }
    return (int)cudaErrorNotSupported;
}

// ------------------------------------------------------- static scratch
// Partial-sum scratch of hmat_matvec_noalloc: a fixed array in the
// library's device image, present on every GPU that loads the library until
// the process exits.  In host code `g_static_scratch` only names the symbol;
// its device address comes from cudaGetSymbolAddress, taken once per device
// (with that device current) and cached.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

int static_scratch_address(int device, void** ptr) {
    static std::mutex mu;
    static void* cached[128] = {};
    if (device < 0 || device >= 128) return (int)cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!cached[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return (int)e;
        cached[device] = p;
    }
    *ptr = cached[device];
    return 0;
}

}  // namespace hm
