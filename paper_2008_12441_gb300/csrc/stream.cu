// Persistent project kernel (Steps 1-2, eq. (prod-vx)) for one right-hand
// side: the memory-bound form of the product, streamed through a
// shared-memory ring by the tensor-memory-access (TMA) engine.
//
// CTA c owns the project tiles [c R, c R + R).  Warp 8 (producer) copies
// the x values of each tile into a ring of eight tile buffers, six tiles
// ahead, and per stage loads one box of V: tile_p slots x RB_l consecutive
// columns of one level's node (at most 32 columns and 24 KB), through that
// level's 2-D tensor map (row = node * s r_l + column), completing on an
// mbarrier with a transaction count; a tile's stages are issued after its
// x has landed.  Warps 0-7 (consumers) own one ring slot each and so take
// every eighth stage: each lane reads 16-byte vectors of the stage's rows
// and the matching x values from shared memory, accumulates every row of
// the stage in increasing slot order, and the warp adds its lanes with a
// reduce-scatter butterfly (31 shuffles for 32 rows); the scaled sum is a
// node sum, or a per-tile partial for a node longer than the tile.
// Step 2 runs at the end of the same kernel: each CTA adds its own tiles'
// partials of a node in tile order, and the CTA whose arrival completes
// the node adds the CTAs' sums in CTA order (a fixed order: results are
// bitwise reproducible run to run on one device).  Stages and x buffers are
// released through mbarriers; only the Step-2 tail synchronises the
// consumer warps.
//
// Every wait is bounded: on timeout the thread sets the status word, skips
// its later waits, and the kernel runs to its end (the producer then waits,
// again bounded, for the copies it issued).
#include <cuda_runtime.h>

#include <cstdint>
#include <utility>

#include "hm_device.h"
#include "hm_once.h"
#include "hm_elem.cuh"

namespace hm {
namespace {

__device__ __forceinline__ unsigned s_addr(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mb_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_addr(bar)), "r"(count));
}
__device__ __forceinline__ void mb_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_addr(bar)));
}
__device__ __forceinline__ void mb_arrive_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_addr(bar)),
                 "r"(bytes));
}
// arrive once this thread's earlier cp.async copies have landed
__device__ __forceinline__ void mb_arrive_cp_async(uint64_t* bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(s_addr(bar)));
}
__device__ __forceinline__ bool mb_try(uint64_t* bar, unsigned parity, unsigned suspend_ns) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(s_addr(bar)), "r"(parity), "r"(suspend_ns));
    return done != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait for the completion of phase `parity` (the thread sleeps in
// try_wait until the phase completes or the suspend hint runs out); false
// once `limit_ns` (two seconds by default) have passed on the global timer.
__device__ __forceinline__ bool mb_wait(uint64_t* bar, unsigned parity,
                                        uint64_t limit_ns = 2000000000ull) {
    if (mb_try(bar, parity, 0)) return true;
    const uint64_t t0 = global_ns();
    for (unsigned it = 0; it < (1u << 30); ++it) {
        if (mb_try(bar, parity, 100000)) return true;
        if ((it & 15) == 15 && global_ns() - t0 > limit_ns) return false;
    }
    return false;
}
// Status word: the first wait that gave up records its site code.
__device__ __forceinline__ void report_status(int* status, int code) { atomicCAS(status, 0, code); }
// global -> shared bulk copy of `bytes` (multiple of 16, both addresses
// 16-byte aligned), completing on `bar`
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            s_addr(dst)),
        "l"(src), "r"(bytes), "r"(s_addr(bar))
        : "memory");
}
// Programmatic dependent launch: let the next kernel of the stream start
// its CTAs early / wait until the previous kernel of the stream has
// completed and its memory is visible (a no-op without such a dependency).
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch with the programmatic-stream-serialization attribute: the kernel
// may start while the previous kernel of the stream is finishing and must
// call pdl_wait() before it reads what that kernel wrote.
template <typename... P, typename... Args>
cudaError_t launch_pdl(bool pdl, void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args&&... args) {
    if (!pdl) {
        kernel<<<grid, block, smem, st>>>(std::forward<Args>(args)...);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// 2-D tensor-map box at (x, y) -> shared memory, completing on `bar`
__device__ __forceinline__ void tma_load_2d(void* dst, const void* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
        "%3}], [%4];" ::"r"(s_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(s_addr(bar))
        : "memory");
}
// one element of 4 or 8 bytes, zero-filled when !valid
template <int B>
__device__ __forceinline__ void cp_async_elem(void* dst, const void* src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(s_addr(dst)), "l"(src), "n"(B),
                 "r"(valid ? B : 0));
}

// Sums of the rows of a stage over groups of LPR lanes (LPR a power of two
// dividing 32): each lane holds M partial sums (M a power of two, M <= LPR),
// one per row it took part in.  The first log2(M) butterfly steps split the
// rows between the two halves of the lanes exchanging (the half with lane
// bit `off` clear keeps the lower rows), the rest are plain butterfly steps
// inside the group.  Row m's total ends on the lanes of the group with
// (lane % LPR) / (LPR / M) == m.
template <typename A, int M, int LPR>
__device__ __forceinline__ A group_sum_rows(A (&v)[M], int lane) {
    int off = LPR / 2;
#pragma unroll
    for (int Mc = M; Mc > 1; Mc >>= 1, off >>= 1) {
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int m = 0; m < Mc / 2; ++m) {
            const A send = upper ? v[m] : v[m + Mc / 2];
            const A keep = upper ? v[m + Mc / 2] : v[m];
            v[m] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    A r = v[0];
#pragma unroll
    for (; off > 0; off >>= 1) r += __shfl_xor_sync(0xffffffffu, r, off);
    return r;
}

// Persistent project kernel.  Warps 0..kProjWarps-1 consume, warp kProjWarps
// produces; ring slot s belongs to consumer warp s (kProjStages ==
// kProjWarps), so every slot's phases are waited on by one warp in order.
constexpr int kProjWarps = 8;
constexpr int kProjStages = kProjWarps;
constexpr int kProjThreads = 32 * (kProjWarps + 1);
constexpr int kProjXBuf = 8;                     // x buffers (one tile each)
constexpr int kProjXAhead = kProjXBuf - 2;       // tiles of x loaded ahead of the stages
constexpr size_t kProjStageBytes = 24 * 1024;    // bytes of one stage (all parts)
constexpr size_t kProjSmemMax = 212 * 1024;
constexpr int kLastCap = 256;                    // nodes a CTA completes, listed for Step 2
// Stages of one tile (the same for every tile): per level, s r_l / RB_l
// boxes of RB_l consecutive columns.
constexpr int kMaxStageTab = 2048;

// stage table entry: level (or expand segment) in bits 0-4, box rows in
// bits 5-11, first column in bits 12-31
__device__ __forceinline__ unsigned pack_stage(int l, int col0, int rows) {
    return (unsigned)l | ((unsigned)rows << 5) | ((unsigned)col0 << 12);
}
__device__ __forceinline__ void unpack_stage(unsigned info, int& l, int& col0, int& rows) {
    l = (int)(info & 0x1fu);
    rows = (int)((info >> 5) & 0x7fu);
    col0 = (int)(info >> 12);
}

// Dot products of the `rows` rows of one stage (rows of `rowb` bytes, CH
// 16-byte chunks each; split storage: low parts `part_bytes` further on)
// with the tile's x values xt.  Lane group grp = lane / LPR takes rows grp,
// grp + 32/LPR, ...; lane sub = lane % LPR chunks sub, sub + LPR, ... in
// increasing order.  Returns row slot j's sum on the lanes of the group
// with sub / (LPR / MJ) == j (row grp + (32/LPR) j).
template <int ST, int LPR, int MR>
__device__ __forceinline__ typename Tr<ST>::A stage_rows_dot(const unsigned char* stg, size_t part_bytes,
                                                            unsigned rowb, int CH,
                                                            const typename Tr<ST>::A* xt, int rows,
                                                            int lane) {
    using A = typename Tr<ST>::A;
    constexpr int VEC = Tr<ST>::VEC;
    constexpr int RPP = 32 / LPR;
    constexpr int MJ = MR / RPP;
    static_assert(MJ >= 1 && MJ <= LPR, "rows per lane");
    const int sub = lane % LPR, grp = lane / LPR;
    A acc[MJ];
#pragma unroll
    for (int j = 0; j < MJ; ++j) acc[j] = A(0);
    for (int c = sub; c < CH; c += LPR) {
        A xv[VEC];
#pragma unroll
        for (int w = 0; w < (int)(VEC * sizeof(A) / 16); ++w) {
            union { float4 v; A e[16 / sizeof(A)]; } cv;
            cv.v = reinterpret_cast<const float4*>(xt + c * VEC)[w];
#pragma unroll
            for (int e = 0; e < (int)(16 / sizeof(A)); ++e) xv[w * (16 / sizeof(A)) + e] = cv.e[e];
        }
#pragma unroll
        for (int j = 0; j < MJ; ++j) {
            const int r = grp + RPP * j;
            if (r < rows) {
                const uint4 hi = reinterpret_cast<const uint4*>(stg + (size_t)r * rowb)[c];
                uint4 lo = hi;
                if constexpr (ST == ST_BF16X2)
                    lo = reinterpret_cast<const uint4*>(stg + part_bytes + (size_t)r * rowb)[c];
                A one[1] = {acc[j]};
                DotStep<ST, 1, 0>::go(hi, lo, xv, one);
                acc[j] = one[0];
            }
        }
    }
    return group_sum_rows<A, MJ, LPR>(acc, lane);
}

// Destination in T of column `col` of level l for tile t: the node sum when
// the node is one tile, else the tile's partial sum.
__device__ __forceinline__ int64_t proj_dest(const DevLevel& L, int sr, int64_t t, int64_t node, int col) {
    return L.nsub > 1 ? L.part_off + t * sr + col : L.fin_off + node * sr + col;
}

template <int ST, int LPR>
__global__ void __launch_bounds__(kProjThreads, 1)
    project_stream_kernel(const MatvecArgs a, int ntile, int R, int RB, int Q) {
    using Trs = Tr<ST>;
    using A = typename Trs::A;
    using E = typename Trs::E;
    constexpr bool SPLIT = ST == ST_BF16X2;
    constexpr int PARTS = SPLIT ? 2 : 1;
    constexpr int S = kProjStages;
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ uint64_t full[S], empty[S], xfull[kProjXBuf], xempty[kProjXBuf];
    __shared__ int s_last_l[kLastCap], s_last_j[kLastCap], s_nlast;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tile = (int)a.tile_p;
    const unsigned rowb = (unsigned)tile * sizeof(E);     // bytes of one row (one part)
    const int CH = (int)(rowb / 16);                      // 16-byte chunks of a row
    // a stage: PARTS boxes of up to RB rows, each starting on 128 bytes
    const size_t part_bytes = ((size_t)RB * rowb + 127) / 128 * 128;
    const size_t stage_bytes = part_bytes * PARTS;
    // dynamic shared memory: ring [S] | x [kProjXBuf][tile] | stage table [Q]
    A* xs = reinterpret_cast<A*>(sm + (size_t)S * stage_bytes);
    unsigned* stagetab = reinterpret_cast<unsigned*>(xs + (size_t)kProjXBuf * tile);
    const int t_begin = blockIdx.x * R;
    const int t_end = min(t_begin + R, ntile);
    const int ntl = max(t_end - t_begin, 0);
    pdl_launch_dependents();   // the expand kernel may take SMs as this grid drains

    if (tid == 0) {
        for (int q = 0; q < S; ++q) {
            mb_init(&full[q], 1);
            mb_init(&empty[q], 1);
        }
        for (int q = 0; q < kProjXBuf; ++q) {
            mb_init(&xfull[q], 32);      // 32 lanes' x copies (or bulk copy + 31 arrivals)
            mb_init(&xempty[q], Q);      // one arrival per stage of the tile
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
        int q = 0;
        for (int l = 1; l <= a.nf; ++l) {
            const int sr = a.s * a.lv[l].r, rb = a.lv[l].tma_rb;
            for (int c = 0; rb > 0 && c < sr; c += rb) stagetab[q++] = pack_stage(l, c, rb);
        }
    }
    __syncthreads();

    if (warp == kProjWarps) {
        // ------------------------------------------------------ producer
        int fail = 0;                 // site code of the first wait that gave up
        const bool xbulk = a.map == nullptr && a.ldx == 1 &&
                           (reinterpret_cast<uintptr_t>(a.x) & 15) == 0;
        const A* __restrict__ x = static_cast<const A*>(a.x);
        const unsigned char* maps = static_cast<const unsigned char*>(a.tmaps);
        // x of tile u into buffer u % kProjXBuf, once the tile that used the
        // buffer before has been consumed
        auto load_x = [&](int u) {
            const int xb = u % kProjXBuf;
            if (!fail && u >= kProjXBuf &&
                !mb_wait(&xempty[xb], (unsigned)((u / kProjXBuf) - 1) & 1u))
                fail = 0x101;
            const int64_t p0 = (int64_t)(t_begin + u) * tile;
            A* xd = xs + (size_t)xb * tile;
            if (xbulk) {
                if (lane == 0) {
                    mb_arrive_tx(&xfull[xb], (unsigned)(tile * sizeof(A)));
                    bulk_copy(xd, x + p0, (unsigned)(tile * sizeof(A)), &xfull[xb]);
                } else {
                    mb_arrive(&xfull[xb]);
                }
            } else {
                for (int e = lane; e < tile; e += 32) {
                    const int64_t row = a.map ? a.map[p0 + e] : p0 + e;
                    const bool v = row >= 0;
                    cp_async_elem<(int)sizeof(A)>(xd + e, v ? x + row * a.ldx : x, v);
                }
                mb_arrive_cp_async(&xfull[xb]);
            }
        };
        for (int u = 0; u < min(kProjXAhead, ntl); ++u) load_x(u);
        for (int u = 0; u < ntl; ++u) {
            if (u + kProjXAhead < ntl) load_x(u + kProjXAhead);
            const int xb = u % kProjXBuf;
            // the stages of tile u are issued once its x has landed, so a
            // consumer that sees a stage full also sees the tile's x
            if (!fail && !mb_wait(&xfull[xb], (unsigned)(u / kProjXBuf) & 1u)) fail = 0x102;
            const int64_t p0 = (int64_t)(t_begin + u) * tile;
            for (int q = 0; q < Q; ++q) {
                const int g = u * Q + q, s = g % S;
                if (!fail && g >= S && !mb_wait(&empty[s], (unsigned)((g / S) - 1) & 1u)) fail = 0x103;
                if (lane == 0) {
                    const unsigned info = stagetab[q];
                    int l, col0, rows;
                    unpack_stage(info, l, col0, rows);
                    const DevLevel& L = a.lv[l];
                    const int64_t node = p0 / L.n;
                    const int inoff = (int)(p0 - node * L.n);
                    const int y0 = (int)(node * a.s * L.r + col0);
                    unsigned char* stg = sm + (size_t)s * stage_bytes;
                    mb_arrive_tx(&full[s], (unsigned)rows * rowb * PARTS);
                    tma_load_2d(stg, maps + (size_t)l * kTensorMapBytes, inoff, y0, &full[s]);
                    if constexpr (SPLIT)
                        tma_load_2d(stg + part_bytes, maps + ((size_t)(kMaxLevels + 1) + l) * kTensorMapBytes,
                                    inoff, y0, &full[s]);
                }
                __syncwarp();
            }
        }
        // wait (bounded) for the last use of every stage and x buffer, so
        // that no copy into this CTA's shared memory is still in flight
        if (lane == 0) {
            const int total = ntl * Q;
            for (int g = max(total - S, 0); g < total; ++g)
                if (!mb_wait(&full[g % S], (unsigned)(g / S) & 1u) && !fail) fail = 0x104;
            for (int u = max(ntl - kProjXBuf, 0); u < ntl; ++u)
                if (!mb_wait(&xfull[u % kProjXBuf], (unsigned)(u / kProjXBuf) & 1u) && !fail) fail = 0x105;
        }
        if (fail) report_status(a.status, fail);
        return;
    }

    // ---------------------------------------------------------- consumers
    // warp w takes the stages g = w, w + S, ... (ring slot w)
    int fail = 0;
    A* __restrict__ T = static_cast<A*>(a.T);
    const int total = ntl * Q;
    for (int g = warp; g < total; g += S) {
        const int u = g / Q, q = g - u * Q;
        if (!fail && !mb_wait(&full[warp], (unsigned)(g / S) & 1u)) fail = 0x106;
        const unsigned info = stagetab[q];
        int l, col0, rows;
        unpack_stage(info, l, col0, rows);
        const unsigned char* stg = sm + (size_t)warp * stage_bytes;
        const A* xt = xs + (size_t)(u % kProjXBuf) * tile;
        A sum;
        int MJ;
        if (rows <= 8) {
            sum = stage_rows_dot<ST, LPR, 8>(stg, part_bytes, rowb, CH, xt, rows, lane);
            MJ = 8 * LPR / 32;
        } else if (rows <= 16) {
            sum = stage_rows_dot<ST, LPR, 16>(stg, part_bytes, rowb, CH, xt, rows, lane);
            MJ = 16 * LPR / 32;
        } else {
            sum = stage_rows_dot<ST, LPR, 32>(stg, part_bytes, rowb, CH, xt, rows, lane);
            MJ = 32 * LPR / 32;
        }
        // the stage and the tile's x are no longer read
        __syncwarp();
        if (lane == 0) {
            mb_arrive(&empty[warp]);
            mb_arrive(&xempty[u % kProjXBuf]);
        }
        const int sub = lane % LPR, step = LPR / MJ;
        const int r = lane / LPR + (32 / LPR) * (sub / step);
        if (sub % step == 0 && r < rows) {
            const DevLevel& L = a.lv[l];
            const int sr = a.s * L.r;
            const int64_t t = t_begin + u;
            const int64_t node = t * tile / L.n;
            const int col = col0 + r;
            const A sc = (A)factor_scale<ST>(a.scV, L, a.s, node, col);
            T[proj_dest(L, sr, t, node, col)] = sum * sc;
        }
    }

    // ------------------------------------------------ Step 2 (fixed order)
    // Nodes longer than a tile, all levels at once: (A) this CTA adds its
    // own tiles' partials of each node it touches (tile order) into the slot
    // of its first such tile; (B) it adds its tile count to the node's
    // arrival counter, and the CTA whose arrival completes the count lists
    // the node and zeroes the counter for the next product; (C) it adds the
    // CTAs' sums of every listed node in CTA order into the node sum.
    constexpr int CT = kProjWarps * 32;
    const int ctid = tid;
    auto consumers_sync = [] { asm volatile("bar.sync 1, %0;" ::"n"(kProjWarps * 32) : "memory"); };
    // node sum of node j of level l from the CTAs' sums, columns col0, col0 + step, ...
    auto node_sum = [&](int l, int j, int col0, int step) {
        const DevLevel& L = a.lv[l];
        const int sr = a.s * L.r, nsub = L.nsub;
        const int c0 = j * nsub / R, c1 = ((j + 1) * nsub - 1) / R;
        for (int col = col0; col < sr; col += step) {
            A v = A(0);
            for (int c = c0; c <= c1; ++c) {
                const int tf = max(c * R, j * nsub);
                v += __ldcg(T + L.part_off + (int64_t)tf * sr + col);
            }
            T[L.fin_off + (int64_t)j * sr + col] = v;
        }
    };
    if (ctid == 0) s_nlast = 0;
    __threadfence();
    consumers_sync();
    int* cnt = a.cnt;
    // (A)
    for (int l = 1; l <= a.nf && ntl > 0; ++l) {
        const DevLevel& L = a.lv[l];
        if (L.nsub <= 1 || L.r == 0) continue;
        const int sr = a.s * L.r, nsub = L.nsub;
        const int j0 = t_begin / nsub, j1 = (t_end - 1) / nsub;
        const int items = (j1 - j0 + 1) * sr;
        for (int it = ctid; it < items; it += CT) {
            const int j = j0 + it / sr, col = it % sr;
            const int ta = max(t_begin, j * nsub), tb = min(t_end, (j + 1) * nsub);
            A* p = T + L.part_off + (int64_t)ta * sr + col;
            A v = __ldcg(p);
            for (int t = ta + 1; t < tb; ++t) v += __ldcg(T + L.part_off + (int64_t)t * sr + col);
            *p = v;
        }
    }
    __threadfence();
    consumers_sync();
    // (B)
    for (int l = 1; l <= a.nf && ntl > 0; ++l) {
        const DevLevel& L = a.lv[l];
        if (L.nsub <= 1 || L.r == 0) continue;
        const int nsub = L.nsub;
        const int j0 = t_begin / nsub, j1 = (t_end - 1) / nsub;
        for (int j = j0 + ctid; j <= j1; j += CT) {
            const int ta = max(t_begin, j * nsub), tb = min(t_end, (j + 1) * nsub);
            int* c = cnt + L.cnt_off + j;
            if (atomicAdd(c, tb - ta) + (tb - ta) == nsub) {
                __threadfence();
                *c = 0;
                const int e = atomicAdd(&s_nlast, 1);
                if (e < kLastCap) {
                    s_last_l[e] = l;
                    s_last_j[e] = j;
                } else {
                    node_sum(l, j, 0, 1);       // list full: this thread alone
                }
            }
        }
    }
    consumers_sync();
    // (C) items (listed node, column), flattened
    const int nl = min(s_nlast, kLastCap);
    int total_items = 0;
    for (int e = 0; e < nl; ++e) total_items += a.s * a.lv[s_last_l[e]].r;
    for (int it = ctid; it < total_items; it += CT) {
        int e = 0, off = it;
        while (off >= a.s * a.lv[s_last_l[e]].r) {
            off -= a.s * a.lv[s_last_l[e]].r;
            ++e;
        }
        node_sum(s_last_l[e], s_last_j[e], off, 1 << 30);
    }
    if (fail) report_status(a.status, fail);
}

template <int ST, int LPR>
int launch_project_stream(const MatvecArgs& a, cudaStream_t st, int grid, size_t smem, int ntile, int R,
                          int RB, int Q) {
    static DeviceFlags attr;
    const cudaError_t e = attr.once([] {
        return cudaFuncSetAttribute(project_stream_kernel<ST, LPR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kProjSmemMax);
    });
    if (e != cudaSuccess) return (int)e;
    project_stream_kernel<ST, LPR><<<grid, kProjThreads, smem, st>>>(a, ntile, R, RB, Q);
    count_launches(1);
    return (int)cudaGetLastError();
}

template <int ST>
int stream_run(const MatvecArgs& a, cudaStream_t st) {
    using Trs = Tr<ST>;
    using E = typename Trs::E;
    using A = typename Trs::A;
    const int parts = ST == ST_BF16X2 ? 2 : 1;
    const int64_t tile = a.tile_p;
    const int RB = stream_stage_rows(tile, (int)sizeof(E), parts);
    const int64_t CH = tile * (int64_t)sizeof(E) / 16;
    if (CH < 16 || tile * (int64_t)sizeof(E) % 16 != 0 || a.cnt == nullptr) return kStreamNotEligible;
    int64_t Q = 0;
    for (int l = 1; l <= a.nf; ++l) {
        const DevLevel& L = a.lv[l];
        if (L.r == 0) continue;
        const int sr = a.s * L.r;
        if (L.n < tile || L.tma_rb < 1 || L.tma_rb > RB || sr % L.tma_rb != 0 || sr >= (1 << 20))
            return kStreamNotEligible;
        Q += sr / L.tma_rb;
    }
    if (Q == 0 || Q > kMaxStageTab) return kStreamNotEligible;
    const size_t rowb = (size_t)tile * sizeof(E);
    const size_t stage = ((size_t)RB * rowb + 127) / 128 * 128 * parts;
    const size_t smem = (size_t)kProjStages * stage + (size_t)kProjXBuf * tile * sizeof(A) +
                        (size_t)Q * sizeof(unsigned);
    if (stage > kProjStageBytes + 128 * parts || smem > kProjSmemMax) return kStreamNotEligible;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
    const int ntile = (int)(a.Np / a.tile_p);
    const int R = (ntile + sms - 1) / sms;
    const int grid = (ntile + R - 1) / R;
    return CH >= 32 ? launch_project_stream<ST, 32>(a, st, grid, smem, ntile, R, RB, (int)Q)
                    : launch_project_stream<ST, 16>(a, st, grid, smem, ntile, R, RB, (int)Q);
}

// ------------------------------------------------------------------ expand
// Persistent expand kernel (Steps 3-5, eqs. (prod-yuz), (prod-ydz)) for one
// right-hand side.  CTA c owns the expand tiles (kExpandStreamTile slots)
// [c R, c R + R).  The columns of a tile are the G columns of its
// near-field group's dense block, then the s r_l columns of U^l of its
// target node per level; each is a run of the tile's slots, so the
// product is y_tile = sum over columns of (column) x (weight).
//   warp 8 (producer): per stage one box of D or of one level's U (tile
//     slots x RB columns) through the tensor maps, ring of S stages;
//   warp 9 (weights): per tile the column weights -- x of the group (times
//     the dense scale) and, per level, the sums t_{i<-j} of the target's
//     siblings at the slot of the target (Steps 3-4; times the U scales) --
//     into a double buffer; then, one tile behind, the sum of the four
//     groups' partial outputs in group order, stored to y;
//   warps 0-7 (consumers): four groups of two warps; stage g (counted over
//     the CTA's tiles) belongs to group g mod 4 and the ring depth is a
//     multiple of four, so every slot is used by one group only; a group's
//     64 threads accumulate 4 slots each
//     over the stage's columns in order.
// Compensated summation: a stage's columns (at most 64, one near-field
// block or one level's U) are added plainly; the stage sums are added to a
// thread's running sum with TwoSum and their rounding errors kept apart,
// the four groups' sums likewise in group order, and the errors are added
// once at the end (the level sums are compensated).
// The summation order is fixed, so results are bitwise reproducible.  The
// kernel is launched as a programmatic dependent of the project side: only
// the weights warp reads what those kernels wrote, after pdl_wait().
// TwoSum (Knuth): s + e == a + b exactly, s = fl(a + b).
template <typename A>
__device__ __forceinline__ void two_sum(A a, A b, A& s, A& e) {
    s = a + b;
    const A bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}

// Coordinates of node i of level l on the ideal-domain boxes (bit b of
// coordinate c is bit d b + c of i), and back.
__device__ __forceinline__ void dnode_coords(int64_t i, int d, int l, int* c) {
    c[0] = c[1] = c[2] = 0;
    for (int b = 0; b < l; ++b)
        for (int k = 0; k < d; ++k) c[k] |= (int)((i >> (d * b + k)) & 1) << b;
}
__device__ __forceinline__ int64_t dnode_index(const int* c, int d, int l) {
    int64_t i = 0;
    for (int b = 0; b < l; ++b)
        for (int k = 0; k < d; ++k) i |= (int64_t)((c[k] >> b) & 1) << (d * b + k);
    return i;
}
// Standard admissibility: the group at near-field slot k of group g0 (the
// 3^d touching boxes, offsets in increasing (e_{d-1}, ..., e_0) order) of
// level lv, or -1 outside the domain.
__device__ __forceinline__ int64_t near_group(int64_t g0, int k, int d, int lv) {
    int c[3];
    dnode_coords(g0, d, lv, c);
    const int side = 1 << lv;
    for (int a = 0; a < d; ++a) {
        c[a] += k % 3 - 1;
        k /= 3;
        if (c[a] < 0 || c[a] >= side) return -1;
    }
    return dnode_index(c, d, lv);
}

constexpr int kMaxStages = 16;
constexpr int kExpGroups = 4;
constexpr int kExpConsumerWarps = 2 * kExpGroups;
constexpr int kExpThreads = 32 * (kExpConsumerWarps + 2);
constexpr int kExpPT = kExpandStreamTile / 64;   // slots per consumer thread
constexpr size_t kExpSmemMax = 215 * 1024;

__device__ __forceinline__ unsigned pack_exp_stage(int seg, int col0, int rows) { return pack_stage(seg, col0, rows); }

// kExpPT consecutive decoded elements of storage kind K from shared memory
template <int K, typename A>
__device__ __forceinline__ void lds_dec(const unsigned char* p, A (&o)[kExpPT]) {
    using TK = Tr<K>;
    typename TK::E e[kExpPT];
    constexpr int B = kExpPT * (int)sizeof(typename TK::E);
    if constexpr (B == 32) {
        const uint4 u0 = reinterpret_cast<const uint4*>(p)[0], u1 = reinterpret_cast<const uint4*>(p)[1];
        memcpy(e, &u0, 16);
        memcpy(reinterpret_cast<char*>(e) + 16, &u1, 16);
    } else if constexpr (B == 16) {
        const uint4 u = *reinterpret_cast<const uint4*>(p);
        memcpy(e, &u, 16);
    } else if constexpr (B == 8) {
        const uint2 u = *reinterpret_cast<const uint2*>(p);
        memcpy(e, &u, 8);
    } else {
        const unsigned u = *reinterpret_cast<const unsigned*>(p);
        memcpy(e, &u, 4);
    }
#pragma unroll
    for (int v = 0; v < kExpPT; ++v) o[v] = (A)TK::dec(e[v]);
}

template <int ST>
__global__ void __launch_bounds__(kExpThreads, 1)
    expand_stream_kernel(const MatvecArgs a, int ntile, int R, int S, int Q, int K) {
    using A = typename Tr<ST>::A;
    using E = typename Tr<ST>::E;
    constexpr int DST = DenseKind<ST>::value;
    using ED = typename Tr<DST>::E;
    constexpr bool SPLIT = ST == ST_BF16X2;
    constexpr int PARTS = SPLIT ? 2 : 1;
    constexpr int TE = kExpandStreamTile;
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ uint64_t full[kMaxStages], empty[kMaxStages];
    __shared__ uint64_t wfull[2], wempty[2], rfull[2], rempty[2];
    __shared__ int woff[kMaxLevels + 1];     // first weight of a segment (0: near field)

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int G = (int)a.G;
    const int NCOL = a.nnb * G;          // near-field columns of a group (nnb source groups)
    const int nc = a.s + 1;
    // a stage: PARTS boxes of up to 16 KB / PARTS, each on 128 bytes
    const size_t part_bytes = (16 * 1024) / PARTS;
    const size_t stage_bytes = part_bytes * PARTS;
    // dynamic shared memory: ring | weights [2][K] | partials [2][groups][sum, error][TE] | stage table [Q]
    A* wbuf = reinterpret_cast<A*>(sm + (size_t)S * stage_bytes);
    A* red = wbuf + 2 * K;
    unsigned* stagetab = reinterpret_cast<unsigned*>(red + 2 * kExpGroups * 2 * TE);
    const int t_begin = blockIdx.x * R;
    const int t_end = min(t_begin + R, ntile);
    const int ntl = max(t_end - t_begin, 0);

    if (tid == 0) {
        for (int q = 0; q < S; ++q) {
            mb_init(&full[q], 1);
            mb_init(&empty[q], 2);
        }
        for (int q = 0; q < 2; ++q) {
            mb_init(&wfull[q], 32);
            mb_init(&wempty[q], kExpConsumerWarps);
            mb_init(&rfull[q], kExpConsumerWarps);
            mb_init(&rempty[q], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
        int q = 0, w = 0;
        const int rbd = a.tma_rb_d;
        woff[0] = 0;
        for (int c = 0; c < NCOL; c += rbd) stagetab[q++] = pack_exp_stage(0, c, rbd);
        w = NCOL;
        for (int l = a.nf; l >= 1; --l) {
            const int sr = a.s * a.lv[l].r, rb = a.lv[l].tma_rb_u;
            woff[l] = w;
            w += sr;
            for (int c = 0; rb > 0 && c < sr; c += rb) stagetab[q++] = pack_exp_stage(l, c, rb);
        }
    }
    __syncthreads();

    if (warp == kExpConsumerWarps) {
        // ------------------------------------------------------ producer
        int fail = 0;                 // site code of the first wait that gave up
        if (lane == 0) {
            const unsigned char* maps = static_cast<const unsigned char*>(a.tmaps_u);
            for (int u = 0; u < ntl; ++u) {
                const int64_t e0 = (int64_t)(t_begin + u) * TE;
                for (int q = 0; q < Q; ++q) {
                    const int g = u * Q + q, s = g % S;
                    if (!fail && g >= S && !mb_wait(&empty[s], (unsigned)((g / S) - 1) & 1u)) fail = 0x201;
                    const unsigned info = stagetab[q];
                    int seg, col0, rows;
                    unpack_stage(info, seg, col0, rows);
                    int x, y;
                    unsigned bytes;
                    if (seg == 0) {
                        const int64_t g0 = e0 / G;
                        x = (int)(e0 - g0 * G);
                        y = (int)(g0 * NCOL + col0);
                        bytes = (unsigned)(rows * TE * sizeof(ED));
                    } else {
                        const DevLevel& L = a.lv[seg];
                        const int64_t i = e0 / L.n;
                        x = (int)(e0 - i * L.n);
                        y = (int)(i * a.s * L.r + col0);
                        bytes = (unsigned)(rows * TE * sizeof(E));
                    }
                    unsigned char* stg = sm + (size_t)s * stage_bytes;
                    mb_arrive_tx(&full[s], bytes * PARTS);
                    tma_load_2d(stg, maps + ((size_t)2 * (kMaxLevels + 1) + seg) * kTensorMapBytes, x, y, &full[s]);
                    if constexpr (SPLIT)
                        tma_load_2d(stg + part_bytes, maps + ((size_t)3 * (kMaxLevels + 1) + seg) * kTensorMapBytes,
                                    x, y, &full[s]);
                }
            }
            const int total = ntl * Q;
            for (int g = max(total - S, 0); g < total; ++g)
                if (!mb_wait(&full[g % S], (unsigned)(g / S) & 1u) && !fail) fail = 0x202;
        }
        if (fail) report_status(a.status, fail);
    } else if (warp == kExpConsumerWarps + 1) {
        // ------------------------------------------------------ weights, output
        int fail = 0;                 // site code of the first wait that gave up
        const A* __restrict__ x = static_cast<const A*>(a.x);
        const A* __restrict__ T = static_cast<const A*>(a.T);
        A* __restrict__ y = static_cast<A*>(a.y);
        auto combine = [&](int u) {
            // partial outputs of tile u -> y
            const int xb = u & 1;
            if (!fail && !mb_wait(&rfull[xb], (unsigned)(u >> 1) & 1u)) fail = 0x203;
            const int64_t e0 = (int64_t)(t_begin + u) * TE;
            const A* rp = red + (size_t)xb * kExpGroups * 2 * TE;
            for (int p = lane; p < TE; p += 32) {
                A v = rp[p], c = rp[TE + p];
#pragma unroll
                for (int gq = 1; gq < kExpGroups; ++gq) {
                    A e;
                    two_sum(v, rp[gq * 2 * TE + p], v, e);
                    c += e + rp[gq * 2 * TE + TE + p];
                }
                v += c;
                const int64_t slot = e0 + p;
                const int64_t dst = a.map ? a.map[slot] : slot;
                if (dst >= 0) y[dst * a.ldy] = v;
            }
            __syncwarp();
            if (lane == 0) mb_arrive(&rempty[xb]);
        };
        pdl_wait();                // node sums of the project / Step-2 kernels
        for (int u = 0; u < ntl; ++u) {
            const int xb = u & 1;
            const int64_t e0 = (int64_t)(t_begin + u) * TE;
            if (!fail && u >= 2 && !mb_wait(&wempty[xb], (unsigned)((u >> 1) - 1) & 1u)) fail = 0x204;
            A* w = wbuf + (size_t)xb * K;
            // near field: x of the group's source groups (times the dense scale)
            const int64_t g0 = e0 / G;
            A dsc = A(1);
            if constexpr (DST == ST_BF16) dsc = (A)a.scD[g0];
            for (int k = 0; k < a.nnb; ++k) {
                const int64_t gs = a.adm ? near_group(g0, k, a.d, a.nf) : g0;
                for (int b = lane; b < G; b += 32) {
                    const int64_t slot = gs * G + b;
                    const int64_t src = gs < 0 ? -1 : a.map ? a.map[slot] : slot;
                    w[k * G + b] = src >= 0 ? x[src * a.ldx] * dsc : A(0);
                }
            }
            // Steps 3-4: target node i of each level reads, for its q-th
            // partner j (weak: other sibling; standard: interaction-list
            // slot), the sums of source j at j's slot for i
            for (int l = 1; l <= a.nf; ++l) {
                const DevLevel& L = a.lv[l];
                const int r = L.r, sr = a.s * r;
                if (sr == 0) continue;
                const int64_t i = e0 / L.n;
                A* wl = w + woff[l];
                if (!a.adm) {
                    const int ci = (int)(i % nc);
                    for (int col = lane; col < sr; col += 32) {
                        const int qp = col / r, cr = col - qp * r;
                        const int cj = qp < ci ? qp : qp + 1;
                        const int64_t j = i - ci + cj;
                        const int qv = ci < cj ? ci : ci - 1;
                        wl[col] = T[(L.fin_off + j * sr + qv * r + cr) * a.kc] *
                                  (A)factor_scale<ST>(a.scU, L, a.s, i, col);
                    }
                } else {
                    int c[3];
                    dnode_coords(i, a.d, l, c);
                    const int pc = (c[0] & 1) | (c[1] & 1) << 1 | (c[2] & 1) << 2;
                    const int side = 1 << l;
                    for (int col = lane; col < sr; col += 32) {
                        const int qp = col / r, cr = col - qp * r;
                        const int pk = a.stencil[pc * a.s + qp];
                        int cj[3];
                        bool in = true;
                        for (int k = 0; k < 3; ++k) {
                            cj[k] = c[k] + ((pk >> (4 * k)) & 15) - 4;
                            in = in && (k >= a.d || (cj[k] >= 0 && cj[k] < side));
                        }
                        A v = A(0);
                        if (in) {
                            const int64_t j = dnode_index(cj, a.d, l);
                            const int qv = pk >> 12;
                            v = T[(L.fin_off + j * sr + qv * r + cr) * a.kc] *
                                (A)factor_scale<ST>(a.scU, L, a.s, i, col);
                        }
                        wl[col] = v;
                    }
                }
            }
            __syncwarp();
            mb_arrive(&wfull[xb]);
            if (u >= 1) combine(u - 1);
        }
        if (ntl >= 1) combine(ntl - 1);
        if (fail) report_status(a.status, fail);
    } else {
        // ------------------------------------------------------ consumers
        int fail = 0;                 // site code of the first wait that gave up
        const int grp = warp >> 1;
        const int pt = ((warp & 1) * 32 + lane) * kExpPT;    // first slot of this thread
        for (int u = 0; u < ntl; ++u) {
            const int xb = u & 1;
            if (!fail && !mb_wait(&wfull[xb], (unsigned)(u >> 1) & 1u)) fail = 0x205;
            const A* w = wbuf + (size_t)xb * K;
            A acc[kExpPT], cmp[kExpPT];
#pragma unroll
            for (int v = 0; v < kExpPT; ++v) acc[v] = cmp[v] = A(0);
            // stage g = u Q + q belongs to group g mod 4: with a ring depth that
            // is a multiple of four, every use of a slot belongs to one group,
            // which waits for its phases in order (no wait can pass on the
            // slot's previous phase while another group's box is in flight)
            const int q0 = (int)(((int64_t)grp - (int64_t)u * Q) % kExpGroups + kExpGroups) % kExpGroups;
            for (int q = q0; q < Q; q += kExpGroups) {
                const int g = u * Q + q, s = g % S;
                if (!fail && !mb_wait(&full[s], (unsigned)(g / S) & 1u)) fail = 0x206;
                const unsigned info = stagetab[q];
                int seg, col0, rows;
                unpack_stage(info, seg, col0, rows);
                const unsigned char* stg = sm + (size_t)s * stage_bytes;
                const A* wc = w + woff[seg] + col0;
                A part[kExpPT];
#pragma unroll
                for (int v = 0; v < kExpPT; ++v) part[v] = A(0);
                if (seg == 0) {
                    for (int c = 0; c < rows; ++c) {
                        A dv[kExpPT];
                        lds_dec<DST>(stg + ((size_t)c * TE + pt) * sizeof(ED), dv);
                        if constexpr (SPLIT) {
                            A lv[kExpPT];
                            lds_dec<DST>(stg + part_bytes + ((size_t)c * TE + pt) * sizeof(ED), lv);
#pragma unroll
                            for (int v = 0; v < kExpPT; ++v) dv[v] += lv[v];
                        }
                        const A wv = wc[c];
#pragma unroll
                        for (int v = 0; v < kExpPT; ++v) part[v] += dv[v] * wv;
                    }
                } else {
                    for (int c = 0; c < rows; ++c) {
                        A uv[kExpPT];
                        lds_dec<ST>(stg + ((size_t)c * TE + pt) * sizeof(E), uv);
                        if constexpr (SPLIT) {
                            A lv[kExpPT];
                            lds_dec<ST>(stg + part_bytes + ((size_t)c * TE + pt) * sizeof(E), lv);
#pragma unroll
                            for (int v = 0; v < kExpPT; ++v) uv[v] += lv[v];
                        }
                        const A wv = wc[c];
#pragma unroll
                        for (int v = 0; v < kExpPT; ++v) part[v] += uv[v] * wv;
                    }
                }
#pragma unroll
                for (int v = 0; v < kExpPT; ++v) {
                    A e;
                    two_sum(acc[v], part[v], acc[v], e);
                    cmp[v] += e;
                }
                __syncwarp();
                if (lane == 0) mb_arrive(&empty[s]);
            }
            // partial output of this group for the tile
            if (!fail && u >= 2 && !mb_wait(&rempty[xb], (unsigned)((u >> 1) - 1) & 1u)) fail = 0x207;
            A* rp = red + ((size_t)xb * kExpGroups + grp) * 2 * TE + pt;
#pragma unroll
            for (int v = 0; v < kExpPT; ++v) {
                rp[v] = acc[v];
                rp[TE + v] = cmp[v];
            }
            __syncwarp();
            if (lane == 0) {
                mb_arrive(&rfull[xb]);
                mb_arrive(&wempty[xb]);
            }
        }
        if (fail) report_status(a.status, fail);
    }
}

template <int ST>
int expand_run(const MatvecArgs& a, cudaStream_t st) {
    using A = typename Tr<ST>::A;
    const int64_t G = a.G, NCOL = (int64_t)a.nnb * G;
    if (G % kExpandStreamTile != 0 || NCOL >= (1 << 20) || a.tma_rb_d < 1 || NCOL % a.tma_rb_d != 0)
        return kStreamNotEligible;
    int64_t Q = NCOL / a.tma_rb_d, K = NCOL;
    for (int l = 1; l <= a.nf; ++l) {
        const DevLevel& L = a.lv[l];
        if (L.r == 0) continue;
        const int sr = a.s * L.r;
        if (L.n < kExpandStreamTile || L.tma_rb_u < 1 || sr % L.tma_rb_u != 0 || sr >= (1 << 20))
            return kStreamNotEligible;
        Q += sr / L.tma_rb_u;
        K += sr;
    }
    if (Q > kMaxStageTab) return kStreamNotEligible;
    const size_t stage = 16 * 1024;
    const size_t fixed = 2 * (size_t)K * sizeof(A) + 4 * (size_t)kExpGroups * kExpandStreamTile * sizeof(A) +
                         (size_t)Q * sizeof(unsigned);
    if (fixed + 4 * stage > kExpSmemMax) return kStreamNotEligible;
    int S = (int)((kExpSmemMax - fixed) / stage);
    S = S > 12 ? 12 : S;
    S = S / kExpGroups * kExpGroups;       // slots owned by one group each (see the consumers)
    const size_t smem = (size_t)S * stage + fixed;
    static DeviceFlags attr;
    {
        const cudaError_t e = attr.once([&] {
            return cudaFuncSetAttribute(expand_stream_kernel<ST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kExpSmemMax);
        });
        if (e != cudaSuccess) return (int)e;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
    const int ntile = (int)(a.Np / kExpandStreamTile);
    const int R = (ntile + sms - 1) / sms;
    const int grid = (ntile + R - 1) / R;
    // starts while the project side finishes: the producer streams D and U
    // (read-only) at once, the weights warp waits for the node sums
    e = launch_pdl(a.pdl != 0, expand_stream_kernel<ST>, dim3(grid), dim3(kExpThreads), smem, st, a, ntile, R, S, (int)Q,
                   (int)K);
    count_launches(1);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaGetLastError();
}

// Self-test of the device error path: one thread waits, with a limit of
// `limit_ns`, on an mbarrier whose phase nothing completes; the wait gives
// up and the kernel sets the status word to 1 and returns.
__global__ void wait_selftest_kernel(int* status, uint64_t limit_ns) {
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    mb_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
    if (!mb_wait(&bar, 0, limit_ns)) atomicExch(status, 1);
    mb_arrive(&bar);   // complete the phase before the CTA exits
}

}  // namespace

int stream_project(const MatvecArgs& a, void* stream) {
    if (a.k != 1 || a.kc != 1 || !a.status || !a.tmaps || a.nf < 1) return kStreamNotEligible;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (a.store) {
        case ST_F64: return stream_run<ST_F64>(a, st);
        case ST_F32: return stream_run<ST_F32>(a, st);
        case ST_BF16: return stream_run<ST_BF16>(a, st);
        case ST_BF16X2: return stream_run<ST_BF16X2>(a, st);
        case ST_FP8: return stream_run<ST_FP8>(a, st);
    }
    return kStreamNotEligible;
}

int stream_expand(const MatvecArgs& a, void* stream) {
    if (a.k != 1 || a.kc != 1 || !a.status || !a.tmaps_u || a.Np % kExpandStreamTile != 0) return kStreamNotEligible;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (a.store) {
        case ST_F64: return expand_run<ST_F64>(a, st);
        case ST_F32: return expand_run<ST_F32>(a, st);
        case ST_BF16: return expand_run<ST_BF16>(a, st);
        case ST_BF16X2: return expand_run<ST_BF16X2>(a, st);
        case ST_FP8: return expand_run<ST_FP8>(a, st);
    }
    return kStreamNotEligible;
}

int wait_selftest(int* status, uint64_t limit_ns, void* stream) {
    wait_selftest_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(status, limit_ns);
    count_launches(1);
    return (int)cudaGetLastError();
}

}  // namespace hm
