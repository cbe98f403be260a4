// Persistent project kernel (Steps 1-2, eq. (prod-vx)) for one right-hand
// side: the memory-bound form of the product, streamed through a
// shared-memory ring by the tensor-memory-access (TMA) engine.
//
// CTA c owns the project tiles [c R, c R + R).  Warp 8 (producer) stages the
// x values of every tile into a double buffer and, per stage, loads one box
// of V: tile_p slots x RB_l consecutive columns of one level's node, through
// that level's 2-D tensor map (row = node * s r_l + column), completing on an
// mbarrier with a transaction count.  Warps 0-7 (consumers) take the rows of
// a stage in turn: each lane reads 16-byte vectors of the row and the
// matching x values from shared memory, accumulates in increasing slot
// order, and the warp adds its lanes with a butterfly; the scaled sum is a
// node sum, or a per-tile partial for a node longer than the tile; a second
// launch adds every such node's partials (Step 2, node_step2).  No CTA-wide
// barrier interrupts the stream: stages and x buffers are released through
// mbarriers.  Per row and per node this is the arithmetic of the cached
// project kernel and its last-CTA reduction, so both give bitwise equal
// sums.
//
// Every wait is bounded: on timeout the thread sets the status word, skips
// its later waits, and the kernel runs to its end (the producer then waits,
// again bounded, for the copies it issued).
#include <cuda_runtime.h>

#include <cstdint>

#include "hm_device.h"
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
// after 2^20 tries or two seconds.
__device__ __forceinline__ bool mb_wait(uint64_t* bar, unsigned parity) {
    if (mb_try(bar, parity, 0)) return true;
    const uint64_t t0 = global_ns();
    for (int it = 0; it < (1 << 20); ++it) {
        if (mb_try(bar, parity, 100000)) return true;
        if (global_ns() - t0 > 2000000000ull) return false;
    }
    return false;
}
// global -> shared bulk copy of `bytes` (multiple of 16, both addresses
// 16-byte aligned), completing on `bar`
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            s_addr(dst)),
        "l"(src), "r"(bytes), "r"(s_addr(bar))
        : "memory");
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

// Warp sums of MR rows (MR a power of two, lane-distributed partial sums in
// v).  The first log2(MR) butterfly steps split the rows between the two
// halves of the lanes exchanging (the half with lane bit `off` clear keeps
// the lower rows), the rest are plain butterfly steps.  Every lane value is
// the same expression as in the full butterfly of one row (a_i + a_j equals
// a_j + a_i exactly), so row m's sum is bitwise that of the butterfly; it
// ends on the lanes with lane / (32 / MR) == m.
template <typename A, int MR>
__device__ __forceinline__ A warp_sum_rows(A (&v)[MR], int lane) {
    int off = 16;
#pragma unroll
    for (int M = MR; M > 1; M >>= 1, off >>= 1) {
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int m = 0; m < M / 2; ++m) {
            const A send = upper ? v[m] : v[m + M / 2];
            const A keep = upper ? v[m + M / 2] : v[m];
            v[m] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    A r = v[0];
#pragma unroll
    for (; off > 0; off >>= 1) r += __shfl_xor_sync(0xffffffffu, r, off);
    return r;
}

constexpr int kConsumerWarps = 16;
constexpr int kRowsPerWarp = 4;            // stage rows <= 64 = 16 warps x 4
constexpr int kStreamThreads = 32 * (kConsumerWarps + 1);
constexpr int kMaxStages = 16;
constexpr size_t kRingBytes = 192 * 1024;
constexpr size_t kStreamSmemMax = 210 * 1024;

// Stages of one tile (the same for every tile): per level, s r_l / RB_l
// boxes of RB_l consecutive columns.  Per tile and level the producer
// records the node, its first slot inside the node and the destination of
// column 0 (kept with the x buffer of the tile).
constexpr int kMaxStageTab = 2048;

__device__ __forceinline__ unsigned pack_stage(int l, int col0, int rows) {
    return (unsigned)l | ((unsigned)col0 << 8) | ((unsigned)rows << 20);
}

struct LevelBase {
    int64_t node;
    int64_t dbase;    // destination in T of column 0
    int64_t y0;       // tensor-map row of column 0 (node * s r_l)
    int64_t inoff;    // first slot of the tile inside the node
};

template <int ST, int MR>
__global__ void __launch_bounds__(kStreamThreads, 1)
    project_stream_kernel(const MatvecArgs a, int ntile, int R, int RB, int S, int Q) {
    using Trs = Tr<ST>;
    using A = typename Trs::A;
    using E = typename Trs::E;
    constexpr int VEC = Trs::VEC;
    constexpr bool SPLIT = ST == ST_BF16X2;
    constexpr int PARTS = SPLIT ? 2 : 1;
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ uint64_t full[kMaxStages], empty[kMaxStages], xfull[2], xempty[2];
    __shared__ LevelBase lb[2][kMaxLevels + 1];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tile = (int)a.tile_p;
    const unsigned rowb = (unsigned)tile * sizeof(E);     // bytes of one row (one part)
    // a stage: PARTS boxes of up to RB rows, each starting on 128 bytes
    const size_t part_bytes = ((size_t)RB * rowb + 127) / 128 * 128;
    const size_t stage_bytes = part_bytes * PARTS;
    // dynamic shared memory: ring | x [2][tile] | stage table [Q]
    A* xs = reinterpret_cast<A*>(sm + (size_t)S * stage_bytes);
    unsigned* stagetab = reinterpret_cast<unsigned*>(xs + 2 * tile);
    const int t_begin = blockIdx.x * R;
    const int t_end = min(t_begin + R, ntile);
    const int ntl = max(t_end - t_begin, 0);

    if (tid == 0) {
        for (int q = 0; q < S; ++q) {
            mb_init(&full[q], 1);
            mb_init(&empty[q], kConsumerWarps);
        }
        for (int q = 0; q < 2; ++q) {
            mb_init(&xfull[q], 33);    // 32 lanes' x copies + the level bases
            mb_init(&xempty[q], kConsumerWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
        int q = 0;
        for (int l = 1; l <= a.nf; ++l) {
            const int sr = a.s * a.lv[l].r, rb = a.lv[l].tma_rb;
            for (int c = 0; rb > 0 && c < sr; c += rb) stagetab[q++] = pack_stage(l, c, rb);
        }
    }
    __syncthreads();

    if (warp == kConsumerWarps) {
        // ------------------------------------------------------ producer
        bool ok = true;
        const bool xbulk = a.map == nullptr && a.ldx == 1 &&
                           (reinterpret_cast<uintptr_t>(a.x) & 15) == 0;
        const A* __restrict__ x = static_cast<const A*>(a.x);
        const unsigned char* maps = static_cast<const unsigned char*>(a.tmaps);
        for (int u = 0; u < ntl; ++u) {
            const int t = t_begin + u;
            const int64_t p0 = (int64_t)t * tile;
            const int xb = u & 1;
            if (ok && u >= 2 && !mb_wait(&xempty[xb], (unsigned)((u >> 1) - 1) & 1u)) ok = false;
            for (int l = 1 + lane; l <= a.nf; l += 32) {
                const DevLevel& L = a.lv[l];
                const int64_t sr = (int64_t)a.s * L.r;
                LevelBase b;
                b.node = p0 / L.n;
                b.inoff = p0 - b.node * L.n;
                b.y0 = b.node * sr;
                b.dbase = L.nsub > 1 ? L.part_off + (int64_t)t * sr : L.fin_off + b.node * sr;
                lb[xb][l] = b;
            }
            __syncwarp();
            if (lane == 0) mb_arrive(&xfull[xb]);
            A* xd = xs + xb * tile;
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
            for (int q = 0; q < Q; ++q) {
                const int g = u * Q + q, s = g % S;
                if (ok && g >= S && !mb_wait(&empty[s], (unsigned)((g / S) - 1) & 1u)) ok = false;
                if (lane == 0) {
                    const unsigned info = stagetab[q];
                    const int l = (int)(info & 0xffu), col0 = (int)((info >> 8) & 0xfffu);
                    const int rows = (int)(info >> 20);
                    const LevelBase& b = lb[xb][l];
                    unsigned char* stg = sm + (size_t)s * stage_bytes;
                    mb_arrive_tx(&full[s], (unsigned)rows * rowb * PARTS);
                    tma_load_2d(stg, maps + (size_t)l * kTensorMapBytes, (int)b.inoff, (int)(b.y0 + col0),
                                &full[s]);
                    if constexpr (SPLIT)
                        tma_load_2d(stg + part_bytes,
                                    maps + ((size_t)(kMaxLevels + 1) + l) * kTensorMapBytes, (int)b.inoff,
                                    (int)(b.y0 + col0), &full[s]);
                }
                __syncwarp();
            }
        }
        // wait (bounded) for the last use of every stage and x buffer, so
        // that no copy into this CTA's shared memory is still in flight
        if (lane == 0) {
            const int total = ntl * Q;
            for (int g = max(total - S, 0); g < total; ++g)
                if (!mb_wait(&full[g % S], (unsigned)(g / S) & 1u)) ok = false;
            for (int u = max(ntl - 2, 0); u < ntl; ++u)
                if (!mb_wait(&xfull[u & 1], (unsigned)(u >> 1) & 1u)) ok = false;
        }
        if (!ok) atomicExch(a.status, 1);
    } else {
        // ------------------------------------------------------ consumers
        bool ok = true;
        A* __restrict__ T = static_cast<A*>(a.T);
        for (int u = 0; u < ntl; ++u) {
            const int xb = u & 1;
            if (ok && !mb_wait(&xfull[xb], (unsigned)(u >> 1) & 1u)) ok = false;
            const A* xt = xs + xb * tile;
            for (int q = 0; q < Q; ++q) {
                const int g = u * Q + q, s = g % S;
                if (ok && !mb_wait(&full[s], (unsigned)(g / S) & 1u)) ok = false;
                const unsigned info = stagetab[q];
                const int l = (int)(info & 0xffu), col0 = (int)((info >> 8) & 0xfffu);
                const int rows = (int)(info >> 20);
                const unsigned char* stg = sm + (size_t)s * stage_bytes;
                // rows warp, warp + 16, ... of the stage together: one x
                // vector per step serves all of them
                const uint4* vh[MR];
                const uint4* vl[MR];
                A acc[MR];
#pragma unroll
                for (int m = 0; m < MR; ++m) {
                    const int r = warp + m * kConsumerWarps;
                    vh[m] = reinterpret_cast<const uint4*>(stg + (size_t)r * rowb);
                    vl[m] = reinterpret_cast<const uint4*>(stg + part_bytes + (size_t)r * rowb);
                    acc[m] = A(0);
                }
                for (int i = lane * VEC; i < tile; i += 32 * VEC) {
                    A xv[VEC];
#pragma unroll
                    for (int w = 0; w < (int)(VEC * sizeof(A) / 16); ++w) {
                        union { float4 v; A e[16 / sizeof(A)]; } cv;
                        cv.v = reinterpret_cast<const float4*>(xt + i)[w];
#pragma unroll
                        for (int e = 0; e < (int)(16 / sizeof(A)); ++e) xv[w * (16 / sizeof(A)) + e] = cv.e[e];
                    }
#pragma unroll
                    for (int m = 0; m < MR; ++m) {
                        if (warp + m * kConsumerWarps < rows) {
                            const uint4 hi = vh[m][i / VEC];
                            uint4 lo = hi;
                            if constexpr (SPLIT) lo = vl[m][i / VEC];
                            A one[1] = {acc[m]};
                            DotStep<ST, 1, 0>::go(hi, lo, xv, one);
                            acc[m] = one[0];
                        }
                    }
                }
                const A sum = warp_sum_rows<A, MR>(acc, lane);
                {
                    const int m = lane / (32 / MR);
                    const int r = warp + m * kConsumerWarps;
                    if (lane % (32 / MR) == 0 && r < rows) {
                        const LevelBase& b = lb[xb][l];
                        const int col = col0 + r;
                        const A sc = (A)factor_scale<ST>(a.scV, a.lv[l], a.s, b.node, col);
                        T[(b.dbase + col) * a.kc] = sum * sc;
                    }
                }
                __syncwarp();
                if (lane == 0) mb_arrive(&empty[s]);
            }
            // this warp is done with the x buffer and level bases of the tile
            __syncwarp();
            if (lane == 0) mb_arrive(&xempty[xb]);
        }
        if (!ok && lane == 0) atomicExch(a.status, 1);
    }
}

// Step 2 after the streamed project: one CTA of 256 threads per node longer
// than the tile adds the node's per-tile partials (node_step2, the order of
// the cached kernel's last-CTA reduction).  grid: sum over those levels of
// their node counts.
template <typename A>
__global__ void __launch_bounds__(256) project_step2_kernel(const MatvecArgs a) {
    __shared__ A red[256];
    int64_t b = blockIdx.x;
    for (int l = 1; l <= a.nf; ++l) {
        const DevLevel& L = a.lv[l];
        if (L.nsub <= 1 || L.r == 0) continue;
        const int64_t nodes = a.Np / L.n;
        if (b >= nodes) {
            b -= nodes;
            continue;
        }
        node_step2<A>(a, L, b, (int)threadIdx.x, red, [] { __syncthreads(); });
        return;
    }
}

template <int ST>
int stream_run(const MatvecArgs& a, cudaStream_t st) {
    using Trs = Tr<ST>;
    using E = typename Trs::E;
    using A = typename Trs::A;
    const int parts = ST == ST_BF16X2 ? 2 : 1;
    const int64_t tile = a.tile_p;
    const int RB = stream_stage_rows(tile, (int)sizeof(E), parts);
    int64_t Q = 0;
    for (int l = 1; l <= a.nf; ++l) {
        const DevLevel& L = a.lv[l];
        if (L.r == 0) continue;
        const int sr = a.s * L.r;
        if (L.n < tile || L.tma_rb < 1 || L.tma_rb > RB || sr % L.tma_rb != 0 || sr > 4095)
            return kStreamNotEligible;
        Q += sr / L.tma_rb;
    }
    if (Q == 0 || Q > kMaxStageTab) return kStreamNotEligible;
    const size_t rowb = (size_t)tile * sizeof(E);
    const size_t stage = ((size_t)RB * rowb + 127) / 128 * 128 * parts;
    int S = (int)(kRingBytes / stage);
    S = S > kMaxStages ? kMaxStages : S;
    if (S < 2) return kStreamNotEligible;
    const size_t smem = (size_t)S * stage + 2 * (size_t)tile * sizeof(A) + (size_t)Q * sizeof(unsigned);
    if (smem > kStreamSmemMax) return kStreamNotEligible;
    static bool done = false;
    if (!done) {
        const cudaError_t e = cudaFuncSetAttribute(project_stream_kernel<ST, kRowsPerWarp>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)kStreamSmemMax);
        if (e != cudaSuccess) return (int)e;
        done = true;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
    const int ntile = (int)(a.Np / a.tile_p);
    const int R = (ntile + sms - 1) / sms;
    const int grid = (ntile + R - 1) / R;
    project_stream_kernel<ST, kRowsPerWarp><<<grid, kStreamThreads, smem, st>>>(a, ntile, R, RB, S, (int)Q);
    e = cudaGetLastError();
    if (e != cudaSuccess) return (int)e;
    int64_t nodes = 0;
    for (int l = 1; l <= a.nf; ++l)
        if (a.lv[l].nsub > 1 && a.lv[l].r > 0) nodes += a.Np / a.lv[l].n;
    if (nodes > 0) project_step2_kernel<A><<<(unsigned)nodes, 256, 0, st>>>(a);
    return (int)cudaGetLastError();
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

}  // namespace hm
