// Tensor-core (tcgen05) kernels of the H-matrix-vector product for several
// right-hand sides, where both steps are dense contractions:
//
//   project (Step 1, eq. (prod-vx)):  T_seg[cols x k] = V_seg^T X_seg
//     A = V^T tile (M = columns of one level, padded to 128; K = slots),
//     K-major straight from the [column][slot] layout;  B = X tile (K = slots,
//     N = k), staged and transposed once per tile.  The per-tile partial sums
//     and the last-CTA reduction (Step 2) are those of the CUDA-core kernel.
//   expand (Steps 3-5, eqs. (prod-yuz), (prod-ydz)):
//     Y_tile[slots x k] = D_g X_g + sum_l U_l T_l
//     A = dense block / U tile (M = slots, K = columns), MN-major straight from
//     the [column][slot] layouts;  B = x of the group / summed t of the target
//     nodes (K x N = k), converted to bf16 per K block.
//
// Operands are bf16 (kind::f16, float accumulation in tensor memory).  Split
// storage runs three MMAs per step (A_hi B_hi + A_hi B_lo + A_lo B_hi, with x
// and t split the same way); e4m3 factors are widened to bf16 while staged.
// One thread issues the MMAs; tcgen05.commit arrives on an mbarrier per
// shared-memory stage; every wait is bounded and reports through a status
// word instead of hanging; tensor memory is always released.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "hm_device.h"

namespace hm {
namespace {

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor, no swizzle: core matrices of 8 rows x 16
// bytes; lbo = byte distance of core matrices adjacent along K, sbo = along
// M (or N).
__device__ __forceinline__ uint64_t smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= 1ull << 46;   // descriptor version of this architecture
    return d;
}

// Shared-memory matrix descriptor, 128-byte swizzle (the layout a tensor
// map with CU_TENSOR_MAP_SWIZZLE_128B writes; base 1024-byte aligned).
// K-major: rows of 128 bytes (64 bf16 along K), sbo = 1024 between groups of
// eight rows, a K step of 16 advances the start by 32 bytes.  MN-major:
// rows of 64 bf16 along M per K index, lbo = distance between 64-element M
// atoms, sbo = 1024 between groups of eight K rows.
__device__ __forceinline__ uint64_t smem_desc_sw128(unsigned addr, unsigned lbo, unsigned sbo) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= 1ull << 46;
    d |= 2ull << 61;   // swizzle mode: 128 bytes
    return d;
}

// 2-D tensor-map box at (x, y) -> shared memory, completing on `bar`
__device__ __forceinline__ void tma_load_2d(void* dst, const void* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
        "%3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Instruction descriptor: bf16 x bf16 -> f32, M x N, A K-major or MN-major,
// B K-major.
__device__ __forceinline__ unsigned idesc_bf16(int M, int N, bool a_mn_major) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn_major ? 1u : 0u) << 15) |
           ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(unsigned dtmem, uint64_t adesc, uint64_t bdesc,
                                         unsigned idesc, unsigned accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar)));
}

__device__ __forceinline__ void bar_init(uint64_t* bar, unsigned count = 1) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void bar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)));
}
// arrive on `bar` once this thread's earlier cp.async copies have landed
__device__ __forceinline__ void bar_arrive_cp_async(uint64_t* bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)));
}

__device__ __forceinline__ bool bar_try(uint64_t* bar, unsigned parity, unsigned suspend_ns) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity), "r"(suspend_ns));
    return done != 0;
}
// Bounded wait for completion `parity` of an mbarrier (the thread sleeps in
// try_wait until the phase completes or the hint runs out); false after
// 2^20 tries or two seconds.
__device__ __forceinline__ bool bar_wait(uint64_t* bar, unsigned parity) {
    if (bar_try(bar, parity, 0)) return true;
    uint64_t t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (int it = 0; it < (1 << 20); ++it) {
        if (bar_try(bar, parity, 100000)) return true;
        uint64_t t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > 2000000000ull) return false;
    }
    return false;
}

__device__ __forceinline__ void tmem_alloc(unsigned* dst, unsigned ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(dst)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;"); }

// 16 consecutive f32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16]) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%"
        "14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 bytes, or 16 zero bytes when !valid (nothing is read then)
__device__ __forceinline__ void cp_async16_z(void* smem, const void* gmem, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(smem)), "l"(gmem),
                 "r"(valid ? 16 : 0));
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;"); }
// AND over the 128 producer threads at named barrier 1
__device__ __forceinline__ bool producers_all(bool v) {
    unsigned r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.and.pred p, 1, 128, q;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(r)
        : "r"(v ? 1u : 0u));
    return r != 0;
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N));
}

__device__ __forceinline__ uint16_t bf16_bits(float v) {
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    return *reinterpret_cast<const uint16_t*>(&b);
}
__device__ __forceinline__ float bf16_val(uint16_t u) { return __uint_as_float((uint32_t)u << 16); }

// 16 e4m3 values -> 16 bf16 (exact: every e4m3 value is a bf16 value)
__device__ __forceinline__ void fp8x16_to_bf16(const uint4& v, uint4& lo8, uint4& hi8) {
    const unsigned w[4] = {v.x, v.y, v.z, v.w};
    unsigned o[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const unsigned pair = (w[q >> 1] >> (16 * (q & 1))) & 0xffffu;
        const __half2_raw h =
            __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)pair, __NV_E4M3);
        const float2 f = __half22float2(__half2(h));
        o[q] = (unsigned)bf16_bits(f.x) | ((unsigned)bf16_bits(f.y) << 16);
    }
    lo8 = make_uint4(o[0], o[1], o[2], o[3]);
    hi8 = make_uint4(o[4], o[5], o[6], o[7]);
}

constexpr int kProducers = 128;            // warps 0-3: copies, then the epilogue
constexpr int kThreads = kProducers + 32;  // warp 4: tensor memory and MMA issue
constexpr int kStages = 4;
constexpr int kNPMax = 64;                 // prepared B operands hold 64 right-hand sides

// Prepared B operands in global memory (bf16, K-major core matrices, 64
// rows): the project kernel writes its x tile (64 rows x tile_p slots) to
// `xprep` at tile * 64 * tile_p elements; the prep kernel writes the summed t
// of every target node (64 rows x sr_pad columns) to `ttprep` at level
// offset + node * 64 * sr_pad.  Core (n/8, k/8) of a K x 64 operand with K
// columns sits at (n/8) * K * 8 + (k/8) * 64 elements, row n%8 at 8 more.
__device__ __forceinline__ int64_t core_elem(int n, int k, int K) {
    return (int64_t)(n >> 3) * K * 8 + (k >> 3) * 64 + (n & 7) * 8 + (k & 7);
}

// ------------------------------------------------- x prep
// x of every project tile as the bf16 K-major B operand (64 rows, tile_p
// slots, core matrices; rows n >= k are zero), plus the low parts for split
// storage.  One thread per (tile, 8-slot group, row n); consecutive threads
// take consecutive n, so each of the eight loads of a warp reads consecutive
// x values of one slot.
template <bool SPLIT>
__global__ void __launch_bounds__(256) tc_xprep_kernel(const MatvecArgs a, int np) {
    const int tile = (int)a.tile_p;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per_tile = (int64_t)(tile / 8) * np;
    const int64_t t = e / per_tile;
    if (t >= a.Np / tile) return;
    const int rem = (int)(e - t * per_tile);
    const int k8 = rem / np, n = rem - k8 * np;
    const float* __restrict__ x = static_cast<const float*>(a.x);
    unsigned hw[4], lw[4];
#pragma unroll
    for (int q = 0; q < 8; q += 2) {
        float v[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int64_t slot = t * tile + k8 * 8 + q + u;
            const int64_t row = a.map ? a.map[slot] : slot;
            v[u] = (row >= 0 && n < a.k) ? __ldg(x + row * a.ldx + n) : 0.f;
        }
        const uint16_t h0 = bf16_bits(v[0]), h1 = bf16_bits(v[1]);
        hw[q / 2] = (unsigned)h0 | ((unsigned)h1 << 16);
        if constexpr (SPLIT)
            lw[q / 2] = (unsigned)bf16_bits(v[0] - bf16_val(h0)) | ((unsigned)bf16_bits(v[1] - bf16_val(h1)) << 16);
    }
    const int64_t at = t * kNPMax * tile + core_elem(n, k8 * 8, tile);
    *reinterpret_cast<uint4*>(static_cast<uint16_t*>(a.xprep) + at) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    if constexpr (SPLIT)
        *reinterpret_cast<uint4*>(static_cast<uint16_t*>(a.xprep_lo) + at) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
}

// global -> shared bulk copy completing on an mbarrier (both addresses
// 16-byte aligned, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void bar_arrive_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes));
}

// ------------------------------------------------- persistent project
// CTA c owns the tiles [c R, c R + R).  Warps 0-3 produce (the prepared x
// tile of every tile into a double buffer by one bulk copy; 128-column x
// 64-slot chunks of V into a ring), warps 4-7 flush accumulators, warp 8
// issues the MMAs.  Accumulator (level, column block) keeps adding across
// the range's tiles while they stay in one node of that level; it is
// flushed when the node ends or the range ends: a node sum if the node lies
// inside the range, else a partial at the tile where the covered part starts
// (tc_reduce_kernel adds those).  Within a tile the coarsest level goes
// first, so the flush of the finest level overlaps the next tile's coarse
// MMAs.
constexpr int kPThreads = 288;
constexpr int kMaxAcc = 8;

template <int ST, int NP, int S>
__global__ void __launch_bounds__(kPThreads) tc_project_persistent(const MatvecArgs a, unsigned tcols,
                                                                   int ntile, int R) {
    constexpr bool SPLIT = ST == ST_BF16X2;
    constexpr int KC = 64;
    constexpr unsigned ALBO = 128, ASBO = (KC / 8) * 128;
    constexpr unsigned ABYTES = 16 * ASBO;
    constexpr unsigned STAGE = (SPLIT ? 2 : 1) * ABYTES;
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ uint64_t full[S], empty[S], xfull[2], xempty[2], afull[kMaxAcc], aempty[kMaxAcc];
    __shared__ unsigned s_tmem;
    __shared__ int s_acc[kMaxLevels + 2];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tile = (int)a.tile_p;
    const int t_begin = blockIdx.x * R;
    const int t_end = min(t_begin + R, ntile);
    const unsigned BSBO = (unsigned)(tile / 8) * 128;
    const unsigned XB = (unsigned)NP * tile * 2;            // one x buffer (hi)
    unsigned char* Xb = sm + (size_t)S * STAGE;              // [2][hi (+lo)]
    float* __restrict__ T = static_cast<float*>(a.T);
    const int nchunk = tile / KC;

    if (tid == 0) {
        for (int q = 0; q < S; ++q) {
            bar_init(&full[q], kProducers);
            bar_init(&empty[q], 1);
        }
        for (int q = 0; q < 2; ++q) {
            bar_init(&xfull[q], 1);
            bar_init(&xempty[q], 1);
        }
        for (int q = 0; q < kMaxAcc; ++q) {
            bar_init(&afull[q], 1);
            bar_init(&aempty[q], kProducers);
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
        int acc = 0;
        for (int l = 1; l <= a.nf; ++l) {
            s_acc[l] = acc;
            acc += (a.s * a.lv[l].r + 127) / 128;
        }
        s_acc[a.nf + 1] = acc;
    }
    if (warp == 8) tmem_alloc(&s_tmem, tcols);
    fence_before();
    __syncthreads();
    fence_after();
    const unsigned tmem = s_tmem;
    const int nacc = s_acc[a.nf + 1];
    const int per_tile = nacc * nchunk;
    // does level l close its accumulators after tile t?
    auto flushes = [&](int l, int t) {
        return t == t_end - 1 || ((int64_t)(t + 1) * tile) % a.lv[l].n == 0;
    };

    if (warp < 4) {
        // ------------------------------------------------------ producers
        bool ok = true;
        int item = 0;
        for (int t = t_begin; t < t_end; ++t) {
            const int u = t - t_begin;
            const int xb = u & 1;
            unsigned char* X = Xb + (size_t)xb * (SPLIT ? 2 : 1) * XB;
            unsigned char* Xlo = X + XB;
            const int64_t p0 = (int64_t)t * tile;
            // the tile's x rows (prepared by tc_xprep_kernel): one bulk copy
            if (tid == 0) {
                if (ok && u >= 2 && !bar_wait(&xempty[xb], (unsigned)((u / 2) - 1) & 1u)) ok = false;
                const uint16_t* xs = static_cast<const uint16_t*>(a.xprep) + (int64_t)t * kNPMax * tile;
                bar_arrive_tx(&xfull[xb], (SPLIT ? 2u : 1u) * XB);
                bulk_g2s(X, xs, XB, &xfull[xb]);
                if constexpr (SPLIT)
                    bulk_g2s(Xlo, static_cast<const uint16_t*>(a.xprep_lo) + (int64_t)t * kNPMax * tile, XB,
                             &xfull[xb]);
            }
            // every producer reaches this barrier; a failed wait anywhere stops all
            ok = producers_all(ok);
            if (!ok) break;
            // V chunks of this tile: levels coarse to fine
            for (int it = 0; it < per_tile; ++it, ++item) {
                const int s = item % S;
                if (ok && item >= S && !bar_wait(&empty[s], (unsigned)((item / S) - 1) & 1u)) ok = false;
                if (!ok) continue;
                const int blk = it / nchunk, kc = it - blk * nchunk;
                int l = 1;
                while (s_acc[l + 1] <= blk) ++l;
                const int cb = blk - s_acc[l];
                const DevLevel& L = a.lv[l];
                const int sr = a.s * L.r;
                const int64_t node = p0 / L.n;
                const int64_t base = L.fac_off + node * (int64_t)sr * L.n + (p0 - node * L.n) +
                                     (int64_t)cb * 128 * L.n + kc * KC;
                unsigned char* A = sm + (size_t)s * STAGE;
                unsigned char* Alo = A + ABYTES;
                for (int e = tid; e < 128 * (KC / 8); e += kProducers) {
                    const int row = e >> 3, k8 = e & 7;
                    const unsigned aoff = (row >> 3) * ASBO + k8 * ALBO + (row & 7) * 16;
                    const bool valid = cb * 128 + row < sr;
                    const int64_t elem = valid ? base + (int64_t)row * L.n + k8 * 8 : 0;
                    if constexpr (ST == ST_FP8) {
                        uint4 lo8 = make_uint4(0, 0, 0, 0), hi8;
                        if (valid) {
                            const uint2 raw = __ldg(reinterpret_cast<const uint2*>(
                                static_cast<const uint8_t*>(a.V) + elem));
                            fp8x16_to_bf16(make_uint4(raw.x, raw.y, 0, 0), lo8, hi8);
                        }
                        *reinterpret_cast<uint4*>(A + aoff) = lo8;
                    } else {
                        cp_async16_z(A + aoff, static_cast<const uint16_t*>(a.V) + elem, valid);
                        if constexpr (SPLIT)
                            cp_async16_z(Alo + aoff, static_cast<const uint16_t*>(a.V_lo) + elem, valid);
                    }
                }
                if constexpr (ST == ST_FP8) {
                    fence_async_smem();
                    bar_arrive(&full[s]);
                } else {
                    bar_arrive_cp_async(&full[s]);
                }
            }
        }
        if (!ok && lane == 0) atomicExch(a.status, 1);
    } else if (warp < 8) {
        // ------------------------------------------------------ epilogue
        const int ew = warp - 4;
        int nfl[kMaxAcc];
        for (int q = 0; q < kMaxAcc; ++q) nfl[q] = 0;
        bool ok = true;
        for (int t = t_begin; t < t_end && ok; ++t) {
            const int64_t p0 = (int64_t)t * tile;
            for (int l = 1; l <= a.nf && ok; ++l) {
                if (!flushes(l, t)) continue;
                const DevLevel& L = a.lv[l];
                const int sr = a.s * L.r;
                const int64_t node = p0 / L.n;
                const int64_t nstart = node * L.n / tile, nend = (node + 1) * L.n / tile;   // tiles
                const bool whole = nstart >= t_begin && nend <= t_end;
                const int64_t pslot = nstart > t_begin ? nstart : t_begin;
                for (int cb = 0; cb < s_acc[l + 1] - s_acc[l]; ++cb) {
                    const int ai = s_acc[l] + cb;
                    if (!bar_wait(&afull[ai], (unsigned)nfl[ai] & 1u)) ok = false;
                    ok = __all_sync(0xffffffffu, ok);
                    if (!ok) break;
                    fence_after();
                    const int col = cb * 128 + ew * 32 + lane;
                    float sc = 1.f;
                    if constexpr (ST == ST_BF16) sc = col < sr ? a.scV[L.sc_off + node * a.s + col / L.r] : 0.f;
                    if constexpr (ST == ST_FP8) sc = col < sr ? a.scV[L.sc_off + node * sr + col] : 0.f;
                    float* dst = whole ? T + (L.fin_off + node * sr + col) * a.kc
                                       : T + (L.part_off + pslot * sr + col) * a.kc;
                    for (int c0 = 0; c0 < NP; c0 += 16) {
                        float v[16];
                        tmem_ld16(tmem + ((unsigned)(ew * 32) << 16) + (unsigned)ai * NP + c0, v);
                        if (col < sr)
#pragma unroll
                            for (int j = 0; j < 16; ++j)
                                if (c0 + j < a.k) dst[c0 + j] = v[j] * sc;
                    }
                    fence_before();
                    bar_arrive(&aempty[ai]);
                    ++nfl[ai];
                }
            }
        }
        if (!ok && lane == 0) atomicExch(a.status, 1);
    } else if (lane == 0) {
        // ------------------------------------------------------ MMA issue
        const unsigned idesc = idesc_bf16(128, NP, false);
        bool fresh[kMaxAcc];
        int nfl[kMaxAcc];
        for (int q = 0; q < kMaxAcc; ++q) {
            fresh[q] = true;
            nfl[q] = 0;
        }
        bool ok = true;
        int item = 0;
        for (int t = t_begin; t < t_end && ok; ++t) {
            const int u = t - t_begin;
            const int xb = u & 1;
            unsigned char* X = Xb + (size_t)xb * (SPLIT ? 2 : 1) * XB;
            unsigned char* Xlo = X + XB;
            if (!bar_wait(&xfull[xb], (unsigned)(u / 2) & 1u)) { ok = false; break; }
            for (int it = 0; it < per_tile; ++it, ++item) {
                const int s = item % S;
                const int blk = it / nchunk, kc = it - blk * nchunk;
                if (kc == 0 && fresh[blk] && nfl[blk] > 0 &&
                    !bar_wait(&aempty[blk], (unsigned)(nfl[blk] - 1) & 1u)) { ok = false; break; }
                if (!bar_wait(&full[s], (unsigned)(item / S) & 1u)) { ok = false; break; }
                fence_async_smem();
                fence_after();
                unsigned char* A = sm + (size_t)s * STAGE;
                unsigned char* Alo = A + ABYTES;
                const unsigned d = tmem + (unsigned)blk * NP;
#pragma unroll
                for (int ks = 0; ks < KC / 16; ++ks) {
                    const unsigned ak = smem_u32(A) + ks * 2 * ALBO;
                    const unsigned ak_lo = smem_u32(Alo) + ks * 2 * ALBO;
                    const int kslot = kc * KC + ks * 16;
                    const unsigned bk = smem_u32(X) + (kslot / 8) * 128;
                    const unsigned bk_lo = smem_u32(Xlo) + (kslot / 8) * 128;
                    const unsigned acc = (fresh[blk] && kc == 0 && ks == 0) ? 0u : 1u;
                    mma_bf16(d, smem_desc(ak, ALBO, ASBO), smem_desc(bk, 128, BSBO), idesc, acc);
                    if constexpr (SPLIT) {
                        mma_bf16(d, smem_desc(ak, ALBO, ASBO), smem_desc(bk_lo, 128, BSBO), idesc, 1u);
                        mma_bf16(d, smem_desc(ak_lo, ALBO, ASBO), smem_desc(bk, 128, BSBO), idesc, 1u);
                    }
                }
                fresh[blk] = false;
                mma_commit(&empty[s]);
            }
            if (!ok) break;
            mma_commit(&xempty[xb]);
            for (int l = 1; l <= a.nf; ++l) {
                if (!flushes(l, t)) continue;
                for (int ai = s_acc[l]; ai < s_acc[l + 1]; ++ai) {
                    mma_commit(&afull[ai]);
                    fresh[ai] = true;
                    ++nfl[ai];
                }
            }
        }
        if (!ok) atomicExch(a.status, 1);
    }
    cp_async_wait_all();
    fence_before();
    __syncthreads();
    if (warp == 8) tmem_dealloc(tmem, tcols);
}

// ------------------------------------------------- project, TMA operands
// As tc_project_persistent (ranges of R tiles, accumulators per (level,
// 128-column block) kept across the range's tiles inside a node, flushed
// at node or range ends), for bf16 and split bf16 storage, with every
// operand moved by the copy engines: per 64-slot chunk of a tile the x
// chunk (NP/8 bulk copies of 1 KB from the prepared x) and, per
// accumulator block, one tensor-map box of V (64 slots x 128 columns, or
// the level's remaining s r_l mod 128 columns; accumulator rows past the
// box are never stored) in the 128-byte swizzle the MMA reads directly.
//   warp 0: producer (one thread), warp 1: tensor memory + MMA issue (one
//   thread), warps 2-5: epilogue (tensor-memory lane quarter = warp % 4).
constexpr int kTmaThreads = 192;
constexpr int kXRing = 3;

template <int ST, int NP>
__global__ void __launch_bounds__(kTmaThreads, 1)
    tc_project_tma(const MatvecArgs a, unsigned tcols, int ntile, int R, int S) {
    constexpr bool SPLIT = ST == ST_BF16X2;
    constexpr int PARTS = SPLIT ? 2 : 1;
    constexpr unsigned ABOX = 128 * 128;                   // one V box: 128 rows x 128 bytes
    constexpr unsigned STAGE = PARTS * ABOX;
    constexpr unsigned XPART = NP * 64 * 2;                // x chunk: NP rows x 64 slots
    constexpr unsigned XCH = PARTS * XPART;
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ uint64_t full[16], empty[16], xfull[kXRing], xempty[kXRing], afull[kMaxAcc], aempty[kMaxAcc];
    __shared__ unsigned s_tmem;
    __shared__ int s_acc[kMaxLevels + 2];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tile = (int)a.tile_p;
    const int t_begin = blockIdx.x * R;
    const int t_end = min(t_begin + R, ntile);
    unsigned char* xring = sm + (size_t)S * STAGE;
    float* __restrict__ T = static_cast<float*>(a.T);
    const int nchunk = tile / 64;

    if (tid == 0) {
        for (int q = 0; q < S; ++q) {
            bar_init(&full[q], 1);
            bar_init(&empty[q], 1);
        }
        for (int q = 0; q < kXRing; ++q) {
            bar_init(&xfull[q], 1);
            bar_init(&xempty[q], 1);
        }
        for (int q = 0; q < kMaxAcc; ++q) {
            bar_init(&afull[q], 1);
            bar_init(&aempty[q], 128);
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
        int acc = 0;
        for (int l = 1; l <= a.nf; ++l) {
            s_acc[l] = acc;
            acc += (a.s * a.lv[l].r + 127) / 128;
        }
        s_acc[a.nf + 1] = acc;
    }
    if (warp == 1) tmem_alloc(&s_tmem, tcols);
    fence_before();
    __syncthreads();
    fence_after();
    const unsigned tmem = s_tmem;
    const int nacc = s_acc[a.nf + 1];
    auto flushes = [&](int l, int t) {
        return t == t_end - 1 || ((int64_t)(t + 1) * tile) % a.lv[l].n == 0;
    };

    if (warp == 0) {
        // ------------------------------------------------------ producer
        bool ok = true;
        if (lane == 0) {
            const unsigned char* maps = static_cast<const unsigned char*>(a.tmaps_tc);
            int g = 0, xc = 0;
            for (int t = t_begin; t < t_end && ok; ++t) {
                const int64_t p0 = (int64_t)t * tile;
                for (int kc = 0; kc < nchunk && ok; ++kc, ++xc) {
                    const int xi = xc % kXRing;
                    if (xc >= kXRing && !bar_wait(&xempty[xi], (unsigned)((xc / kXRing) - 1) & 1u)) { ok = false; break; }
                    unsigned char* X = xring + (size_t)xi * XCH;
                    bar_arrive_tx(&xfull[xi], XCH);
                    const int64_t xo = (int64_t)t * kNPMax * tile + kc * 512;
                    for (int ng = 0; ng < NP / 8; ++ng) {
                        bulk_g2s(X + ng * 1024, static_cast<const uint16_t*>(a.xprep) + xo + (int64_t)ng * tile * 8,
                                 1024, &xfull[xi]);
                        if constexpr (SPLIT)
                            bulk_g2s(X + XPART + ng * 1024,
                                     static_cast<const uint16_t*>(a.xprep_lo) + xo + (int64_t)ng * tile * 8, 1024,
                                     &xfull[xi]);
                    }
                    for (int l = 1; l <= a.nf; ++l) {
                        const DevLevel& L = a.lv[l];
                        const int sr = a.s * L.r;
                        const int64_t node = p0 / L.n;
                        const int x = (int)(p0 - node * L.n) + kc * 64;
                        for (int cb = 0; cb < s_acc[l + 1] - s_acc[l]; ++cb, ++g) {
                            const int s = g % S;
                            if (g >= S && !bar_wait(&empty[s], (unsigned)((g / S) - 1) & 1u)) { ok = false; break; }
                            const int rows = sr - cb * 128 < 128 ? sr - cb * 128 : 128;
                            const int kind = rows == 128 ? kMapVSw : kMapVSwRem;
                            unsigned char* A = sm + (size_t)s * STAGE;
                            bar_arrive_tx(&full[s], (unsigned)rows * 128 * PARTS);
                            const int y = (int)(node * sr + cb * 128);
                            tma_load_2d(A, maps + ((size_t)kind * (kMaxLevels + 1) + l) * kTensorMapBytes, x, y,
                                        &full[s]);
                            if constexpr (SPLIT)
                                tma_load_2d(A + ABOX, maps + ((size_t)(kind + 1) * (kMaxLevels + 1) + l) * kTensorMapBytes,
                                            x, y, &full[s]);
                        }
                        if (!ok) break;
                    }
                }
            }
            // copies still in flight into this CTA's shared memory
            for (int q = (g > S ? g - S : 0); q < g; ++q) bar_wait(&full[q % S], (unsigned)(q / S) & 1u);
            for (int q = (xc > kXRing ? xc - kXRing : 0); q < xc; ++q)
                bar_wait(&xfull[q % kXRing], (unsigned)(q / kXRing) & 1u);
        }
        if (!ok && lane == 0) atomicExch(a.status, 1);
    } else if (warp == 1) {
        // ------------------------------------------------------ MMA issue
        if (lane == 0) {
            const unsigned idesc = idesc_bf16(128, NP, false);
            bool fresh[kMaxAcc];
            int nfl[kMaxAcc];
            for (int q = 0; q < kMaxAcc; ++q) {
                fresh[q] = true;
                nfl[q] = 0;
            }
            bool ok = true;
            int g = 0, xc = 0;
            for (int t = t_begin; t < t_end && ok; ++t) {
                for (int kc = 0; kc < nchunk && ok; ++kc, ++xc) {
                    const int xi = xc % kXRing;
                    if (!bar_wait(&xfull[xi], (unsigned)(xc / kXRing) & 1u)) { ok = false; break; }
                    const unsigned char* X = xring + (size_t)xi * XCH;
                    for (int ai = 0; ai < nacc; ++ai, ++g) {
                        const int s = g % S;
                        if (kc == 0 && fresh[ai] && nfl[ai] > 0 &&
                            !bar_wait(&aempty[ai], (unsigned)(nfl[ai] - 1) & 1u)) { ok = false; break; }
                        if (!bar_wait(&full[s], (unsigned)(g / S) & 1u)) { ok = false; break; }
                        fence_after();
                        const unsigned A = smem_u32(sm + (size_t)s * STAGE);
                        const unsigned B = smem_u32(X);
                        const unsigned d = tmem + (unsigned)ai * NP;
#pragma unroll
                        for (int ks = 0; ks < 4; ++ks) {
                            const uint64_t ad = smem_desc_sw128(A + ks * 32, 16, 1024);
                            const uint64_t bd = smem_desc(B + ks * 256, 128, 1024);
                            const unsigned accf = (fresh[ai] && kc == 0 && ks == 0) ? 0u : 1u;
                            mma_bf16(d, ad, bd, idesc, accf);
                            if constexpr (SPLIT) {
                                mma_bf16(d, ad, smem_desc(B + XPART + ks * 256, 128, 1024), idesc, 1u);
                                mma_bf16(d, smem_desc_sw128(A + ABOX + ks * 32, 16, 1024), bd, idesc, 1u);
                            }
                        }
                        if (kc == 0) fresh[ai] = false;
                        mma_commit(&empty[s]);
                    }
                    if (!ok) break;
                    mma_commit(&xempty[xi]);
                }
                if (!ok) break;
                for (int l = 1; l <= a.nf; ++l) {
                    if (!flushes(l, t)) continue;
                    for (int ai = s_acc[l]; ai < s_acc[l + 1]; ++ai) {
                        mma_commit(&afull[ai]);
                        fresh[ai] = true;
                        ++nfl[ai];
                    }
                }
            }
            if (!ok) atomicExch(a.status, 1);
        }
    } else {
        // ------------------------------------------------------ epilogue
        const int q4 = warp & 3;                        // tensor-memory lane quarter
        int nfl[kMaxAcc];
        for (int q = 0; q < kMaxAcc; ++q) nfl[q] = 0;
        bool ok = true;
        for (int t = t_begin; t < t_end && ok; ++t) {
            const int64_t p0 = (int64_t)t * tile;
            for (int l = 1; l <= a.nf && ok; ++l) {
                if (!flushes(l, t)) continue;
                const DevLevel& L = a.lv[l];
                const int sr = a.s * L.r;
                const int64_t node = p0 / L.n;
                const int64_t nstart = node * L.n / tile, nend = (node + 1) * L.n / tile;   // tiles
                const bool whole = nstart >= t_begin && nend <= t_end;
                const int64_t pslot = nstart > t_begin ? nstart : t_begin;
                for (int cb = 0; cb < s_acc[l + 1] - s_acc[l]; ++cb) {
                    const int ai = s_acc[l] + cb;
                    if (!bar_wait(&afull[ai], (unsigned)nfl[ai] & 1u)) ok = false;
                    ok = __all_sync(0xffffffffu, ok);
                    if (!ok) break;
                    fence_after();
                    const int col = cb * 128 + q4 * 32 + lane;
                    float sc = 1.f;
                    if constexpr (ST == ST_BF16) sc = col < sr ? a.scV[L.sc_off + node * a.s + col / L.r] : 0.f;
                    float* dst = whole ? T + (L.fin_off + node * sr + col) * a.kc
                                       : T + (L.part_off + pslot * sr + col) * a.kc;
                    for (int c0 = 0; c0 < NP; c0 += 16) {
                        float v[16];
                        tmem_ld16(tmem + ((unsigned)(q4 * 32) << 16) + (unsigned)ai * NP + c0, v);
                        if (col < sr)
#pragma unroll
                            for (int j = 0; j < 16; ++j)
                                if (c0 + j < a.k) dst[c0 + j] = v[j] * sc;
                    }
                    fence_before();
                    bar_arrive(&aempty[ai]);
                    ++nfl[ai];
                }
            }
        }
        if (!ok && lane == 0) atomicExch(a.status, 1);
    }
    fence_before();
    __syncthreads();
    if (warp == 1) tmem_dealloc(tmem, tcols);
}

// -------------------------------------------------------- Step 2 (k > 1)
// Node sums of the levels whose nodes span several ranges of the persistent
// project kernel (ranges of R tiles; a node inside one range already has its
// sum).  The partials of a spanning node sit at its first tile and at every
// range start inside it, and are added in increasing tile order, one item
// (column, right-hand side) per thread.  Work is enumerated by range
// boundary: boundary b (tile b R, 0 < b < ranges) lying strictly inside node
// j of a level is that node's owner when it is the node's first such
// boundary.  grid: levels x (ranges - 1) x ceil(items / kRedThreads).
constexpr int kRedThreads = 256;
__global__ void __launch_bounds__(kRedThreads) tc_reduce_kernel(const MatvecArgs a, int nranges, int chunks) {
    float* __restrict__ T = static_cast<float*>(a.T);
    const int R = a.tc_range;
    const int64_t per_level = (int64_t)(nranges - 1) * chunks;
    int64_t b = blockIdx.x;
    const int lvl = (int)(b / per_level) + 1;
    b -= (int64_t)(lvl - 1) * per_level;
    const int64_t bnd = b / chunks + 1;
    const int chunk = (int)(b % chunks);
    if (lvl > a.nf) return;
    const DevLevel& L = a.lv[lvl];
    if (L.nsub <= 1 || L.r == 0) return;
    const int64_t tl = L.nsub, tb = bnd * R;
    const int64_t node = tb / tl, t0 = node * tl, t1 = t0 + tl;
    if (tb == t0 || (bnd - 1) * R > t0) return;                  // not inside, or not the first
    const int sr = a.s * L.r;
    const int items = sr * a.kc;
    const int item = chunk * kRedThreads + threadIdx.x;
    if (item >= items) return;
    const int64_t stride = (int64_t)sr * a.kc;
    const float* src = T + L.part_off * a.kc + item;
    float sum = __ldcg(src + t0 * stride);
    int64_t t = tb;
#pragma unroll 4
    for (; t < t1; t += R) sum += __ldcg(src + t * stride);
    T[(L.fin_off + node * sr) * a.kc + item] = sum;
}

// ---------------------------------------------------------------- t prep
// Steps 3-4: for every level and target node i, the summed t_{i<-j} of its
// siblings (times the U scales), as a bf16 K-major operand of sr_pad columns.
template <int ST>
__global__ void tc_tt_prep_kernel(const MatvecArgs a) {
    constexpr bool SPLIT = ST == ST_BF16X2;
    const float* __restrict__ T = static_cast<const float*>(a.T);
    uint16_t* out = static_cast<uint16_t*>(a.ttprep);
    uint16_t* out_lo = static_cast<uint16_t*>(a.ttprep_lo);
    const int nc = a.s + 1;
    const int np = (a.k + 15) / 16 * 16;
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int l = 1; l <= a.nf; ++l) {
        const DevLevel& L = a.lv[l];
        const int r = L.r, sr = a.s * r, srp = (sr + 15) / 16 * 16;
        const int64_t nodes = a.Np / L.n;
        const int64_t items = nodes * np * (srp / 8);     // one core row (8 columns) each
        if (e >= items) {
            e -= items;
            continue;
        }
        const int64_t i = e / (np * (srp / 8));
        const int rem = (int)(e - i * (np * (srp / 8)));
        const int k8 = rem / np, n = rem - k8 * np;       // right-hand side fastest: coalesced T reads
        const int ci = (int)(i % nc);
        unsigned hw[4], lw[4];
#pragma unroll
        for (int t = 0; t < 8; t += 2) {
            float v[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int col = k8 * 8 + t + u;
                v[u] = 0.f;
                if (col < sr && n < a.k) {
                    const int qp = col / r, cr = col - qp * r;
                    const int cj = qp < ci ? qp : qp + 1;
                    const int64_t j = i - ci + cj;
                    const int qv = ci < cj ? ci : ci - 1;
                    v[u] = T[(L.fin_off + j * sr + qv * r + cr) * a.kc + n];
                    if constexpr (ST == ST_BF16) v[u] *= a.scU[L.sc_off + i * a.s + qp];
                    if constexpr (ST == ST_FP8) v[u] *= a.scU[L.sc_off + i * sr + col];
                }
            }
            const uint16_t h0 = bf16_bits(v[0]), h1 = bf16_bits(v[1]);
            hw[t / 2] = (unsigned)h0 | ((unsigned)h1 << 16);
            if constexpr (SPLIT)
                lw[t / 2] = (unsigned)bf16_bits(v[0] - bf16_val(h0)) |
                            ((unsigned)bf16_bits(v[1] - bf16_val(h1)) << 16);
        }
        const int64_t at = L.tt_off + i * kNPMax * srp + core_elem(n, k8 * 8, srp);
        *reinterpret_cast<uint4*>(out + at) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        if constexpr (SPLIT) *reinterpret_cast<uint4*>(out_lo + at) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        return;
    }
}

// ------------------------------------------------------------------ expand
// CTA = MT tiles of 128 slots inside one near-field group (one node per
// level).  K = [near field: G columns][level nf: sr_pad]...[level 1]; blocks
// of KB columns never cross a segment.  Producers copy A (MN-major, from the
// [column][slot] layouts) and B (from xprep / ttprep) with cp.async through a
// 4-stage ring; one thread issues the MMAs; the producers read the
// accumulators out and write y.
template <int ST, int NP, int MT>
__global__ void __launch_bounds__(kThreads) tc_expand_kernel(const MatvecArgs a) {
    constexpr bool SPLIT = ST == ST_BF16X2;
    constexpr int KB = SPLIT ? 16 : 32;     // 20 KB stages: two CTAs per SM
    constexpr unsigned ALBO = 128, ASBO = (KB / 8) * 128;
    constexpr unsigned ATILE = 16 * ASBO;
    constexpr unsigned ABYTES = MT * ATILE;
    constexpr unsigned BSBO = (KB / 8) * 128, BBYTES = NP * KB * 2;
    constexpr unsigned STAGE = (SPLIT ? 2 : 1) * (ABYTES + BBYTES);
    // two accumulators per M-tile: low-rank levels, and the near field (which
    // gets its group's dense-block scale at readout)
    constexpr unsigned TCOLS = (2 * MT * NP) <= 32 ? 32 : (2 * MT * NP) <= 64 ? 64
                             : (2 * MT * NP) <= 128 ? 128 : 256;
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ uint64_t full[kStages], empty[kStages], accum;
    __shared__ unsigned s_tmem;
    __shared__ int s_seg[kMaxLevels + 2];      // first block of each segment
    __shared__ int64_t s_abase[kMaxLevels + 1];
    __shared__ int64_t s_node[kMaxLevels + 1];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int TE = 128 * MT;
    const int64_t e0 = (int64_t)blockIdx.x * TE;
    const int64_t G = a.G;
    const int64_t g = e0 / G;
    const int tile = (int)a.tile_p;

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            bar_init(&full[s], kProducers);
            bar_init(&empty[s], 1);
        }
        bar_init(&accum, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
        // segment q: 0 = near field, q >= 1 = level nf + 1 - q
        int b = 0;
        s_seg[0] = 0;
        b += (int)((G + KB - 1) / KB);
        for (int q = 1; q <= a.nf; ++q) {
            s_seg[q] = b;
            const int srp = (a.s * a.lv[a.nf + 1 - q].r + 15) / 16 * 16;
            b += (srp + KB - 1) / KB;
        }
        s_seg[a.nf + 1] = b;
    }
    if (tid <= a.nf) {
        if (tid == 0) {
            s_abase[0] = g * G * G + (e0 - g * G);
            s_node[0] = g;
        } else {
            const DevLevel& L = a.lv[tid];
            const int64_t i = e0 / L.n;
            s_abase[tid] = L.fac_off + i * (int64_t)a.s * L.r * L.n + (e0 - i * L.n);
            s_node[tid] = i;
        }
    }
    if (warp == 4) tmem_alloc(&s_tmem, TCOLS);
    fence_before();
    __syncthreads();
    fence_after();
    const unsigned tmem = s_tmem;
    const int nblk = s_seg[a.nf + 1];
    bool ok = true;

    if (warp < 4) {
        // ---- producers
        for (int b = 0; b < nblk; ++b) {
            const int s = b % kStages;
            if (b >= kStages && ok && !bar_wait(&empty[s], (unsigned)((b / kStages) - 1) & 1u)) ok = false;
            if (!ok) break;
            int q = 0;
            while (s_seg[q + 1] <= b) ++q;
            const int c0 = (b - s_seg[q]) * KB;
            const int l = q == 0 ? 0 : a.nf + 1 - q;
            const int sr = q == 0 ? (int)G : a.s * a.lv[l].r;
            const int srp = q == 0 ? (int)G : (sr + 15) / 16 * 16;
            const int kb = min(KB, srp - c0);
            const int64_t stride = q == 0 ? G : a.lv[l].n;
            const int64_t abase = s_abase[l] + (int64_t)c0 * stride;
            unsigned char* A = sm + (size_t)s * STAGE;
            unsigned char* Alo = A + ABYTES;
            unsigned char* B = A + (SPLIT ? 2 : 1) * ABYTES;
            unsigned char* Blo = B + BBYTES;
            const bool fp8_a = ST == ST_FP8 && q > 0;
            // A: KB columns x TE slots, chunk = 8 slots of one column
            constexpr int M8 = 16 * MT;
            for (int e = tid; e < KB * M8; e += kProducers) {
                const int kc = e / M8, m8 = e - kc * M8;
                const unsigned aoff = (m8 >> 4) * ATILE + (m8 & 15) * ASBO + (kc >> 3) * ALBO + (kc & 7) * 16;
                const bool valid = kc < kb && c0 + kc < sr;
                const int64_t elem = valid ? abase + (int64_t)kc * stride + m8 * 8 : 0;
                if (fp8_a) {
                    uint4 lo8 = make_uint4(0, 0, 0, 0), hi8;
                    if (valid) {
                        const uint2 raw = __ldg(reinterpret_cast<const uint2*>(
                            static_cast<const uint8_t*>(a.U) + elem));
                        fp8x16_to_bf16(make_uint4(raw.x, raw.y, 0, 0), lo8, hi8);
                    }
                    *reinterpret_cast<uint4*>(A + aoff) = lo8;
                } else {
                    const void* src = q == 0 ? a.D : a.U;
                    const void* srcl = q == 0 ? a.D_lo : a.U_lo;
                    cp_async16_z(A + aoff, static_cast<const uint16_t*>(src) + elem, valid);
                    if constexpr (SPLIT) cp_async16_z(Alo + aoff, static_cast<const uint16_t*>(srcl) + elem, valid);
                }
            }
            // B: NP rows x KB columns, chunk = one core row (8 columns)
            for (int e = tid; e < NP * (KB / 8); e += kProducers) {
                const int n = e / (KB / 8), k8 = e - n * (KB / 8);
                const unsigned boff = (n >> 3) * BSBO + k8 * 128 + (n & 7) * 16;
                const bool valid = k8 * 8 < kb;
                int64_t at = 0;
                if (valid) {
                    if (q == 0) {
                        const int64_t gs = g * G + c0 + k8 * 8;           // slot of the column
                        const int64_t t = gs / tile;
                        at = t * kNPMax * tile + core_elem(n, (int)(gs - t * tile), tile);
                    } else {
                        at = a.lv[l].tt_off + s_node[l] * kNPMax * srp + core_elem(n, c0 + k8 * 8, srp);
                    }
                }
                const uint16_t* src = static_cast<const uint16_t*>(q == 0 ? a.xprep : a.ttprep);
                cp_async16_z(B + boff, src + at, valid);
                if constexpr (SPLIT) {
                    const uint16_t* srcl = static_cast<const uint16_t*>(q == 0 ? a.xprep_lo : a.ttprep_lo);
                    cp_async16_z(Blo + boff, srcl + at, valid);
                }
            }
            if (fp8_a) {
                cp_async_wait_all();
                fence_async_smem();
                bar_arrive(&full[s]);
            } else {
                bar_arrive_cp_async(&full[s]);
            }
        }
        // ---- epilogue: lane = slot
        if (ok && !bar_wait(&accum, 0)) ok = false;
        ok = __all_sync(0xffffffffu, ok);
        fence_after();
        if (ok) {
            float* __restrict__ y = static_cast<float*>(a.y);
            constexpr int DST = ST == ST_FP8 ? ST_BF16 : ST;
            const float dsc = DST == ST_BF16 ? a.scD[g] : 1.f;
            for (int mt = 0; mt < MT; ++mt) {
                const int64_t slot = e0 + mt * 128 + warp * 32 + lane;
                const int64_t dst = a.map ? a.map[slot] : slot;
                for (int c0 = 0; c0 < NP; c0 += 16) {
                    float v[16], w[16];
                    const unsigned row = tmem + ((unsigned)(warp * 32) << 16);
                    tmem_ld16(row + mt * NP + c0, v);
                    tmem_ld16(row + (MT + mt) * NP + c0, w);
                    if (dst >= 0)
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (c0 + j < a.k) y[dst * a.ldy + c0 + j] = dsc * w[j] + v[j];
                }
            }
        } else if (lane == 0) {
            atomicExch(a.status, 1);
        }
    } else if (lane == 0) {
        // ---- MMA issue
        const unsigned idesc = idesc_bf16(128, NP, true);
        for (int b = 0; b < nblk; ++b) {
            const int s = b % kStages;
            if (!bar_wait(&full[s], (unsigned)(b / kStages) & 1u)) {
                atomicExch(a.status, 1);
                break;
            }
            fence_async_smem();
            fence_after();
            int q = 0;
            while (s_seg[q + 1] <= b) ++q;
            const int c0 = (b - s_seg[q]) * KB;
            const int srp = q == 0 ? (int)G : (a.s * a.lv[a.nf + 1 - q].r + 15) / 16 * 16;
            const int kb = min(KB, srp - c0);
            unsigned char* A = sm + (size_t)s * STAGE;
            unsigned char* Alo = A + ABYTES;
            unsigned char* B = A + (SPLIT ? 2 : 1) * ABYTES;
            unsigned char* Blo = B + BBYTES;
            for (int ks = 0; ks < kb / 16; ++ks) {
                const unsigned bk = smem_u32(B) + ks * 2 * 128;
                const unsigned bk_lo = smem_u32(Blo) + ks * 2 * 128;
#pragma unroll
                for (int mt = 0; mt < MT; ++mt) {
                    const unsigned ak = smem_u32(A) + mt * ATILE + ks * 2 * ALBO;
                    const unsigned ak_lo = smem_u32(Alo) + mt * ATILE + ks * 2 * ALBO;
                    // near field (segment 0) and levels in separate accumulators
                    const unsigned d = tmem + (q == 0 ? MT + mt : mt) * NP;
                    const int first = q == 0 ? 0 : s_seg[1];
                    const unsigned acc = (b > first || ks > 0) ? 1u : 0u;
                    mma_bf16(d, smem_desc(ak, ALBO, ASBO), smem_desc(bk, 128, BSBO), idesc, acc);
                    if constexpr (SPLIT) {
                        mma_bf16(d, smem_desc(ak, ALBO, ASBO), smem_desc(bk_lo, 128, BSBO), idesc, 1u);
                        mma_bf16(d, smem_desc(ak_lo, ALBO, ASBO), smem_desc(bk, 128, BSBO), idesc, 1u);
                    }
                }
            }
            mma_commit(&empty[s]);
        }
        mma_commit(&accum);
    }
    cp_async_wait_all();
    fence_before();
    __syncthreads();
    if (warp == 4) tmem_dealloc(tmem, TCOLS);
}

// tensor-memory columns of the project kernel: every (level, column block)
// accumulator at once, NP columns each (power of two, at least 32)
unsigned project_tcols(const MatvecArgs& a, int NP) {
    int blocks = 0;
    for (int l = 1; l <= a.nf; ++l) blocks += (a.s * a.lv[l].r + 127) / 128;
    const unsigned need = (unsigned)(blocks * NP);
    unsigned c = 32;
    while (c < need) c *= 2;
    return c;
}

template <int ST, int NP, int MT>
int run_expand(const MatvecArgs& a, cudaStream_t st) {
    constexpr bool SPLIT = ST == ST_BF16X2;
    constexpr int KB = SPLIT ? 16 : 32;
    const size_t stage = (SPLIT ? 2 : 1) * ((size_t)MT * 16 * (KB / 8) * 128 + (size_t)NP * KB * 2);
    const size_t smem = kStages * stage;
    static bool done = false;
    if (!done) {
        const cudaError_t e = cudaFuncSetAttribute(tc_expand_kernel<ST, NP, MT>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return (int)e;
        done = true;
    }
    const unsigned grid = (unsigned)(a.Np / (128 * MT));
    tc_expand_kernel<ST, NP, MT><<<grid, kThreads, smem, st>>>(a);
    return (int)cudaGetLastError();
}


// TMA-fed project (bf16 family, swizzled V maps present); ring depth S
template <int ST, int NP>
int run_project_tma(const MatvecArgs& a0, cudaStream_t st, int R, int grid, int ntile) {
    constexpr bool SPLIT = ST == ST_BF16X2;
    constexpr size_t STAGE = (SPLIT ? 2 : 1) * 128 * 128;
    constexpr size_t XCH = (SPLIT ? 2 : 1) * (size_t)NP * 64 * 2;
    const size_t budget = 220 * 1024 - kXRing * XCH;
    int S = (int)(budget / STAGE);
    S = S > 16 ? 16 : S;
    if (S < 3) return (int)cudaErrorInvalidConfiguration;
    const size_t smem = (size_t)S * STAGE + kXRing * XCH;
    static bool done = false;
    if (!done) {
        const cudaError_t e = cudaFuncSetAttribute(tc_project_tma<ST, NP>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, 222 * 1024);
        if (e != cudaSuccess) return (int)e;
        done = true;
    }
    tc_project_tma<ST, NP><<<grid, kTmaThreads, smem, st>>>(a0, project_tcols(a0, NP), ntile, R, S);
    return (int)cudaGetLastError();
}

template <int ST, int NP>
int run_project(const MatvecArgs& a0, cudaStream_t st) {
    constexpr bool SPLIT = ST == ST_BF16X2;
    constexpr int S = SPLIT ? 3 : 4;
    const size_t smem = (size_t)S * (SPLIT ? 2 : 1) * 16 * 1024 + 2 * (SPLIT ? 2 : 1) * (size_t)NP * a0.tile_p * 2;
    static bool done = false;
    if (!done) {
        const cudaError_t e = cudaFuncSetAttribute(tc_project_persistent<ST, NP, S>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, 226 * 1024);
        if (e != cudaSuccess) return (int)e;
        done = true;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
    const int ntile = (int)(a0.Np / a0.tile_p);
    const int R = (ntile + sms - 1) / sms;
    const int grid = (ntile + R - 1) / R;
    MatvecArgs a = a0;
    a.tc_range = R;
    {
        const int64_t items = (int64_t)ntile * (a.tile_p / 8) * NP;
        tc_xprep_kernel<SPLIT><<<(unsigned)((items + 255) / 256), 256, 0, st>>>(a, NP);
    }
    if constexpr (ST == ST_BF16 || ST == ST_BF16X2) {
        if (a.tmaps_tc) {
            const int rc = run_project_tma<ST, NP>(a, st, R, grid, ntile);
            if (rc != 0) return rc;
        } else {
            tc_project_persistent<ST, NP, S><<<grid, kPThreads, smem, st>>>(a, project_tcols(a, NP), ntile, R);
        }
    } else {
        tc_project_persistent<ST, NP, S><<<grid, kPThreads, smem, st>>>(a, project_tcols(a, NP), ntile, R);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return (int)e;
    // Step 2 for the levels whose nodes span several ranges
    int chunks = 1;
    bool any = false;
    for (int l = 1; l <= a.nf; ++l)
        if (a.lv[l].nsub > 1 && a.lv[l].r > 0) {
            any = true;
            chunks = std::max(chunks, (a.s * a.lv[l].r * a.kc + kRedThreads - 1) / kRedThreads);
        }
    const int64_t rblocks = any && grid > 1 ? (int64_t)a.nf * (grid - 1) * chunks : 0;
    if (rblocks > 0) tc_reduce_kernel<<<(unsigned)rblocks, kRedThreads, 0, st>>>(a, grid, chunks);
    // Steps 3-4: summed t of every target node, bf16
    int64_t items = 0;
    const int np = (a.k + 15) / 16 * 16;
    for (int l = 1; l <= a.nf; ++l) {
        const int srp = (a.s * a.lv[l].r + 15) / 16 * 16;
        items += (a.Np / a.lv[l].n) * np * (srp / 8);
    }
    const unsigned pgrid = (unsigned)((items + 255) / 256);
    if (pgrid > 0) tc_tt_prep_kernel<ST><<<pgrid, 256, 0, st>>>(a);
    return (int)cudaGetLastError();
}

template <int ST, int NP>
int tc_launch_np(int which, const MatvecArgs& a, cudaStream_t st) {
    if (which == 0) return a.nf > 0 ? run_project<ST, NP>(a, st) : 0;
    if (a.G % 256 == 0 && a.Np % 256 == 0) return run_expand<ST, NP, 2>(a, st);
    return run_expand<ST, NP, 1>(a, st);
}

template <int ST>
int tc_launch_st(int which, const MatvecArgs& a, cudaStream_t st) {
    const int np = (a.k + 15) / 16 * 16;
    switch (np) {
        case 16: return tc_launch_np<ST, 16>(which, a, st);
        case 32: return tc_launch_np<ST, 32>(which, a, st);
        case 48: return tc_launch_np<ST, 48>(which, a, st);
        case 64: return tc_launch_np<ST, 64>(which, a, st);
    }
    return (int)cudaErrorInvalidValue;
}

}  // namespace

bool tc_eligible(const MatvecArgs& a) {
    if (a.store != ST_BF16 && a.store != ST_BF16X2 && a.store != ST_FP8) return false;
    if (!a.xprep || !a.ttprep || !a.status) return false;
    if (a.nf < 1 || a.k > kNPMax) return false;
    if (a.G % 128 != 0 || a.Np % 128 != 0 || a.tile_p % 64 != 0) return false;
    if (a.G % a.tile_p != 0) return false;                 // near field = whole x tiles
    for (int l = 1; l <= a.nf; ++l)
        if (a.lv[l].n < a.tile_p) return false;            // a project tile lies in one node
    if (project_tcols(a, (a.k + 15) / 16 * 16) > 512) return false;
    int nacc = 0;
    for (int l = 1; l <= a.nf; ++l) nacc += (a.s * a.lv[l].r + 127) / 128;
    if (nacc > kMaxAcc) return false;
    const bool split = a.store == ST_BF16X2;
    const size_t psm = (size_t)(split ? 3 : 4) * (split ? 2 : 1) * 16 * 1024 +
                       2 * (split ? 2 : 1) * (size_t)kNPMax * a.tile_p * 2;
    return psm <= 226 * 1024;
}

int tc_launch(int which, const MatvecArgs& a, int* /*status*/, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (a.store) {
        case ST_BF16: return tc_launch_st<ST_BF16>(which, a, st);
        case ST_BF16X2: return tc_launch_st<ST_BF16X2>(which, a, st);
        case ST_FP8: return tc_launch_st<ST_FP8>(which, a, st);
    }
    return (int)cudaErrorNotSupported;
}

}  // namespace hm
