// Tensor-core (tcgen05) kernels of the H-matrix-vector product for several
// right-hand sides, where both steps are dense contractions.  One product
// is four launches:
//
//   tc_xprep_kernel: x of every project tile as the bf16 B operand (64
//     rows per 64-slot chunk, chunk-major, rows past k zero; split storage
//     also the low parts).
//   project (Step 1, eq. (prod-vx)): T_seg[cols x k] = V_seg^T X_seg per
//     level and 128-column block, A = V (K-major, straight from the
//     [column][slot] layout), B = the prepared x.  Persistent CTAs own
//     ranges of R tiles; accumulators stay in tensor memory across a
//     range's tiles inside one node and are flushed at node or range ends
//     (a node sum, or a partial at the range start).  tc_project_tma moves
//     every operand with the copy engines (tensor-map boxes of V in the
//     128-byte swizzle, one bulk copy per x chunk);
//     tc_project_persistent is the cp.async form for geometries without the
//     swizzled maps.
//     A node sum goes straight to its target's bf16 B operand of the
//     expand (Steps 3-4, tt_store: the sums t_{i<-j} of i's siblings, times
//     i's U scales); a partial goes to the partial-sum buffer.
//   tc_reduce_kernel (Steps 2-4): the sums of the nodes that span ranges,
//     from their partials in increasing tile order, to the B operand.
//   expand (Step 5, eqs. (prod-yuz), (prod-ydz)):
//     Y_tile[slots x k] = D_g X_g + sum_l U_l T_l, A = D or U^l (MN-major,
//     from the [column][slot] layouts), B = the prepared x or t.
//     tc_expand_tma: tensor-map boxes and bulk copies, double-buffered
//     accumulators so a tile's epilogue overlaps the next tile's MMAs;
//     tc_expand_kernel is the cp.async form.
//
// Operands are bf16 (kind::f16, float accumulation in tensor memory).  Split
// storage runs three MMAs per step (A_hi B_hi + A_hi B_lo + A_lo B_hi, with x
// and t split the same way); e4m3 factors arrive raw and converter warps
// widen them to bf16 (exactly) in shared memory.  One thread issues the
// MMAs; tcgen05.commit arrives on an mbarrier per shared-memory stage; every
// wait is bounded and reports through a status word instead of hanging;
// tensor memory is always released.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "hm_device.h"
#include "hm_once.h"

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

// Bring a tensor map (in global memory) into the copy engine's descriptor
// cache ahead of its first use.
__device__ __forceinline__ void prefetch_map(const void* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(map) : "memory");
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
// try_wait until the phase completes or the hint runs out); false once two
// seconds have passed on the global timer.
__device__ __forceinline__ bool bar_wait(uint64_t* bar, unsigned parity) {
    if (bar_try(bar, parity, 0)) return true;
    uint64_t t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (unsigned it = 0; it < (1u << 30); ++it) {
        if (bar_try(bar, parity, 100000)) return true;
        if ((it & 15) == 15) {
            uint64_t t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            if (t - t0 > 2000000000ull) return false;
        }
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

// The same load without the wait: several loads go out back to back, then
// one tmem_ld_wait; regs_ready ties every register to that wait (an empty
// asm after it, so that no use of a register moves above the wait).
__device__ __forceinline__ void tmem_ld16_issue(unsigned taddr, unsigned (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%"
        "14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void regs_ready(unsigned (&r)[16]) {
#pragma unroll
    for (int i = 0; i < 16; ++i) asm volatile("" : "+r"(r[i]));
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
// rows, chunk-major): the x of project tile t (64 rows x tile_p slots) at
// t * 64 * tile_p elements of `xprep`, the summed t of target node i of
// level l (64 rows x s r_l columns padded to a multiple of 64) at
// tt_off_l + i * 64 * srp64 of `ttprep`.  Within a region, K chunk c (64
// columns) is 64 x 64 contiguous elements; in it core (n/8, k/8) of 8 x 8
// sits at (n/8) * 512 + (k/8) * 64, row n%8 at 8 more -- so the first NP
// rows of a chunk are NP * 64 contiguous elements, one bulk copy, and in
// shared memory core rows along K are 128 bytes apart, row groups 1 KB.
__device__ __forceinline__ int64_t prep_elem(int n, int k) {
    return (int64_t)(k >> 6) * 4096 + (n >> 3) * 512 + ((k & 63) >> 3) * 64 + (n & 7) * 8 + (k & 7);
}

// Steps 3-4 for one value: the sum t of source node j at level L, column
// col (block qv of sibling slot, entry cr), right-hand side n, V scale
// applied, goes to the target node i it is meant for (i reads j's sums at
// j's slot for i) as element (n, k = qp r + cr) of i's prepared bf16 B
// operand, times i's U scale; split storage also the low part.  The padding
// columns k >= s r_l of a region are never written (they stay zero from the
// allocation).
// tt_route: the element of (row 0, k) in i's region and i's U scale, for
// one column of source j; tt_put: one value at row n.
template <int ST>
__device__ __forceinline__ void tt_route(const MatvecArgs& a, const DevLevel& L, int64_t j, int col, int64_t& at0,
                                         float& scale) {
    const int nc = a.s + 1, r = L.r, sr = a.s * r;
    const int cj = (int)(j % nc);
    const int qv = col / r, cr = col - qv * r;
    const int ci = qv < cj ? qv : qv + 1;
    const int64_t i = j - cj + ci;
    const int qp = cj < ci ? cj : cj - 1;
    const int k = qp * r + cr;
    scale = 1.f;
    if constexpr (ST == ST_BF16) scale = a.scU[L.sc_off + i * a.s + qp];
    if constexpr (ST == ST_FP8) scale = a.scU[L.sc_off + i * sr + k];
    const int srp = (sr + 63) / 64 * 64;
    at0 = L.tt_off + i * kNPMax * srp + prep_elem(0, k);
}
template <int ST>
__device__ __forceinline__ void tt_put(const MatvecArgs& a, int64_t at0, int n, float v) {
    const int64_t at = at0 + (n >> 3) * 512 + (n & 7) * 8;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    static_cast<__nv_bfloat16*>(a.ttprep)[at] = h;
    if constexpr (ST == ST_BF16X2)
        static_cast<__nv_bfloat16*>(a.ttprep_lo)[at] = __float2bfloat16_rn(v - __bfloat162float(h));
}
template <int ST>
__device__ __forceinline__ void tt_store(const MatvecArgs& a, const DevLevel& L, int64_t j, int col, int n,
                                         float v) {
    int64_t at0;
    float scale;
    tt_route<ST>(a, L, j, col, at0, scale);
    tt_put<ST>(a, at0, n, v * scale);
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
    // one block per (tile, 256 items): no 64-bit divisions
    const int per_tile = (tile / 8) * np;                  // a multiple of 256 / gcd: see the launch
    const int blocks_per_tile = (per_tile + 255) / 256;
    const int t = (int)(blockIdx.x / blocks_per_tile);
    const int rem = (int)(blockIdx.x - (unsigned)t * blocks_per_tile) * 256 + (int)threadIdx.x;
    if (rem >= per_tile) return;
    const int k8 = rem / np, n = rem - k8 * np;
    const float* __restrict__ x = static_cast<const float*>(a.x);
    unsigned hw[4], lw[4];
#pragma unroll
    for (int q = 0; q < 8; q += 2) {
        float v[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int64_t slot = (int64_t)t * tile + k8 * 8 + q + u;
            const int64_t row = a.map ? a.map[slot] : slot;
            v[u] = (row >= 0 && n < a.k) ? __ldg(x + row * a.ldx + n) : 0.f;
        }
        const uint16_t h0 = bf16_bits(v[0]), h1 = bf16_bits(v[1]);
        hw[q / 2] = (unsigned)h0 | ((unsigned)h1 << 16);
        if constexpr (SPLIT)
            lw[q / 2] = (unsigned)bf16_bits(v[0] - bf16_val(h0)) | ((unsigned)bf16_bits(v[1] - bf16_val(h1)) << 16);
    }
    const int64_t at = (int64_t)t * kNPMax * tile + prep_elem(n, k8 * 8);
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
// flushed when the node ends or the range ends: a node sum (routed to its
// targets' B operand) if the node lies inside the range, else a partial at
// the tile where the covered part starts (tc_reduce_kernel adds those and
// routes the sums).  Within a tile the coarsest level goes first, so the
// flush of the finest level overlaps the next tile's coarse MMAs.
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
    const unsigned XB = (unsigned)NP * tile * 2;            // one x buffer (hi): tile / 64 chunks
    constexpr unsigned XCHUNK = NP * 64 * 2;
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
    // accumulation segments: a.tc_seg tiles from the range start (the last
    // one shorter); accumulators are flushed at segment and node ends
    const int F = a.tc_seg > 0 ? a.tc_seg : R;
    auto seg_begin = [&](int t) { return t_begin + (t - t_begin) / F * F; };
    // does level l close its accumulators after tile t?
    auto flushes = [&](int l, int t) {
        return t == t_end - 1 || (t + 1 - t_begin) % F == 0 || ((int64_t)(t + 1) * tile) % a.lv[l].n == 0;
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
                for (int c = 0; c < tile / 64; ++c) {
                    bulk_g2s(X + c * XCHUNK, xs + c * 4096, XCHUNK, &xfull[xb]);
                    if constexpr (SPLIT)
                        bulk_g2s(Xlo + c * XCHUNK,
                                 static_cast<const uint16_t*>(a.xprep_lo) + (int64_t)t * kNPMax * tile + c * 4096,
                                 XCHUNK, &xfull[xb]);
                }
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
        if (!ok && lane == 0) atomicCAS(a.status, 0, 0x301);
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
                const int64_t sb = seg_begin(t), se = min(sb + F, (int64_t)t_end);
                const bool whole = nstart >= sb && nend <= se;
                const int64_t pslot = nstart > sb ? nstart : sb;
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
                    float* dst = T + (L.part_off + pslot * sr + col) * a.kc;
                    const bool vec = (a.kc % 4 == 0);
                    int64_t tat = 0;
                    float tsc = 0.f;
                    if (whole && col < sr) {
                        tt_route<ST>(a, L, node, col, tat, tsc);
                        tsc *= sc;
                    }
                    for (int c0 = 0; c0 < NP; c0 += 16) {
                        float v[16];
                        tmem_ld16(tmem + ((unsigned)(ew * 32) << 16) + (unsigned)ai * NP + c0, v);
                        if (col >= sr) continue;
                        if (whole) {
                            // a node sum: straight to its target's B operand
#pragma unroll
                            for (int j = 0; j < 16; ++j)
                                if (c0 + j < a.k) tt_put<ST>(a, tat, c0 + j, v[j] * tsc);
                            continue;
                        }
#pragma unroll
                        for (int j = 0; j < 16; j += 4) {
                            if (vec && c0 + j + 4 <= a.k) {
                                *reinterpret_cast<float4*>(dst + c0 + j) =
                                    make_float4(v[j] * sc, v[j + 1] * sc, v[j + 2] * sc, v[j + 3] * sc);
                            } else {
#pragma unroll
                                for (int q = 0; q < 4; ++q)
                                    if (c0 + j + q < a.k) dst[c0 + j + q] = v[j + q] * sc;
                            }
                        }
                    }
                    fence_before();
                    bar_arrive(&aempty[ai]);
                    ++nfl[ai];
                }
            }
        }
        if (!ok && lane == 0) atomicCAS(a.status, 0, 0x301);
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
                    const unsigned bo = (kslot >> 6) * XCHUNK + ((kslot & 63) >> 3) * 128;
                    const unsigned bk = smem_u32(X) + bo;
                    const unsigned bk_lo = smem_u32(Xlo) + bo;
                    const unsigned acc = (fresh[blk] && kc == 0 && ks == 0) ? 0u : 1u;
                    mma_bf16(d, smem_desc(ak, ALBO, ASBO), smem_desc(bk, 128, 1024), idesc, acc);
                    if constexpr (SPLIT) {
                        mma_bf16(d, smem_desc(ak, ALBO, ASBO), smem_desc(bk_lo, 128, 1024), idesc, 1u);
                        mma_bf16(d, smem_desc(ak_lo, ALBO, ASBO), smem_desc(bk, 128, 1024), idesc, 1u);
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
        if (!ok) atomicCAS(a.status, 0, 0x301);
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
// chunk (one bulk copy from the prepared x) and, per
// accumulator block, one tensor-map box of V (64 slots x 128 columns, or
// the level's remaining s r_l mod 128 columns; accumulator rows past the
// box are never stored) in the 128-byte swizzle the MMA reads directly.
//   warp 0: producer (one thread), warp 1: tensor memory + MMA issue (one
//   thread), warps 2-5: epilogue (tensor-memory lane quarter = warp % 4).
// e4m3 storage: the boxes of V arrive raw (64 bytes x rows) in a ring of
// their own; warps 6-9 widen them to bf16 (exact) in the swizzled layout,
// one row per thread, and release the stage to the MMA.
constexpr int kTmaThreads = 192;
constexpr int kTmaThreadsF8 = 320;
constexpr int kRawRingMax = 16;            // raw e4m3 ring slots (at most)
constexpr int kXRing = 3;
constexpr int kTmaStagesMax = 32;

template <int ST, int NP>
__global__ void __launch_bounds__(ST == ST_FP8 ? kTmaThreadsF8 : kTmaThreads, 1)
    tc_project_tma(const MatvecArgs a, unsigned tcols, int ntile, int R, int S, unsigned ABOX, int cps, int SR,
                   unsigned RAWB, int XR) {
    constexpr bool SPLIT = ST == ST_BF16X2;
    constexpr bool F8 = ST == ST_FP8;
    constexpr int PARTS = SPLIT ? 2 : 1;
    // ABOX: bytes of the largest V box (rows x 128 bytes, a multiple of 1 KB);
    // a stage holds cps consecutive 64-slot chunks: [part][chunk] boxes
    const unsigned STAGE = PARTS * cps * ABOX;
    constexpr unsigned XPART = NP * 64 * 2;                // x chunk: NP rows x 64 slots
    const unsigned XCH = PARTS * cps * XPART;             // an x ring slot: [part][chunk]
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ uint64_t full[kTmaStagesMax], empty[kTmaStagesMax], xfull[kXRing], xempty[kXRing],
        afull[kMaxAcc], aempty[kMaxAcc];
    // raw e4m3 ring: SR slots of cps boxes of RAWB bytes (the largest box's
    // rows x 64 bytes)
    __shared__ uint64_t rfull[F8 ? kRawRingMax : 1], rempty[F8 ? kRawRingMax : 1];
    __shared__ unsigned s_tmem;
    __shared__ int s_acc[kMaxLevels + 2];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tile = (int)a.tile_p;
    const int t_begin = blockIdx.x * R;
    const int t_end = min(t_begin + R, ntile);
    unsigned char* xring = sm + (size_t)S * STAGE;
    unsigned char* rawring = xring + (size_t)XR * XCH;           // e4m3: SR slots of cps raw boxes
    float* __restrict__ T = static_cast<float*>(a.T);
    const int nchunk = tile / 64;

    if (tid == 0) {
        for (int q = 0; q < S; ++q) {
            bar_init(&full[q], F8 ? 4 : 1);
            bar_init(&empty[q], 1);
        }
        if constexpr (F8)
            for (int q = 0; q < SR; ++q) {
                bar_init(&rfull[q], 1);
                bar_init(&rempty[q], 4);
            }
        for (int q = 0; q < XR; ++q) {
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
    // accumulation segments: a.tc_seg tiles from the range start (the last
    // one shorter); accumulators are flushed at segment and node ends
    const int F = a.tc_seg > 0 ? a.tc_seg : R;
    auto seg_begin = [&](int t) { return t_begin + (t - t_begin) / F * F; };
    auto flushes = [&](int l, int t) {
        return t == t_end - 1 || (t + 1 - t_begin) % F == 0 || ((int64_t)(t + 1) * tile) % a.lv[l].n == 0;
    };

    if (warp == 0) {
        // ------------------------------------------------------ producer
        bool ok = true;
        if (lane == 0) {
            const unsigned char* maps = static_cast<const unsigned char*>(a.tmaps_tc);
            for (int l = 1; l <= a.nf; ++l) {
                const int sr = a.s * a.lv[l].r;
                if (sr == 0) continue;
                for (int part = 0; part < (F8 ? 1 : PARTS); ++part) {
                    const int k0 = F8 ? kMapV8 : kMapVSw + part, k1 = F8 ? kMapV8Rem : kMapVSwRem + part;
                    prefetch_map(maps + ((size_t)k0 * (kMaxLevels + 1) + l) * kTensorMapBytes);
                    if (sr % 128 != 0) prefetch_map(maps + ((size_t)k1 * (kMaxLevels + 1) + l) * kTensorMapBytes);
                }
            }
            int g = 0, xc = 0;
            for (int t = t_begin; t < t_end && ok; ++t) {
                const int64_t p0 = (int64_t)t * tile;
                for (int kc = 0; kc < nchunk && ok; kc += cps, ++xc) {
                    const int xi = xc % XR;
                    if (xc >= XR && !bar_wait(&xempty[xi], (unsigned)((xc / XR) - 1) & 1u)) { ok = false; break; }
                    unsigned char* X = xring + (size_t)xi * XCH;
                    bar_arrive_tx(&xfull[xi], XCH);
                    for (int c = 0; c < cps; ++c) {
                        const int64_t xo = (int64_t)t * kNPMax * tile + (int64_t)(kc + c) * 4096;
                        bulk_g2s(X + c * XPART, static_cast<const uint16_t*>(a.xprep) + xo, XPART, &xfull[xi]);
                        if constexpr (SPLIT)
                            bulk_g2s(X + (cps + c) * XPART, static_cast<const uint16_t*>(a.xprep_lo) + xo, XPART,
                                     &xfull[xi]);
                    }
                    for (int l = 1; l <= a.nf; ++l) {
                        const DevLevel& L = a.lv[l];
                        const int sr = a.s * L.r;
                        const int64_t node = p0 / L.n;
                        const int x = (int)(p0 - node * L.n) + kc * 64;
                        for (int cb = 0; cb < s_acc[l + 1] - s_acc[l]; ++cb, ++g) {
                            const int rows = sr - cb * 128 < 128 ? sr - cb * 128 : 128;
                            const int y = (int)(node * sr + cb * 128);
                            if constexpr (F8) {
                                const int rs = g % SR;
                                if (g >= SR && !bar_wait(&rempty[rs], (unsigned)((g / SR) - 1) & 1u)) { ok = false; break; }
                                bar_arrive_tx(&rfull[rs], (unsigned)(rows * 64 * cps));
                                for (int c = 0; c < cps; ++c)
                                    tma_load_2d(rawring + ((size_t)rs * cps + c) * RAWB,
                                                maps + ((size_t)(rows == 128 ? kMapV8 : kMapV8Rem) * (kMaxLevels + 1) + l) *
                                                           kTensorMapBytes,
                                                x + c * 64, y, &rfull[rs]);
                                continue;
                            }
                            const int s = g % S;
                            if (g >= S && !bar_wait(&empty[s], (unsigned)((g / S) - 1) & 1u)) { ok = false; break; }
                            const int kind = rows == 128 ? kMapVSw : kMapVSwRem;
                            unsigned char* A = sm + (size_t)s * STAGE;
                            bar_arrive_tx(&full[s], (unsigned)(rows * 128 * PARTS * cps));
                            for (int c = 0; c < cps; ++c) {
                                tma_load_2d(A + c * ABOX, maps + ((size_t)kind * (kMaxLevels + 1) + l) * kTensorMapBytes,
                                            x + c * 64, y, &full[s]);
                                if constexpr (SPLIT)
                                    tma_load_2d(A + (cps + c) * ABOX,
                                                maps + ((size_t)(kind + 1) * (kMaxLevels + 1) + l) * kTensorMapBytes,
                                                x + c * 64, y, &full[s]);
                            }
                        }
                        if (!ok) break;
                    }
                }
            }
            // copies still in flight into this CTA's shared memory
            if constexpr (F8) {
                for (int q = (g > SR ? g - SR : 0); q < g; ++q) bar_wait(&rfull[q % SR], (unsigned)(q / SR) & 1u);
            } else {
                for (int q = (g > S ? g - S : 0); q < g; ++q) bar_wait(&full[q % S], (unsigned)(q / S) & 1u);
            }
            for (int q = (xc > XR ? xc - XR : 0); q < xc; ++q)
                bar_wait(&xfull[q % XR], (unsigned)(q / XR) & 1u);
        }
        if (!ok && lane == 0) atomicCAS(a.status, 0, 0x302);
    } else if (warp == 1) {
        // ------------------------------------------------------ MMA issue
        if (lane == 0) {
            const unsigned idesc = idesc_bf16(128, NP, false);
            // per accumulator, in registers: no MMA since the last flush
            // (fresh), flushed at least once (used), parity of the flushes
            unsigned fresh = 0xffu, used = 0u, par = 0u;
            bool ok = true;
            int g = 0, xc = 0;
            for (int t = t_begin; t < t_end && ok; ++t) {
                for (int kc = 0; kc < nchunk && ok; kc += cps, ++xc) {
                    const int xi = xc % XR;
                    if (!bar_wait(&xfull[xi], (unsigned)(xc / XR) & 1u)) { ok = false; break; }
                    const unsigned char* X = xring + (size_t)xi * XCH;
                    for (int ai = 0; ai < nacc; ++ai, ++g) {
                        const int s = g % S;
                        const unsigned bit = 1u << ai;
                        // wait for the epilogue to drain the flushed accumulator
                        if (kc == 0 && (fresh & used & bit) &&
                            !bar_wait(&aempty[ai], ((par >> ai) & 1u) ^ 1u)) { ok = false; break; }
                        if (!bar_wait(&full[s], (unsigned)(g / S) & 1u)) { ok = false; break; }
                        fence_after();
                        const unsigned A0 = smem_u32(sm + (size_t)s * STAGE);
                        const unsigned B0 = smem_u32(X);
                        const unsigned d = tmem + (unsigned)ai * NP;
                        for (int c = 0; c < cps; ++c) {
                            const unsigned A = A0 + c * ABOX, B = B0 + c * XPART;
#pragma unroll
                            for (int ks = 0; ks < 4; ++ks) {
                                const uint64_t ad = smem_desc_sw128(A + ks * 32, 16, 1024);
                                const uint64_t bd = smem_desc(B + ks * 256, 128, 1024);
                                const unsigned accf = ((fresh & bit) && kc == 0 && c == 0 && ks == 0) ? 0u : 1u;
                                mma_bf16(d, ad, bd, idesc, accf);
                                if constexpr (SPLIT) {
                                    mma_bf16(d, ad, smem_desc(B0 + (cps + c) * XPART + ks * 256, 128, 1024), idesc, 1u);
                                    mma_bf16(d, smem_desc_sw128(A0 + (cps + c) * ABOX + ks * 32, 16, 1024), bd, idesc,
                                             1u);
                                }
                            }
                        }
                        if (kc == 0) fresh &= ~bit;
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
                        fresh |= 1u << ai;
                        used |= 1u << ai;
                        par ^= 1u << ai;
                    }
                }
            }
            if (!ok) atomicCAS(a.status, 0, 0x302);
        }
    } else if (F8 && warp >= 6) {
        // ------------------------------------------------------ e4m3 -> bf16
        bool ok = true;
        const int row = (warp - 6) * 32 + lane;
        int g = 0;
        for (int t = t_begin; t < t_end && ok; ++t)
            for (int kc = 0; kc < nchunk && ok; kc += cps)
                for (int ai = 0; ai < nacc && ok; ++ai, ++g) {
                    const int rs = g % SR, s = g % S;
                    if (!bar_wait(&rfull[rs], (unsigned)(g / SR) & 1u)) ok = false;
                    if (ok && g >= S && !bar_wait(&empty[s], (unsigned)((g / S) - 1) & 1u)) ok = false;
                    ok = __all_sync(0xffffffffu, ok);
                    if (!ok) break;
                    // rows of this accumulator's box: a stage chunk holds ABOX
                    // bytes (the largest box), so rows past the box are not
                    // written (the accumulator rows they feed are never stored)
                    int l = 1;
                    while (s_acc[l + 1] <= ai) ++l;
                    const int brows = min(128, a.s * a.lv[l].r - (ai - s_acc[l]) * 128);
                    for (int c = 0; c < cps && row < brows; ++c) {
                        const uint4* src =
                            reinterpret_cast<const uint4*>(rawring + ((size_t)rs * cps + c) * RAWB + row * 64);
                        unsigned char* dst = sm + (size_t)s * STAGE + c * ABOX + row * 128;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            uint4 lo8, hi8;
                            fp8x16_to_bf16(src[q], lo8, hi8);
                            // 16-byte chunk j of the row goes to chunk j ^ (row % 8) (128-byte swizzle)
                            *reinterpret_cast<uint4*>(dst + (((2 * q) ^ (row & 7)) << 4)) = lo8;
                            *reinterpret_cast<uint4*>(dst + (((2 * q + 1) ^ (row & 7)) << 4)) = hi8;
                        }
                    }
                    fence_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        bar_arrive(&rempty[rs]);
                        bar_arrive(&full[s]);
                    }
                }
        if (!ok && lane == 0) atomicCAS(a.status, 0, 0x305);
    } else {
        // ------------------------------------------------------ epilogue
        const int q4 = warp & 3;                        // tensor-memory lane quarter
        unsigned par = 0u;                               // parity of each accumulator's flushes
        bool ok = true;
        for (int t = t_begin; t < t_end && ok; ++t) {
            const int64_t p0 = (int64_t)t * tile;
            for (int l = 1; l <= a.nf && ok; ++l) {
                if (!flushes(l, t)) continue;
                const DevLevel& L = a.lv[l];
                const int sr = a.s * L.r;
                const int64_t node = p0 / L.n;
                const int64_t nstart = node * L.n / tile, nend = (node + 1) * L.n / tile;   // tiles
                const int64_t sb = seg_begin(t), se = min(sb + F, (int64_t)t_end);
                const bool whole = nstart >= sb && nend <= se;
                const int64_t pslot = nstart > sb ? nstart : sb;
                for (int cb = 0; cb < s_acc[l + 1] - s_acc[l]; ++cb) {
                    const int ai = s_acc[l] + cb;
                    if (!bar_wait(&afull[ai], (par >> ai) & 1u)) ok = false;
                    ok = __all_sync(0xffffffffu, ok);
                    if (!ok) break;
                    fence_after();
                    const int col = cb * 128 + q4 * 32 + lane;
                    float sc = 1.f;
                    if constexpr (ST == ST_BF16) sc = col < sr ? a.scV[L.sc_off + node * a.s + col / L.r] : 0.f;
                    if constexpr (ST == ST_FP8) sc = col < sr ? a.scV[L.sc_off + node * sr + col] : 0.f;
                    float* dst = T + (L.part_off + pslot * sr + col) * a.kc;
                    const bool vec = (a.kc % 4 == 0);
                    int64_t tat = 0;
                    float tsc = 0.f;
                    if (whole && col < sr) {
                        tt_route<ST>(a, L, node, col, tat, tsc);
                        tsc *= sc;
                    }
                    // every chunk of the accumulator at once, one wait, and
                    // the accumulator goes back to the MMAs before the stores
                    unsigned rr[NP / 16][16];
#pragma unroll
                    for (int c = 0; c < NP / 16; ++c)
                        tmem_ld16_issue(tmem + ((unsigned)(q4 * 32) << 16) + (unsigned)ai * NP + c * 16, rr[c]);
                    tmem_ld_wait();
#pragma unroll
                    for (int c = 0; c < NP / 16; ++c) regs_ready(rr[c]);
                    fence_before();
                    bar_arrive(&aempty[ai]);
                    par ^= 1u << ai;
#pragma unroll
                    for (int c = 0; c < NP / 16; ++c) {
                        const int c0 = c * 16;
                        float v[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(rr[c][j]);
                        if (col >= sr) continue;
                        if (whole) {
                            // a node sum: straight to its target's B operand
#pragma unroll
                            for (int j = 0; j < 16; ++j)
                                if (c0 + j < a.k) tt_put<ST>(a, tat, c0 + j, v[j] * tsc);
                            continue;
                        }
#pragma unroll
                        for (int j = 0; j < 16; j += 4) {
                            if (vec && c0 + j + 4 <= a.k) {
                                *reinterpret_cast<float4*>(dst + c0 + j) =
                                    make_float4(v[j] * sc, v[j + 1] * sc, v[j + 2] * sc, v[j + 3] * sc);
                            } else {
#pragma unroll
                                for (int q = 0; q < 4; ++q)
                                    if (c0 + j + q < a.k) dst[c0 + j + q] = v[j + q] * sc;
                            }
                        }
                    }
                }
            }
        }
        if (!ok && lane == 0) atomicCAS(a.status, 0, 0x302);
    }
    fence_before();
    __syncthreads();
    if (warp == 1) tmem_dealloc(tmem, tcols);
}

// -------------------------------------------------------- Step 2 (k > 1)
// Node sums of the levels' nodes that span accumulation segments of the
// persistent project kernels (ranges of a.tc_range tiles, each cut into
// segments of a.tc_seg tiles from its start; a node inside one segment
// already has its sum).  The partials of a spanning node sit at its first
// tile and at every segment start inside it, and are added in increasing
// tile order, one item (column, right-hand side) per thread.  grid: the
// nodes (level by level) of the levels whose nodes span several tiles,
// times `chunks` blocks of kRedThreads items.
constexpr int kRedThreads = 256;
// The nodes that span segments, listed by the host (level << 24 | node), in
// the launch's parameters: blocks exist only for them.
constexpr int kMaxSpans = 1024;
struct SpanList {
    int n;
    unsigned e[kMaxSpans];
};
template <int ST>
__global__ void __launch_bounds__(kRedThreads) tc_reduce_kernel(const MatvecArgs a, int chunks,
                                                                 const SpanList spans) {
    float* __restrict__ T = static_cast<float*>(a.T);
    const int R = a.tc_range;
    const int F = a.tc_seg > 0 ? a.tc_seg : R;
    const int b = (int)(blockIdx.x / chunks);
    const int chunk = (int)(blockIdx.x % chunks);
    if (b >= spans.n) return;
    const int lvl = (int)(spans.e[b] >> 24);
    if (lvl < 1 || lvl > a.nf) return;
    const DevLevel& L = a.lv[lvl];
    if (L.nsub <= 1 || L.r == 0) return;
    const int node = (int)(spans.e[b] & 0xFFFFFFu), t0 = node * L.nsub, t1 = t0 + L.nsub;
    if ((int64_t)t1 * a.tile_p > a.Np) return;
    // the first segment start after t0: within t0's range, or the next range
    const int c0 = t0 / R;
    int next = c0 * R + ((t0 - c0 * R) / F + 1) * F;
    if (next >= c0 * R + R) next = (c0 + 1) * R;
    if (next >= t1) return;                    // inside one segment: sum already stored
    const int sr = a.s * L.r;
    const int items = sr * a.kc;
    const int item = chunk * kRedThreads + threadIdx.x;
    if (item >= items) return;
    const int64_t stride = (int64_t)sr * a.kc;
    const float* src = T + L.part_off * a.kc + item;
    // partials at t0 and at the segment starts in (t0, t1), increasing
    // (range by range, F apart); partial p goes to accumulator p mod 8 and
    // eight loads are in flight at a time; the accumulators are added in a
    // fixed tree
    float acc[8];
    acc[0] = __ldcg(src + (int64_t)t0 * stride);
#pragma unroll
    for (int q = 1; q < 8; ++q) acc[q] = 0.f;
    int c = next / R, s = next;
    while (s < t1) {
        int ts[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            ts[q] = s;
            if (s < t1) {
                s += F;
                if (s >= (c + 1) * R) s = ++c * R;
            }
        }
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = ts[q] < t1 ? __ldcg(src + (int64_t)ts[q] * stride) : 0.f;
        // partials 1 + 8 m + q: accumulator (q + 1) mod 8
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[(q + 1) & 7] += v[q];
    }
    const float sum = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
    const int col = item / a.kc, n = item - col * a.kc;
    if (n < a.k) tt_store<ST>(a, L, node, col, n, sum);
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
                        at = t * kNPMax * tile + prep_elem(n, (int)(gs - t * tile));
                    } else {
                        const int srp64 = (sr + 63) / 64 * 64;
                        at = a.lv[l].tt_off + s_node[l] * kNPMax * srp64 + prep_elem(n, c0 + k8 * 8);
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
            atomicCAS(a.status, 0, 0x303);
        }
    } else if (lane == 0) {
        // ---- MMA issue
        const unsigned idesc = idesc_bf16(128, NP, true);
        for (int b = 0; b < nblk; ++b) {
            const int s = b % kStages;
            if (!bar_wait(&full[s], (unsigned)(b / kStages) & 1u)) {
                atomicCAS(a.status, 0, 0x303);
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

template <int ST, int NP, int MT>
int run_expand(const MatvecArgs& a, cudaStream_t st);

// ------------------------------------------------- expand, TMA operands
// Steps 3-5 for bf16 and split bf16 storage with every operand moved by the
// copy engines.  CTA c owns the 128-slot expand tiles [c R, c R + R).  Per
// tile the K columns are the G columns of its near-field group, then per
// level the s r_l columns of its target node; per stage of KB columns:
//   A = two tensor-map boxes (slots 0-63, 64-127 of the tile) of D or U^l in
//       the 128-byte swizzle, MN-major (a remainder box rounded up to 16
//       columns: the extra columns meet the zero padding of t, or the
//       copy engine's zero fill past the array);
//   B = the matching chunk of the prepared x (near field) or of the summed t
//       of the target node (levels): one bulk copy.
// Near field and levels accumulate apart (the near field takes its group's
// dense scale at readout), in two tensor-memory buffers alternating between
// tiles so that the epilogue of a tile overlaps the next tile's MMAs.
//   warp 0: producer (one thread), warp 1: tensor memory + MMA issue, warps
//   2-5: epilogue (slot = 32 (warp % 4) + lane).
template <int ST, int NP>
__global__ void __launch_bounds__(ST == ST_FP8 ? kTmaThreadsF8 : kTmaThreads, 1)
    tc_expand_tma(const MatvecArgs a, int ntile, int R, int S, int SR) {
    constexpr bool SPLIT = ST == ST_BF16X2;
    constexpr bool F8 = ST == ST_FP8;           // U arrives raw and is widened by warps 6-9
    constexpr int PARTS = SPLIT ? 2 : 1;
    constexpr int KB = 64;
    constexpr unsigned ABOX = 64 * KB * 2;                 // one box: KB columns x 64 slots
    constexpr unsigned APART = 2 * ABOX;
    constexpr unsigned BPART = NP * KB * 2;
    constexpr unsigned STAGE = PARTS * (APART + BPART);
    constexpr unsigned TCOLS = 4 * NP <= 32 ? 32 : 4 * NP <= 64 ? 64 : 4 * NP <= 128 ? 128 : 256;
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ uint64_t full[16], empty[16], afull[2], aempty[2];
    // raw e4m3 ring: SR slots of two boxes of 4 KB (64 columns x 64 slots)
    constexpr unsigned RAWST = 2 * 64 * 64;
    __shared__ uint64_t rfull[F8 ? kRawRingMax : 1], rempty[F8 ? kRawRingMax : 1];
    __shared__ unsigned s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t G = a.G;
    const int tile_p = (int)a.tile_p;
    const int t_begin = blockIdx.x * R;
    const int t_end = min(t_begin + R, ntile);

    unsigned char* rawring = sm + (size_t)S * STAGE;        // e4m3 only
    if (tid == 0) {
        for (int q = 0; q < S; ++q) {
            bar_init(&full[q], F8 ? 5 : 1);                   // e4m3: the copies + four converter warps
            bar_init(&empty[q], 1);
        }
        for (int q = 0; q < 2; ++q) {
            bar_init(&afull[q], 1);
            bar_init(&aempty[q], 128);
        }
        if constexpr (F8)
            for (int q = 0; q < SR; ++q) {
                bar_init(&rfull[q], 1);
                bar_init(&rempty[q], 4);
            }
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 1) tmem_alloc(&s_tmem, TCOLS);
    fence_before();
    __syncthreads();
    fence_after();
    const unsigned tmem = s_tmem;

    if (warp == 0) {
        // ------------------------------------------------------ producer
        bool ok = true;
        if (lane == 0) {
            const unsigned char* maps = static_cast<const unsigned char*>(a.tmaps_tc);
            auto map = [&](int kind, int l) { return maps + ((size_t)kind * (kMaxLevels + 1) + l) * kTensorMapBytes; };
            for (int part = 0; part < PARTS; ++part) prefetch_map(map(kMapUSw + part, 0));
            for (int l = 1; l <= a.nf; ++l) {
                const int sr = a.s * a.lv[l].r;
                if (sr == 0) continue;
                const bool rem = ((sr + 15) / 16 * 16) % KB != 0;
                for (int part = 0; part < (F8 ? 1 : PARTS); ++part) {
                    prefetch_map(map(F8 ? kMapU8 : kMapUSw + part, l));
                    if (rem) prefetch_map(map(F8 ? kMapU8Rem : kMapUSwRem + part, l));
                }
            }
            int g = 0, gr = 0;                                 // stages, raw e4m3 stages
            for (int t = t_begin; t < t_end && ok; ++t) {
                const int64_t e0 = (int64_t)t * 128;
                const int64_t grp = e0 / G;
                // segment 0: near field; segment l: level l (finest first)
                for (int seg = 0; seg <= a.nf && ok; ++seg) {
                    const int l = seg == 0 ? 0 : a.nf + 1 - seg;
                    const int sr = l == 0 ? (int)G : a.s * a.lv[l].r;
                    if (sr == 0) continue;
                    const int srp = l == 0 ? (int)G : (sr + 15) / 16 * 16;
                    const int srp64 = (srp + 63) / 64 * 64;
                    const int64_t node = l == 0 ? grp : e0 / a.lv[l].n;
                    const int x = (int)(e0 - node * (l == 0 ? G : a.lv[l].n));
                    for (int c0 = 0; c0 < srp; c0 += KB, ++g) {
                        const int s = g % S;
                        if (g >= S && !bar_wait(&empty[s], (unsigned)((g / S) - 1) & 1u)) { ok = false; break; }
                        const int kb = srp - c0 < KB ? srp - c0 : KB;
                        const bool rem = kb < KB;
                        unsigned char* A = sm + (size_t)s * STAGE;
                        unsigned char* B = A + PARTS * APART;
                        const int y = (int)(node * sr + c0);
                        const bool raw = F8 && l > 0;
                        if (raw) {
                            // U boxes raw into the e4m3 ring; the converters fill A
                            const int rs = gr % SR;
                            if (gr >= SR && !bar_wait(&rempty[rs], (unsigned)((gr / SR) - 1) & 1u)) { ok = false; break; }
                            bar_arrive_tx(&rfull[rs], 2u * 64 * kb);
                            const void* mp = map(rem ? kMapU8Rem : kMapU8, l);
                            tma_load_2d(rawring + (size_t)rs * RAWST, mp, x, y, &rfull[rs]);
                            tma_load_2d(rawring + (size_t)rs * RAWST + 64 * 64, mp, x + 64, y, &rfull[rs]);
                            ++gr;
                        }
                        bar_arrive_tx(&full[s], (unsigned)PARTS * ((raw ? 0u : 2u * 64 * kb * 2) + BPART));
                        for (int part = 0; part < PARTS; ++part) {
                            if (!raw) {
                                const void* mp = map((rem ? kMapUSwRem : kMapUSw) + part, l);
                                tma_load_2d(A + part * APART, mp, x, y, &full[s]);
                                tma_load_2d(A + part * APART + ABOX, mp, x + 64, y, &full[s]);
                            }
                            // B: the chunk's NP rows, one bulk copy (zero columns past s r_l)
                            const uint16_t* src;
                            int64_t at0;
                            if (l == 0) {
                                const int64_t slot = grp * G + c0;
                                const int64_t tp = slot / tile_p;
                                src = static_cast<const uint16_t*>(part ? a.xprep_lo : a.xprep);
                                at0 = tp * kNPMax * tile_p + ((slot - tp * tile_p) >> 6) * 4096;
                            } else {
                                src = static_cast<const uint16_t*>(part ? a.ttprep_lo : a.ttprep);
                                at0 = a.lv[l].tt_off + node * kNPMax * srp64 + (c0 >> 6) * 4096;
                            }
                            bulk_g2s(B + part * BPART, src + at0, BPART, &full[s]);
                        }
                    }
                }
            }
            if constexpr (F8)
                for (int q = (gr > SR ? gr - SR : 0); q < gr; ++q) bar_wait(&rfull[q % SR], (unsigned)(q / SR) & 1u);
            for (int q = (g > S ? g - S : 0); q < g; ++q) bar_wait(&full[q % S], (unsigned)(q / S) & 1u);
        }
        if (!ok && lane == 0) atomicCAS(a.status, 0, 0x304);
    } else if (warp == 1) {
        // ------------------------------------------------------ MMA issue
        if (lane == 0) {
            const unsigned idesc = idesc_bf16(128, NP, true);
            bool ok = true;
            int g = 0;
            for (int t = t_begin; t < t_end && ok; ++t) {
                const int u = t - t_begin, ab = u & 1;
                if (u >= 2 && !bar_wait(&aempty[ab], (unsigned)((u >> 1) - 1) & 1u)) { ok = false; break; }
                bool lr_fresh = true;                  // no MMA into the levels' accumulator yet
                for (int seg = 0; seg <= a.nf && ok; ++seg) {
                    const int l = seg == 0 ? 0 : a.nf + 1 - seg;
                    const int sr = l == 0 ? (int)G : a.s * a.lv[l].r;
                    if (sr == 0) continue;
                    const int srp = l == 0 ? (int)G : (sr + 15) / 16 * 16;
                    const unsigned d = tmem + (unsigned)(ab * 2 + (seg == 0 ? 1 : 0)) * NP;
                    for (int c0 = 0; c0 < srp; c0 += KB, ++g) {
                        const int s = g % S;
                        if (!bar_wait(&full[s], (unsigned)(g / S) & 1u)) { ok = false; break; }
                        fence_after();
                        const int kb = srp - c0 < KB ? srp - c0 : KB;
                        const unsigned A = smem_u32(sm + (size_t)s * STAGE);
                        const unsigned B = A + PARTS * APART;
                        for (int ks = 0; ks < kb / 16; ++ks) {
                            const uint64_t ad = smem_desc_sw128(A + ks * 2048, ABOX, 1024);
                            const uint64_t bd = smem_desc(B + ks * 256, 128, 1024);
                            // first step of the near field / of the first level with rank
                            const bool first = seg == 0 ? (c0 == 0 && ks == 0) : lr_fresh;
                            lr_fresh = lr_fresh && seg == 0;
                            mma_bf16(d, ad, bd, idesc, first ? 0u : 1u);
                            if constexpr (SPLIT) {
                                mma_bf16(d, ad, smem_desc(B + BPART + ks * 256, 128, 1024), idesc, 1u);
                                mma_bf16(d, smem_desc_sw128(A + APART + ks * 2048, ABOX, 1024), bd, idesc, 1u);
                            }
                        }
                        mma_commit(&empty[s]);
                    }
                }
                if (!ok) break;
                mma_commit(&afull[ab]);
            }
            if (!ok) atomicCAS(a.status, 0, 0x304);
        }
    } else if (F8 && warp >= 6) {
        // ------------------------------------------------------ e4m3 -> bf16 (U)
        // thread = (box, column): 64 raw slots -> one 128-byte swizzled row
        bool ok = true;
        const int ct = (warp - 6) * 32 + lane, box = ct >> 6, col = ct & 63;
        int g = 0, gr = 0;
        for (int t = t_begin; t < t_end && ok; ++t) {
            for (int seg = 0; seg <= a.nf && ok; ++seg) {
                const int l = seg == 0 ? 0 : a.nf + 1 - seg;
                const int sr = l == 0 ? (int)G : a.s * a.lv[l].r;
                if (sr == 0) continue;
                const int srp = l == 0 ? (int)G : (sr + 15) / 16 * 16;
                for (int c0 = 0; c0 < srp && ok; c0 += KB, ++g) {
                    const int s = g % S;
                    // the slot's previous use must be consumed before this use's
                    // arrivals (also for near-field stages, which need no widening)
                    if (g >= S && !bar_wait(&empty[s], (unsigned)((g / S) - 1) & 1u)) ok = false;
                    ok = __all_sync(0xffffffffu, ok);
                    if (!ok) break;
                    if (l > 0) {
                        const int rs = gr % SR;
                        if (!bar_wait(&rfull[rs], (unsigned)(gr / SR) & 1u)) ok = false;
                        ok = __all_sync(0xffffffffu, ok);
                        if (!ok) break;
                        const uint4* src =
                            reinterpret_cast<const uint4*>(rawring + (size_t)rs * RAWST + box * 64 * 64 + col * 64);
                        unsigned char* dst = sm + (size_t)s * STAGE + box * ABOX + col * 128;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            uint4 lo8, hi8;
                            fp8x16_to_bf16(src[q], lo8, hi8);
                            *reinterpret_cast<uint4*>(dst + (((2 * q) ^ (col & 7)) << 4)) = lo8;
                            *reinterpret_cast<uint4*>(dst + (((2 * q + 1) ^ (col & 7)) << 4)) = hi8;
                        }
                        fence_async_smem();
                        __syncwarp();
                        if (lane == 0) bar_arrive(&rempty[rs]);
                        ++gr;
                    }
                    __syncwarp();
                    if (lane == 0) bar_arrive(&full[s]);
                }
            }
        }
        if (!ok && lane == 0) atomicCAS(a.status, 0, 0x306);
    } else {
        // ------------------------------------------------------ epilogue
        const int q4 = warp & 3;
        float* __restrict__ y = static_cast<float*>(a.y);
        bool ok = true;
        for (int t = t_begin; t < t_end && ok; ++t) {
            const int u = t - t_begin, ab = u & 1;
            if (!bar_wait(&afull[ab], (unsigned)(u >> 1) & 1u)) ok = false;
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            fence_after();
            const int64_t e0 = (int64_t)t * 128;
            const float dsc = (ST == ST_BF16 || ST == ST_FP8) ? a.scD[e0 / G] : 1.f;
            const int64_t slot = e0 + q4 * 32 + lane;
            const int64_t dst = a.map ? a.map[slot] : slot;
            const unsigned row = tmem + ((unsigned)(q4 * 32) << 16);
            float* yr = dst >= 0 ? y + dst * a.ldy : y;
            const bool vec = (a.ldy % 4 == 0) && ((reinterpret_cast<uintptr_t>(y) & 15) == 0);
            // both accumulators at once, one wait, and the buffer goes back
            // to the MMAs before the stores
            unsigned rv[NP / 16][16], rw[NP / 16][16];
#pragma unroll
            for (int c = 0; c < NP / 16; ++c) {
                tmem_ld16_issue(row + (unsigned)(ab * 2) * NP + c * 16, rv[c]);        // levels
                tmem_ld16_issue(row + (unsigned)(ab * 2 + 1) * NP + c * 16, rw[c]);    // near field
            }
            tmem_ld_wait();
#pragma unroll
            for (int c = 0; c < NP / 16; ++c) {
                regs_ready(rv[c]);
                regs_ready(rw[c]);
            }
            fence_before();
            bar_arrive(&aempty[ab]);
#pragma unroll
            for (int c = 0; c < NP / 16; ++c) {
                const int c0 = c * 16;
                float v[16], w[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    v[j] = __uint_as_float(rv[c][j]);
                    w[j] = __uint_as_float(rw[c][j]);
                }
                if (dst < 0) continue;
#pragma unroll
                for (int j = 0; j < 16; j += 4) {
                    if (vec && c0 + j + 4 <= a.k) {
                        *reinterpret_cast<float4*>(yr + c0 + j) =
                            make_float4(dsc * w[j] + v[j], dsc * w[j + 1] + v[j + 1], dsc * w[j + 2] + v[j + 2],
                                        dsc * w[j + 3] + v[j + 3]);
                    } else {
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (c0 + j + q < a.k) yr[c0 + j + q] = dsc * w[j + q] + v[j + q];
                    }
                }
            }
        }
        if (!ok && lane == 0) atomicCAS(a.status, 0, 0x304);
    }
    fence_before();
    __syncthreads();
    if (warp == 1) tmem_dealloc(tmem, TCOLS);
}

template <int ST, int NP>
int run_expand_tma(const MatvecArgs& a, cudaStream_t st) {
    bool any = false;
    for (int l = 1; l <= a.nf; ++l) any = any || a.lv[l].r > 0;
    if (!any) return run_expand<ST, NP, 1>(a, st);
    constexpr bool SPLIT = ST == ST_BF16X2;
    constexpr int KB = 64;
    constexpr size_t STAGE = (SPLIT ? 2 : 1) * ((size_t)2 * 64 * KB * 2 + (size_t)NP * KB * 2);
    // e4m3: the raw ring reads the U boxes from HBM, so it gets the depth
    // (eight slots, 64 KB) while the bf16 stages keep at least four
    constexpr int SR0 = ST == ST_FP8 ? 8 : 0;
    int S = (int)((size_t)(220 * 1024 - (size_t)SR0 * 2 * 64 * 64) / STAGE);
    S = S > 16 ? 16 : S;
    if (S < 3) return (int)cudaErrorInvalidConfiguration;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
    const int ntile = (int)(a.Np / 128);
    const int R = (ntile + sms - 1) / sms;
    const int grid = (ntile + R - 1) / R;
    // rings no deeper than the stages one CTA streams (64-column chunks of
    // the near field and of every level, per tile)
    int SR = SR0;
    {
        int per_tile = (int)(a.G / 64), raw = 0;
        for (int l = 1; l <= a.nf; ++l) {
            const int sr = a.s * a.lv[l].r;
            const int c = ((sr + 15) / 16 * 16 + 63) / 64;
            per_tile += c;
            raw += c;
        }
        const int64_t need = std::max<int64_t>(2, (int64_t)R * per_tile);
        if (S > need) S = (int)need;
        if (SR > 0) SR = (int)std::max<int64_t>(2, std::min<int64_t>(SR, (int64_t)R * raw));
    }
    const size_t smem = (size_t)S * STAGE + (size_t)SR * 2 * 64 * 64;
    static DeviceFlags attr;
    {
        const cudaError_t e = attr.once([&] {
            return cudaFuncSetAttribute(tc_expand_tma<ST, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        222 * 1024);
        });
        if (e != cudaSuccess) return (int)e;
    }
    tc_expand_tma<ST, NP><<<grid, ST == ST_FP8 ? kTmaThreadsF8 : kTmaThreads, smem, st>>>(a, ntile, R, S, SR);
    count_launches(1);
    return (int)cudaGetLastError();
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
    static DeviceFlags attr;
    {
        const cudaError_t e = attr.once([&] {
            return cudaFuncSetAttribute(tc_expand_kernel<ST, NP, MT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem);
        });
        if (e != cudaSuccess) return (int)e;
    }
    const unsigned grid = (unsigned)(a.Np / (128 * MT));
    tc_expand_kernel<ST, NP, MT><<<grid, kThreads, smem, st>>>(a);
    count_launches(1);
    return (int)cudaGetLastError();
}


// TMA-fed project (bf16 family, swizzled V maps present); ring depth S
template <int ST, int NP>
int run_project_tma(const MatvecArgs& a0, cudaStream_t st, int R, int grid, int ntile) {
    constexpr bool SPLIT = ST == ST_BF16X2;
    // stage = the largest V box in use (many small boxes keep as many bytes in flight)
    int maxrows = 8;
    for (int l = 1; l <= a0.nf; ++l) {
        const int sr = a0.s * a0.lv[l].r;
        maxrows = std::max(maxrows, sr >= 128 ? 128 : sr);
    }
    const unsigned abox = (unsigned)((maxrows * 128 + 1023) / 1024 * 1024);
    // four, else two 64-slot chunks per stage when the tile's chunk count
    // allows and at least four stages still fit (less MMA-issue and barrier
    // work per byte, 512 or 256 contiguous bytes per row of V; with four,
    // two x slots instead of three)
    // e4m3: raw boxes of the largest box's rows x 64 bytes; the raw ring is
    // the one that reads HBM, so it gets the depth (about 72 KB in flight)
    const unsigned rawb = (unsigned)((maxrows * 64 + 127) / 128 * 128);
    int cps = 1, S = 0, SR = 0, XR = kXRing;
    size_t smem = 0;
    for (int c = 4; c >= 1 && S == 0; c /= 2) {
        if ((a0.tile_p / 64) % c != 0) continue;
        const int xr = c == 4 ? 2 : kXRing;
        const size_t STAGE = (SPLIT ? 2 : 1) * (size_t)c * abox;
        const size_t XCH = (SPLIT ? 2 : 1) * (size_t)c * NP * 64 * 2;
        // raw ring depths to try, deepest first (none without e4m3)
        const int sr_hi = ST == ST_FP8 ? (int)std::min<size_t>(kRawRingMax, std::max<size_t>(4, (72 * 1024) / (c * rawb)))
                                       : 0;
        const int sr_lo = ST == ST_FP8 ? 4 : 0;
        for (int sr = sr_hi; sr >= sr_lo && S == 0; --sr) {
            const size_t fixed = xr * XCH + (size_t)sr * c * rawb;
            if (fixed >= 220 * 1024) continue;
            int s = (int)((220 * 1024 - fixed) / STAGE);
            s = s > kTmaStagesMax ? kTmaStagesMax : s;
            if (s < (c == 1 ? 3 : 4)) continue;
            cps = c;
            S = s;
            SR = sr;
            XR = xr;
            smem = (size_t)s * STAGE + fixed;
        }
    }
    if (S == 0) return (int)cudaErrorInvalidConfiguration;
    {
        // rings no deeper than the boxes one CTA streams: small products
        // leave room for more CTAs per SM (other products of a batch)
        int nacc = 0;
        for (int l = 1; l <= a0.nf; ++l) nacc += (a0.s * a0.lv[l].r + 127) / 128;
        const int64_t boxes = (int64_t)R * (a0.tile_p / 64 / cps) * nacc;
        const int need = (int)std::max<int64_t>(2, std::min<int64_t>(boxes, kTmaStagesMax));
        if (S > need) S = need;
        if (SR > need) SR = need;
        const size_t STAGE = (SPLIT ? 2 : 1) * (size_t)cps * abox;
        const size_t XCH = (SPLIT ? 2 : 1) * (size_t)cps * NP * 64 * 2;
        smem = (size_t)S * STAGE + XR * XCH + (size_t)SR * cps * rawb;
        // an MMA reads 128 rows (16 KB) from every box, also where the box
        // holds fewer (the accumulator rows past it are never stored): the
        // last box of the last stage must not read past the allocation
        smem = std::max(smem, (size_t)S * STAGE - abox + 16384);
    }
    static DeviceFlags attr;
    {
        const cudaError_t e = attr.once([&] {
            return cudaFuncSetAttribute(tc_project_tma<ST, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        222 * 1024);
        });
        if (e != cudaSuccess) return (int)e;
    }
    tc_project_tma<ST, NP><<<grid, ST == ST_FP8 ? kTmaThreadsF8 : kTmaThreads, smem, st>>>(
        a0, project_tcols(a0, NP), ntile, R, S, abox, cps, SR, rawb, XR);
    count_launches(1);
    return (int)cudaGetLastError();
}

template <int ST, int NP>
int run_project(const MatvecArgs& a0, cudaStream_t st) {
    constexpr bool SPLIT = ST == ST_BF16X2;
    constexpr int S = SPLIT ? 3 : 4;
    const size_t smem = (size_t)S * (SPLIT ? 2 : 1) * 16 * 1024 + 2 * (SPLIT ? 2 : 1) * (size_t)NP * a0.tile_p * 2;
    static DeviceFlags attr;
    {
        const cudaError_t e = attr.once([&] {
            return cudaFuncSetAttribute(tc_project_persistent<ST, NP, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        226 * 1024);
        });
        if (e != cudaSuccess) return (int)e;
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
    // split storage reaches the FP32 tolerance only with short tensor-memory
    // accumulation chains: flush every four tiles (64 K-steps of 16)
    a.tc_seg = ST == ST_BF16X2 ? std::min(R, 4) : R;
    {
        const int per_tile = (int)(a.tile_p / 8) * NP;
        const int64_t blocks = (int64_t)ntile * ((per_tile + 255) / 256);
        tc_xprep_kernel<SPLIT><<<(unsigned)blocks, 256, 0, st>>>(a, NP);
        count_launches(1);
    }
    if constexpr (ST == ST_BF16 || ST == ST_BF16X2 || ST == ST_FP8) {
        if (a.tmaps_tc) {
            const int rc = run_project_tma<ST, NP>(a, st, R, grid, ntile);
            if (rc != 0) return rc;
        } else {
            tc_project_persistent<ST, NP, S><<<grid, kPThreads, smem, st>>>(a, project_tcols(a, NP), ntile, R);
            count_launches(1);
        }
    } else {
        tc_project_persistent<ST, NP, S><<<grid, kPThreads, smem, st>>>(a, project_tcols(a, NP), ntile, R);
        count_launches(1);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return (int)e;
    // Steps 2-4 for the nodes that span accumulation segments: a node spans
    // when a segment start (a range start, or F tiles after one inside the
    // range) falls strictly inside it; the starts come in increasing order,
    // so each spanning node is listed once
    int chunks = 1;
    for (int l = 1; l <= a.nf; ++l)
        if (a.lv[l].nsub > 1 && a.lv[l].r > 0)
            chunks = std::max(chunks, (a.s * a.lv[l].r * a.kc + kRedThreads - 1) / kRedThreads);
    const int F = a.tc_seg > 0 ? a.tc_seg : R;
    SpanList spans;
    spans.n = 0;
    auto flush = [&]() -> cudaError_t {
        if (spans.n == 0) return cudaSuccess;
        tc_reduce_kernel<ST><<<(unsigned)(spans.n * chunks), kRedThreads, 0, st>>>(a, chunks, spans);
        count_launches(1);
        spans.n = 0;
        return cudaGetLastError();
    };
    for (int l = 1; l <= a.nf; ++l) {
        const DevLevel& L = a.lv[l];
        if (L.nsub <= 1 || L.r == 0) continue;
        int64_t last = -1;
        for (int64_t c = 0; c * R < ntile; ++c)
            for (int64_t s0 = c * R + (c == 0 ? F : 0); s0 < std::min<int64_t>((c + 1) * R, ntile); s0 += F) {
                if (s0 % L.nsub == 0) continue;                  // a node boundary, not inside
                const int64_t j = s0 / L.nsub;
                if (j == last) continue;
                last = j;
                spans.e[spans.n++] = ((unsigned)l << 24) | (unsigned)j;
                if (spans.n == kMaxSpans && (e = flush()) != cudaSuccess) return (int)e;
            }
    }
    if ((e = flush()) != cudaSuccess) return (int)e;
    return (int)cudaGetLastError();
}

template <int ST, int NP>
int tc_launch_np(int which, const MatvecArgs& a, cudaStream_t st) {
    if (which == 0) return a.nf > 0 ? run_project<ST, NP>(a, st) : 0;
    if (a.tmaps_tc) return run_expand_tma<ST, NP>(a, st);
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
