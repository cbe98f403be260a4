// Storage-kind traits and element decoding shared by the CUDA-core kernels
// (device code only; every translation unit gets its own copy).
#pragma once
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "hm_device.h"

namespace hm {
namespace {

// ------------------------------------------------------------ storage kinds
template <int ST>
struct Tr;
template <>
struct Tr<ST_F64> {
    using E = double;
    using A = double;
    static constexpr int VEC = 2;
    static __device__ __forceinline__ A dec(E e) { return e; }
};
template <>
struct Tr<ST_F32> {
    using E = float;
    using A = float;
    static constexpr int VEC = 4;
    static __device__ __forceinline__ A dec(E e) { return e; }
};
template <>
struct Tr<ST_BF16> {
    using E = uint16_t;
    using A = float;
    static constexpr int VEC = 8;
    // bf16 is the upper half of a float's bit pattern
    static __device__ __forceinline__ A dec(E e) { return __uint_as_float((uint32_t)e << 16); }
};
template <>
struct Tr<ST_BF16X2> : Tr<ST_BF16> {};
template <>
struct Tr<ST_FP8> {
    using E = uint8_t;
    using A = float;
    static constexpr int VEC = 16;
    static __device__ __forceinline__ A dec(E e) {
        const __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)e, __NV_E4M3);
        return __half2float(__half(h));
    }
};
// storage of the dense near-field blocks
template <int ST>
struct DenseKind {
    static constexpr int value = ST == ST_FP8 ? ST_BF16 : ST;
};

// N consecutive elements of type E as aligned loads (N * sizeof(E) <= 32).
template <typename E, int N>
__device__ __forceinline__ void raw_load(const E* p, E (&o)[N]) {
    constexpr int B = N * (int)sizeof(E);
    static_assert(B <= 32 && (B & (B - 1)) == 0, "load size");
    if constexpr (B == 32) {
        union { uint4 v[2]; E e[N]; } u;
        u.v[0] = __ldg(reinterpret_cast<const uint4*>(p));
        u.v[1] = __ldg(reinterpret_cast<const uint4*>(p) + 1);
#pragma unroll
        for (int i = 0; i < N; ++i) o[i] = u.e[i];
    } else if constexpr (B == 16) {
        union { uint4 v; E e[N]; } u;
        u.v = __ldg(reinterpret_cast<const uint4*>(p));
#pragma unroll
        for (int i = 0; i < N; ++i) o[i] = u.e[i];
    } else if constexpr (B == 8) {
        union { uint2 v; E e[N]; } u;
        u.v = __ldg(reinterpret_cast<const uint2*>(p));
#pragma unroll
        for (int i = 0; i < N; ++i) o[i] = u.e[i];
    } else if constexpr (B == 4) {
        union { unsigned int v; E e[N]; } u;
        u.v = __ldg(reinterpret_cast<const unsigned int*>(p));
#pragma unroll
        for (int i = 0; i < N; ++i) o[i] = u.e[i];
    } else if constexpr (B == 2) {
        union { unsigned short v; E e[N]; } u;
        u.v = __ldg(reinterpret_cast<const unsigned short*>(p));
#pragma unroll
        for (int i = 0; i < N; ++i) o[i] = u.e[i];
    } else {
        union { unsigned char v; E e[N]; } u;
        u.v = __ldg(reinterpret_cast<const unsigned char*>(p));
        o[0] = u.e[0];
    }
}

// N decoded values at element offset `off` of a factor array (plus its low
// part for split storage).
template <int ST, int N>
__device__ __forceinline__ void load_dec(const void* base, const void* lo, int64_t off,
                                         typename Tr<ST>::A (&o)[N]) {
    using T = Tr<ST>;
    typename T::E raw[N];
    raw_load<typename T::E, N>(static_cast<const typename T::E*>(base) + off, raw);
#pragma unroll
    for (int i = 0; i < N; ++i) o[i] = T::dec(raw[i]);
    if constexpr (ST == ST_BF16X2) {
        typename T::E r2[N];
        raw_load<typename T::E, N>(static_cast<const typename T::E*>(lo) + off, r2);
#pragma unroll
        for (int i = 0; i < N; ++i) o[i] += T::dec(r2[i]);
    }
}

// scale of column `col` of node `node` (block q = col / r)
template <int ST>
__device__ __forceinline__ float factor_scale(const float* sc, const DevLevel& L, int s,
                                              int64_t node, int col) {
    if constexpr (ST == ST_BF16) {
        return sc[L.sc_off + node * s + col / L.r];
    } else if constexpr (ST == ST_FP8) {
        return sc[L.sc_off + node * (int64_t)s * L.r + col];
    } else {
        return 1.f;
    }
}

// Element e (compile-time) of a 16-byte raw vector of storage kind ST.
template <int ST, int e>
__device__ __forceinline__ typename Tr<ST>::A elem16(const uint4& v) {
    const unsigned w[4] = {v.x, v.y, v.z, v.w};
    if constexpr (ST == ST_F64) {
        return __hiloint2double((int)w[2 * e + 1], (int)w[2 * e]);
    } else if constexpr (ST == ST_F32) {
        return __uint_as_float(w[e]);
    } else if constexpr (ST == ST_BF16 || ST == ST_BF16X2) {
        const unsigned u = w[e >> 1];
        return __uint_as_float((e & 1) ? (u & 0xffff0000u) : (u << 16));
    } else {
        const unsigned u = (w[e >> 2] >> (8 * (e & 3))) & 0xffu;
        return Tr<ST_FP8>::dec((uint8_t)u);
    }
}

// Element e of a 16-byte raw vector (e a constant after unrolling).
template <int ST>
__device__ __forceinline__ typename Tr<ST>::A elem_at(const uint4& v, int e) {
    const unsigned w[4] = {v.x, v.y, v.z, v.w};
    if constexpr (ST == ST_F64) {
        return __hiloint2double((int)w[2 * e + 1], (int)w[2 * e]);
    } else if constexpr (ST == ST_F32) {
        return __uint_as_float(w[e]);
    } else if constexpr (ST == ST_BF16 || ST == ST_BF16X2) {
        const unsigned u = w[e >> 1];
        return __uint_as_float((e & 1) ? (u & 0xffff0000u) : (u << 16));
    } else {
        const unsigned u = (w[e >> 2] >> (8 * (e & 3))) & 0xffu;
        return Tr<ST_FP8>::dec((uint8_t)u);
    }
}

template <int ST, int KC, int e>
struct DotStep {
    // acc[c] += element e of (hi [+ lo]) * xv[e * KC + c], then the next element
    static __device__ __forceinline__ void go(const uint4& hi, const uint4& lo,
                                              const typename Tr<ST>::A* xv,
                                              typename Tr<ST>::A (&acc)[KC]) {
        typename Tr<ST>::A v = elem16<ST, e>(hi);
        if constexpr (ST == ST_BF16X2) v += elem16<ST, e>(lo);
#pragma unroll
        for (int c = 0; c < KC; ++c) acc[c] += v * xv[e * KC + c];
        if constexpr (e + 1 < Tr<ST>::VEC) DotStep<ST, KC, e + 1>::go(hi, lo, xv, acc);
    }
};

// Step 2 of one node of level l (nodes longer than the project tile): the
// node's per-tile partial sums are added in a fixed order and written as the
// node sum, by `nthreads` threads (thread `tid`) of which the first 256 take
// part.  Per item (column, right-hand side) and f < F = max(1, 256 / items):
// tiles u = f mod F in increasing order into four interleaved accumulators,
// combined as (s0 + s1) + (s2 + s3); then the F results in order of f
// (through `red`, 256 values).  Up to PF loads (a multiple of 4) are issued
// before their adds (the order of the adds is the same for every PF).  Ends
// with `sync()` when F > 1.
template <typename A, typename Sync, int PF = 16>
__device__ __forceinline__ void node_step2(const MatvecArgs& a, const DevLevel& L, int64_t node,
                                           int tid, A* red, Sync sync) {
    A* __restrict__ T = static_cast<A*>(a.T);
    const int sr = a.s * L.r;
    const int64_t t0 = node * L.nsub;
    const int items = sr * a.k;
    const int F = items >= 256 ? 1 : 256 / items;
    const int64_t stride = (int64_t)sr * a.kc;
    for (int t = tid; t < items * F; t += 256) {
        const int item = t % items, f = t / items;
        const int col = item / a.k, c = item - col * a.k;
        const A* src = T + (L.part_off + t0 * sr + col) * a.kc + c;
        A s0 = A(0), s1 = A(0), s2 = A(0), s3 = A(0);
        // this thread's tiles: u = f + F k, k < nk; k = 4 g + c goes to
        // accumulator c for the full groups g < nk / 4, the rest to s0
        const int nk = f < L.nsub ? (L.nsub - f + F - 1) / F : 0;
        const int full = nk / 4 * 4;
        for (int k0 = 0; k0 < nk; k0 += PF) {
            A v[PF];
#pragma unroll
            for (int q = 0; q < PF; ++q) {
                // unconditional loads (clamped to the thread's last tile) so
                // that all of them are in flight together
                const int k = k0 + q < nk ? k0 + q : nk - 1;
                v[q] = __ldcg(src + (int64_t)(f + k * F) * stride);
            }
#pragma unroll
            for (int q = 0; q < PF; q += 4) {
                if (k0 + q + 3 < full) {
                    s0 += v[q];
                    s1 += v[q + 1];
                    s2 += v[q + 2];
                    s3 += v[q + 3];
                } else {
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (k0 + q + c >= full && k0 + q + c < nk) s0 += v[q + c];
                }
            }
        }
        const A sum = (s0 + s1) + (s2 + s3);
        if (F == 1) T[(L.fin_off + node * sr + col) * a.kc + c] = sum;
        else red[t] = sum;
    }
    if (F > 1) {
        sync();
        for (int item = tid; item < items; item += 256) {
            A sum = A(0);
            for (int f = 0; f < F; ++f) sum += red[f * items + item];
            const int col = item / a.k, c = item - col * a.k;
            T[(L.fin_off + node * sr + col) * a.kc + c] = sum;
        }
        sync();
    }
}

}  // namespace
}  // namespace hm
