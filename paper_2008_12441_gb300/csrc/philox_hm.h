// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11),
// from its published definition: ten rounds of two 32x32->64 products by
// 0xD2511F53 / 0xCD9E8D57, a word swap with key xor, and a Weyl key bump by
// 0x9E3779B9 / 0xBB67AE85 between rounds.
//
// Random block entry (the paper's random H-matrices, Section 5.1; the value
// distribution is this library's choice): uniform on [-1, 1) as the exact
// dyadic (w >> 8 - 2^23) * 2^-23 of word (col & 3) of
//   philox(counter = {row, col >> 2, t, s | level << 24 | kind << 29},
//          key = {seed, seed >> 32}).
// kind: 0 = U factor, 1 = V factor, 2 = dense block, 3 = sketch matrix.
#pragma once
#include <cstdint>

#if defined(__CUDACC__)
#define HM_HD __host__ __device__ __forceinline__
#else
#define HM_HD inline
#endif

namespace hm {

enum { RAND_U = 0, RAND_V = 1, RAND_D = 2, RAND_SKETCH = 3 };

struct U32x4 {
    uint32_t w[4];
};

HM_HD U32x4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                          uint32_t k0, uint32_t k1) {
    for (int round = 0; round < 10; ++round) {
        if (round) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint64_t a = (uint64_t)0xD2511F53u * c0;
        const uint64_t b = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t n0 = (uint32_t)(b >> 32) ^ c1 ^ k0;
        const uint32_t n2 = (uint32_t)(a >> 32) ^ c3 ^ k1;
        c1 = (uint32_t)b;
        c3 = (uint32_t)a;
        c0 = n0;
        c2 = n2;
    }
    U32x4 r;
    r.w[0] = c0; r.w[1] = c1; r.w[2] = c2; r.w[3] = c3;
    return r;
}

HM_HD double dyadic_uniform(uint32_t w) {
    return (double)((int32_t)(w >> 8) - (1 << 23)) * (1.0 / 8388608.0);
}

HM_HD double rand_entry(uint64_t seed, int kind, int level, uint32_t t, uint32_t s,
                        uint32_t row, uint32_t col) {
    const uint32_t c3 = s | ((uint32_t)level << 24) | ((uint32_t)kind << 29);
    U32x4 r = philox4x32_10(row, col >> 2, t, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
    return dyadic_uniform(r.w[col & 3]);
}

// 2^-e(n) with e(n) = ceil(ceil(log2 n) / 2): scale of random entries whose
// product sums over n terms.
HM_HD double rand_scale(int64_t n) {
    int cl = 0;
    while (((int64_t)1 << cl) < n) ++cl;
    const int e = (cl + 1) / 2;
    double s = 1.0;
    for (int i = 0; i < e; ++i) s *= 0.5;
    return s;
}

}  // namespace hm
