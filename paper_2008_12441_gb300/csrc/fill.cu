// Random-filled H-matrices generated on the device, straight into the
// device layout (the paper's benchmark matrices, Section 5.1: random dense
// and low-rank blocks).  Each entry is the counter-based Philox4x32-10
// value of its block, row and column (philox_hm.h), exactly as the host
// builder computes it, so a device-filled handle equals a host-filled one
// bit for bit; no float64 master copy is built.  Used for unpadded trees
// (every leaf holds exactly m_pad points: the paper's grids) under weak
// admissibility, in FP32 or FP64 storage.
#include <cuda_runtime.h>

#include <cstdint>

#include "hm_device.h"
#include "philox_hm.h"

namespace hm {
namespace {

// One level of U (kind RAND_U, target side) or V (kind RAND_V, source side):
// node p, column q r + c, row a (position inside the node).  The partner of
// p in sibling slot q is its q-th other sibling; the block is (target,
// source) = (p, partner) for U and (partner, p) for V.
template <typename T>
__global__ void fill_factor_kernel(T* __restrict__ dst, int kind, uint64_t seed, int level, int64_t nodes,
                                   int64_t n, int s, int r, double scale) {
    const int64_t total = nodes * s * r * n;
    const int nc = s + 1;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = e % n;
        const int64_t col = (e / n) % ((int64_t)s * r);
        const int64_t p = e / (n * s * r);
        const int q = (int)(col / r), c = (int)(col % r);
        const int cp = (int)(p % nc);
        const int cq = q < cp ? q : q + 1;
        const int64_t partner = p - cp + cq;
        const uint32_t t = (uint32_t)(kind == RAND_U ? p : partner);
        const uint32_t sidx = (uint32_t)(kind == RAND_U ? partner : p);
        dst[e] = (T)(scale * rand_entry(seed, kind, level, t, sidx, (uint32_t)a, (uint32_t)c));
    }
}

// Near-field group g (G slots, column b contiguous over the target slots p).
// Leaf pairs (reading A): leaves of m slots, entry of leaf pair
// (g nc + p / m, g nc + b / m) at (p mod m, b mod m), level `lev` = L;
// otherwise (reading B) the group's diagonal leaf block itself, lev = L.
template <typename T>
__global__ void fill_dense_kernel(T* __restrict__ dst, uint64_t seed, int lev, int64_t groups, int64_t G,
                                  int64_t m, int nc, int leaf_pairs, double scale) {
    const int64_t total = groups * G * G;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = e % G;
        const int64_t b = (e / G) % G;
        const int64_t g = e / (G * G);
        uint32_t lt, ls, at, as;
        if (leaf_pairs) {
            lt = (uint32_t)(g * nc + p / m);
            ls = (uint32_t)(g * nc + b / m);
            at = (uint32_t)(p % m);
            as = (uint32_t)(b % m);
        } else {
            lt = ls = (uint32_t)g;
            at = (uint32_t)p;
            as = (uint32_t)b;
        }
        dst[e] = (T)(scale * rand_entry(seed, RAND_D, lev, lt, ls, at, as));
    }
}

unsigned fill_grid(int64_t total) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess)
        sms = 148;
    const int64_t want = (total + 255) / 256;
    const int64_t cap = (int64_t)sms * 16;
    return (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

int fill_random_factor(void* dst, bool f64, int kind, uint64_t seed, int level, int64_t nodes, int64_t n, int s,
                       int r, double scale) {
    const int64_t total = nodes * s * r * n;
    if (total <= 0) return 0;
    const unsigned grid = fill_grid(total);
    if (f64)
        fill_factor_kernel<double><<<grid, 256>>>(static_cast<double*>(dst), kind, seed, level, nodes, n, s, r, scale);
    else
        fill_factor_kernel<float><<<grid, 256>>>(static_cast<float*>(dst), kind, seed, level, nodes, n, s, r, scale);
    count_launches(1);
    return (int)cudaGetLastError();
}

int fill_random_dense(void* dst, bool f64, uint64_t seed, int lev, int64_t groups, int64_t G, int64_t m, int nc,
                      int leaf_pairs, double scale) {
    const int64_t total = groups * G * G;
    if (total <= 0) return 0;
    const unsigned grid = fill_grid(total);
    if (f64)
        fill_dense_kernel<double><<<grid, 256>>>(static_cast<double*>(dst), seed, lev, groups, G, m, nc, leaf_pairs,
                                                 scale);
    else
        fill_dense_kernel<float><<<grid, 256>>>(static_cast<float*>(dst), seed, lev, groups, G, m, nc, leaf_pairs,
                                                scale);
    count_launches(1);
    return (int)cudaGetLastError();
}

}  // namespace hm
