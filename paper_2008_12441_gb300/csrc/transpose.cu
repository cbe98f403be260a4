// Transposed copy of the dense near-field blocks for the transposed product
// K^T x.  Group g stores D_g with column b contiguous over the target slots
// (entry (b, p) at g G^2 + b G + p); the copy stores D_g^T the same way, so
// that the expand kernels read it exactly as they read D.  A one-time setup
// step (32 x 32 tiles through shared memory, coalesced reads and writes),
// not part of a product.
#include <cuda_runtime.h>

#include <cstdint>

#include "hm_device.h"

namespace hm {
namespace {

template <typename E>
__global__ void __launch_bounds__(256) transpose_groups_kernel(const E* __restrict__ src, E* __restrict__ dst,
                                                               int64_t G) {
    __shared__ E tile[32][33];
    const int64_t g = blockIdx.z;
    const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    const E* s = src + g * G * G;
    E* d = dst + g * G * G;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int64_t r = r0 + i, c = c0 + threadIdx.x;
        if (r < G && c < G) tile[i][threadIdx.x] = s[r * G + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int64_t r = c0 + i, c = r0 + threadIdx.x;
        if (r < G && c < G) d[r * G + c] = tile[threadIdx.x][i];
    }
}

}  // namespace

int transpose_groups(const void* src, void* dst, int esize, int64_t groups, int64_t G, void* stream) {
    if (groups <= 0 || G <= 0) return 0;
    if (esize != 2 && esize != 4 && esize != 8) return (int)cudaErrorInvalidValue;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const dim3 block(32, 8);
    // at most 65535 groups per launch (grid z)
    for (int64_t g0 = 0; g0 < groups; g0 += 65535) {
        const int64_t ng = groups - g0 < 65535 ? groups - g0 : 65535;
        const dim3 grid((unsigned)((G + 31) / 32), (unsigned)((G + 31) / 32), (unsigned)ng);
        const size_t off = (size_t)g0 * G * G * esize;
        const char* s = static_cast<const char*>(src) + off;
        char* d = static_cast<char*>(dst) + off;
        if (esize == 2)
            transpose_groups_kernel<uint16_t><<<grid, block, 0, st>>>(reinterpret_cast<const uint16_t*>(s),
                                                                      reinterpret_cast<uint16_t*>(d), G);
        else if (esize == 4)
            transpose_groups_kernel<uint32_t><<<grid, block, 0, st>>>(reinterpret_cast<const uint32_t*>(s),
                                                                      reinterpret_cast<uint32_t*>(d), G);
        else
            transpose_groups_kernel<uint64_t><<<grid, block, 0, st>>>(reinterpret_cast<const uint64_t*>(s),
                                                                      reinterpret_cast<uint64_t*>(d), G);
        count_launches(1);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return (int)e;
    }
    return 0;
}

}  // namespace hm
