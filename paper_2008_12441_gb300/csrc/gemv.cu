// The GEMV form of the product, y = alpha K x + beta y (the remark after
// Step 5 of Sec. 4.1): the product goes to the handle's staging, this
// kernel combines it with y.  Elementwise and memory-bound: one read of
// the product, one read and one write of y per element (no read of y when
// beta is zero, so y may hold anything then, as in the BLAS).
#include <cuda_runtime.h>

#include <cstdint>

#include "hm_device.h"

namespace hm {
namespace {

template <typename A>
__global__ void __launch_bounds__(256) axpby_kernel(int64_t n, int k, A alpha, const A* __restrict__ t,
                                                    int64_t ldt, A beta, A* __restrict__ y, int64_t ldy,
                                                    bool read_y) {
    const int64_t total = n * k;
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += step) {
        const int64_t i = e / k;
        const int c = (int)(e - i * k);
        const A v = alpha * t[i * ldt + c];
        A* yp = y + i * ldy + c;
        *yp = read_y ? v + beta * *yp : v;
    }
}

}  // namespace

int axpby(bool f64, int64_t n, int k, double alpha, const void* t, int64_t ldt, double beta, void* y,
          int64_t ldy, void* stream) {
    if (n <= 0 || k <= 0) return 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
    const int64_t total = n * k;
    const int64_t want = (total + 255) / 256;
    const int64_t cap = (int64_t)sms * 8;   // grid-stride beyond eight CTAs per SM
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    const bool read_y = beta != 0.0;
    if (f64)
        axpby_kernel<double><<<grid, 256, 0, st>>>(n, k, alpha, static_cast<const double*>(t), ldt, beta,
                                                  static_cast<double*>(y), ldy, read_y);
    else
        axpby_kernel<float><<<grid, 256, 0, st>>>(n, k, (float)alpha, static_cast<const float*>(t), ldt,
                                                 (float)beta, static_cast<float*>(y), ldy, read_y);
    count_launches(1);
    return (int)cudaGetLastError();
}

}  // namespace hm
