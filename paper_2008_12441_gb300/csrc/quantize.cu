// Host-side rounding of the float64 master factors to the device storage
// formats (round to nearest even, through CUDA's own conversion routines).
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <cstdint>
#include <cstring>

#include "hm_device.h"

namespace hm {

namespace {
uint16_t bf16_bits(double v) {
    const __nv_bfloat16 b = __double2bfloat16(v);
    uint16_t u;
    std::memcpy(&u, &b, 2);
    return u;
}
double bf16_value(uint16_t u) {
    uint32_t w = (uint32_t)u << 16;
    float f;
    std::memcpy(&f, &w, 4);
    return (double)f;
}
}  // namespace

void to_bf16(const double* src, uint16_t* dst, size_t n, double scale_inv) {
    for (size_t i = 0; i < n; ++i) dst[i] = bf16_bits(src[i] * scale_inv);
}

void to_bf16_split(const double* src, uint16_t* hi, uint16_t* lo, size_t n) {
    for (size_t i = 0; i < n; ++i) {
        hi[i] = bf16_bits(src[i]);
        lo[i] = bf16_bits(src[i] - bf16_value(hi[i]));
    }
}

void to_fp8e4m3(const double* src, uint8_t* dst, size_t n, double scale_inv) {
    for (size_t i = 0; i < n; ++i)
        dst[i] = (uint8_t)__nv_cvt_double_to_fp8(src[i] * scale_inv, __NV_SATFINITE, __NV_E4M3);
}

}  // namespace hm
