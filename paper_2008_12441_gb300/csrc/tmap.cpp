// Tensor-memory-access descriptors ("tensor maps") of the factor arrays.
//
// The descriptors are encoded on the host by the driver's
// cuTensorMapEncodeTiled, reached through the runtime's entry-point query
// (so the library does not link the driver library itself).
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "hm_device.h"

namespace hm {

namespace {

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                              CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                              CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
    static std::once_flag once;
    static EncodeFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

}  // namespace

int encode_rows_map(void* map, const void* base, int esize, uint64_t row_len, uint64_t rows,
                    uint32_t box_x, uint32_t box_y, bool swizzle128) {
    static_assert(sizeof(CUtensorMap) == kTensorMapBytes, "tensor map size");
    EncodeFn fn = encode_fn();
    if (!fn) return -1;
    CUtensorMapDataType dt;
    switch (esize) {
        case 1: dt = CU_TENSOR_MAP_DATA_TYPE_UINT8; break;
        case 2: dt = CU_TENSOR_MAP_DATA_TYPE_UINT16; break;
        case 4: dt = CU_TENSOR_MAP_DATA_TYPE_UINT32; break;
        case 8: dt = CU_TENSOR_MAP_DATA_TYPE_UINT64; break;
        default: return -1;
    }
    const cuuint64_t dims[2] = {row_len, rows};
    const cuuint64_t strides[1] = {row_len * (uint64_t)esize};
    const cuuint32_t box[2] = {box_x, box_y};
    const cuuint32_t estr[2] = {1, 1};
    alignas(64) CUtensorMap m;
    const CUresult r = fn(&m, dt, 2, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE,
                          swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return (int)r;
    std::memcpy(map, &m, sizeof(m));
    return 0;
}

}  // namespace hm
