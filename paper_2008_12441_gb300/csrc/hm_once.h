// Per-device one-time setup (kernel attributes such as the dynamic
// shared-memory limit, which the runtime keeps per device).
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

namespace hm {

// The devices (ordinals 0..63) on which a setup step has succeeded.  once()
// runs the step on the current device unless it already succeeded there;
// concurrent first calls may both run it (the steps are idempotent), and
// ordinals from 64 up run it on every call.
class DeviceFlags {
public:
    template <typename F>
    cudaError_t once(F&& fn) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        const uint64_t bit = dev >= 0 && dev < 64 ? (uint64_t)1 << dev : 0;
        if (bit && (bits_.load(std::memory_order_acquire) & bit)) return cudaSuccess;
        e = fn();
        if (e == cudaSuccess && bit) bits_.fetch_or(bit, std::memory_order_acq_rel);
        return e;
    }

private:
    std::atomic<uint64_t> bits_{0};
};

}  // namespace hm
