// Per-device set-up of kernel attributes.
//
// cudaFuncSetAttribute and the occupancy queries act on the current device
// only, so a value that a launcher works out once must be kept per device:
// a process that drives several GPUs (one handle per device, or one handle
// moved between devices) needs each of them set up.
#pragma once
#include <atomic>
#include <cuda_runtime.h>

namespace hh {

// Raise a kernel's dynamic shared-memory limit to `bytes` on the current
// device, once per device (bit d of `done` records device d; devices beyond
// 63 are set up on every call).  Callers racing on one device set the same
// value, so no lock is needed.
template <typename K>
inline cudaError_t smem_attr_once(K kern, size_t bytes, std::atomic<unsigned long long>& done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev >= 0 && dev < 64 ? 1ull << dev : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
    return e;
}

// A per-device integer computed once (e.g. a persistent grid size); 0 means
// not yet known.  Devices beyond 63 recompute it on every call.
struct PerDeviceInt {
    std::atomic<int> v[64];
    PerDeviceInt() {
        for (auto& a : v) a.store(0, std::memory_order_relaxed);
    }
    int get(int dev) const { return dev >= 0 && dev < 64 ? v[dev].load(std::memory_order_acquire) : 0; }
    void set(int dev, int x) {
        if (dev >= 0 && dev < 64) v[dev].store(x, std::memory_order_release);
    }
};

}  // namespace hh
