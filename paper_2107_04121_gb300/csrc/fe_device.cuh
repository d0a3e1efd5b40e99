// Device helpers shared by the libfe kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "fe_internal.h"

// Record a device-detected problem: the first error code wins, the smallest
// element index is kept.  Never traps.
__device__ __forceinline__ void fe_report(unsigned long long *status, int code, long long elem)
{
    atomicCAS(&status[0], 0ull, (unsigned long long)code);
    atomicMin(&status[1], (unsigned long long)elem);
}

template <typename T>
__device__ __forceinline__ T fe_ld(const T *p)
{
    return __ldg(p);
}

// Voigt index of the symmetric pair (i, j): (11,22,33,12,13,23) -> 0..5.
__host__ __device__ __forceinline__ int fe_voigt(int i, int j)
{
    return i == j ? i : (i + j == 1 ? 3 : (i + j == 2 ? 4 : 5));
}

// Launch configuration (resident CTAs per SM times SM count) computed once per
// kernel instantiation and device: kernel attributes are set and occupancy is
// queried on the first launch only, so later launches cost no driver calls
// beyond the launch itself.
struct FeLaunchCache {
    std::atomic<int> ready[64];
    long long value[64];
};

template <typename F>
inline cudaError_t fe_cached_grid(FeLaunchCache &c, F compute, long long *out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && c.ready[dev].load(std::memory_order_acquire)) {
        *out = c.value[dev];
        return cudaSuccess;
    }
    long long v = 0;
    e = compute(dev, &v);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) {
        c.value[dev] = v;
        c.ready[dev].store(1, std::memory_order_release);
    }
    *out = v;
    return cudaSuccess;
}
