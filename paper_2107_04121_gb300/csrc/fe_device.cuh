// Device helpers shared by the libfe kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

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
