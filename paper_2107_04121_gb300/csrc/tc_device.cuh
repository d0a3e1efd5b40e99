// Device pieces of the tcgen05 kernels (5th-generation tensor cores, accumulators in
// tensor memory): the K-major shared-memory operand layout and its descriptors, the
// MMA instruction, tensor-memory loads, mbarrier waits that give up after a bounded
// time, bulk copies to global memory, and the split of float32 values into hi + lo
// operand pairs (TF32 or BF16) of the split-precision ladder.  Inline PTX only.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace {

constexpr long long TC_WAIT_CYCLES = 4000000000ll;  // about two seconds at 2 GHz

enum TcMode { TC_TF32X3 = 0, TC_BF16X3 = 1, TC_BF16 = 2 };

// K-major, non-swizzled canonical layout: 8-row x 16-byte core matrices; the
// K chunks of one 8-row group are adjacent (LBO = 128 B), 8-row groups follow
// each other (SBO = all K chunks of a group).
template <int EB, int KPAD, int ROWS>
struct OpLayout {
    static constexpr int CHUNK = 16 / EB;         // K values per core-matrix row
    static constexpr int KCHUNKS = KPAD / CHUNK;  // 16-byte K chunks per row
    static constexpr int LBO = 128;
    static constexpr int SBO = KCHUNKS * 128;
    static constexpr int BYTES = (ROWS / 8) * SBO;
    __device__ static int offset(int m, int k)
    {
        return (m >> 3) * SBO + (k / CHUNK) * LBO + (m & 7) * 16 + (k % CHUNK) * EB;
    }
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory matrix descriptor: start address, LBO, SBO (all >> 4),
// descriptor version 1 (bits 46-47), no base offset, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, int lbo, int sbo)
{
    uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= 1ull << 46;
    return d;
}

// Instruction descriptor of kind::tf32 / kind::f16: FP32 accumulator (bits 4-5),
// A and B formats (bits 7-9, 10-12: 1 = BF16, 2 = TF32), both K-major,
// N >> 3 (bits 17-22), M >> 4 (bits 24-28).
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt, int m, int n)
{
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// One MMA of M x N x K (K = 8 TF32 or 16 BF16 values) into tensor memory at d_tmem,
// accumulating when `accumulate` is non-zero.
template <int MODE, int M, int N>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate)
{
    static_assert(M == 128 && N % 16 == 0 && N >= 16 && N <= 256, "cta_group::1 shapes with M = 128");
    if constexpr (MODE == TC_TF32X3) {
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(instr_desc(2, M, N)), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(instr_desc(1, M, N)), "r"(accumulate)
            : "memory");
    }
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void bulk_store(void *gdst, const void *ssrc, unsigned bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(smem_u32(ssrc)),
                 "r"(bytes)
                 : "memory");
}

// split x into hi + lo in the operand format; returns the two 32-bit or 16-bit patterns
template <int MODE>
__device__ __forceinline__ void split(float x, uint32_t &hi, uint32_t &lo)
{
    if constexpr (MODE == TC_TF32X3) {
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(x));
        const float r = x - __uint_as_float(hi);
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lo) : "f"(r));
    } else {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
        hi = (uint32_t)__bfloat16_as_ushort(h);
        lo = (uint32_t)__bfloat16_as_ushort(l);
    }
}

// Two values in bf16 (x1 in the upper half, x0 in the lower), with the bf16
// rounding of the residuals x - hi in lo: hi + lo carries about 16 bits of x.
__device__ __forceinline__ uint32_t pack_bf16x2(float x1, float x0)
{
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(x1), "f"(x0));
    return r;
}

__device__ __forceinline__ void split_bf16x2(float x1, float x0, uint32_t &hi, uint32_t &lo)
{
    hi = pack_bf16x2(x1, x0);
    const float h0 = __uint_as_float(hi << 16), h1 = __uint_as_float(hi & 0xffff0000u);
    lo = pack_bf16x2(x1 - h1, x0 - h0);
}

__device__ __forceinline__ void named_sync(int id, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Wait on an mbarrier phase, giving up after TC_WAIT_CYCLES or when the CTA aborts.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, volatile int *abort_flag)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag || clock64() - t0 > TC_WAIT_CYCLES) return false;
    }
    return true;
}

// The same wait bounded by time alone (the drain of an aborting CTA).
__device__ __forceinline__ bool mbar_wait_cycles(uint32_t bar, uint32_t parity)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > TC_WAIT_CYCLES) return false;
    }
    return true;
}


}  // namespace
