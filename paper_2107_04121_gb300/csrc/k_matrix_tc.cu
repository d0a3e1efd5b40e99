// Matrix mode on the 5th-generation tensor cores (tcgen05, accumulators in
// tensor memory) for vector Q2 linear elasticity with Lame materials, in the
// split-precision ladder of the library: TF32 x3, BF16 x3 (operands split
// x = hi + lo, products hi*hi + hi*lo + lo*hi, FP32 accumulation) and raw BF16.
// Element matrices of the form 'IK,s(i:j)->I,s(k:l)->K' (Sec. 5.3.3 of
// Cimrman, arXiv 2107.04121), Algorithm 2 of the paper.
//
// Per element the contraction is the Gram matrix of the scaled physical
// gradients, A = X^T X with X[q][(j,a)] = sqrt(w_q det J_q) G_q[j][a]
// (Q = 27 quadrature points, 81 columns (j,a)), followed by the Lame epilogue
//   K[(i,a),(k,b)] = lambda A_ik[a][b] + mu A_ik[b][a] + mu delta_ik sum_j A_jj[a][b].
// A is one tcgen05 MMA chain of M = 128 (rows (j,a) -> 32 j + a), N = 96,
// K = 32 (points, zero padded).  Because A is a Gram matrix, one operand
// buffer serves as both the A and the B operand (K-major, no swizzle).
//
// One CTA of four warps per element at a time:
//   (a) stage sqrt(w det J) J^-1 of the element (FP32 copy of the FP64 geometry)
//   (b) build X = (sqrt(w det J) J^-T grad_xi phi), split into hi/lo operands
//   (c) one thread issues the MMAs and commits them to an mbarrier
//   (d) all threads wait on the mbarrier (bounded; a timeout is reported)
//   (e) warps 0-2 load their 32 accumulator lanes (rows j = warp) from tensor
//       memory and publish them to shared memory
//   (f) each thread forms one row of K_e, which needs the transposed block
//       A_ik[b][a] and the diagonal blocks from the other warps
//   (g) the 26,244-byte element matrix is written by one bulk copy
#include <cuda_bf16.h>

#include "fe_device.cuh"

namespace {

constexpr int TC_N = 27, TC_Q = 27;
constexpr int TC_THREADS = 128;
constexpr int TC_M = 128;        // MMA rows
constexpr int TC_NCOL = 96;      // MMA columns
constexpr int TC_KPAD = 32;      // quadrature points, padded
constexpr int TC_TMEM_COLS = 128;
constexpr int TC_NROW = 3 * TC_N;  // 81
constexpr long long TC_WAIT_CYCLES = 4000000000ll;  // about two seconds at 2 GHz

enum TcMode { TC_TF32X3 = 0, TC_BF16X3 = 1, TC_BF16 = 2 };

// K-major, non-swizzled canonical layout: 8-row x 16-byte core matrices; the
// K chunks of one 8-row group are adjacent (LBO = 128 B), 8-row groups follow
// each other (SBO = all K chunks of a group).
template <int EB>
struct OpLayout {
    static constexpr int CHUNK = 16 / EB;         // K values per core-matrix row
    static constexpr int KCHUNKS = TC_KPAD / CHUNK;  // 8 (4-byte) or 4 (2-byte)
    static constexpr int LBO = 128;
    static constexpr int SBO = KCHUNKS * 128;
    static constexpr int BYTES = (TC_M / 8) * SBO;  // 16 KB or 8 KB
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
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt)
{
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(TC_NCOL >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

template <int MODE>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate)
{
    if constexpr (MODE == TC_TF32X3) {
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(instr_desc(2)), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(instr_desc(1)), "r"(accumulate)
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

// One operand tile of phase (b): this lane's node a and points q of its 4-byte
// segment, for the three gradient rows j.  All shared-memory reads happen
// before the stores (the buffers do not alias).
template <int MODE, int SEGV, int CHUNK>
__device__ __forceinline__ void operand_tile(const float *__restrict__ dp, const float *__restrict__ jw, int a, int q0,
                                             unsigned char *__restrict__ hi, unsigned char *__restrict__ lo,
                                             const int *__restrict__ off)
{
    uint32_t hv[3] = {0, 0, 0}, lv[3] = {0, 0, 0};
    float x[SEGV][3];
#pragma unroll
    for (int v = 0; v < SEGV; ++v) {
        const int q = q0 + v;
        const bool ok = a < TC_N && q < TC_Q;
        const int qq = ok ? q : 0, aa = ok ? a : 0;
        const float d0 = dp[qq * 3 * TC_N + aa], d1 = dp[qq * 3 * TC_N + TC_N + aa],
                    d2 = dp[qq * 3 * TC_N + 2 * TC_N + aa];
        float J[9];
#pragma unroll
        for (int t = 0; t < 9; ++t) J[t] = jw[qq * 9 + t];
#pragma unroll
        for (int j = 0; j < 3; ++j) x[v][j] = ok ? d0 * J[j] + d1 * J[3 + j] + d2 * J[6 + j] : 0.0f;
    }
#pragma unroll
    for (int v = 0; v < SEGV; ++v)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            uint32_t h, l;
            split<MODE>(x[v][j], h, l);
            hv[j] |= h << (16 * v);
            lv[j] |= l << (16 * v);
        }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        *reinterpret_cast<uint32_t *>(hi + off[j]) = hv[j];
        if constexpr (MODE != TC_BF16) *reinterpret_cast<uint32_t *>(lo + off[j]) = lv[j];
    }
}

// Row (i, a) of K_e, k-th column block: lambda A_ik[a][.] + mu A_ik[.][a]
// (+ mu trace for k = i), read from the exchange buffer before any store.
template <int STRIDE>
__device__ __forceinline__ void k_row_block(const float *own, const float *__restrict__ trc,
                                            const float *__restrict__ o1, const float *__restrict__ o2, bool diag,
                                            float lam, float mu, float *__restrict__ out)
{
    float t[TC_N];
#pragma unroll
    for (int b = 0; b < TC_N; ++b) t[b] = trc[b * STRIDE];
    if (diag) {
#pragma unroll
        for (int b = 0; b < TC_N; ++b) t[b] = fmaf(mu, own[b] + o1[b] + o2[b], mu * t[b]) + lam * own[b];
    } else {
#pragma unroll
        for (int b = 0; b < TC_N; ++b) t[b] = fmaf(lam, own[b], mu * t[b]);
    }
#pragma unroll
    for (int b = 0; b < TC_N; ++b) out[b] = t[b];
}

template <int MODE>
struct TcSmem {
    static constexpr int EB = MODE == TC_TF32X3 ? 4 : 2;
    using L = OpLayout<EB>;
    static constexpr int HI = 0;
    static constexpr int LO = L::BYTES;
    // the exchange buffer [3][3][27][33] floats reuses the operand buffers,
    // which are dead once the MMAs have completed
    static constexpr int EX = 0;
    static constexpr int EX_STRIDE = 33;
    static constexpr int EX_BYTES = 9 * TC_N * EX_STRIDE * 4;
    static constexpr int OPEX = (2 * L::BYTES > EX_BYTES ? 2 * L::BYTES : EX_BYTES + 15) / 16 * 16;
    static constexpr int KS = OPEX;                                    // K staging: 6561 + 4 floats
    static constexpr int KS_BYTES = (TC_NROW * TC_NROW + 4) * 4;
    static constexpr int JW = (KS + KS_BYTES + 15) / 16 * 16;          // sqrt(w det J) J^-1: 27 x 9 floats
    static constexpr int DP = JW + TC_Q * 9 * 4;                       // grad_xi phi: 27 x 3 x 27 floats
    static constexpr int MISC = (DP + TC_Q * 3 * TC_N * 4 + 15) / 16 * 16;  // mbarrier, tmem slot, lambda/mu, flag
    static constexpr int BYTES = MISC + 32;
};

// Prefetched geometry of one element: 27 x 9 J^-1 entries, 27 weights, the Lame pair.
constexpr int TC_PF = (TC_Q * 9 + TC_THREADS - 1) / TC_THREADS;  // 2 per thread

template <int MODE>
__global__ void __launch_bounds__(TC_THREADS) k_matrix_tc(const float *__restrict__ jinv,
                                                         const float *__restrict__ wdetj,
                                                         const float *__restrict__ dphi, long long E,
                                                         const double *__restrict__ lame, float *__restrict__ K,
                                                         unsigned long long *__restrict__ status)
{
    using P = TcSmem<MODE>;
    using L = typename P::L;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *opHi = smem + P::HI;
    unsigned char *opLo = smem + P::LO;
    float *ex = reinterpret_cast<float *>(smem + P::EX);
    float *ks = reinterpret_cast<float *>(smem + P::KS);
    float *sJw = reinterpret_cast<float *>(smem + P::JW);
    float *sDp = reinterpret_cast<float *>(smem + P::DP);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + P::MISC);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + P::MISC + 8);
    float *sLM = reinterpret_cast<float *>(smem + P::MISC + 16);
    int *abort_flag = reinterpret_cast<int *>(smem + P::MISC + 24);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int i = tid; i < TC_Q * 3 * TC_N; i += TC_THREADS) sDp[i] = dphi[i];
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *abort_flag = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // prefetch registers: this thread's share of the next element's geometry
    float pj[TC_PF], pw[TC_PF];
    double plm = 0.0;
    auto prefetch = [&](long long e) {
        if (e >= E) return;
#pragma unroll
        for (int u = 0; u < TC_PF; ++u) {
            const int t = tid + u * TC_THREADS;
            if (t < TC_Q * 9) {
                pj[u] = jinv[e * TC_Q * 9 + t];
                pw[u] = wdetj[e * TC_Q + t / 9];
            }
        }
        if (tid < 2) plm = lame[2 * e + tid];
    };
    prefetch(blockIdx.x);

    uint32_t phase = 0;
    for (long long e = blockIdx.x; e < E; e += gridDim.x, phase ^= 1) {
        // (a) geometry of the element, then start fetching the next one
#pragma unroll
        for (int u = 0; u < TC_PF; ++u) {
            const int t = tid + u * TC_THREADS;
            if (t < TC_Q * 9) sJw[t] = sqrtf(pw[u]) * pj[u];
        }
        if (tid < 2) sLM[tid] = (float)plm;
        prefetch(e + gridDim.x);
        __syncthreads();

        // (b) X[(j,a)][q] = sum_k dphi[q][k][a] sqrt(w) Jinv[q][k][j], split into hi/lo.
        // Lane (r, seg) of a tile owns node a = 8 g + r and the points of its 4-byte
        // segment; it writes the same position of the three row blocks j, so every
        // warp store covers one 128-byte core matrix.  Padding (a >= 27, q >= 27) is
        // written as zero: the buffer held the previous element's exchange data.
        {
            constexpr int SEGV = 4 / P::EB;  // K values per 4-byte segment: 1 (tf32) or 2 (bf16)
            constexpr int NCH = TC_KPAD / L::CHUNK;
            const int r = lane >> 2, seg = lane & 3;
            static_assert((4 * NCH) % 4 == 0, "tiles split evenly over the four warps");
#pragma unroll
            for (int it = 0; it < NCH; ++it) {
                const int tile = warp + 4 * it;
                const int g = tile / NCH, c = tile % NCH;
                const int a = 8 * g + r, q0 = c * L::CHUNK + seg * SEGV;
                const int off[3] = {L::offset(a, q0), L::offset(32 + a, q0), L::offset(64 + a, q0)};
                operand_tile<MODE, SEGV, L::CHUNK>(sDp, sJw, a, q0, opHi, opLo, off);
            }
        }
        fence_async_smem();  // operand writes -> tensor-core (async) proxy
        __syncthreads();

        // (c) MMA chain: D = sum over K steps of hi*hi (+ hi*lo + lo*hi)
        if (tid == 0) {
            tc_fence_after();
            constexpr int KSTEP_BYTES = 2 * L::LBO;  // one MMA consumes two 16-byte K chunks
            constexpr int NSTEP = TC_KPAD / (2 * L::CHUNK);
            const uint32_t hi = smem_u32(opHi), lo = smem_u32(opLo);
#pragma unroll
            for (int s = 0; s < NSTEP; ++s) {
                const uint64_t dh = smem_desc(hi + s * KSTEP_BYTES, L::LBO, L::SBO);
                mma<MODE>(tmem, dh, dh, s > 0 ? 1u : 0u);
                if constexpr (MODE != TC_BF16) {
                    const uint64_t dl = smem_desc(lo + s * KSTEP_BYTES, L::LBO, L::SBO);
                    mma<MODE>(tmem, dh, dl, 1u);
                    mma<MODE>(tmem, dl, dh, 1u);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(mbar))
                         : "memory");
        }

        // (d) wait for the accumulator (bounded by time)
        {
            const long long t0 = clock64();
            bool ok = false;
            while (!(ok = mbar_try_wait(smem_u32(mbar), phase)) && clock64() - t0 < TC_WAIT_CYCLES) {
            }
            if (!ok) {
                *abort_flag = 1;
                fe_report(status, FE_ERR_TIMEOUT, e);
            }
        }
        tc_fence_after();
        __syncthreads();
        if (*abort_flag) break;

        // (e) accumulator rows (j = warp, a = lane) stay in registers and are
        // published to the exchange buffer ex[j][l][a][b] (over the operands)
        float d[TC_NCOL];
        if (warp < 3) {
            const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16);
            tmem_ld32(taddr, d);
            tmem_ld32(taddr + 32, d + 32);
            tmem_ld32(taddr + 64, d + 64);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (lane < TC_N) {
#pragma unroll
                for (int l = 0; l < 3; ++l)
#pragma unroll
                    for (int b = 0; b < TC_N; ++b) ex[((warp * 3 + l) * TC_N + lane) * P::EX_STRIDE + b] = d[32 * l + b];
            }
        }
        tc_fence_before();
        if (tid == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");  // staging drained
        __syncthreads();

        // (f) row (i = warp, a = lane) of K_e into the staging buffer
        const float *dst0 = K + e * (long long)(TC_NROW * TC_NROW);
        const int shift = (int)(((unsigned long long)dst0 % 16) / 4);
        float *kst = ks + shift;
        if (warp < 3 && lane < TC_N) {
            const int i = warp, a = lane;
            const float lam = sLM[0], mu = sLM[1];
            float *row = kst + (i * TC_N + a) * TC_NROW;
            const float *o1 = ex + ((((i + 1) % 3) * 4) * TC_N + a) * P::EX_STRIDE;  // A_jj[a][.] of the other warps
            const float *o2 = ex + ((((i + 2) % 3) * 4) * TC_N + a) * P::EX_STRIDE;
#pragma unroll
            for (int k = 0; k < 3; ++k)
                k_row_block<P::EX_STRIDE>(d + 32 * k,                                    // A_ik[a][.] (registers)
                                          ex + ((i * 3 + k) * TC_N) * P::EX_STRIDE + a,  // A_ik[.][a]
                                          o1, o2, k == i, lam, mu, row + k * TC_N);
        }
        fence_async_smem();
        __syncthreads();

        // (g) one bulk copy per element matrix (scalar head/tail to reach 16-byte alignment)
        if (tid == 0) {
            float *dst = K + e * (long long)(TC_NROW * TC_NROW);
            constexpr int LEN = TC_NROW * TC_NROW;
            const int head = (4 - shift) % 4;
            const int body = (LEN - head) / 4 * 4;
            for (int t = 0; t < head; ++t) dst[t] = kst[t];
            for (int t = head + body; t < LEN; ++t) dst[t] = kst[t];
            bulk_store(dst + head, kst + head, (unsigned)(body * 4));
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
    }
    if (tid == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS)
                     : "memory");
}

template <int MODE>
cudaError_t launch_tc(const fe_geometry_h *g, fe_material_args mat, void *K, int sm_count,
                      unsigned long long *status, cudaStream_t s)
{
    using P = TcSmem<MODE>;
    static_assert(P::BYTES <= 227 * 1024, "shared memory plan too large");
    auto kern = k_matrix_tc<MODE>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, P::BYTES);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (err != cudaSuccess) return err;
    // resident CTAs per SM: shared memory (228 KB per SM, 1 KB reserved per CTA),
    // registers, and the 512 tensor-memory columns of which every CTA holds TC_TMEM_COLS
    int dev = 0, smem_sm = 0, regs_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaFuncAttributes fa{};
    err = cudaFuncGetAttributes(&fa, kern);
    if (err != cudaSuccess) return err;
    int per_sm = smem_sm / (P::BYTES + 1024);
    const int by_regs = regs_sm / (((fa.numRegs + 7) / 8 * 8) * TC_THREADS);
    if (by_regs < per_sm) per_sm = by_regs;
    if (per_sm * TC_TMEM_COLS > 512) per_sm = 512 / TC_TMEM_COLS;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long blocks = (long long)per_sm * sm_count;
    if (blocks > g->mesh.n_elems) blocks = g->mesh.n_elems;
    kern<<<(unsigned)blocks, TC_THREADS, P::BYTES, s>>>(g->d_jinv32, g->d_wdetj32, g->d_dphi32, g->mesh.n_elems,
                                                        mat.data, (float *)K, status);
    return cudaGetLastError();
}

}  // namespace

cudaError_t fe_launch_matrix_tc(const fe_geometry_h *g, const fe_form_h *f, fe_material_args mat, fe_precision prec,
                                void *K, int sm_count, unsigned long long *status, cudaStream_t s)
{
    if (g->mesh.n_elems == 0) return cudaSuccess;
    if (f->kind != FK_ELASTICITY || mat.kind != FE_MAT_LAME || g->N != TC_N || g->Q != TC_Q)
        return cudaErrorNotSupported;
    switch (prec) {
    case FE_TF32X3: return launch_tc<TC_TF32X3>(g, mat, K, sm_count, status, s);
    case FE_BF16X3: return launch_tc<TC_BF16X3>(g, mat, K, sm_count, status, s);
    case FE_BF16: return launch_tc<TC_BF16>(g, mat, K, sm_count, status, s);
    default: return cudaErrorNotSupported;
    }
}
