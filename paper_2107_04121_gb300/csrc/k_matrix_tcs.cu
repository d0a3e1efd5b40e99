// Matrix mode on the 5th-generation tensor cores for P3 tetrahedra (20 nodes, the
// 35-point Grundmann-Moller rule of index 3), TF32 x3: Lame elasticity
// ('IK,s(i:j)->I,s(k:l)->K', Sec. 5.3.3 of Cimrman, arXiv 2107.04121) and the weighted
// scalar Laplacian ('0,0.i,0.i'), Algorithm 2.
//
// The element matrix is again built from the Gram blocks A_jl[a][b] =
// sum_q w_q det J_q G_q[j][a] G_q[l][b]; the Lame epilogue is
//   K_ik[a][b] = lambda A_ik[a][b] + mu A_ik[b][a] + mu delta_ik sum_j A_jj[a][b],
// the Laplacian K = c sum_j A_jj.  The rule has negative weights, so the Gram trick
// of the hexahedra (both operands scaled by sqrt(w det J)) needs a sign: the points
// are ordered positive weights first (slots [0, KPOS), padded with zeros to a multiple
// of 8), then negative ones (slots [KPOS, KPOS + KNEG)), both operands carry
// sqrt(|w det J|), and the MMAs of the negative slots take as A operand a copy of X
// with its sign flipped (hi and lo both negated, exactly), so that one accumulator
// sums X_pos^T X_pos - X_neg^T X_neg.
//
// Rows (j, a) of the operand are 32 j + a (a < 20; the rest of each block and rows
// 96-127 are zero or unread), one M = 128 tile against the 96 columns of the three
// blocks, 5 K steps x 3 products into 96 tensor-memory columns (128 allocated), so
// three CTAs of 4 warps share an SM and overlap one another's phases.  Per element:
// (a) sqrt(|w det J|) J^-1 per slot, (b) the operand and its negated copy, (c) one
// thread issues the MMAs and waits (bounded) for their commit, (d) warps 0-2 read the
// tensor-memory rows of block j (lane b holds row b of A_jk = column b of K_jk, K
// being symmetric), publish them, and write K_e into a staging area with consecutive
// lanes on consecutive columns; one bulk copy writes it.  The exchange area and the
// staging reuse the operand buffer once the MMAs are done.
#include <type_traits>

#include "fe_device.cuh"
#include "tc_device.cuh"

namespace {

constexpr int TS_THREADS = 128;
constexpr int TS_TMEM_COLS = 128;  // 96 used
constexpr int TS_JW = 12;          // floats per slot of the staged sqrt(|w det J|) J^-1
constexpr int TS_EXA = 100;        // floats per row of a warp's published accumulator rows (96 + 4)
enum TsForm { TS_ELAST = 0, TS_LAPL = 1 };

// Slot -> quadrature point (or -1) of the K dimension, by value in the kernel's parameters.
struct TsSlots {
    signed char q[64];
};

template <int N, int KPOS, int KNEG>
struct TsSmem {
    static constexpr int KP = KPOS + KNEG;
    using L = OpLayout<4, KP, 128>;      // X: 128 rows x KP slots (TF32)
    using LN = OpLayout<4, KNEG, 128>;   // -X over the negative slots
    static constexpr int XHI = 0, XLO = L::BYTES, NHI = 2 * L::BYTES, NLO = NHI + LN::BYTES;
    static constexpr int OP_BYTES = NLO + LN::BYTES;
    // reused once the MMAs are done
    static constexpr int EXA = 0;                                  // [3][32][TS_EXA]
    static constexpr int STG = EXA + 3 * 32 * TS_EXA * 4;          // (3N)^2 + 4 floats
    static_assert(STG + (9 * N * N + 4) * 4 <= OP_BYTES, "exchange and staging fit the operand buffer");
    static constexpr int JR = (OP_BYTES + 15) / 16 * 16;          // [Q][9] J^-1 of the element
    static constexpr int WR = JR + 64 * 9 * 4;                     // [Q] w det J
    static constexpr int SL = WR + 64 * 4;                         // [64] slot -> point
    static constexpr int LM = SL + 64 * 4;
    static constexpr int MISC = (LM + 16 + 15) / 16 * 16;          // mbarrier, tmem slot, abort flag
    static constexpr int BYTES = MISC + 16;
};

template <int N, int Q, int KPOS, int KNEG, int FORM>
__global__ void __launch_bounds__(TS_THREADS, 3)
    k_matrix_tcs(const float *__restrict__ jinv, const float *__restrict__ wdetj, const float *__restrict__ dphi,
                 long long E, const double *__restrict__ mat, float *__restrict__ K,
                 unsigned long long *__restrict__ status, const TsSlots slots)
{
    using P = TsSmem<N, KPOS, KNEG>;
    using L = typename P::L;
    using LN = typename P::LN;
    constexpr int KP = P::KP;
    constexpr int NR = FORM == TS_ELAST ? 3 * N : N;  // rows (and columns) of K_e
    extern __shared__ __align__(1024) unsigned char smem[];
    float *sJr = reinterpret_cast<float *>(smem + P::JR);
    float *sWr = reinterpret_cast<float *>(smem + P::WR);
    int *sSl = reinterpret_cast<int *>(smem + P::SL);
    float *sLM = reinterpret_cast<float *>(smem + P::LM);
    uint64_t *mma_bar = reinterpret_cast<uint64_t *>(smem + P::MISC);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + P::MISC + 8);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + P::MISC + 12);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int k = tid; k < 64; k += TS_THREADS) sSl[k] = slots.q[k];
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mma_bar)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *abort_flag = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TS_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t tlane = (uint32_t)(32 * warp) << 16;

    // the element's J^-1, w det J and material, loaded into registers one element ahead
    constexpr int NPF = (Q * 9 + TS_THREADS - 1) / TS_THREADS;
    float pj[NPF], pw = 0.0f;
    double pm = 0.0;
    auto prefetch = [&](long long e) {
        if (e >= E) return;
#pragma unroll
        for (int k = 0; k < NPF; ++k) {
            const int t = tid + k * TS_THREADS;
            if (t < Q * 9) pj[k] = jinv[e * (Q * 9) + t];
        }
        if (tid < Q) pw = wdetj[e * Q + tid];
        if constexpr (FORM == TS_ELAST) {
            if (tid < 2) pm = mat[2 * e + tid];
        } else {
            if (tid == 0) pm = mat ? mat[e] : 1.0;
        }
    };
    prefetch(blockIdx.x);

    int n = 0;
    bool issued = false;
    for (long long e = blockIdx.x; e < E; e += gridDim.x, ++n) {
        // the operand buffer holds the previous staging: its bulk copy must have been read
        if (tid == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        __syncthreads();
        if (*abort_flag) break;
        // (a) the element's geometry and material to shared memory, the next element's loads
#pragma unroll
        for (int k = 0; k < NPF; ++k) {
            const int t = tid + k * TS_THREADS;
            if (t < Q * 9) sJr[t] = pj[k];
        }
        if (tid < Q) sWr[tid] = pw;
        if (tid < 2) sLM[tid] = (float)pm;
        prefetch(e + gridDim.x);
        __syncthreads();
        // (b) X[(j,a)][k] split into TF32 hi/lo, and -X over the negative slots.  Warp w
        // takes the chunks of 4 slots c = w, w + 4, ...: lane (r, kk) takes slot
        // k = 4 c + kk (its sqrt(|w det J|) J^-1 in registers) and the nodes a = 8 ga + r,
        // each reference gradient serving the three rows (j, a); zeros for padding
        {
            unsigned char *xhi = smem + P::XHI, *xlo = smem + P::XLO, *nhi = smem + P::NHI, *nlo = smem + P::NLO;
            const int r = lane >> 2, kk = lane & 3;
            for (int c = warp; c < KP / 4; c += TS_THREADS / 32) {
                const int k = 4 * c + kk, q = sSl[k];
                float jq[9];
                const float sw = q >= 0 ? sqrtf(fabsf(sWr[q])) : 0.0f;
#pragma unroll
                for (int t = 0; t < 9; ++t) jq[t] = q >= 0 ? sw * sJr[q * 9 + t] : 0.0f;
                const float *dq = dphi + (q >= 0 ? q : 0) * 3 * N;
                float dv[4][3];
#pragma unroll
                for (int ga = 0; ga < 4; ++ga) {
                    const int a = 8 * ga + r;
                    const bool ok = a < N && q >= 0;
#pragma unroll
                    for (int m = 0; m < 3; ++m) dv[ga][m] = ok ? __ldg(dq + m * N + a) : 0.0f;
                }
#pragma unroll
                for (int ga = 0; ga < 4; ++ga)
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const float x = dv[ga][0] * jq[j] + dv[ga][1] * jq[3 + j] + dv[ga][2] * jq[6 + j];
                        uint32_t h, l;
                        split<TC_TF32X3>(x, h, l);
                        const int row = 32 * j + 8 * ga + r;
                        const int off = L::offset(row, k);
                        *reinterpret_cast<uint32_t *>(xhi + off) = h;
                        *reinterpret_cast<uint32_t *>(xlo + off) = l;
                        if (k >= KPOS) {
                            const int offn = LN::offset(row, k - KPOS);
                            *reinterpret_cast<uint32_t *>(nhi + offn) = h ^ 0x80000000u;  // -hi, -lo exactly
                            *reinterpret_cast<uint32_t *>(nlo + offn) = l ^ 0x80000000u;
                        }
                    }
            }
        }
        fence_async_smem();  // operand writes -> tensor-core (async) proxy
        __syncthreads();
        // (c) D = sum over positive slots X^T X + sum over negative slots (-X)^T X
        if (tid == 0) {
            tc_fence_after();
            constexpr int KSTEP_BYTES = 2 * L::LBO;  // 8 slots per MMA
            const uint32_t xh = smem_u32(smem + P::XHI), xl = smem_u32(smem + P::XLO);
            const uint32_t nh = smem_u32(smem + P::NHI), nl = smem_u32(smem + P::NLO);
#pragma unroll
            for (int s2 = 0; s2 < KP / 8; ++s2) {
                const bool neg = s2 >= KPOS / 8;
                const uint64_t bh = smem_desc(xh + s2 * KSTEP_BYTES, L::LBO, L::SBO);
                const uint64_t bl = smem_desc(xl + s2 * KSTEP_BYTES, L::LBO, L::SBO);
                const uint64_t ah = neg ? smem_desc(nh + (s2 - KPOS / 8) * KSTEP_BYTES, LN::LBO, LN::SBO) : bh;
                const uint64_t al = neg ? smem_desc(nl + (s2 - KPOS / 8) * KSTEP_BYTES, LN::LBO, LN::SBO) : bl;
                mma<TC_TF32X3, 128, 96>(tmem, ah, bh, s2 > 0 ? 1u : 0u);
                mma<TC_TF32X3, 128, 96>(tmem, ah, bl, 1u);
                mma<TC_TF32X3, 128, 96>(tmem, al, bh, 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(mma_bar))
                         : "memory");
            issued = true;
            if (!mbar_wait_bounded(smem_u32(mma_bar), n & 1, abort_flag)) {
                *abort_flag = 1;
                fe_report(status, FE_ERR_TIMEOUT, e);
            } else {
                issued = false;
            }
        }
        __syncthreads();
        if (*abort_flag) break;
        tc_fence_after();

        // (d) warp j < 3 publishes rows b of block j (all 96 columns)
        float *exa = reinterpret_cast<float *>(smem + P::EXA);
        float v[32];
        if (warp < 3) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                tmem_ld32(tmem + tlane + 32 * k, v);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    reinterpret_cast<float4 *>(exa + (warp * 32 + lane) * TS_EXA + 32 * k)[c] =
                        make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
            }
        }
        __syncthreads();
        float *dstg = K + e * (long long)(NR * NR);
        const int shift = (int)(((unsigned long long)dstg % 16) / 4);
        float *stg = reinterpret_cast<float *>(smem + P::STG) + shift;
        if constexpr (FORM == TS_ELAST) {
            // K_jk[a][b] = lambda A_jk[a][b] + mu A_jk[b][a] (+ mu sum_l A_ll[a][b] when k = j):
            // lane b holds A_jk[b][.] in tensor memory; A_jk[a][b] is row a of the published block
            const float lam = sLM[0], mu = sLM[1];
            if (warp < 3) {
                const int j = warp, b = lane;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    tmem_ld32(tmem + tlane + 32 * k, v);  // v[a] = A_jk[b][a]
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (b < N) {
#pragma unroll
                        for (int a = 0; a < N; ++a) {
                            float val = fmaf(lam, exa[(32 * j + a) * TS_EXA + 32 * k + b], mu * v[a]);
                            if (k == j)
                                val = fmaf(mu, exa[a * TS_EXA + b] + exa[(32 + a) * TS_EXA + 32 + b] +
                                                   exa[(64 + a) * TS_EXA + 64 + b],
                                           val);
                            stg[(N * j + a) * NR + N * k + b] = val;
                        }
                    }
                }
            }
        } else {
            const float cw = sLM[0];
            for (int t = tid; t < N * N; t += TS_THREADS) {
                const int a = t / N, b = t % N;
                stg[t] = cw * (exa[a * TS_EXA + b] + exa[(32 + a) * TS_EXA + 32 + b] + exa[(64 + a) * TS_EXA + 64 + b]);
            }
        }
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            constexpr int LEN = NR * NR;
            const int head = (4 - shift) % 4;
            const int body = (LEN - head) / 4 * 4;
            for (int t = 0; t < head; ++t) dstg[t] = stg[t];
            for (int t = head + body; t < LEN; ++t) dstg[t] = stg[t];
            bulk_store(dstg + head, stg + head, (unsigned)(body * 4));
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
        tc_fence_before();  // this element's tensor-memory loads before the next MMAs
    }
    // an aborting CTA frees its tensor memory only after the MMAs it issued are done
    if (issued) mbar_wait_cycles(smem_u32(mma_bar), n & 1);
    if (tid == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TS_TMEM_COLS)
                     : "memory");
}

// P3: 20 nodes, 35 points, 24 positive and 11 negative weights (16 slots)
constexpr int TS_P3_N = 20, TS_P3_Q = 35, TS_P3_KPOS = 24, TS_P3_KNEG = 16;

template <int FORM>
cudaError_t launch_tcs(const fe_geometry_h *g, fe_material_args mat, void *K, int sm_count,
                       unsigned long long *status, cudaStream_t s)
{
    using P = TsSmem<TS_P3_N, TS_P3_KPOS, TS_P3_KNEG>;
    auto kern = k_matrix_tcs<TS_P3_N, TS_P3_Q, TS_P3_KPOS, TS_P3_KNEG, FORM>;
    static FeLaunchCache cache;
    long long per_sm = 0;
    cudaError_t err = fe_cached_grid(
        cache,
        [&](int dev, long long *v) {
            cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, P::BYTES);
            if (e2 != cudaSuccess) return e2;
            e2 = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
            if (e2 != cudaSuccess) return e2;
            // resident CTAs per SM from shared memory (1 KB reserved per CTA), registers
            // (whole warps per sub-partition) and the 512 tensor-memory columns; the
            // runtime's occupancy calculator reports one CTA per SM for this kernel
            int smem_sm = 0, regs_sm = 0;
            cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
            cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
            cudaFuncAttributes fa{};
            e2 = cudaFuncGetAttributes(&fa, kern);
            if (e2 != cudaSuccess) return e2;
            int nb = smem_sm / (P::BYTES + 1024);
            const int warp_regs = (fa.numRegs * 32 + 255) / 256 * 256;
            const int by_regs = 4 * ((regs_sm / 4) / warp_regs) / (TS_THREADS / 32);
            if (by_regs < nb) nb = by_regs;
            if (nb > 512 / TS_TMEM_COLS) nb = 512 / TS_TMEM_COLS;
            if (nb < 1) return cudaErrorInvalidConfiguration;
            *v = nb;
            return cudaSuccess;
        },
        &per_sm);
    if (err != cudaSuccess) return err;
    long long blocks = per_sm * sm_count;
    if (blocks > g->mesh.n_elems) blocks = g->mesh.n_elems;
    TsSlots slots;
    for (int k = 0; k < 64; ++k) slots.q[k] = g->slot_q[k];
    kern<<<(unsigned)blocks, TS_THREADS, P::BYTES, s>>>(g->d_jinv32, g->d_wdetj32, g->d_dphi32, g->mesh.n_elems,
                                                        mat.data, (float *)K, status, slots);
    return cudaGetLastError();
}

}  // namespace

bool fe_matrix_tcs_supported(const fe_geometry_h *g, const fe_form_h *f, fe_precision prec)
{
    if (prec != FE_TF32X3 || g->N != TS_P3_N || g->Q != TS_P3_Q) return false;
    if (g->n_wpos > TS_P3_KPOS || g->n_wneg > TS_P3_KNEG) return false;
    // the slot table pads the positive group to the kernel's KPOS
    if ((g->n_wpos + 7) / 8 * 8 != TS_P3_KPOS) return false;
    const bool lame = f->kind == FK_ELASTICITY && f->mat == FE_MAT_LAME && !f->mat_transposed;
    return lame || (f->kind == FK_LAPLACE && f->ncomp == 1);
}

cudaError_t fe_launch_matrix_tcs(const fe_geometry_h *g, const fe_form_h *f, fe_material_args mat,
                                 fe_precision prec, void *K, int sm_count, unsigned long long *status,
                                 cudaStream_t s)
{
    if (g->mesh.n_elems == 0) return cudaSuccess;
    if (!fe_matrix_tcs_supported(g, f, prec)) return cudaErrorNotSupported;
    if (f->kind == FK_ELASTICITY) {
        if (mat.kind != FE_MAT_LAME) return cudaErrorNotSupported;
        return launch_tcs<TS_ELAST>(g, mat, K, sm_count, status, s);
    }
    return launch_tcs<TS_LAPL>(g, mat, K, sm_count, status, s);
}
