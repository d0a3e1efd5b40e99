// Matrix mode on the 5th-generation tensor cores for vector Q3 linear elasticity
// (64-node hexahedra, 4 x 4 x 4 Gauss points) with Lame materials, TF32 x3
// (operands split x = hi + lo, products hi*hi + hi*lo + lo*hi, FP32 accumulation in
// tensor memory): the form 'IK,s(i:j)->I,s(k:l)->K' of Sec. 5.3.3 of Cimrman,
// arXiv 2107.04121, Algorithm 2.
//
// As for Q2 (k_matrix_tc.cu), the contraction is the Gram matrix A = X^T X of the
// scaled physical gradients X[q][(j,a)] = sqrt(w_q det J_q) G_q[j][a] -- here 64
// points and 192 columns (j,a) -- followed by the Lame epilogue
//   K_ik[a][b] = lambda A_ik[a][b] + mu A_ik[b][a] + mu delta_ik sum_j A_jj[a][b].
// A has 192 rows, so it takes two MMA tiles of M = 128: rows 0-127 (j = 0, 1) and
// rows 128-255 (j = 2, then 64 rows of padding whose results are not read), each
// against all 192 columns: 8 K steps x 3 products per tile, into tensor-memory
// columns [0, 192) and [256, 448).  The 448 columns leave room for one CTA per SM.
//
// One element at a time per CTA (8 warps):
//   (a) sqrt(w det J) J^-1 of the 64 points to shared memory;
//   (b) every warp builds its share of the hi/lo operand (K-major core matrices,
//       each store of a warp one 8-row x 4-point core matrix of 128 bytes);
//   (c) one thread issues both MMA chains and commits them to an mbarrier;
//   (d) epilogue.  Warp w reads the tensor-memory lanes of its quarter w % 4: the
//       warps of quarters 0-1 hold the rows of the blocks j = 0 (first tile) and
//       j = 2 (second tile), those of quarters 2-3 the block j = 1; warp w / 4
//       picks the column half.  A lane holds a row b of A_ik, i.e. (K being
//       symmetric) column b of K_ik, so it writes the staged row block of K_e one
//       row a at a time with consecutive lanes on consecutive columns.  The
//       diagonal blocks A_jj are published for sum_j A_jj, an off-diagonal block
//       A_ik goes through a transposition buffer for its A_ik[a][b] term.  Each
//       group of four warps stages a 64 x 192 row block of K_e (contiguous in
//       global memory) and writes it with one bulk copy; the group of quarters
//       0-1 does the row blocks 0 and 2, the other group the row block 1.
// The weighted scalar Laplacian and mass matrix of the same elements ('0,0.i,0.i',
// '0,i,i', per-element c) take the same kernel (FORM): the Laplacian is
// c sum_j A_jj, for which the MMAs compute only the diagonal blocks (first tile
// against columns 0-127, second tile against columns 128-191); the mass matrix
// is the Gram matrix of sqrt(w det J) phi (64 rows, one tile against 64 columns).
// Both write a 64 x 64 K_e with one bulk copy.  The pair mode is elasticity that
// also writes the weighted Laplacian of the same elements, c sum_j A_jj, from the
// diagonal blocks its epilogue publishes anyway (staged and copied out by the warp
// group with one row block, into a second output).
//
// The exchange area and group 0-1's staging reuse the operand buffer once the
// MMAs are done, so the next element's operands are built after those bulk
// copies have been read.  Every mbarrier wait is bounded: a timeout is reported
// as FE_ERR_TIMEOUT and the CTA drains its MMAs and frees tensor memory.
#include <type_traits>

#include "fe_device.cuh"
#include "tc_device.cuh"

namespace {

constexpr int T6_N = 64, T6_Q = 64;     // nodes, points
constexpr int T6_ROWS = 3 * T6_N;       // 192 rows (j, a) of A and of K_e
constexpr int T6_OPROWS = 256;          // operand rows: two M = 128 tiles
constexpr int T6_THREADS = 256;
constexpr int T6_TMEM_COLS = 512;       // tiles at columns 0 and 256 (192 each)
constexpr int T6_EX = 68;               // floats per row of the exchange blocks (16-byte rows)
constexpr int T6_JW = 12;               // floats per point of the staged sqrt(w det J) J^-1
constexpr int T6_BAR_G0 = 1, T6_BAR_G1 = 2;  // named barriers of the two warp groups
enum T6Form { T6_ELAST = 0, T6_LAPL = 1, T6_MASS = 2, T6_PAIR = 3 };

struct T6Smem {
    using L = OpLayout<4, T6_Q, T6_OPROWS>;         // TF32 operands: 64 KB each
    static constexpr int HI = 0, LO = L::BYTES;       // [0, 128 KB)
    // reused once the MMAs are done:
    static constexpr int EXD = 0;                                       // [3][64][68] diagonal blocks
    static constexpr int EXT0 = EXD + 3 * T6_N * T6_EX * 4;             // [64][68] transposition, group 0
    static constexpr int STG0 = EXT0 + T6_N * T6_EX * 4;                // [64][192] (+4) staging, group 0
    static constexpr int STG_BYTES = (T6_N * T6_ROWS + 4) * 4;
    static_assert(STG0 + STG_BYTES <= 2 * L::BYTES, "exchange and staging fit the operand buffer");
    static constexpr int EXT1 = 2 * L::BYTES;                           // group 1's own buffers
    static constexpr int STG1 = EXT1 + T6_N * T6_EX * 4;
    static constexpr int JW = STG1 + STG_BYTES;                         // [64][12]
    static constexpr int LM = JW + T6_Q * T6_JW * 4;                    // lambda, mu
    static constexpr int MISC = (LM + 16 + 15) / 16 * 16;               // mbarrier, tmem slot, abort flag
    static constexpr int BYTES = MISC + 16;
    static constexpr int LSTG = BYTES;                                  // pair mode: [64][64] (+4) Laplacian
    static constexpr int BYTES_PAIR = LSTG + (T6_N * T6_N + 4) * 4;
    static_assert(BYTES_PAIR <= 227 * 1024, "pair mode fits one CTA");
};

// 32 consecutive floats of an exchange row as eight 16-byte stores.
__device__ __forceinline__ void store_row32(float *dst, const float *v)
{
#pragma unroll
    for (int c = 0; c < 8; ++c)
        reinterpret_cast<float4 *>(dst)[c] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
}

template <int FORM>
__global__ void __launch_bounds__(T6_THREADS, 1)
    k_matrix_tc64(const float *__restrict__ jinv, const float *__restrict__ wdetj, const float *__restrict__ dphi,
                  const float *__restrict__ phi, long long E, const double *__restrict__ lame,
                  float *__restrict__ K, unsigned long long *__restrict__ status, const double *__restrict__ coef,
                  float *__restrict__ K2)
{
    constexpr bool ELAST = FORM == T6_ELAST || FORM == T6_PAIR;
    constexpr int NR = ELAST ? T6_ROWS : T6_N;  // rows (and columns) of K_e
    using P = T6Smem;
    using L = P::L;
    extern __shared__ __align__(1024) unsigned char smem[];
    float *sJw = reinterpret_cast<float *>(smem + P::JW);
    float *sLM = reinterpret_cast<float *>(smem + P::LM);
    uint64_t *mma_bar = reinterpret_cast<uint64_t *>(smem + P::MISC);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + P::MISC + 8);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + P::MISC + 12);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int sp = warp & 3, half = warp >> 2;  // tensor-memory lane quarter, column half
    const int grp = sp >> 1;                    // 0: row blocks 0 and 2; 1: row block 1
    const bool issuer = tid == 0, copier = lane == 0 && half == 0 && (sp & 1) == 0;  // warp 0 or 2

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mma_bar)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *abort_flag = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(T6_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t tlane = (uint32_t)(32 * sp) << 16;  // this warp's lane quarter

    // the element's J^-1 and w det J are loaded into registers one element ahead
    constexpr int NPF = (T6_Q * 9 + T6_THREADS - 1) / T6_THREADS;  // 3 per thread
    float pj[NPF], pw[NPF];
    double plm = 0.0;
    auto prefetch = [&](long long e) {
        if (e >= E) return;
#pragma unroll
        for (int k = 0; k < NPF; ++k) {
            const int t = tid + k * T6_THREADS;
            if (t < T6_Q * 9) {
                if constexpr (FORM != T6_MASS) pj[k] = jinv[e * (T6_Q * 9) + t];
                pw[k] = wdetj[e * T6_Q + t / 9];
            }
        }
        if constexpr (ELAST) {
            if (tid < 2) plm = lame[2 * e + tid];
            if (FORM == T6_PAIR && tid == 2) plm = coef ? coef[e] : 1.0;
        } else {
            if (tid == 0) plm = lame ? lame[e] : 1.0;
        }
    };
    prefetch(blockIdx.x);

    int n = 0;
    bool issued = false;  // the issuer: MMAs committed to mma_bar and not yet waited for
    for (long long e = blockIdx.x; e < E; e += gridDim.x, ++n) {
        // the operand buffer holds group 0's staging and the exchange area: its
        // bulk copies must have been read before the operands are rebuilt
        if (copier) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        __syncthreads();
        if (*abort_flag) break;
        // (a) sqrt(w det J) J^-1 and the Lame pair, then the next element's loads
#pragma unroll
        for (int k = 0; k < NPF; ++k) {
            const int t = tid + k * T6_THREADS;
            if (t < T6_Q * 9) {
                if constexpr (FORM == T6_MASS) {
                    if (t % 9 == 0) sJw[(t / 9) * T6_JW] = sqrtf(pw[k]);  // sqrt(w det J) alone
                } else {
                    sJw[(t / 9) * T6_JW + t % 9] = sqrtf(pw[k]) * pj[k];
                }
            }
        }
        if (tid < (FORM == T6_PAIR ? 3 : 2)) sLM[tid] = (float)plm;
        prefetch(e + gridDim.x);
        __syncthreads();
        // (b, c) X[(j,a)][q] split into TF32 hi/lo, then the MMAs, in two halves of
        // the points: the second half is built while the first half's MMAs run.
        // In half hk, warp w builds the chunk of points 4 (8 hk + w) ... + 3: lane
        // (r, kk) takes point q = 4 (8 hk + w) + kk and, for the nodes a = 8 ig + r,
        // the three rows (j, a); the reference gradients of (q, a) are read once (read-
        // only cache; 48 KB, the same for every element) and serve the three rows.
        constexpr int KSTEP_BYTES = 2 * L::LBO;  // one MMA consumes two 16-byte K chunks (8 points)
        constexpr int NSTEP = T6_Q / (2 * L::CHUNK);
        static_assert(T6_Q / 8 == T6_THREADS / 32, "one chunk of 4 points per warp and half");
        for (int hk = 0; hk < 2; ++hk) {
            unsigned char *hi = smem + P::HI, *lo = smem + P::LO;
            const int r = lane >> 2, kk = lane & 3;
            const int q = 4 * ((T6_Q / 8) * hk + warp) + kk;
            if constexpr (FORM == T6_MASS) {
                // rows a: sqrt(w det J) phi_a(q)
                const float sw = sJw[q * T6_JW];
                const float *pq = phi + q * T6_N + r;
#pragma unroll 4
                for (int ig = 0; ig < T6_N / 8; ++ig) {
                    uint32_t h, l;
                    split<TC_TF32X3>(sw * __ldg(pq + 8 * ig), h, l);
                    const int off = L::offset(8 * ig + r, q);
                    *reinterpret_cast<uint32_t *>(hi + off) = h;
                    *reinterpret_cast<uint32_t *>(lo + off) = l;
                }
            } else {
            float jq[9];
#pragma unroll
            for (int t = 0; t < 9; ++t) jq[t] = sJw[q * T6_JW + t];
            const float *dq = dphi + q * 3 * T6_N + r;
#pragma unroll 4
            for (int ig = 0; ig < T6_N / 8; ++ig) {
                const int a = 8 * ig + r;
                const float d0 = __ldg(dq + 8 * ig), d1 = __ldg(dq + T6_N + 8 * ig), d2 = __ldg(dq + 2 * T6_N + 8 * ig);
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const float x = d0 * jq[j] + d1 * jq[3 + j] + d2 * jq[6 + j];
                    uint32_t h, l;
                    split<TC_TF32X3>(x, h, l);
                    const int off = L::offset(T6_N * j + a, q);
                    *reinterpret_cast<uint32_t *>(hi + off) = h;
                    *reinterpret_cast<uint32_t *>(lo + off) = l;
                }
            }
            }
            fence_async_smem();  // operand writes -> tensor-core (async) proxy
            __syncthreads();
            if (issuer) {
                tc_fence_after();
                const uint32_t hs = smem_u32(smem + P::HI), ls = smem_u32(smem + P::LO);
                // one chain of 3 products per K step: rows from `arow`, columns from `brow`
                auto chain = [&](uint32_t d_tmem, uint32_t arow, uint32_t brow, auto ncols) {
                    constexpr int NC = decltype(ncols)::value;
#pragma unroll
                    for (int s2 = hk * NSTEP / 2; s2 < (hk + 1) * NSTEP / 2; ++s2) {
                        const uint64_t ah = smem_desc(hs + arow + s2 * KSTEP_BYTES, L::LBO, L::SBO);
                        const uint64_t al = smem_desc(ls + arow + s2 * KSTEP_BYTES, L::LBO, L::SBO);
                        const uint64_t bh = smem_desc(hs + brow + s2 * KSTEP_BYTES, L::LBO, L::SBO);
                        const uint64_t bl = smem_desc(ls + brow + s2 * KSTEP_BYTES, L::LBO, L::SBO);
                        mma<TC_TF32X3, 128, NC>(d_tmem, ah, bh, s2 > 0 ? 1u : 0u);
                        mma<TC_TF32X3, 128, NC>(d_tmem, ah, bl, 1u);
                        mma<TC_TF32X3, 128, NC>(d_tmem, al, bh, 1u);
                    }
                };
                const uint32_t row128 = (uint32_t)(16 * L::SBO);  // byte offset of operand row 128
                if constexpr (ELAST) {
                    chain(tmem, 0u, 0u, std::integral_constant<int, T6_ROWS>{});
                    chain(tmem + 256, row128, 0u, std::integral_constant<int, T6_ROWS>{});
                } else if constexpr (FORM == T6_LAPL) {
                    // diagonal blocks only: rows 0-127 x columns 0-127, rows 128-191 x columns 128-191
                    chain(tmem, 0u, 0u, std::integral_constant<int, 128>{});
                    chain(tmem + 256, row128, row128, std::integral_constant<int, T6_N>{});
                } else {
                    chain(tmem, 0u, 0u, std::integral_constant<int, T6_N>{});
                }
                if (hk == 1) {
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
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
            }
        }
        __syncthreads();
        if (*abort_flag) break;
        tc_fence_after();

        // (d) epilogue
        if constexpr (ELAST) {
        // (d) epilogue
        const float lam = sLM[0], mu = sLM[1];
        float *exd = reinterpret_cast<float *>(smem + P::EXD);
        float *ext = reinterpret_cast<float *>(smem + (grp ? P::EXT1 : P::EXT0));
        float v[32];
        // the diagonal blocks A_jj: row b (this lane), columns of this warp's half
        {
            const int bl = 32 * (sp & 1) + lane;  // row within the block
            const int jd = grp ? 1 : 0;
            tmem_ld32(tmem + tlane + 64 * jd + 32 * half, v);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            store_row32(exd + (jd * T6_N + bl) * T6_EX + 32 * half, v);
            if (!grp) {
                tmem_ld32(tmem + 256 + tlane + 128 + 32 * half, v);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                store_row32(exd + (2 * T6_N + bl) * T6_EX + 32 * half, v);
            }
        }
        __syncthreads();
        // row blocks: group 0 does i = 0 then 2, group 1 does i = 1
        const int bar = grp ? T6_BAR_G1 : T6_BAR_G0;
        const int nblk = grp ? 1 : 2;
        for (int bi = 0; bi < nblk; ++bi) {
            const int i = grp ? 1 : 2 * bi;
            const uint32_t tbase = tmem + (i == 2 ? 256u : 0u) + tlane;
            const int bl = 32 * (sp & 1) + lane;  // this lane: row b of block i = column b of K_i.
            float *dstg = K + e * (long long)(T6_ROWS * T6_ROWS) + (long long)i * T6_N * T6_ROWS;
            const int shift = (int)(((unsigned long long)dstg % 16) / 4);
            float *stg = reinterpret_cast<float *>(smem + (grp ? P::STG1 : P::STG0)) + shift;
            if (bi > 0) {  // group 0's staging of row block 0 must have been read
                if (copier) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                named_sync(bar, 128);
            }
            for (int k = 0; k < 3; ++k) {
                tmem_ld32(tbase + 64 * k + 32 * half, v);  // v[t] = A_ik[b][32 half + t]
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (k == i) {
                    // K_ii[a][b] = (lambda + mu) A_ii[b][a] + mu sum_j A_jj[b][a], a = 32 half + t
                    const float *d0 = exd + (0 * T6_N + bl) * T6_EX + 32 * half;
                    const float *d1 = exd + (1 * T6_N + bl) * T6_EX + 32 * half;
                    const float *d2 = exd + (2 * T6_N + bl) * T6_EX + 32 * half;
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const float4 x0 = reinterpret_cast<const float4 *>(d0)[c];
                        const float4 x1 = reinterpret_cast<const float4 *>(d1)[c];
                        const float4 x2 = reinterpret_cast<const float4 *>(d2)[c];
                        v[4 * c] = fmaf(lam + mu, v[4 * c], mu * (x0.x + x1.x + x2.x));
                        v[4 * c + 1] = fmaf(lam + mu, v[4 * c + 1], mu * (x0.y + x1.y + x2.y));
                        v[4 * c + 2] = fmaf(lam + mu, v[4 * c + 2], mu * (x0.z + x1.z + x2.z));
                        v[4 * c + 3] = fmaf(lam + mu, v[4 * c + 3], mu * (x0.w + x1.w + x2.w));
                    }
                } else {
                    // K_ik[a][b] = lambda A_ik[a][b] + mu A_ik[b][a]: the first term from
                    // the block published row-major (rows a) by the group's warps
                    store_row32(ext + bl * T6_EX + 32 * half, v);
                    named_sync(bar, 128);
#pragma unroll
                    for (int t = 0; t < 32; ++t) v[t] = fmaf(lam, ext[(32 * half + t) * T6_EX + bl], mu * v[t]);
                    named_sync(bar, 128);  // the buffer is read before the next block's publication
                }
#pragma unroll
                for (int t = 0; t < 32; ++t) stg[(32 * half + t) * T6_ROWS + 64 * k + bl] = v[t];
            }
            fence_async_smem();
            named_sync(bar, 128);
            if (copier) {
                constexpr int LEN = T6_N * T6_ROWS;
                const int head = (4 - shift) % 4;
                const int body = (LEN - head) / 4 * 4;
                for (int t = 0; t < head; ++t) dstg[t] = stg[t];
                for (int t = head + body; t < LEN; ++t) dstg[t] = stg[t];
                bulk_store(dstg + head, stg + head, (unsigned)(body * 4));
                asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            }
        }
        if constexpr (FORM == T6_PAIR) {
            // the group with one row block: K_L[a][b] = c sum_j A_jj[a][b] from the
            // published diagonal blocks (intact until the next element's operands)
            if (grp) {
                const float cw = sLM[2];
                float *dl = K2 + e * (long long)(T6_N * T6_N);
                const int sh = (int)(((unsigned long long)dl % 16) / 4);
                float *sl = reinterpret_cast<float *>(smem + P::LSTG) + sh;
                const int gt = 64 * half + 32 * (sp - 2) + lane;  // 0 .. 127 within the group
                const int b2 = gt & 63, a0 = (gt >> 6) * 32;      // column b2, rows a0 .. a0 + 31
#pragma unroll 8
                for (int t = 0; t < 32; ++t) {
                    const int a2 = a0 + t;
                    sl[a2 * T6_N + b2] = cw * (exd[(0 * T6_N + a2) * T6_EX + b2] + exd[(1 * T6_N + a2) * T6_EX + b2] +
                                               exd[(2 * T6_N + a2) * T6_EX + b2]);
                }
                fence_async_smem();
                named_sync(T6_BAR_G1, 128);
                if (copier) {
                    constexpr int LEN = T6_N * T6_N;
                    const int head = (4 - sh) % 4;
                    const int body = (LEN - head) / 4 * 4;
                    for (int t = 0; t < head; ++t) dl[t] = sl[t];
                    for (int t = head + body; t < LEN; ++t) dl[t] = sl[t];
                    bulk_store(dl + head, sl + head, (unsigned)(body * 4));
                    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                }
            }
        }
        } else {
            // Laplacian K = c sum_j A_jj, mass matrix K = c A_00: 64 x 64, one bulk copy
            const float cw = sLM[0];
            float *dstg = K + e * (long long)(NR * NR);
            const int shift = (int)(((unsigned long long)dstg % 16) / 4);
            float *stg = reinterpret_cast<float *>(smem + P::STG0) + shift;
            float v[32];
            const int bl = 32 * (sp & 1) + lane;  // row b of the block held by this lane
            if constexpr (FORM == T6_MASS) {
                if (sp < 2) {  // A_00 is symmetric: lane b writes column b of K
                    tmem_ld32(tmem + tlane + 32 * half, v);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int t = 0; t < 32; ++t) stg[(32 * half + t) * T6_N + bl] = cw * v[t];
                }
            } else {
                float *exd = reinterpret_cast<float *>(smem + P::EXD);
                if (sp < 2) {  // A_00 (first tile) and A_22 (second tile, its columns 0-63)
                    tmem_ld32(tmem + tlane + 32 * half, v);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    store_row32(exd + (0 * T6_N + bl) * T6_EX + 32 * half, v);
                    tmem_ld32(tmem + 256 + tlane + 32 * half, v);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    store_row32(exd + (2 * T6_N + bl) * T6_EX + 32 * half, v);
                } else {  // A_11: first tile, rows 64-127, columns 64-127
                    tmem_ld32(tmem + tlane + 64 + 32 * half, v);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    store_row32(exd + (1 * T6_N + bl) * T6_EX + 32 * half, v);
                }
                __syncthreads();
                const int b2 = tid & 63, a0 = (tid >> 6) * 16;  // column b2, rows a0 .. a0 + 15
#pragma unroll
                for (int t = 0; t < 16; ++t) {
                    const int a2 = a0 + t;
                    stg[a2 * T6_N + b2] = cw * (exd[(0 * T6_N + a2) * T6_EX + b2] + exd[(1 * T6_N + a2) * T6_EX + b2] +
                                                exd[(2 * T6_N + a2) * T6_EX + b2]);
                }
            }
            fence_async_smem();
            __syncthreads();
            if (tid == 0) {
                constexpr int LEN = T6_N * T6_N;
                const int head = (4 - shift) % 4;
                const int body = (LEN - head) / 4 * 4;
                for (int t = 0; t < head; ++t) dstg[t] = stg[t];
                for (int t = head + body; t < LEN; ++t) dstg[t] = stg[t];
                bulk_store(dstg + head, stg + head, (unsigned)(body * 4));
                asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            }
        }
        tc_fence_before();  // this element's tensor-memory loads before the next MMAs
    }
    // an aborting CTA frees its tensor memory only after the MMAs it issued are done
    if (issued) mbar_wait_cycles(smem_u32(mma_bar), n & 1);
    if (copier) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(T6_TMEM_COLS)
                     : "memory");
}

template <int FORM>
cudaError_t launch_tc64(const fe_geometry_h *g, fe_material_args mat, void *K, int sm_count,
                        unsigned long long *status, cudaStream_t s, const double *coef = nullptr,
                        void *K2 = nullptr)
{
    auto kern = k_matrix_tc64<FORM>;
    constexpr int BYTES = FORM == T6_PAIR ? T6Smem::BYTES_PAIR : T6Smem::BYTES;
    static FeLaunchCache cache;
    long long per_sm = 0;
    cudaError_t err = fe_cached_grid(
        cache,
        [&](int, long long *v) {
            cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, BYTES);
            if (e2 != cudaSuccess) return e2;
            *v = 1;  // up to 448 of the 512 tensor-memory columns: one CTA per SM
            return cudaSuccess;
        },
        &per_sm);
    if (err != cudaSuccess) return err;
    long long blocks = per_sm * sm_count;
    if (blocks > g->mesh.n_elems) blocks = g->mesh.n_elems;
    kern<<<(unsigned)blocks, T6_THREADS, BYTES, s>>>(g->d_jinv32, g->d_wdetj32, g->d_dphi32, g->d_phi32,
                                                     g->mesh.n_elems, mat.data, (float *)K, status, coef, (float *)K2);
    return cudaGetLastError();
}

}  // namespace

cudaError_t fe_launch_matrix_tc64(const fe_geometry_h *g, const fe_form_h *f, fe_material_args mat,
                                  fe_precision prec, void *K, int sm_count, unsigned long long *status,
                                  cudaStream_t s)
{
    if (g->mesh.n_elems == 0) return cudaSuccess;
    if (g->N != T6_N || g->Q != T6_Q || prec != FE_TF32X3) return cudaErrorNotSupported;
    if (f->kind == FK_ELASTICITY && mat.kind == FE_MAT_LAME) return launch_tc64<T6_ELAST>(g, mat, K, sm_count, status, s);
    if (f->kind == FK_LAPLACE && f->ncomp == 1) return launch_tc64<T6_LAPL>(g, mat, K, sm_count, status, s);
    if (f->kind == FK_MASS && f->ncomp == 1) return launch_tc64<T6_MASS>(g, mat, K, sm_count, status, s);
    return cudaErrorNotSupported;
}

bool fe_matrix_tc64_pair_supported(const fe_geometry_h *g)
{
    return g->N == T6_N && g->Q == T6_Q && g->d_jinv32 && g->d_dphi32;
}

cudaError_t fe_launch_matrix_tc64_pair(const fe_geometry_h *g, const double *lame, void *K, const double *coef,
                                       void *K2, int sm_count, unsigned long long *status, cudaStream_t s)
{
    if (g->mesh.n_elems == 0) return cudaSuccess;
    if (!fe_matrix_tc64_pair_supported(g)) return cudaErrorNotSupported;
    fe_material_args mat{};
    mat.kind = FE_MAT_LAME;
    mat.data = lame;
    return launch_tc64<T6_PAIR>(g, mat, K, sm_count, status, s, coef, K2);
}
