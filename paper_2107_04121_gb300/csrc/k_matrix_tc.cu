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
// Warp-specialised pipeline, two operand buffers and two accumulators per CTA:
//   producer warps 3-5, element n into buffer n % 2:
//     (a) stage sqrt(w det J) J^-1 of the element (FP32 copy of the FP64 geometry)
//     (b) build X = sqrt(w det J) J^-T grad_xi phi, split into hi/lo operands
//     (c) one thread issues the MMAs and commits them to full[n % 2]
//   consumer warps 0-2, element n from buffer n % 2:
//     (d) wait full[n % 2] (bounded; a timeout is reported, never trapped)
//     (e) load accumulator rows j = warp (lanes a) from tensor memory and
//         publish the diagonal block A_jj and one off-diagonal block A_j,j+1
//         to the exchange area, which reuses the operand buffer
//     (f) K is symmetric: warp i forms the diagonal block K_ii (which needs
//         the other warps' diagonal blocks) and the off-diagonal block
//         K_i,i+1 (which needs its own transposed block A_i,i+1[b][a]), and
//         writes K_i+1,i = K_i,i+1^T as columns
//     (g) the 26,244-byte element matrix is written by one bulk copy, and
//         empty[n % 2] hands the buffer and the accumulator back
// so the operand build and MMAs of element n+1 overlap the epilogue of n.
//
// The weighted weak Laplacian of the same elements ('0,0.i,0.i', per-element c) is
// the sum of the diagonal blocks of the same Gram matrix, K[a][b] = c sum_j A_jj[a][b]
// (FORM = TC_LAPL): the operands and the MMA chain are those of elasticity, the
// epilogue adds the three diagonal blocks published by the consumer warps and
// writes the 27 x 27 matrix.  FORM = TC_PAIR (TF32x3) is elasticity that also writes
// that Laplacian of the same elements, with its own coefficient, into a second
// output: both from one Gram matrix.
//
// With a stale float32-only deferred geometry (Q2, 3x3x3 Gauss points) two
// more warps per CTA compute the FP64 geometry themselves, one element at a time
// (lanes = 1-D lines of the collocation stages of the geometry kernel, same
// roundings, same bits): each stores the float32 J^-1 and w det J of the handle
// and puts sqrt(w det J) J^-1 and the Lame pair into a ring
// of shared-memory slots that replaces phase (a).  The geometry is bound by the
// FP64 units, the rest of the kernel by shared memory and HBM, so the two overlap
// instead of running one after the other.  On GB300 every SM sub-partition has
// its own FP64 unit, which takes about 64 cycles per warp-instruction whatever
// the number of active lanes, and the warps of co-resident CTAs sit on the
// sub-partitions in turn, so that six geometry warps share four units unevenly;
// element n of a CTA goes to its geometry warp n % 2.  (Claiming elements from a
// grid-wide counter, with the producers taking whichever slot is filled first,
// measured 4% slower: shared memory, not the FP64 units, sets the pace.)
#include "fe_device.cuh"
#include "geometry_body.cuh"
#include "tc_device.cuh"

namespace {

constexpr int TC_N = 27, TC_Q = 27;
constexpr int TC_M = 128;        // MMA rows
constexpr int TC_NCOL = 96;      // MMA columns
constexpr int TC_KPAD = 32;      // quadrature points, padded
constexpr int TC_TMEM_COLS = 128;
constexpr int TC_NROW = 3 * TC_N;  // 81
constexpr int TC_JW_STRIDE = 12;  // floats per point of the staged sqrt(w det J) J^-1 (16-byte rows)
constexpr int TC_EX_STRIDE = 28;  // floats per row of the exchange blocks (16-byte rows, conflict-free float4)
enum TcForm { TC_ELAST = 0, TC_LAPL = 1, TC_PAIR = 2 };  // Lame elasticity, weighted Laplacian, both
constexpr int TC_NGEO = 2;  // geometry warps per CTA (GEO)

// Diagonal block of K_e for row (i, a): own A_ii[a][.] from registers, the
// other warps' diagonal blocks from the exchange area; all reads before stores.
template <int STRIDE>
__device__ __forceinline__ void diag_block(const float *own, const float *__restrict__ d1,
                                           const float *__restrict__ d2, float lam, float mu,
                                           float *__restrict__ out)
{
    static_assert(STRIDE % 4 == 0, "exchange rows must be 16-byte aligned");
    float t[28];
#pragma unroll
    for (int c = 0; c < 7; ++c) {
        const float4 x = reinterpret_cast<const float4 *>(d1)[c], y = reinterpret_cast<const float4 *>(d2)[c];
        t[4 * c] = x.x + y.x;
        t[4 * c + 1] = x.y + y.y;
        t[4 * c + 2] = x.z + y.z;
        t[4 * c + 3] = x.w + y.w;
    }
#pragma unroll
    for (int b = 0; b < TC_N; ++b) out[b] = fmaf(lam + 2.0f * mu, own[b], mu * t[b]);
}

// Off-diagonal block K_ik of row (i, a) and its mirror column K_ki[.][a]:
// v[b] = lambda A_ik[a][b] + mu A_ik[b][a], written to the row and to the column.
template <int STRIDE>
__device__ __forceinline__ void offdiag_block(const float *own, const float *__restrict__ trc, float lam, float mu,
                                              float *__restrict__ row, float *__restrict__ col)
{
    float t[TC_N];
#pragma unroll
    for (int b = 0; b < TC_N; ++b) t[b] = trc[b * STRIDE];
#pragma unroll
    for (int b = 0; b < TC_N; ++b) t[b] = fmaf(lam, own[b], mu * t[b]);
#pragma unroll
    for (int b = 0; b < TC_N; ++b) row[b] = t[b];
#pragma unroll
    for (int b = 0; b < TC_N; ++b) col[b * TC_NROW] = t[b];
}

// The two accumulator blocks a consumer warp uses are in registers: d[0..31] =
// its diagonal block A_II, d[32..63] = A_I,I+1.  28 columns per block (the last
// is padding) go to the exchange area as 16-byte stores.
__device__ __forceinline__ void publish_blocks(const float *d, float *__restrict__ e0, float *__restrict__ e1)
{
#pragma unroll
    for (int c = 0; c < 7; ++c)
        reinterpret_cast<float4 *>(e0)[c] = make_float4(d[4 * c], d[4 * c + 1], d[4 * c + 2], d[4 * c + 3]);
#pragma unroll
    for (int c = 0; c < 7; ++c)
        reinterpret_cast<float4 *>(e1)[c] =
            make_float4(d[32 + 4 * c], d[32 + 4 * c + 1], d[32 + 4 * c + 2], d[32 + 4 * c + 3]);
}

// Blocks K_ii and K_i,i+1 of row (i, a) and the mirror column of K_i+1,i.
template <int STRIDE>
__device__ __forceinline__ void epilogue_rows(int I, const float *d, const float *ex, int a, float lam, float mu,
                                              float *kst)
{
    const int Kb = I == 2 ? 0 : I + 1, Mb = I == 0 ? 2 : I - 1;
    // K_ii[a][b] = (lambda + mu) A_ii[a][b] + mu (A_ii + A_kk + A_mm)[a][b]
    diag_block<STRIDE>(d, ex + ((Kb * 2) * TC_N + a) * STRIDE, ex + ((Mb * 2) * TC_N + a) * STRIDE, lam, mu,
                       kst + (I * TC_N + a) * TC_NROW + I * TC_N);
    // K_ik[a][b] = lambda A_ik[a][b] + mu A_ik[b][a]; K_ki[b][a] = K_ik[a][b]
    offdiag_block<STRIDE>(d + 32, ex + ((I * 2 + 1) * TC_N) * STRIDE + a, lam, mu,
                          kst + (I * TC_N + a) * TC_NROW + Kb * TC_N, kst + (Kb * TC_N) * TC_NROW + I * TC_N + a);
}

template <int MODE, bool GEO>
struct TcSmem {
    static constexpr int EB = MODE == TC_TF32X3 ? 4 : 2;
    using L = OpLayout<EB, TC_KPAD, TC_M>;
    // per buffer: hi and lo operands; the exchange area [3 warps][2 blocks][27][28]
    // floats of the epilogue reuses them once the buffer's MMAs have completed
    static constexpr int EX_STRIDE = TC_EX_STRIDE;
    static constexpr int EX_BYTES = 6 * TC_N * EX_STRIDE * 4;
    static constexpr int BUF = ((2 * L::BYTES > EX_BYTES ? 2 * L::BYTES : EX_BYTES) + 1023) / 1024 * 1024;
    static constexpr int HI = 0;
    static constexpr int LO = L::BYTES;
    static constexpr int KS = 2 * BUF;                                  // K staging: 6561 + 4 floats
    static constexpr int KS_BYTES = (TC_NROW * TC_NROW + 4) * 4;
    // grad_xi phi (27 x 3 x 27 floats) is read into the producers' registers before
    // the first element, and the first K staging write waits for the first MMA:
    // the table lives in the staging area
    static constexpr int DP = KS;
    static_assert(TC_Q * 3 * TC_N * 4 <= KS_BYTES, "reference gradients fit the staging area");
    // sqrt(w det J) J^-1 of the elements in flight: [2][27][12] filled by the
    // producers, or (GEO) a ring of RING slots [27][12] + (lambda, mu, pad) filled
    // by the geometry warp
    static constexpr int RING = GEO ? 6 : 0;                            // a multiple of TC_NGEO
    static constexpr int SLOT = TC_Q * TC_JW_STRIDE + 4;               // floats per ring slot
    static constexpr int JW = (KS + KS_BYTES + 15) / 16 * 16;
    static constexpr int JW_BYTES = GEO ? RING * SLOT * 4 : 2 * TC_Q * TC_JW_STRIDE * 4;
    static constexpr int LM = JW + JW_BYTES;                            // [2][2] lambda, mu
    // GEO: FP64 stage buffers of each geometry warp [4][81] (x / points, two
    // interpolation stages, J over the last three) and their tables B[9], Dq[9 + 4], w[27]
    static constexpr int GS = (LM + 16 + 15) / 16 * 16;
    static constexpr int GS_WARP = 4 * 3 * TC_N;                        // doubles per geometry warp
    static constexpr int GT = GS + (GEO ? TC_NGEO * GS_WARP * 8 : 0);
    static constexpr int GT_LEN = 9 + 9 + GEO_DQ_EXTRA + TC_Q;
    // full[2], empty[2], tmem slot, abort flag, accfree[2]; GEO: geo_full[RING], geo_empty[RING]
    static constexpr int MISC = (GT + (GEO ? GT_LEN * 8 : 0) + 15) / 16 * 16;
    static constexpr int GFULL = MISC + 64, GEMPTY = GFULL + 8 * RING;
    static constexpr int BYTES = MISC + 64 + 16 * RING;
    // TC_PAIR: the Laplacian's staging (27 x 27 + 4 floats) and its coefficient [2]
    static constexpr int LS = (BYTES + 15) / 16 * 16;
    static constexpr int LC = (LS + (TC_N * TC_N + 4) * 4 + 15) / 16 * 16;
    static constexpr int BYTES_PAIR = LC + 16;
    // accumulators in tensor memory: one when three CTAs fit an SM (the MMAs of
    // element n+1 wait only for element n's read-out; the other CTAs hide it),
    // two when only two CTAs fit (512 columns per SM)
    static constexpr int NACC = 3 * (BYTES + 1024) <= 228 * 1024 ? 1 : 2;
};

constexpr int TC_CONS = 96;               // consumer threads (warps 0-2)
constexpr int TC_PROD = 96;               // producer threads (warps 3-5)
constexpr int TC_THREADS_WS = TC_CONS + TC_PROD;
constexpr int TC_BAR_PROD = 1, TC_BAR_CONS = 2;  // named barriers

// The arrays of the geometry warp (GEO): the mesh, the FP64 tables of the
// collocation stages and the handle's float32 copy it writes.
struct TcGeoArgs {
    const double *coords;
    const int32_t *conn;
    long long n_nodes;
    const double *b1d, *dq, *w;  // B (3 x 3), Dq (3 x 3) + GEO_DQ_EXTRA, w (27)
    float *jinv_out, *wdetj_out;
};

constexpr int TC_GEO_WARP = 6;  // first geometry warp

template <int MODE, bool GEO, int FORM>
__global__ void __launch_bounds__(TC_THREADS_WS + (GEO ? 32 * TC_NGEO : 0), MODE == TC_TF32X3 ? 2 : 3)
    k_matrix_tc(const float *__restrict__ jinv, const float *__restrict__ wdetj, const float *__restrict__ dphi,
                long long E, const double *__restrict__ lame, float *__restrict__ K,
                unsigned long long *__restrict__ status, const int *__restrict__ hold, TcGeoArgs geo,
                const double *__restrict__ coef, float *__restrict__ K2)
{
    static_assert(FORM != TC_PAIR || (MODE == TC_TF32X3 && !GEO), "the pair runs TF32x3 on a stored geometry");
    constexpr bool ELASTF = FORM != TC_LAPL;  // elasticity (alone or with the Laplacian)
    using P = TcSmem<MODE, GEO>;
    using L = typename P::L;
    constexpr int NTHREADS = TC_THREADS_WS + (GEO ? 32 * TC_NGEO : 0);
    extern __shared__ __align__(1024) unsigned char smem[];
    float *ks = reinterpret_cast<float *>(smem + P::KS);
    float *sJw = reinterpret_cast<float *>(smem + P::JW);
    float *sLM = reinterpret_cast<float *>(smem + P::LM);
    float *sDp = reinterpret_cast<float *>(smem + P::DP);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + P::MISC);       // [2]
    uint64_t *empty = reinterpret_cast<uint64_t *>(smem + P::MISC + 16); // [2]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + P::MISC + 32);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + P::MISC + 36);
    uint64_t *accfree = reinterpret_cast<uint64_t *>(smem + P::MISC + 40);  // [NACC] accumulator read out
    uint64_t *geo_full = reinterpret_cast<uint64_t *>(smem + P::GFULL);    // [RING] slot filled
    uint64_t *geo_empty = reinterpret_cast<uint64_t *>(smem + P::GEMPTY);  // [RING] slot read

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int i = tid; i < TC_Q * 3 * TC_N; i += NTHREADS) sDp[i] = dphi[i];
    if constexpr (GEO) {
        double *gt = reinterpret_cast<double *>(smem + P::GT);
        for (int i = tid; i < P::GT_LEN; i += NTHREADS)
            gt[i] = i < 9 ? geo.b1d[i] : (i < 18 + GEO_DQ_EXTRA ? geo.dq[i - 9] : geo.w[i - 18 - GEO_DQ_EXTRA]);
    }
    if (tid == 0) {
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(full + b)), "r"(1) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(empty + b)), "r"(1) : "memory");
        }
#pragma unroll
        for (int b = 0; b < P::NACC; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(accfree + b)), "r"(1) : "memory");
        for (int b = 0; b < P::RING; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(geo_full + b)), "r"(1) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(geo_empty + b)), "r"(1) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *abort_flag = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(P::NACC * TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (GEO && warp >= TC_GEO_WARP) {
        // ------------------------------------------------------------ geometry
        // one 1-D line per lane; the connectivity is read two elements ahead and
        // the coordinates one, so that no load waits on another
        if constexpr (GEO) {
            const int gw_id = warp - TC_GEO_WARP;
            double *gS = reinterpret_cast<double *>(smem + P::GS) + gw_id * P::GS_WARP;  // [4][81]
            const double *gB = reinterpret_cast<const double *>(smem + P::GT);
            const double *gDq = gB + 9;
            const double *gw = gDq + 9 + GEO_DQ_EXTRA;
            float *ring = reinterpret_cast<float *>(smem + P::JW);
            double px[3] = {0.0, 0.0, 0.0};  // this lane's node of the next element
            double plm = 0.0;                // lanes 27, 28: its lambda, mu
            long long pnode = 0;             // this lane's node index of the element after
            auto fetch_node = [&](long long e) {
                if (e < E && lane < TC_N) pnode = geo.conn[e * TC_N + lane];
            };
            auto fetch = [&](long long e) {  // with pnode = the node of element e
                if (e >= E) return;
                if (lane < TC_N) {
                    const bool ok = (unsigned long long)pnode < (unsigned long long)geo.n_nodes;  // never read outside
                    if (!ok) fe_report(status, FE_ERR_SHAPE, e);
                    const long long nd = ok ? pnode : 0;
#pragma unroll
                    for (int c = 0; c < 3; ++c) px[c] = geo.coords[3 * nd + c];
                } else if (lane < TC_N + 2) {
                    plm = lame[2 * e + lane - TC_N];
                }
            };
            // element n of this CTA goes to geometry warp n % TC_NGEO, ring slot n % RING
            const long long stride = (long long)gridDim.x * TC_NGEO;
            long long e = blockIdx.x + (long long)gw_id * gridDim.x;
            fetch_node(e);
            fetch(e);
            fetch_node(e + stride);
            for (int n = gw_id; e < E; e += stride, n += TC_NGEO) {
                const int sl = n % P::RING;
                float *slot = ring + sl * P::SLOT;
                // the slot is free once the producers have read its previous element
                if (n >= P::RING) {
                    if (lane == 0 &&
                        !mbar_wait_bounded(smem_u32(geo_empty + sl), ((n / P::RING) - 1) & 1, abort_flag)) {
                        *abort_flag = 1;
                        fe_report(status, FE_ERR_TIMEOUT, e);
                    }
                    __syncwarp();
                    if (*abort_flag) break;
                }
                if (lane < TC_N) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) gS[c * TC_N + lane] = px[c];
                }
                const float lm = (float)plm;
                fetch(e + stride);
                fetch_node(e + 2 * stride);
                __syncwarp();
                if (lane < TC_N) geo_lines_x<3, true>(lane, gS, gS + 81, gB);  // contract i
                __syncwarp();
                if (lane < TC_N) geo_lines_y<3, true>(lane, gS + 81, gS + 162, gB);  // contract j
                __syncwarp();
                if (lane < TC_N) geo_lines_z<3, true>(lane, gS + 162, gS, gB);  // contract k: x at the points
                __syncwarp();
                // J on the points: 81 lines, three per lane (the third for lanes < 17)
                geo_lines_jacobian<3, true>(lane, gS, gS + 81, gDq);
                geo_lines_jacobian<3, true>(lane + 32, gS, gS + 81, gDq);
                if (lane + 64 < 3 * TC_N) geo_lines_jacobian<3, true>(lane + 64, gS, gS + 81, gDq);
                __syncwarp();
                if (lane < TC_Q) {
                    float o[9], wd;
                    const double det = geo_point_f32(gS + 81 + lane * 9, gw[lane], o, wd);
                    const int bad = geo_det_status(det);
                    if (bad) fe_report(status, bad, e);
                    const long long idx = e * TC_Q + lane;
#pragma unroll
                    for (int k = 0; k < 9; ++k) geo.jinv_out[idx * 9 + k] = o[k];
                    geo.wdetj_out[idx] = wd;
                    const float sw = sqrtf(wd);
#pragma unroll
                    for (int k = 0; k < 9; ++k) slot[lane * TC_JW_STRIDE + k] = sw * o[k];
                } else if (lane < TC_Q + 2) {
                    slot[TC_Q * TC_JW_STRIDE + lane - TC_Q] = lm;
                }
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(geo_full + sl))
                                            : "memory");
            }
        }
    } else if (warp >= 3) {
        // ------------------------------------------------------------ producer
        const int ptid = tid - TC_CONS, pw = warp - 3;
        constexpr int NPF = (TC_Q * 9 + TC_PROD - 1) / TC_PROD;  // 3 per thread
        float pj[NPF], pwt[NPF];
        double plm = 0.0;
        auto prefetch = [&](long long e) {
            if constexpr (!GEO) {
                if (e >= E) return;
#pragma unroll
                for (int u = 0; u < NPF; ++u) {
                    const int t = ptid + u * TC_PROD;
                    if (t < TC_Q * 9) {
                        pj[u] = jinv[e * TC_Q * 9 + t];
                        pwt[u] = wdetj[e * TC_Q + t / 9];
                    }
                }
                if constexpr (FORM == TC_LAPL) {
                    if (ptid == 0) plm = lame ? lame[e] : 1.0;
                } else {
                    if (ptid < 2) plm = lame[2 * e + ptid];
                    if (FORM == TC_PAIR && ptid == 2) plm = coef ? coef[e] : 1.0;
                }
            }
        };
        prefetch(blockIdx.x);
        constexpr int SEGV = 4 / P::EB;            // points per 4-byte segment: 1 (tf32) or 2 (bf16)
        constexpr int NCH = TC_KPAD / L::CHUNK;    // K chunks: 8 (tf32) or 4 (bf16)
        constexpr int PCH = (NCH + 2) / 3;         // chunks per producer warp
        const int r = lane >> 2, seg = lane & 3;
        float dreg[PCH][4][SEGV][3];
#pragma unroll
        for (int ci = 0; ci < PCH; ++ci)
#pragma unroll
            for (int g = 0; g < 4; ++g)
#pragma unroll
                for (int v = 0; v < SEGV; ++v) {
                    const int q = (pw + 3 * ci) * L::CHUNK + seg * SEGV + v, a = 8 * g + r;
                    const bool ok = q < TC_Q && a < TC_N && pw + 3 * ci < NCH;
#pragma unroll
                    for (int k = 0; k < 3; ++k) dreg[ci][g][v][k] = ok ? sDp[(q * 3 + k) * TC_N + a] : 0.0f;
                }
        int n = 0;
        int last_b = -1;  // thread 0: buffer and phase parity of the last MMA commit
        uint32_t last_parity = 0;
        for (long long e = blockIdx.x; e < E; e += gridDim.x, ++n) {
            const int sl = GEO ? n % (GEO ? P::RING : 1) : 0;  // GEO: ring slot of element n
            if constexpr (GEO) {
                // (a) the geometry warp's ring slot of element n
                if (ptid == 0 && !mbar_wait_bounded(smem_u32(geo_full + sl), (n / (GEO ? P::RING : 1)) & 1,
                                                    abort_flag)) {
                    *abort_flag = 1;
                    fe_report(status, FE_ERR_TIMEOUT, e);
                }
                named_sync(TC_BAR_PROD, TC_PROD);
                if (*abort_flag) break;
            }
            const int b = n & 1;
            unsigned char *opHi = smem + b * P::BUF + P::HI;
            unsigned char *opLo = smem + b * P::BUF + P::LO;
            float *jw = GEO ? sJw + sl * P::SLOT : sJw + b * TC_Q * TC_JW_STRIDE;
            // the buffer and its accumulator are free once element n-2's epilogue is done
            if (n >= 2) {
                if (ptid == 0 && !mbar_wait_bounded(smem_u32(empty + b), ((n >> 1) - 1) & 1, abort_flag)) {
                    *abort_flag = 1;
                    fe_report(status, FE_ERR_TIMEOUT, e);
                }
                named_sync(TC_BAR_PROD, TC_PROD);
                if (*abort_flag) break;
                tc_fence_after();
            }
            if constexpr (GEO) {
                // the Lame pair for the consumers
                if (ptid < 2) sLM[2 * b + ptid] = jw[TC_Q * TC_JW_STRIDE + ptid];
            } else {
                // (a) geometry of the element, then start fetching the next one
#pragma unroll
                for (int u = 0; u < NPF; ++u) {
                    const int t = ptid + u * TC_PROD;
                    if (t < TC_Q * 9) jw[(t / 9) * TC_JW_STRIDE + t % 9] = sqrtf(pwt[u]) * pj[u];
                }
                if (ptid < 2) sLM[2 * b + ptid] = (float)plm;
                if (FORM == TC_PAIR && ptid == 2) reinterpret_cast<float *>(smem + P::LC)[b] = (float)plm;
                prefetch(e + gridDim.x);
                named_sync(TC_BAR_PROD, TC_PROD);
            }

            // (b) X[(j,a)][q] split into hi/lo: lane (r, seg) owns node a = 8 g + r and
            // the points of its 4-byte segment, for the three row blocks j; warp pw
            // takes the K chunks c = pw, pw + 3, ...  The reference gradients of these
            // (q, a) pairs live in registers for the whole kernel; sqrt(w det J) J^-1
            // of a point is read once per chunk.  Valid rows get zeros past the last
            // point (the buffer held the exchange data of element n-2).
#pragma unroll
            for (int ci = 0; ci < PCH; ++ci) {
                const int c = pw + 3 * ci;
                if (c >= NCH) break;
                const int q0 = c * L::CHUNK + seg * SEGV;
                float J[SEGV][12];
#pragma unroll
                for (int v = 0; v < SEGV; ++v) {
                    const int q = q0 + v < TC_Q ? q0 + v : 0;
                    const float4 *jq = reinterpret_cast<const float4 *>(jw + q * TC_JW_STRIDE);
#pragma unroll
                    for (int t = 0; t < 3; ++t) {
                        const float4 x = jq[t];
                        J[v][4 * t] = x.x;
                        J[v][4 * t + 1] = x.y;
                        J[v][4 * t + 2] = x.z;
                        J[v][4 * t + 3] = x.w;
                    }
                }
#pragma unroll
                for (int g = 0; g < 4; ++g) {
                    const int a = 8 * g + r;
                    if (a >= TC_N) continue;
                    // X values of the lane's points (zero past the last point)
                    float x[SEGV][3];
#pragma unroll
                    for (int v = 0; v < SEGV; ++v) {
                        const float *dd = dreg[ci][g][v];
#pragma unroll
                        for (int j = 0; j < 3; ++j)
                            x[v][j] = q0 + v < TC_Q ? dd[0] * J[v][j] + dd[1] * J[v][3 + j] + dd[2] * J[v][6 + j]
                                                    : 0.0f;
                    }
                    uint32_t hv[3], lv[3];
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        if constexpr (MODE == TC_TF32X3) split<MODE>(x[0][j], hv[j], lv[j]);
                        else if constexpr (MODE == TC_BF16X3) split_bf16x2(x[1][j], x[0][j], hv[j], lv[j]);
                        else hv[j] = pack_bf16x2(x[1][j], x[0][j]);
                    }
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const int off = L::offset(32 * j + a, q0);
                        *reinterpret_cast<uint32_t *>(opHi + off) = hv[j];
                        if constexpr (MODE != TC_BF16) *reinterpret_cast<uint32_t *>(opLo + off) = lv[j];
                    }
                }
            }
            fence_async_smem();  // operand writes -> tensor-core (async) proxy
            named_sync(TC_BAR_PROD, TC_PROD);
            if (GEO && ptid == 0)  // the ring slot has been read: back to the geometry warp
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(geo_empty + sl)) : "memory");

            // (c) MMA chain into the accumulator once the consumers have read out
            // element n-1's: D = sum over K steps of hi*hi (+ hi*lo + lo*hi)
            const int acc = n % P::NACC;
            if (ptid == 0) {
                if (n >= P::NACC && !mbar_wait_bounded(smem_u32(accfree + acc), (n / P::NACC - 1) & 1, abort_flag)) {
                    *abort_flag = 1;
                    fe_report(status, FE_ERR_TIMEOUT, e);
                }
            }
            if (ptid == 0 && !*abort_flag) {
                tc_fence_after();
                constexpr int KSTEP_BYTES = 2 * L::LBO;  // one MMA consumes two 16-byte K chunks
                constexpr int NSTEP = TC_KPAD / (2 * L::CHUNK);
                const uint32_t hi = smem_u32(opHi), lo = smem_u32(opLo);
                const uint32_t d_tmem = tmem + acc * TC_TMEM_COLS;
#pragma unroll
                for (int s = 0; s < NSTEP; ++s) {
                    const uint64_t dh = smem_desc(hi + s * KSTEP_BYTES, L::LBO, L::SBO);
                    mma<MODE, TC_M, TC_NCOL>(d_tmem, dh, dh, s > 0 ? 1u : 0u);
                    if constexpr (MODE != TC_BF16) {
                        const uint64_t dl = smem_desc(lo + s * KSTEP_BYTES, L::LBO, L::SBO);
                        mma<MODE, TC_M, TC_NCOL>(d_tmem, dh, dl, 1u);
                        mma<MODE, TC_M, TC_NCOL>(d_tmem, dl, dh, 1u);
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(full + b))
                             : "memory");
                last_b = b;
                last_parity = (uint32_t)((n >> 1) & 1);
            }
        }
        // an aborting CTA frees its tensor memory only after the MMAs it issued are
        // done (a commit completes when all earlier MMAs of the thread have)
        if (ptid == 0 && *abort_flag && last_b >= 0) mbar_wait_cycles(smem_u32(full + last_b), last_parity);
    } else {
        // ------------------------------------------------------------ consumer
        const int ctid = tid;
        if (hold) {
            // test hook: wait on a flag that nothing sets, so that the bounded wait
            // runs out and the abort path is taken
            if (ctid == 0) {
                const long long t0 = clock64();
                while (*(volatile const int *)hold == 0) {
                    if (clock64() - t0 > TC_WAIT_CYCLES) {
                        *abort_flag = 1;
                        fe_report(status, FE_ERR_TIMEOUT, blockIdx.x);
                        break;
                    }
                }
            }
            named_sync(TC_BAR_CONS, TC_CONS);
        }
        int n = 0;
        for (long long e = blockIdx.x; e < E; e += gridDim.x, ++n) {
            const int b = n & 1;
            float *ex = reinterpret_cast<float *>(smem + b * P::BUF);
            // (d) accumulator of element n complete
            if (ctid == 0 && !mbar_wait_bounded(smem_u32(full + b), (n >> 1) & 1, abort_flag)) {
                *abort_flag = 1;
                fe_report(status, FE_ERR_TIMEOUT, e);
            }
            named_sync(TC_BAR_CONS, TC_CONS);
            if (*abort_flag) break;
            tc_fence_after();

            // (e) rows (j = warp, a = lane) of the accumulator: the two blocks this warp
            // uses (A_jj, A_j,j+1) -> registers; the accumulator is then handed back
            // to the producers, and the blocks go to the exchange area
            float d[ELASTF ? 64 : 32];
            {
                const int jn = warp == 2 ? 0 : warp + 1;
                const uint32_t taddr = tmem + (n % P::NACC) * TC_TMEM_COLS + ((uint32_t)(32 * warp) << 16);
                tmem_ld32(taddr + 32 * warp, d);
                if constexpr (ELASTF) tmem_ld32(taddr + 32 * jn, d + 32);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            }
            tc_fence_before();
            named_sync(TC_BAR_CONS, TC_CONS);
            if (ctid == 0)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(accfree + n % P::NACC))
                             : "memory");
            if (lane < TC_N) {
                // ex[w][0] = A_ww, ex[w][1] = A_w,w+1 (rows a, columns b)
                float *e0 = ex + ((warp * 2 + 0) * TC_N + lane) * P::EX_STRIDE;
                if constexpr (ELASTF) {
                    float *e1 = ex + ((warp * 2 + 1) * TC_N + lane) * P::EX_STRIDE;
                    publish_blocks(d, e0, e1);
                } else {
#pragma unroll
                    for (int c = 0; c < 7; ++c)
                        reinterpret_cast<float4 *>(e0)[c] = make_float4(d[4 * c], d[4 * c + 1], d[4 * c + 2], d[4 * c + 3]);
                }
            }
            if (ctid == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");  // staging drained
            named_sync(TC_BAR_CONS, TC_CONS);

            // (f) elasticity: blocks K_ii and K_i,i+1 of row (i = warp, a = lane), and
            // K_i+1,i as columns; Laplacian: row a, columns 4c..4c+3 per item (a, c)
            constexpr int NR = ELASTF ? TC_NROW : TC_N;  // rows (and columns) of K_e
            const float *dst0 = K + e * (long long)(NR * NR);
            const int shift = (int)(((unsigned long long)dst0 % 16) / 4);
            float *kst = ks + shift;
            // the Laplacian c sum_j A_jj (TC_LAPL into kst; TC_PAIR into its own staging)
            float *lst = kst;
            if constexpr (FORM == TC_PAIR)
                lst = reinterpret_cast<float *>(smem + P::LS) +
                      (int)(((unsigned long long)(K2 + e * (long long)(TC_N * TC_N)) % 16) / 4);
            if constexpr (ELASTF) {
                if (lane < TC_N) {
                    const float lam = sLM[2 * b], mu = sLM[2 * b + 1];
                    epilogue_rows<P::EX_STRIDE>(warp, d, ex, lane, lam, mu, kst);
                }
            }
            if constexpr (FORM != TC_ELAST) {
                const float cw = FORM == TC_PAIR ? reinterpret_cast<const float *>(smem + P::LC)[b] : sLM[2 * b];
                for (int it = ctid; it < TC_N * 7; it += TC_CONS) {
                    const int a = it / 7, c = it % 7;
                    const float4 x0 = reinterpret_cast<const float4 *>(ex + (0 * 2 * TC_N + a) * P::EX_STRIDE)[c];
                    const float4 x1 = reinterpret_cast<const float4 *>(ex + (1 * 2 * TC_N + a) * P::EX_STRIDE)[c];
                    const float4 x2 = reinterpret_cast<const float4 *>(ex + (2 * 2 * TC_N + a) * P::EX_STRIDE)[c];
                    const float v[4] = {cw * (x0.x + x1.x + x2.x), cw * (x0.y + x1.y + x2.y),
                                        cw * (x0.z + x1.z + x2.z), cw * (x0.w + x1.w + x2.w)};
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if (4 * c + i < TC_N) lst[a * TC_N + 4 * c + i] = v[i];
                }
            }
            fence_async_smem();
            named_sync(TC_BAR_CONS, TC_CONS);

            // (g) one bulk copy per element matrix; buffer b goes back to the producers
            if (ctid == 0) {
                float *dst = K + e * (long long)(NR * NR);
                constexpr int LEN = NR * NR;
                const int head = (4 - shift) % 4;
                const int body = (LEN - head) / 4 * 4;
                for (int t = 0; t < head; ++t) dst[t] = kst[t];
                for (int t = head + body; t < LEN; ++t) dst[t] = kst[t];
                bulk_store(dst + head, kst + head, (unsigned)(body * 4));
                if constexpr (FORM == TC_PAIR) {
                    float *dl = K2 + e * (long long)(TC_N * TC_N);
                    constexpr int LL = TC_N * TC_N;
                    const int hl = (int)((4 - ((unsigned long long)dl % 16) / 4) % 4);
                    const int bdl = (LL - hl) / 4 * 4;
                    for (int t = 0; t < hl; ++t) dl[t] = lst[t];
                    for (int t = hl + bdl; t < LL; ++t) dl[t] = lst[t];
                    bulk_store(dl + hl, lst + hl, (unsigned)(bdl * 4));
                }
                asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(empty + b)) : "memory");
            }
        }
        if (ctid == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(P::NACC * TC_TMEM_COLS)
                     : "memory");
}

template <int MODE, bool GEO, int FORM>
cudaError_t launch_tc(const fe_geometry_h *g, fe_material_args mat, void *K, int sm_count,
                      unsigned long long *status, const int *hold, cudaStream_t s, const double *coef = nullptr,
                      void *K2 = nullptr)
{
    using P = TcSmem<MODE, GEO>;
    constexpr int SMEM = FORM == TC_PAIR ? P::BYTES_PAIR : P::BYTES;
    static_assert(SMEM <= 227 * 1024, "shared memory plan too large");
    static_assert(MODE == TC_TF32X3 || 3 * (P::BYTES + 1024) <= 228 * 1024, "three CTAs per SM in the BF16 modes");
    constexpr int NTHREADS = TC_THREADS_WS + (GEO ? 32 * TC_NGEO : 0);
    auto kern = k_matrix_tc<MODE, GEO, FORM>;
    // resident CTAs per SM: shared memory (228 KB per SM, 1 KB reserved per CTA),
    // registers, and the 512 tensor-memory columns of which every CTA holds
    // NACC x TC_TMEM_COLS (a persistent CTA waiting for columns would stall in
    // tcgen05.alloc)
    static FeLaunchCache cache;
    long long per_sm = 0;
    cudaError_t err = fe_cached_grid(
        cache,
        [&](int dev, long long *v) {
            cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
            if (e2 != cudaSuccess) return e2;
            e2 = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
            if (e2 != cudaSuccess) return e2;
            int smem_sm = 0, regs_sm = 0;
            cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
            cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
            cudaFuncAttributes fa{};
            e2 = cudaFuncGetAttributes(&fa, kern);
            if (e2 != cudaSuccess) return e2;
            int n = smem_sm / (SMEM + 1024);
            // registers: whole warps in each of the four sub-partitions (regs_sm / 4 each)
            const int warp_regs = (fa.numRegs * 32 + 255) / 256 * 256;
            const int by_regs = 4 * ((regs_sm / 4) / warp_regs) / (NTHREADS / 32);
            if (by_regs < n) n = by_regs;
            if (n * P::NACC * TC_TMEM_COLS > 512) n = 512 / (P::NACC * TC_TMEM_COLS);
            if (n < 1) return cudaErrorInvalidConfiguration;
            *v = n;
            return cudaSuccess;
        },
        &per_sm);
    if (err != cudaSuccess) return err;
    long long blocks = per_sm * sm_count;
    if (blocks > g->mesh.n_elems) blocks = g->mesh.n_elems;
    TcGeoArgs geo{};
    if (GEO) {
        geo.coords = g->mesh.coords;
        geo.conn = g->mesh.conn;
        geo.n_nodes = g->mesh.n_nodes;
        geo.b1d = g->d_b1d;
        geo.dq = g->d_dq;
        geo.w = g->d_w64;
        geo.jinv_out = g->d_jinv32;
        geo.wdetj_out = g->d_wdetj32;
    }
    kern<<<(unsigned)blocks, NTHREADS, SMEM, s>>>(g->d_jinv32, g->d_wdetj32, g->d_dphi32, g->mesh.n_elems,
                                                  mat.data, (float *)K, status, hold, geo, coef, (float *)K2);
    return cudaGetLastError();
}

template <bool GEO, int FORM>
cudaError_t dispatch_tc(const fe_geometry_h *g, fe_material_args mat, fe_precision prec, void *K, int sm_count,
                        unsigned long long *status, const int *hold, cudaStream_t s)
{
    switch (prec) {
    case FE_TF32X3: return launch_tc<TC_TF32X3, GEO, FORM>(g, mat, K, sm_count, status, hold, s);
    case FE_BF16X3: return launch_tc<TC_BF16X3, GEO, FORM>(g, mat, K, sm_count, status, hold, s);
    case FE_BF16: return launch_tc<TC_BF16, GEO, FORM>(g, mat, K, sm_count, status, hold, s);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace

bool fe_matrix_tc_supported(const fe_geometry_h *g, const fe_form_h *f, fe_precision prec)
{
    // P3 tetrahedra with the 35-point Grundmann-Moller rule, TF32x3 (k_matrix_tcs.cu)
    if (g->N == 20 && g->Q == 35) return fe_matrix_tcs_supported(g, f, prec);
    const bool lame = f->kind == FK_ELASTICITY && f->mat == FE_MAT_LAME && !f->mat_transposed;
    // 64-node hexahedra with 64 points, TF32x3 (k_matrix_tc64.cu): Lame elasticity,
    // the scalar Laplacian and the scalar mass matrix
    if (g->N == 64 && g->Q == 64)
        return prec == FE_TF32X3 && (lame || ((f->kind == FK_LAPLACE || f->kind == FK_MASS) && f->ncomp == 1));
    // 27-node hexahedra with 27 points: Lame elasticity, or the (weighted) scalar Laplacian
    if (g->N != TC_N || g->Q != TC_Q) return false;
    return lame || (f->kind == FK_LAPLACE && f->ncomp == 1);
}

bool fe_matrix_tc_geometry_fusable(const fe_geometry_h *g)
{
    // a stale deferred handle keeping only the float32 copy, Q2 with 3 x 3 x 3
    // Gauss points whose middle point is the middle node (collocation stages)
    return g->pending && g->d_dq && g->geo_center && g->n1d == 3 && g->nq1d == 3 && g->N == TC_N &&
           g->Q == TC_Q && g->d_jinv32 && !g->is_view && (g->flags & FE_GEOM_STORE_F32) &&
           !(g->flags & FE_GEOM_STORE_F64);
}

cudaError_t fe_launch_matrix_tc(const fe_geometry_h *g, const fe_form_h *f, fe_material_args mat, fe_precision prec,
                                void *K, int sm_count, unsigned long long *status, const int *hold,
                                bool with_geometry, cudaStream_t s)
{
    if (g->mesh.n_elems == 0) return cudaSuccess;
    if (!fe_matrix_tc_supported(g, f, prec)) return cudaErrorNotSupported;
    if (g->N == 64 || g->N == 20) {
        if (with_geometry || hold) return cudaErrorNotSupported;
        return g->N == 64 ? fe_launch_matrix_tc64(g, f, mat, prec, K, sm_count, status, s)
                          : fe_launch_matrix_tcs(g, f, mat, prec, K, sm_count, status, s);
    }
    const bool elast = f->kind == FK_ELASTICITY;
    if (elast && mat.kind != FE_MAT_LAME) return cudaErrorNotSupported;
    if (with_geometry) {
        if (!elast || !fe_matrix_tc_geometry_fusable(g)) return cudaErrorNotSupported;
        return dispatch_tc<true, TC_ELAST>(g, mat, prec, K, sm_count, status, hold, s);
    }
    return elast ? dispatch_tc<false, TC_ELAST>(g, mat, prec, K, sm_count, status, hold, s)
                 : dispatch_tc<false, TC_LAPL>(g, mat, prec, K, sm_count, status, hold, s);
}

bool fe_matrix_tc_pair_supported(const fe_geometry_h *g)
{
    if (g->N == TC_N && g->Q == TC_Q) return g->d_jinv32 && g->d_dphi32;
    return fe_matrix_tc64_pair_supported(g);
}

cudaError_t fe_launch_matrix_tc_pair(const fe_geometry_h *g, const double *lame, void *K, const double *coef,
                                     void *K2, int sm_count, unsigned long long *status, cudaStream_t s)
{
    if (g->mesh.n_elems == 0) return cudaSuccess;
    if (!fe_matrix_tc_pair_supported(g)) return cudaErrorNotSupported;
    if (g->N != TC_N) return fe_launch_matrix_tc64_pair(g, lame, K, coef, K2, sm_count, status, s);
    fe_material_args mat{};
    mat.kind = FE_MAT_LAME;
    mat.data = lame;
    return launch_tc<TC_TF32X3, false, TC_PAIR>(g, mat, K, sm_count, status, nullptr, s, coef, K2);
}
