// Device code of the SIMT matrix mode (Algorithm 2 of Cimrman, arXiv
// 2107.04121): shared-memory plan, tile loads and the per-element-group body
// matrix_group, shared by the standalone matrix kernel (k_matrix.cu) and the
// batched persistent kernel (k_batch.cu).  See k_matrix.cu for the design.
#pragma once

#include "fe_device.cuh"

namespace {

__host__ __device__ constexpr int gcd_const(int a, int b) { return b == 0 ? a : gcd_const(b, a % b); }

// Padded position of node a inside its group of T: groups start on 16 bytes,
// except FP32 pairs, which are read as float2 and need only 8.
template <int T, typename S>
__host__ __device__ constexpr int tile_pad()
{
    return T == 2 && sizeof(S) == 4 ? 2 : (T * (int)sizeof(S) + 15) / 16 * 16 / (int)sizeof(S);
}

template <typename S, int T>
struct TileVec {
    // load T consecutive values starting at a 16-byte aligned address
    __device__ __forceinline__ static void load(const S *p, S *v)
    {
#pragma unroll
        for (int x = 0; x < T; ++x) v[x] = p[x];
    }
};
template <>
struct TileVec<float, 3> {
    __device__ __forceinline__ static void load(const float *p, float *v)
    {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        v[0] = q.x;
        v[1] = q.y;
        v[2] = q.z;
    }
};
template <>
struct TileVec<float, 4> {
    __device__ __forceinline__ static void load(const float *p, float *v)
    {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        v[0] = q.x;
        v[1] = q.y;
        v[2] = q.z;
        v[3] = q.w;
    }
};
template <>
struct TileVec<float, 2> {
    __device__ __forceinline__ static void load(const float *p, float *v)
    {
        const float2 q = *reinterpret_cast<const float2 *>(p);
        v[0] = q.x;
        v[1] = q.y;
    }
};
template <>
struct TileVec<double, 2> {
    __device__ __forceinline__ static void load(const double *p, double *v)
    {
        const double2 q = *reinterpret_cast<const double2 *>(p);
        v[0] = q.x;
        v[1] = q.y;
    }
};
template <>
struct TileVec<double, 4> {
    __device__ __forceinline__ static void load(const double *p, double *v)
    {
        const double2 q0 = *reinterpret_cast<const double2 *>(p);
        const double2 q1 = *reinterpret_cast<const double2 *>(p + 2);
        v[0] = q0.x;
        v[1] = q0.y;
        v[2] = q1.x;
        v[3] = q1.y;
    }
};
template <>
struct TileVec<double, 3> {
    __device__ __forceinline__ static void load(const double *p, double *v)
    {
        const double2 q0 = *reinterpret_cast<const double2 *>(p);
        v[0] = q0.x;
        v[1] = q0.y;
        v[2] = p[2];
    }
};

// Output paths of the element matrices:
//   STAGE_DIRECT  scattered stores straight from registers
//   STAGE_FULL    all EPB matrices staged in shared memory, copied out with
//                 coalesced 16-byte stores
//   STAGE_BULK    one component row block (N rows) at a time, double-buffered
//                 in shared memory and written by asynchronous bulk copies
//                 (cp.async.bulk), which overlap with the next block
constexpr int STAGE_DIRECT = 0, STAGE_FULL = 1, STAGE_BULK = 2;

__device__ __forceinline__ void bulk_store(void *gdst, const void *ssrc, unsigned bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst),
                 "r"((unsigned)__cvta_generic_to_shared(ssrc)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void bulk_wait_read()
{
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(PENDING) : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Quadrature rules of the supported (N, Q) pairs: Gauss (hexahedra, positive
// weights) or Grundmann-Moller of index >= 1 (tetrahedra, negative weights).
__host__ __device__ constexpr bool rule_weights_positive(int N, int Q)
{
    return !((N == 4 && Q == 5) || (N == 10 && Q == 15) || (N == 20 && Q == 35));
}

// Shared-memory plan of one CTA (sizes in elements of S).
template <typename S, int N, int Q, int KIND, int T, int EPB, int STAGE>
struct MatrixSmem {
    static constexpr bool GRAD = KIND != FK_MASS;
    static constexpr int V = 16 / (int)sizeof(S);
    static constexpr int TP = tile_pad<T, S>();
    static constexpr int NP = (N / T) * TP;  // padded node count
    static constexpr int G_SIZE = GRAD ? EPB * Q * 3 * NP : Q * NP;
    static constexpr int NROW_MAX = (KIND == FK_LAPLACE ? 1 : 3) * N;
    // bulk staging slot: one row block of one element, +16 bytes of alignment shift
    static constexpr int SLOT = (N * NROW_MAX + V + V - 1) / V * V;
    // staged matrices, +16 bytes to shift the chunk onto the global alignment
    static constexpr int K_SIZE = STAGE == STAGE_FULL   ? EPB * NROW_MAX * NROW_MAX + V
                                  : STAGE == STAGE_BULK ? 2 * EPB * SLOT
                                                        : 0;
    static constexpr int GK = G_SIZE > K_SIZE ? G_SIZE : K_SIZE;  // K staging reuses the G buffer
    static constexpr int J_OFF = GK;
    static constexpr int W_OFF = J_OFF + EPB * Q * 9;
    static constexpr int C_OFF = W_OFF + EPB * Q;
    static constexpr int D_OFF = C_OFF + EPB * 81;      // reference gradients (Q, 3, N), loaded once
    // tables above 16 KB (Q3: 48 KB) stay in global memory (read through L1 by the
    // gradient build), so that the plan leaves room for more resident CTAs
    static constexpr bool REF_SMEM = GRAD && Q * 3 * N * (int)sizeof(S) <= 16384;
    static constexpr int TOTAL = D_OFF + (REF_SMEM ? Q * 3 * N : 0);
    static constexpr size_t BYTES = sizeof(S) * (size_t)TOTAL;
};

// One group of ne <= EPB consecutive elements starting at e0, computed by the
// THREADS threads of the CTA (one upper-triangle tile per thread; threads past
// ne * NU only join the barriers).  The reference gradients must already be in
// the plan's D region (matrix_load_ref) when the plan keeps them there
// (REF_SMEM); otherwise they are read from dphi.  MATK: 0 scalar coefficient (or none),
// 1 Lame pair, 2 general D (6x6 Voigt).  LAP2 (Lame elasticity, bulk staging): the
// weighted scalar Laplacian of the same elements, c sum_j A_jj, is written to K2 from
// the same Gram blocks (c from mat2, 1 where mat2 is NULL).
template <typename S, int N, int Q, int KIND, int MATK, int T, int EPB, int THREADS, int STAGE, bool LAP2 = false>
__device__ __forceinline__ void matrix_group(const S *__restrict__ jinv, const S *__restrict__ wdetj,
                                             const S *__restrict__ phi, const S *__restrict__ dphi, long long e0,
                                             int ne, int ncomp,
                                             const double *__restrict__ mat, int mat_t, S *__restrict__ K,
                                             unsigned char *smem_raw, S *__restrict__ K2 = nullptr,
                                             const double *__restrict__ mat2 = nullptr)
{
    static_assert(!LAP2 || (KIND == FK_ELASTICITY && MATK == 1 && STAGE == STAGE_BULK),
                  "the shared-Gram Laplacian rides on the bulk-staged Lame elasticity");
    using P = MatrixSmem<S, N, Q, KIND, T, EPB, STAGE>;
    constexpr bool GRAD = P::GRAD;
    constexpr int TP = P::TP, NP = P::NP, NT = N / T, NU = NT * (NT + 1) / 2;
    // Gauss rules (hexahedra) have positive weights: both Gram operands carry
    // sqrt(w det J).  Grundmann-Moller rules (the tetrahedron pairs) have negative
    // weights: the gradients stay unscaled and one operand takes w det J.
    constexpr bool SQW = rule_weights_positive(N, Q);
    constexpr int NDIR = KIND == FK_ELASTICITY ? 3 : 1;
    S *sm = reinterpret_cast<S *>(smem_raw);
    S *sG = sm;
    S *sK = sm;
    S *sJ = sm + P::J_OFF;
    S *sW = sm + P::W_OFF;
    S *sC = sm + P::C_OFF;
    const S *sD = P::REF_SMEM ? sm + P::D_OFF : dphi;
    const int nrow = ncomp * N;
    {
        if constexpr (STAGE == STAGE_BULK)
            if (threadIdx.x == 0) bulk_wait_read<0>();  // staging (aliased with G) has been read out
        __syncthreads();  // previous iteration's copy-out has finished reading sK
        if constexpr (GRAD)
            for (int i = threadIdx.x; i < ne * Q * 9; i += THREADS) sJ[i] = jinv[e0 * Q * 9 + i];
        for (int i = threadIdx.x; i < ne * Q; i += THREADS) sW[i] = wdetj[e0 * Q + i];
        if constexpr (MATK == 2) {
            for (int i = threadIdx.x; i < ne * 81; i += THREADS) {
                const int el = i / 81, t = i % 81;
                const int ii = t / 27, jj = (t / 9) % 3, kk = (t / 3) % 3, ll = t % 3;
                const int I = fe_voigt(ii, jj), Kv = fe_voigt(kk, ll);
                const long long e = e0 + el;
                sC[i] = (S)(mat_t ? mat[e * 36 + Kv * 6 + I] : mat[e * 36 + I * 6 + Kv]);
            }
        } else if constexpr (MATK == 1) {
            for (int i = threadIdx.x; i < ne * 2; i += THREADS) sC[i] = (S)mat[e0 * 2 + i];
            if constexpr (LAP2)
                for (int i = threadIdx.x; i < ne; i += THREADS) sC[2 * EPB + i] = mat2 ? (S)mat2[e0 + i] : (S)1;
        } else {
            for (int i = threadIdx.x; i < ne; i += THREADS) sC[i] = mat ? (S)mat[e0 + i] : (S)1;
        }
        if constexpr (!GRAD)
            for (int i = threadIdx.x; i < Q * N; i += THREADS) {
                const int q = i / N, a = i % N;
                sG[q * NP + (a / T) * TP + a % T] = phi[i];
            }
        __syncthreads();
        if constexpr (GRAD) {
            // scaled physical gradients sqrt(w det J) G[el][q][j][a], G = J^-T grad_xi phi,
            // padded node index; the Gram blocks then need no weight in the inner loop
            // (det J > 0 is checked by the geometry kernel; Gauss weights are positive)
            if constexpr (SQW)
                for (int i = threadIdx.x; i < ne * Q; i += THREADS) {
                    const S sw = sqrt(sW[i]);
#pragma unroll
                    for (int t = 0; t < 9; ++t) sJ[i * 9 + t] *= sw;
                }
            __syncthreads();
            // A thread per point looping over the nodes is cheapest, but its lanes are
            // 3 NP words apart: where that stride shares 8 or more banks (Q1, Q3) one
            // (element, point, node) per thread, nodes fastest, keeps the reads of the
            // reference gradients and the writes of G on consecutive banks instead
            constexpr bool BY_NODE = gcd_const(3 * NP, 32) >= 8;
            if constexpr (BY_NODE) {
                for (int i = threadIdx.x; i < ne * Q * N; i += THREADS) {
                    const int a = i % N, eq = i / N, q = eq % Q;
                    const S *Ji = sJ + eq * 9;
                    const S *D0 = sD + q * 3 * N;
                    const S g0 = D0[a], g1 = D0[N + a], g2 = D0[2 * N + a];
                    S *Go = sG + eq * 3 * NP + (a / T) * TP + a % T;
#pragma unroll
                    for (int j = 0; j < 3; ++j) Go[j * NP] = g0 * Ji[j] + g1 * Ji[3 + j] + g2 * Ji[6 + j];
                }
            } else {
                for (int i = threadIdx.x; i < ne * Q; i += THREADS) {
                    const int q = i % Q;
                    S Ji[9];
#pragma unroll
                    for (int t = 0; t < 9; ++t) Ji[t] = sJ[i * 9 + t];
                    const S *D0 = sD + q * 3 * N;
                    S *Go = sG + i * 3 * NP;
#pragma unroll 3
                    for (int a = 0; a < N; ++a) {
                        const S g0 = D0[a], g1 = D0[N + a], g2 = D0[2 * N + a];
                        const int pa = (a / T) * TP + a % T;
#pragma unroll
                        for (int j = 0; j < 3; ++j) Go[j * NP + pa] = g0 * Ji[j] + g1 * Ji[3 + j] + g2 * Ji[6 + j];
                    }
                }
            }
            __syncthreads();
        }

        // ---- accumulate the upper tile triangle in registers: one tile per
        // thread, or (direct stores, no barriers below) as many passes over the
        // tiles as the CTA needs
        constexpr bool MULTI = STAGE == STAGE_DIRECT;
        const int n_pass = MULTI ? (ne * NU + THREADS - 1) / THREADS : 1;
        for (int tile_pass = 0; tile_pass < n_pass; ++tile_pass) {
        const int wi = threadIdx.x + tile_pass * THREADS;
        const bool active = wi < ne * NU;
        int el = 0, ta = 0, tb = 0;
        S acc[NDIR][NDIR][T][T];
#pragma unroll
        for (int j = 0; j < NDIR; ++j)
#pragma unroll
            for (int l = 0; l < NDIR; ++l)
#pragma unroll
                for (int x = 0; x < T; ++x)
#pragma unroll
                    for (int y = 0; y < T; ++y) acc[j][l][x][y] = 0;
        if (active) {
            el = wi / NU;
            int u = wi % NU;
            // u -> (ta, tb), ta <= tb, along the diagonals d = tb - ta: neighbouring
            // threads differ in both tile indices, so neither the tile's rows nor its
            // mirror's rows share a shared-memory bank across a warp
            int d = 0;
            while (u >= NT - d) {
                u -= NT - d;
                ++d;
            }
            ta = u;
            tb = u + d;
            const S *Wq = sW + el * Q;
#pragma unroll 9
            for (int q = 0; q < Q; ++q) {
                const S *Gq = GRAD ? sG + (el * Q + q) * 3 * NP : sG + q * NP;
                S ga[NDIR][T], gb[NDIR][T];
                if constexpr (KIND == FK_LAPLACE) {
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        S va[T], vb[T];
                        TileVec<S, T>::load(Gq + j * NP + ta * TP, va);
                        TileVec<S, T>::load(Gq + j * NP + tb * TP, vb);
                        if constexpr (!SQW)
#pragma unroll
                            for (int x = 0; x < T; ++x) va[x] *= Wq[q];
#pragma unroll
                        for (int x = 0; x < T; ++x)
#pragma unroll
                            for (int y = 0; y < T; ++y) acc[0][0][x][y] = fma(va[x], vb[y], acc[0][0][x][y]);
                    }
                } else {
                    const S wq = GRAD && SQW ? (S)1 : Wq[q];
#pragma unroll
                    for (int j = 0; j < NDIR; ++j) {
                        TileVec<S, T>::load(Gq + j * NP + ta * TP, ga[j]);
                        TileVec<S, T>::load(Gq + j * NP + tb * TP, gb[j]);
                        if constexpr (!GRAD || !SQW)
#pragma unroll
                            for (int x = 0; x < T; ++x) ga[j][x] *= wq;
                    }
#pragma unroll
                    for (int j = 0; j < NDIR; ++j)
#pragma unroll
                        for (int l = 0; l < NDIR; ++l)
#pragma unroll
                            for (int x = 0; x < T; ++x)
#pragma unroll
                                for (int y = 0; y < T; ++y) acc[j][l][x][y] = fma(ga[j][x], gb[l][y], acc[j][l][x][y]);
                }
            }
        }

        // ---- epilogue: element-matrix entries of this tile and its mirror image
        const int a0 = ta * T, b0 = tb * T;
        const bool mirror = ta != tb;
        S lam = 0, mu = 0;
        if constexpr (KIND == FK_ELASTICITY && MATK == 1) {
            lam = sC[el * 2];
            mu = sC[el * 2 + 1];
        }
        // entry (r, c) = ((i, a0+x), (k, b0+y)) of the tile and its mirror entry
        // ((k, b0+y), (i, a0+x)); emit(i, k, x, y, v, vt) receives both values
        auto for_entries = [&](auto &&emit) {
            if constexpr (KIND == FK_ELASTICITY) {
#pragma unroll
                for (int x = 0; x < T; ++x)
#pragma unroll
                    for (int y = 0; y < T; ++y) {
#pragma unroll
                        for (int i = 0; i < 3; ++i)
#pragma unroll
                            for (int k = 0; k < 3; ++k) {
                                S v, vt;
                                if constexpr (MATK == 1) {
                                    v = lam * acc[i][k][x][y] + mu * acc[k][i][x][y];
                                    if (i == k) v += mu * (acc[0][0][x][y] + acc[1][1][x][y] + acc[2][2][x][y]);
                                    vt = v;  // symmetric D: K is symmetric
                                } else {
                                    const S *C = sC + el * 81;  // general D: C_ijkl read from shared memory
                                    v = 0;
                                    vt = 0;
#pragma unroll
                                    for (int j = 0; j < 3; ++j)
#pragma unroll
                                        for (int l = 0; l < 3; ++l) {
                                            v = fma(C[i * 27 + j * 9 + k * 3 + l], acc[j][l][x][y], v);
                                            vt = fma(C[k * 27 + l * 9 + i * 3 + j], acc[j][l][x][y], vt);
                                        }
                                }
                                emit(i, k, x, y, v, vt);
                            }
                    }
            } else {
                const S c = sC[el];
#pragma unroll
                for (int x = 0; x < T; ++x)
#pragma unroll
                    for (int y = 0; y < T; ++y) {
                        const S v = c * acc[0][0][x][y];
                        for (int r = 0; r < ncomp; ++r)
                            for (int s2 = 0; s2 < ncomp; ++s2) emit(r, s2, x, y, r == s2 ? v : (S)0, r == s2 ? v : (S)0);
                    }
            }
        };

        if constexpr (STAGE == STAGE_BULK) {
            // one component row block per pass, double-buffered, drained by bulk copies
            constexpr int V = P::V;
            const int nblk = ncomp;
            const int blk_len = N * nrow;  // elements of one row block of one matrix
            // destination of row block pb of element e_l (pass nblk: the Laplacian into K2)
            auto dst_of = [&](int e_l, int pb) -> S * {
                if (LAP2 && pb == nblk) return K2 + (e0 + e_l) * (long long)(N * N);
                return K + (e0 + e_l) * (long long)nrow * nrow + (long long)pb * blk_len;
            };
            auto shift_of = [&](int e_l, int pb) {
                return (int)(((unsigned long long)dst_of(e_l, pb) % 16) / sizeof(S));
            };
            // entry ((i, a0+x), (k, b0+y)) of the elasticity matrix and of its mirror
            auto kval = [&](int i, int k, int x, int y) -> S {
                if constexpr (MATK == 1) {
                    S v = lam * acc[i][k][x][y] + mu * acc[k][i][x][y];
                    if (i == k) v += mu * (acc[0][0][x][y] + acc[1][1][x][y] + acc[2][2][x][y]);
                    return v;
                } else {
                    const S *C = sC + el * 81;
                    S v = 0;
#pragma unroll
                    for (int j = 0; j < 3; ++j)
#pragma unroll
                        for (int l = 0; l < 3; ++l) v = fma(C[i * 27 + j * 9 + k * 3 + l], acc[j][l][x][y], v);
                    return v;
                }
            };
            auto kval_t = [&](int i, int k, int x, int y) -> S {
                if constexpr (MATK == 1) {
                    return kval(i, k, x, y);
                } else {
                    const S *C = sC + el * 81;
                    S v = 0;
#pragma unroll
                    for (int j = 0; j < 3; ++j)
#pragma unroll
                        for (int l = 0; l < 3; ++l) v = fma(C[k * 27 + l * 9 + i * 3 + j], acc[j][l][x][y], v);
                    return v;
                }
            };
            for (int pb = 0; pb < nblk + (LAP2 ? 1 : 0); ++pb) {
                const int buf = pb & 1;
                if (pb >= 2 && threadIdx.x == 0) bulk_wait_read<1>();  // buffer of pass pb-2 drained
                __syncthreads();  // pass 0: everyone is done reading G
                if (active) {
                    S *slot = sK + (buf * EPB + el) * P::SLOT + shift_of(el, pb);
                    if (LAP2 && pb == nblk) {
                        // c (A_00 + A_11 + A_22) of the tile and its mirror
                        const S c = sC[2 * EPB + el];
#pragma unroll
                        for (int x = 0; x < T; ++x)
#pragma unroll
                            for (int y = 0; y < T; ++y) {
                                const S v = c * (acc[0][0][x][y] + acc[1][1][x][y] + acc[2][2][x][y]);
                                slot[(a0 + x) * N + b0 + y] = v;
                                if (mirror) slot[(b0 + y) * N + a0 + x] = v;
                            }
                    } else if constexpr (KIND == FK_ELASTICITY) {
                        // rows of block pb: direct entries with i == pb, mirror entries with k == pb
#pragma unroll
                        for (int pc = 0; pc < 3; ++pc) {
                            if (pc != pb) continue;
#pragma unroll
                            for (int x = 0; x < T; ++x)
#pragma unroll
                                for (int y = 0; y < T; ++y)
#pragma unroll
                                    for (int k = 0; k < 3; ++k) slot[(a0 + x) * nrow + k * N + b0 + y] = kval(pc, k, x, y);
                            if (mirror)
#pragma unroll
                                for (int y = 0; y < T; ++y)
#pragma unroll
                                    for (int x = 0; x < T; ++x)
#pragma unroll
                                        for (int i = 0; i < 3; ++i)
                                            slot[(b0 + y) * nrow + i * N + a0 + x] = kval_t(i, pc, x, y);
                        }
                    } else {
                        for_entries([&](int i, int k, int x, int y, S v, S vt) {
                            if (i == pb) slot[(a0 + x) * nrow + k * N + b0 + y] = v;
                            if (mirror && k == pb) slot[(b0 + y) * nrow + i * N + a0 + x] = vt;
                        });
                    }
                }
                fence_proxy_async();  // make the staged values visible to the bulk-copy engine
                __syncthreads();
                if (threadIdx.x == 0) {
                    const int len = LAP2 && pb == nblk ? N * N : blk_len;
                    for (int e_l = 0; e_l < ne; ++e_l) {
                        const int sh = shift_of(e_l, pb);
                        const S *src = sK + (buf * EPB + e_l) * P::SLOT + sh;
                        S *dst = dst_of(e_l, pb);
                        const int head = (V - sh) % V < len ? (V - sh) % V : len;
                        const int body = (len - head) / V * V;
                        for (int t = 0; t < head; ++t) dst[t] = src[t];
                        for (int t = head + body; t < len; ++t) dst[t] = src[t];
                        if (body > 0) bulk_store(dst + head, src + head, (unsigned)(body * sizeof(S)));
                    }
                    bulk_commit();
                }
            }
        } else {
            S *Kst = nullptr;
            long long kbase = 0;
            int shift = 0;
            if constexpr (STAGE == STAGE_FULL) {
                __syncthreads();  // everyone is done reading G: reuse the buffer for K
                kbase = e0 * (long long)nrow * nrow;
                // stage at the same offset modulo 16 bytes as the global destination
                shift = (int)(((unsigned long long)(K + kbase) % 16) / sizeof(S));
                Kst = sK + shift;
            }
            auto put = [&](int r, int c, S v) {
                if constexpr (STAGE == STAGE_FULL)
                    Kst[(long long)el * nrow * nrow + r * nrow + c] = v;
                else
                    K[(e0 + el) * (long long)nrow * nrow + (long long)r * nrow + c] = v;
            };
            if (active)
                for_entries([&](int i, int k, int x, int y, S v, S vt) {
                    put(i * N + a0 + x, k * N + b0 + y, v);
                    if (mirror) put(k * N + b0 + y, i * N + a0 + x, vt);
                });
            if constexpr (STAGE == STAGE_FULL) {
                __syncthreads();
                // coalesced 16-byte streaming stores of the ne contiguous matrices
                constexpr int V = 16 / (int)sizeof(S);
                const long long total = (long long)ne * nrow * nrow;
                const int head = (int)((V - shift) % V);  // scalars before the first aligned vector
                S *Kg = K + kbase;
                for (int i = threadIdx.x; i < head && i < total; i += THREADS) Kg[i] = Kst[i];
                const long long nvec = (total - head) / V;
                const float4 *src = reinterpret_cast<const float4 *>(Kst + head);
                float4 *dst = reinterpret_cast<float4 *>(Kg + head);
                for (long long i = threadIdx.x; i < nvec; i += THREADS) __stcs(dst + i, src[i]);
                for (long long i = head + nvec * V + threadIdx.x; i < total; i += THREADS) Kg[i] = Kst[i];
            }
        }
        }  // tile passes
    }
}

template <typename S, int N, int Q, int KIND, int T, int EPB, int THREADS, int STAGE>
__device__ __forceinline__ void matrix_load_ref(const S *__restrict__ dphi, unsigned char *smem_raw)
{
    using P = MatrixSmem<S, N, Q, KIND, T, EPB, STAGE>;
    if constexpr (P::REF_SMEM) {
        S *sD = reinterpret_cast<S *>(smem_raw) + P::D_OFF;
        for (int i = threadIdx.x; i < Q * 3 * N; i += THREADS) sD[i] = dphi[i];
    }
}


}  // namespace
