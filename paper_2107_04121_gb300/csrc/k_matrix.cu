// Matrix mode (Algorithm 2 of Cimrman, arXiv 2107.04121) on CUDA cores, FP64
// or FP32.  Element matrices of
//   weak Laplacian   K[a][b]         = c sum_q wdetJ G_q[j][a] G_q[j][b]
//   mass / dot       K[(r,a)][(s,b)] = c delta_rs sum_q wdetJ phi_q[a] phi_q[b]
//   elasticity       K[(i,a)][(k,b)] = sum_q wdetJ B_I(i,a) D_IK B_K(k,b)
// (Sec. 5.3 einsums 'cq,cqjd,cqje->cde', 'cq,qd,ir,qe,is->crdse' and
// 'cq,cqje,rjI,cqIK,cqlf,slK->cresf').
//
// Design.  The elasticity contraction is rewritten exactly (up to rounding) as
// the Gram blocks A_jl[a][b] = sum_q wdetJ G_q[j][a] G_q[l][b] followed by a
// per-node-pair epilogue K[(i,a)][(k,b)] = sum_jl C_ijkl A_jl[a][b] with the
// 4th-order tensor C_ijkl = D[V(i,j)][V(k,l)] (V = Voigt index), which is
// what the 0/1 selector Psg of Sec. 5.3.3 encodes; the sparsity of Psg that
// the paper's einsum leaves unused costs nothing here.  For Lame materials
// the epilogue is lambda A_ik + mu A_ki + mu delta_ik tr A.
//
// A CTA takes EPB consecutive elements: it stages J^-1 and wdetJ (one
// contiguous block, element-outermost layout) and forms the physical gradients
// G = J^-T grad_xi phi in shared memory, with every T-node group padded to a
// 16-byte boundary so that a thread fetches its T gradients with one vector
// load.  Element matrices are symmetric, so each thread owns one T x T node
// tile of the upper tile triangle (all nine direction pairs for elasticity,
// T*T*9 register accumulators) and writes it and its mirror image.  The
// finished matrices are staged in shared memory (over the dead G buffer) and
// streamed to HBM with coalesced 16-byte stores that bypass L2 residency
// (st.global.cs), since K_e is written once and never re-read here.
#include "matrix_body.cuh"

namespace {

template <typename S, int N, int Q, int KIND, int MATK, int T, int EPB, int THREADS, int STAGE>
__global__ void __launch_bounds__(THREADS) k_matrix_sym(const S *__restrict__ jinv, const S *__restrict__ wdetj,
                                                        const S *__restrict__ dphi, const S *__restrict__ phi,
                                                        long long E, int ncomp, const double *__restrict__ mat,
                                                        int mat_t, S *__restrict__ K)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    matrix_load_ref<S, N, Q, KIND, T, EPB, THREADS, STAGE>(dphi, smem_raw);
    for (long long e0 = (long long)blockIdx.x * EPB; e0 < E; e0 += (long long)gridDim.x * EPB) {
        const int ne = (int)((E - e0) < EPB ? (E - e0) : EPB);
        matrix_group<S, N, Q, KIND, MATK, T, EPB, THREADS, STAGE>(jinv, wdetj, phi, dphi, e0, ne, ncomp, mat, mat_t, K,
                                                                   smem_raw);
    }
    if constexpr (STAGE == STAGE_BULK)
        if (threadIdx.x == 0) bulk_wait_read<0>();  // shared memory must outlive the copies' reads
}

template <typename S, int N, int Q, int KIND, int MATK, int T, int EPB, int THREADS, int STAGE>
cudaError_t launch_sym(const fe_geometry_h *g, const fe_form_h *f, fe_material_args mat, void *K, int sm_count,
                       cudaStream_t s)
{
    using P = MatrixSmem<S, N, Q, KIND, T, EPB, STAGE>;
    static_assert(STAGE == STAGE_DIRECT || EPB * (N / T) * (N / T + 1) / 2 <= THREADS, "one tile per thread");
    static_assert(P::BYTES <= 227 * 1024, "shared memory plan exceeds one CTA's limit");
    auto kern = k_matrix_sym<S, N, Q, KIND, MATK, T, EPB, THREADS, STAGE>;
    static FeLaunchCache cache;
    long long per_sm = 0;
    cudaError_t err = fe_cached_grid(
        cache,
        [&](int, long long *v) {
            cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P::BYTES);
            if (e2 != cudaSuccess) return e2;
            int n = 0;
            e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, THREADS, P::BYTES);
            if (e2 != cudaSuccess) return e2;
            if (n < 1) return cudaErrorInvalidConfiguration;
            *v = n;
            return cudaSuccess;
        },
        &per_sm);
    if (err != cudaSuccess) return err;
    const long long E = g->mesh.n_elems;
    long long blocks = (E + EPB - 1) / EPB;
    const long long cap = per_sm * sm_count * 4;
    if (blocks > cap) blocks = cap;
    const bool f64 = sizeof(S) == 8;
    const S *jinv = f64 ? (const S *)g->d_jinv64 : (const S *)g->d_jinv32;
    const S *wdetj = f64 ? (const S *)g->d_wdetj64 : (const S *)g->d_wdetj32;
    const S *dphi = f64 ? (const S *)g->d_dphi64 : (const S *)g->d_dphi32;
    const S *phi = f64 ? (const S *)g->d_phi64 : (const S *)g->d_phi32;
    kern<<<(unsigned)blocks, THREADS, P::BYTES, s>>>(jinv, wdetj, dphi, phi, E, f->ncomp, mat.data, mat.transposed,
                                                      (S *)K);
    return cudaGetLastError();
}

// Tile shapes: T x T node tiles, EPB elements per CTA, one upper-triangle tile
// per thread; Laplace/mass (L) and elasticity (E) configured separately.
// K is staged in shared memory unless it would not fit.
template <typename S, int N, int Q, int T_L, int EPB_L, int THR_L, int STAGE_L, int T_E, int EPB_E, int THR_E,
          int STAGE_E>
cudaError_t dispatch_nq(const fe_geometry_h *g, const fe_form_h *f, fe_material_args mat, void *K, int sm,
                        cudaStream_t s)
{
    switch (f->kind) {
    case FK_LAPLACE: return launch_sym<S, N, Q, FK_LAPLACE, 0, T_L, EPB_L, THR_L, STAGE_L>(g, f, mat, K, sm, s);
    case FK_MASS: return launch_sym<S, N, Q, FK_MASS, 0, T_L, EPB_L, THR_L, STAGE_L>(g, f, mat, K, sm, s);
    case FK_ELASTICITY:
        if (mat.kind == FE_MAT_LAME)
            return launch_sym<S, N, Q, FK_ELASTICITY, 1, T_E, EPB_E, THR_E, STAGE_E>(g, f, mat, K, sm, s);
        return launch_sym<S, N, Q, FK_ELASTICITY, 2, T_E, EPB_E, THR_E, STAGE_E>(g, f, mat, K, sm, s);
    }
    return cudaErrorInvalidValue;
}

template <typename S>
cudaError_t dispatch(const fe_geometry_h *g, const fe_form_h *f, fe_material_args mat, void *K, int sm,
                     cudaStream_t s)
{
    const int N = g->N, Q = g->Q;
    constexpr bool D = sizeof(S) == 8;
    constexpr int B = STAGE_BULK;
    // Q1: 2x2 tiles, 10 upper tiles per element, 12 elements per CTA
    if (N == 8 && Q == 8) return dispatch_nq<S, 8, 8, 2, 12, 128, B, 2, 12, 128, B>(g, f, mat, K, sm, s);
    if (N == 8 && Q == 27) return dispatch_nq<S, 8, 27, 2, 12, 128, B, 2, 12, 128, B>(g, f, mat, K, sm, s);
    // Q2: 3x3 tiles, 45 upper tiles per element, 2 elements per 96-thread CTA
    if (N == 27 && Q == 27) return dispatch_nq<S, 27, 27, 3, 2, 96, B, 3, 2, 96, B>(g, f, mat, K, sm, s);
    if (N == 27 && Q == 64) return dispatch_nq<S, 27, 64, 3, 2, 96, B, 3, 2, 96, B>(g, f, mat, K, sm, s);
    // Q3: 4x4 tiles (136 per element) for the scalar forms; elasticity 2x2 tiles
    // (528 per element, 36 accumulators: 17 warps per SM instead of the 5 of 4x4
    // tiles with 144, measured 0.90 against 1.14 ms for 8,000 elements in FP32);
    // FP64 elasticity writes directly (a 64 x 192 FP64 row block per buffer would
    // not fit)
    // tetrahedra: P1 2x2 tiles (3 per element), P2 2x2 tiles (15 per element),
    // P3 2x2 tiles (55 per element, 4 elements per CTA: measured 0.23 / 0.074 /
    // 0.34 ms against 0.29 / 0.12 / 0.45 ms with 4x4 tiles and 8 elements for the
    // Laplace / mass / elasticity matrices of 40,000 elements in FP32; FP64:
    // 4x4 tiles, elasticity 2x2)
    if (N == 4 && Q == 5) return dispatch_nq<S, 4, 5, 2, 32, 96, B, 2, 32, 96, B>(g, f, mat, K, sm, s);
    if (N == 10 && Q == 15) return dispatch_nq<S, 10, 15, 2, 8, 128, B, 2, 8, 128, B>(g, f, mat, K, sm, s);
    if (N == 20 && Q == 35) {
        if constexpr (D)
            return dispatch_nq<S, 20, 35, 4, 8, 128, B, 2, 2, 128, B>(g, f, mat, K, sm, s);
        else
            return dispatch_nq<S, 20, 35, 2, 4, 256, B, 2, 4, 256, B>(g, f, mat, K, sm, s);
    }
    if (N == 64 && Q == 64) {
        if constexpr (D)
            return dispatch_nq<S, 64, 64, 4, 1, 160, B, 2, 1, 544, STAGE_DIRECT>(g, f, mat, K, sm, s);
        else
            return dispatch_nq<S, 64, 64, 4, 1, 160, B, 2, 1, 544, B>(g, f, mat, K, sm, s);
    }
    return cudaErrorInvalidValue;
}

// Lame elasticity and the weighted scalar Laplacian of the same elements from one
// set of Gram blocks: K_L = c sum_j A_jj is the trace the Lame epilogue already
// forms, written as a fourth bulk-staged row block into K2 (FP32).
template <int N, int Q, int T, int EPB, int THREADS>
__global__ void __launch_bounds__(THREADS) k_matrix_pair(const float *__restrict__ jinv, const float *__restrict__ wdetj,
                                                         const float *__restrict__ dphi, long long E,
                                                         const double *__restrict__ lame, float *__restrict__ K,
                                                         const double *__restrict__ coef, float *__restrict__ K2)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    matrix_load_ref<float, N, Q, FK_ELASTICITY, T, EPB, THREADS, STAGE_BULK>(dphi, smem_raw);
    for (long long e0 = (long long)blockIdx.x * EPB; e0 < E; e0 += (long long)gridDim.x * EPB) {
        const int ne = (int)((E - e0) < EPB ? (E - e0) : EPB);
        matrix_group<float, N, Q, FK_ELASTICITY, 1, T, EPB, THREADS, STAGE_BULK, true>(
            jinv, wdetj, nullptr, dphi, e0, ne, 3, lame, 0, K, smem_raw, K2, coef);
    }
    if (threadIdx.x == 0) bulk_wait_read<0>();  // shared memory must outlive the copies' reads
}

template <int N, int Q, int T, int EPB, int THREADS>
cudaError_t launch_pair(const fe_geometry_h *g, const double *lame, float *K, const double *coef, float *K2,
                        int sm_count, cudaStream_t s)
{
    using P = MatrixSmem<float, N, Q, FK_ELASTICITY, T, EPB, STAGE_BULK>;
    static_assert(EPB * (N / T) * (N / T + 1) / 2 <= THREADS, "one tile per thread");
    static_assert(P::BYTES <= 227 * 1024, "shared memory plan exceeds one CTA's limit");
    auto kern = k_matrix_pair<N, Q, T, EPB, THREADS>;
    static FeLaunchCache cache;
    long long per_sm = 0;
    cudaError_t err = fe_cached_grid(
        cache,
        [&](int, long long *v) {
            cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P::BYTES);
            if (e2 != cudaSuccess) return e2;
            int n = 0;
            e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, THREADS, P::BYTES);
            if (e2 != cudaSuccess) return e2;
            if (n < 1) return cudaErrorInvalidConfiguration;
            *v = n;
            return cudaSuccess;
        },
        &per_sm);
    if (err != cudaSuccess) return err;
    const long long E = g->mesh.n_elems;
    long long blocks = (E + EPB - 1) / EPB;
    const long long cap = per_sm * sm_count * 4;
    if (blocks > cap) blocks = cap;
    kern<<<(unsigned)blocks, THREADS, P::BYTES, s>>>(g->d_jinv32, g->d_wdetj32, g->d_dphi32, E, lame, K, coef, K2);
    return cudaGetLastError();
}

}  // namespace

bool fe_supported_nq(int N, int Q)
{
    return (N == 8 && (Q == 8 || Q == 27)) || (N == 27 && (Q == 27 || Q == 64)) || (N == 64 && Q == 64) ||
           // P1, P2, P3 tetrahedra with the Grundmann-Moller rules of index p (5, 15, 35 points)
           (N == 4 && Q == 5) || (N == 10 && Q == 15) || (N == 20 && Q == 35);
}

cudaError_t fe_launch_matrix_simt(const fe_geometry_h *g, const fe_form_h *f, fe_material_args mat, bool f64,
                                  void *K, int sm_count, cudaStream_t s)
{
    if (g->mesh.n_elems == 0) return cudaSuccess;
    return f64 ? dispatch<double>(g, f, mat, K, sm_count, s) : dispatch<float>(g, f, mat, K, sm_count, s);
}

bool fe_matrix_pair_supported(const fe_geometry_h *g)
{
    return fe_supported_nq(g->N, g->Q) && g->d_jinv32 && g->d_dphi32;
}

cudaError_t fe_launch_matrix_pair(const fe_geometry_h *g, const double *lame, void *K, const double *coef, void *K2,
                                  int sm_count, cudaStream_t s)
{
    if (g->mesh.n_elems == 0) return cudaSuccess;
    if (!fe_matrix_pair_supported(g)) return cudaErrorNotSupported;
    float *Ke = (float *)K, *Kl = (float *)K2;
    const int N = g->N, Q = g->Q;
    // the elasticity tiles of the FP32 dispatch above
    if (N == 8 && Q == 8) return launch_pair<8, 8, 2, 12, 128>(g, lame, Ke, coef, Kl, sm_count, s);
    if (N == 8 && Q == 27) return launch_pair<8, 27, 2, 12, 128>(g, lame, Ke, coef, Kl, sm_count, s);
    if (N == 27 && Q == 27) return launch_pair<27, 27, 3, 2, 96>(g, lame, Ke, coef, Kl, sm_count, s);
    if (N == 27 && Q == 64) return launch_pair<27, 64, 3, 2, 96>(g, lame, Ke, coef, Kl, sm_count, s);
    if (N == 4 && Q == 5) return launch_pair<4, 5, 2, 32, 96>(g, lame, Ke, coef, Kl, sm_count, s);
    if (N == 10 && Q == 15) return launch_pair<10, 15, 2, 8, 128>(g, lame, Ke, coef, Kl, sm_count, s);
    if (N == 20 && Q == 35) return launch_pair<20, 35, 2, 4, 256>(g, lame, Ke, coef, Kl, sm_count, s);
    if (N == 64 && Q == 64) return launch_pair<64, 64, 2, 1, 544>(g, lame, Ke, coef, Kl, sm_count, s);
    return cudaErrorNotSupported;
}
