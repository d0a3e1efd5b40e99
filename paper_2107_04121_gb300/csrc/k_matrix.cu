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
// contiguous block, element-outermost layout), forms the physical gradients
// G = J^-T grad_xi phi in shared memory, and each thread accumulates a TA x TB
// node-pair tile (all nine direction pairs for elasticity) in registers.
#include "fe_device.cuh"

namespace {

template <typename T, int N, int Q, int KIND, int TA, int TB, int EPB, int THREADS>
__global__ void __launch_bounds__(THREADS) k_matrix_simt(const T *__restrict__ jinv, const T *__restrict__ wdetj,
                                                         const T *__restrict__ dphi, const T *__restrict__ phi,
                                                         long long E, int ncomp, fe_material_kind mkind,
                                                         const double *__restrict__ mat, int mat_t,
                                                         T *__restrict__ K)
{
    constexpr int NTA = N / TA, NTB = N / TB, NT = NTA * NTB;
    constexpr bool GRAD = KIND != FK_MASS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sG = reinterpret_cast<T *>(smem_raw);          // GRAD: [EPB][Q][3][N]; MASS: phi [Q][N]
    T *sJ = sG + (GRAD ? EPB * Q * 3 * N : Q * N);    // [EPB][Q][9]
    T *sW = sJ + EPB * Q * 9;                         // [EPB][Q]
    T *sC = sW + EPB * Q;                             // [EPB][81] elasticity tensor or [EPB] coefficient

    const int nrow = ncomp * N;
    for (long long e0 = (long long)blockIdx.x * EPB; e0 < E; e0 += (long long)gridDim.x * EPB) {
        const int ne = (int)((E - e0) < EPB ? (E - e0) : EPB);
        __syncthreads();
        // stage J^-1, wdetJ (contiguous) and the material
        if (GRAD)
            for (int i = threadIdx.x; i < ne * Q * 9; i += THREADS) sJ[i] = jinv[e0 * Q * 9 + i];
        for (int i = threadIdx.x; i < ne * Q; i += THREADS) sW[i] = wdetj[e0 * Q + i];
        if constexpr (KIND == FK_ELASTICITY) {
            for (int i = threadIdx.x; i < ne * 81; i += THREADS) {
                const int el = i / 81, t = i % 81;
                const int ii = t / 27, jj = (t / 9) % 3, kk = (t / 3) % 3, ll = t % 3;
                double c;
                const long long e = e0 + el;
                if (mkind == FE_MAT_LAME) {
                    const double lam = mat[2 * e], mu = mat[2 * e + 1];
                    c = lam * (ii == jj) * (kk == ll) + mu * ((ii == kk) * (jj == ll) + (ii == ll) * (jj == kk));
                } else {
                    const int I = fe_voigt(ii, jj), Kv = fe_voigt(kk, ll);
                    c = mat_t ? mat[e * 36 + Kv * 6 + I] : mat[e * 36 + I * 6 + Kv];
                }
                sC[i] = (T)c;
            }
        } else {
            for (int i = threadIdx.x; i < ne; i += THREADS) sC[i] = mat ? (T)mat[e0 + i] : (T)1;
        }
        if (!GRAD)
            for (int i = threadIdx.x; i < Q * N; i += THREADS) sG[i] = phi[i];
        __syncthreads();
        if (GRAD) {
            // G[el][q][j][a] = sum_k dphi[q][k][a] Jinv[el][q][k][j]
            for (int i = threadIdx.x; i < ne * Q * N; i += THREADS) {
                const int a = i % N, q = (i / N) % Q, el = i / (N * Q);
                const T g0 = dphi[(q * 3 + 0) * N + a], g1 = dphi[(q * 3 + 1) * N + a],
                        g2 = dphi[(q * 3 + 2) * N + a];
                const T *Ji = sJ + (el * Q + q) * 9;
                T *Go = sG + ((el * Q + q) * 3) * N + a;
#pragma unroll
                for (int j = 0; j < 3; ++j) Go[j * N] = g0 * Ji[j] + g1 * Ji[3 + j] + g2 * Ji[6 + j];
            }
            __syncthreads();
        }

        for (int wi = threadIdx.x; wi < ne * NT; wi += THREADS) {
            const int el = wi / NT, tile = wi % NT;
            const int a0 = (tile / NTB) * TA, b0 = (tile % NTB) * TB;
            const T *Wq = sW + el * Q;
            T *Ke = K + (e0 + el) * (long long)nrow * nrow;
            if constexpr (KIND == FK_ELASTICITY) {
                T acc[3][3][TA][TB];
#pragma unroll
                for (int j = 0; j < 3; ++j)
#pragma unroll
                    for (int l = 0; l < 3; ++l)
#pragma unroll
                        for (int x = 0; x < TA; ++x)
#pragma unroll
                            for (int y = 0; y < TB; ++y) acc[j][l][x][y] = 0;
                const T *Ge = sG + el * Q * 3 * N;
                for (int q = 0; q < Q; ++q) {
                    const T wq = Wq[q];
                    const T *Gq = Ge + q * 3 * N;
                    T ga[3][TA], gb[3][TB];
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
#pragma unroll
                        for (int x = 0; x < TA; ++x) ga[j][x] = wq * Gq[j * N + a0 + x];
#pragma unroll
                        for (int y = 0; y < TB; ++y) gb[j][y] = Gq[j * N + b0 + y];
                    }
#pragma unroll
                    for (int j = 0; j < 3; ++j)
#pragma unroll
                        for (int l = 0; l < 3; ++l)
#pragma unroll
                            for (int x = 0; x < TA; ++x)
#pragma unroll
                                for (int y = 0; y < TB; ++y) acc[j][l][x][y] = fma(ga[j][x], gb[l][y], acc[j][l][x][y]);
                }
                const T *C = sC + el * 81;
                if (mkind == FE_MAT_LAME) {
                    const T lam = C[0 * 27 + 0 * 9 + 1 * 3 + 1];   // C_0011 = lambda
                    const T mu = C[0 * 27 + 1 * 9 + 0 * 3 + 1];    // C_0101 = mu
#pragma unroll
                    for (int x = 0; x < TA; ++x)
#pragma unroll
                        for (int y = 0; y < TB; ++y) {
                            const T tr = acc[0][0][x][y] + acc[1][1][x][y] + acc[2][2][x][y];
#pragma unroll
                            for (int i = 0; i < 3; ++i)
#pragma unroll
                                for (int k = 0; k < 3; ++k) {
                                    T v = lam * acc[i][k][x][y] + mu * acc[k][i][x][y];
                                    if (i == k) v += mu * tr;
                                    Ke[(long long)(i * N + a0 + x) * nrow + k * N + b0 + y] = v;
                                }
                        }
                } else {
#pragma unroll
                    for (int x = 0; x < TA; ++x)
#pragma unroll
                        for (int y = 0; y < TB; ++y)
#pragma unroll
                            for (int i = 0; i < 3; ++i)
#pragma unroll
                                for (int k = 0; k < 3; ++k) {
                                    T v = 0;
#pragma unroll
                                    for (int j = 0; j < 3; ++j)
#pragma unroll
                                        for (int l = 0; l < 3; ++l) v = fma(C[i * 27 + j * 9 + k * 3 + l], acc[j][l][x][y], v);
                                    Ke[(long long)(i * N + a0 + x) * nrow + k * N + b0 + y] = v;
                                }
                }
            } else {
                T acc[TA][TB];
#pragma unroll
                for (int x = 0; x < TA; ++x)
#pragma unroll
                    for (int y = 0; y < TB; ++y) acc[x][y] = 0;
                for (int q = 0; q < Q; ++q) {
                    const T wq = Wq[q];
                    if constexpr (KIND == FK_LAPLACE) {
                        const T *Gq = sG + (el * Q + q) * 3 * N;
#pragma unroll
                        for (int j = 0; j < 3; ++j) {
                            T ga[TA], gb[TB];
#pragma unroll
                            for (int x = 0; x < TA; ++x) ga[x] = wq * Gq[j * N + a0 + x];
#pragma unroll
                            for (int y = 0; y < TB; ++y) gb[y] = Gq[j * N + b0 + y];
#pragma unroll
                            for (int x = 0; x < TA; ++x)
#pragma unroll
                                for (int y = 0; y < TB; ++y) acc[x][y] = fma(ga[x], gb[y], acc[x][y]);
                        }
                    } else {
                        const T *Pq = sG + q * N;
                        T pa[TA], pb[TB];
#pragma unroll
                        for (int x = 0; x < TA; ++x) pa[x] = wq * Pq[a0 + x];
#pragma unroll
                        for (int y = 0; y < TB; ++y) pb[y] = Pq[b0 + y];
#pragma unroll
                        for (int x = 0; x < TA; ++x)
#pragma unroll
                            for (int y = 0; y < TB; ++y) acc[x][y] = fma(pa[x], pb[y], acc[x][y]);
                    }
                }
                const T c = sC[el];
                for (int r = 0; r < ncomp; ++r)
                    for (int s2 = 0; s2 < ncomp; ++s2)
#pragma unroll
                        for (int x = 0; x < TA; ++x)
#pragma unroll
                            for (int y = 0; y < TB; ++y)
                                Ke[(long long)(r * N + a0 + x) * nrow + s2 * N + b0 + y] = (r == s2) ? c * acc[x][y] : (T)0;
            }
        }
    }
}

template <typename T, int N, int Q, int KIND, int TA, int TB, int EPB, int THREADS>
cudaError_t launch_simt(const fe_geometry_h *g, const fe_form_h *f, fe_material_args mat, void *K, int sm_count,
                        cudaStream_t s)
{
    constexpr bool GRAD = KIND != FK_MASS;
    const size_t smem = sizeof(T) * ((GRAD ? (size_t)EPB * Q * 3 * N : (size_t)Q * N) + (size_t)EPB * Q * 9 +
                                     (size_t)EPB * Q + (size_t)EPB * 81);
    auto kern = k_matrix_simt<T, N, Q, KIND, TA, TB, EPB, THREADS>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long E = g->mesh.n_elems;
    long long blocks = (E + EPB - 1) / EPB;
    const long long cap = (long long)per_sm * sm_count * 8;
    if (blocks > cap) blocks = cap;
    const bool f64 = sizeof(T) == 8;
    const T *jinv = f64 ? (const T *)g->d_jinv64 : (const T *)g->d_jinv32;
    const T *wdetj = f64 ? (const T *)g->d_wdetj64 : (const T *)g->d_wdetj32;
    const T *dphi = f64 ? (const T *)g->d_dphi64 : (const T *)g->d_dphi32;
    const T *phi = f64 ? (const T *)g->d_phi64 : (const T *)g->d_phi32;
    kern<<<(unsigned)blocks, THREADS, smem, s>>>(jinv, wdetj, dphi, phi, E, f->ncomp, mat.kind, mat.data,
                                                  mat.transposed, (T *)K);
    return cudaGetLastError();
}

template <typename T>
cudaError_t dispatch(const fe_geometry_h *g, const fe_form_h *f, fe_material_args mat, void *K, int sm,
                     cudaStream_t s)
{
    const int N = g->N, Q = g->Q;
#define FE_CASE(NN, QQ, TA_, TB_, EPB_L, EPB_E, THR)                                                                 \
    if (N == NN && Q == QQ) {                                                                                       \
        switch (f->kind) {                                                                                          \
        case FK_LAPLACE: return launch_simt<T, NN, QQ, FK_LAPLACE, TA_, TB_, EPB_L, THR>(g, f, mat, K, sm, s);       \
        case FK_MASS: return launch_simt<T, NN, QQ, FK_MASS, TA_, TB_, EPB_L, THR>(g, f, mat, K, sm, s);             \
        case FK_ELASTICITY: return launch_simt<T, NN, QQ, FK_ELASTICITY, TA_, TB_, EPB_E, THR>(g, f, mat, K, sm, s); \
        }                                                                                                           \
    }
    FE_CASE(8, 8, 2, 2, 8, 8, 128)
    FE_CASE(8, 27, 2, 2, 8, 4, 128)
    FE_CASE(27, 27, 3, 3, 3, 3, 256)
    FE_CASE(27, 64, 3, 3, 2, 1, 256)
    // 4 x 4 FP64 tiles would need 288 accumulator registers: halve TB there
    FE_CASE(64, 64, 4, (sizeof(T) == 8 ? 2 : 4), 1, 1, 256)
#undef FE_CASE
    return cudaErrorInvalidValue;
}

}  // namespace

bool fe_supported_nq(int N, int Q)
{
    return (N == 8 && (Q == 8 || Q == 27)) || (N == 27 && (Q == 27 || Q == 64)) || (N == 64 && Q == 64);
}

cudaError_t fe_launch_matrix_simt(const fe_geometry_h *g, const fe_form_h *f, fe_material_args mat, bool f64,
                                  void *K, int sm_count, cudaStream_t s)
{
    if (g->mesh.n_elems == 0) return cudaSuccess;
    return f64 ? dispatch<double>(g, f, mat, K, sm_count, s) : dispatch<float>(g, f, mat, K, sm_count, s);
}
