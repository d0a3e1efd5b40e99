// Residual mode (Algorithm 1 of Cimrman, arXiv 2107.04121): the element DOFs
// are gathered from the global vector through the connectivity, the integrand
// is evaluated at each quadrature point and integrated with w det J:
//   weak Laplacian  r[a]     = c sum_q wdetJ G_q[j][a] (grad u_h)_j
//   mass / dot      r[(i,a)] = c sum_q wdetJ phi_q[a] u_h,i
//   elasticity      r[(i,a)] = sum_q wdetJ G_q[j][a] sigma_ij(u_h),  sigma = D e(u_h)
// (the residual-mode einsums of Sec. 5.3, e.g. 'cq,qd,ir,qe,cie->crd').
//
// Design.  The physical gradients are never formed: with G = J^-T grad_xi phi,
//   grad u_h = (sum_b u_b grad_xi phi_b) J^-1            (phase 1, per (e, q))
//   r[(i,a)]  = sum_q sum_m F_q[i][m] d phi_a / d xi_m,
//   F_q[i][m] = wdetJ sum_j sigma_ij (J^-1)_mj          (phase 2, per (e, a))
// so each element reads only J^-1 and w det J (40 bytes per quadrature point
// in FP32) besides its DOFs, while the reference gradients (shared by all
// elements) stay in shared memory.
#include "fe_device.cuh"

namespace {

template <typename T, int N, int Q, int KIND, int EPB, int THREADS>
__global__ void __launch_bounds__(THREADS) k_residual(const T *__restrict__ jinv, const T *__restrict__ wdetj,
                                                      const T *__restrict__ dphi, const T *__restrict__ phi,
                                                      const int32_t *__restrict__ conn, long long E, int ncomp,
                                                      fe_material_kind mkind, const double *__restrict__ mat,
                                                      int mat_t, const T *__restrict__ u, T *__restrict__ r,
                                                      long long n_nodes, unsigned long long *__restrict__ status)
{
    constexpr bool GRAD = KIND != FK_MASS;
    constexpr int NC = KIND == FK_ELASTICITY ? 3 : (KIND == FK_LAPLACE ? 1 : 3);  // max components
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sB = reinterpret_cast<T *>(smem_raw);  // GRAD: dphi (Q,3,N); MASS: phi (Q,N)
    T *sJ = sB + (GRAD ? Q * 3 * N : Q * N);   // [EPB][Q][9]
    T *sW = sJ + EPB * Q * 9;                  // [EPB][Q]
    T *sU = sW + EPB * Q;                      // [EPB][NC][N]
    T *sF = sU + EPB * NC * N;                 // [EPB][Q][NC][3]
    T *sM = sF + EPB * Q * NC * 3;             // [EPB][36] material (D, Voigt) or [EPB] coefficient

    for (int i = threadIdx.x; i < (GRAD ? Q * 3 * N : Q * N); i += THREADS) sB[i] = GRAD ? dphi[i] : phi[i];
    for (long long e0 = (long long)blockIdx.x * EPB; e0 < E; e0 += (long long)gridDim.x * EPB) {
        const int ne = (int)((E - e0) < EPB ? (E - e0) : EPB);
        __syncthreads();
        if (GRAD)
            for (int i = threadIdx.x; i < ne * Q * 9; i += THREADS) sJ[i] = jinv[e0 * Q * 9 + i];
        for (int i = threadIdx.x; i < ne * Q; i += THREADS) sW[i] = wdetj[e0 * Q + i];
        for (int i = threadIdx.x; i < ne * N; i += THREADS) {
            const int el = i / N, a = i % N;
            const long long node = conn[(e0 + el) * N + a];
            const bool ok = (unsigned long long)node < (unsigned long long)n_nodes;  // never read outside u
            if (!ok) fe_report(status, FE_ERR_SHAPE, e0 + el);
            for (int c = 0; c < ncomp; ++c) sU[(el * NC + c) * N + a] = ok ? u[node * ncomp + c] : (T)0;
        }
        if constexpr (KIND == FK_ELASTICITY) {
            for (int i = threadIdx.x; i < ne * 36; i += THREADS) {
                const int el = i / 36, I = (i % 36) / 6, K = i % 6;
                const long long e = e0 + el;
                double d;
                if (mkind == FE_MAT_LAME)
                    d = (I < 3 && K < 3 ? mat[2 * e] : 0.0) + (I == K ? (I < 3 ? 2.0 : 1.0) * mat[2 * e + 1] : 0.0);
                else
                    d = mat_t ? mat[e * 36 + K * 6 + I] : mat[e * 36 + I * 6 + K];
                sM[i] = (T)d;
            }
        } else {
            for (int i = threadIdx.x; i < ne; i += THREADS) sM[i] = mat ? (T)mat[e0 + i] : (T)1;
        }
        __syncthreads();

        // phase 1: fluxes at the quadrature points
        for (int wi = threadIdx.x; wi < ne * Q; wi += THREADS) {
            const int el = wi / Q, q = wi % Q;
            const T wd = sW[el * Q + q];
            T *F = sF + (el * Q + q) * NC * 3;
            if constexpr (KIND == FK_MASS) {
                const T *P = sB + q * N;
                const T c = sM[el];
                for (int i = 0; i < ncomp; ++i) {
                    const T *ui = sU + (el * NC + i) * N;
                    T s = 0;
#pragma unroll 9
                    for (int b = 0; b < N; ++b) s = fma(P[b], ui[b], s);
                    F[i] = c * wd * s;
                }
            } else {
                const T *Ji = sJ + (el * Q + q) * 9;
                const T *D0 = sB + q * 3 * N;
                // reference gradients g[i][m] = sum_b u_ib d phi_b / d xi_m
                T g[NC][3];
#pragma unroll
                for (int i = 0; i < NC; ++i) {
                    const T *ui = sU + (el * NC + i) * N;
                    T s0 = 0, s1 = 0, s2 = 0;
#pragma unroll 9
                    for (int b = 0; b < N; ++b) {
                        const T ub = ui[b];
                        s0 = fma(ub, D0[b], s0);
                        s1 = fma(ub, D0[N + b], s1);
                        s2 = fma(ub, D0[2 * N + b], s2);
                    }
                    g[i][0] = s0;
                    g[i][1] = s1;
                    g[i][2] = s2;
                }
                // physical gradient H[i][j] = sum_m g[i][m] Jinv[m][j]
                T H[NC][3];
#pragma unroll
                for (int i = 0; i < NC; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) H[i][j] = g[i][0] * Ji[j] + g[i][1] * Ji[3 + j] + g[i][2] * Ji[6 + j];
                T S[NC][3];  // wdetJ * flux in physical coordinates
                if constexpr (KIND == FK_LAPLACE) {
                    const T c = sM[el] * wd;
#pragma unroll
                    for (int j = 0; j < 3; ++j) S[0][j] = c * H[0][j];
                } else {
                    const T *Dm = sM + el * 36;
                    T eps[6] = {H[0][0], H[1][1], H[2][2], H[0][1] + H[1][0], H[0][2] + H[2][0], H[1][2] + H[2][1]};
                    T sig[6];
#pragma unroll
                    for (int I = 0; I < 6; ++I) {
                        T s = 0;
#pragma unroll
                        for (int K = 0; K < 6; ++K) s = fma(Dm[I * 6 + K], eps[K], s);
                        sig[I] = wd * s;
                    }
#pragma unroll
                    for (int i = 0; i < 3; ++i)
#pragma unroll
                        for (int j = 0; j < 3; ++j) S[i][j] = sig[fe_voigt(i, j)];
                }
                // pull back: F[i][m] = sum_j S[i][j] Jinv[m][j]
#pragma unroll
                for (int i = 0; i < NC; ++i)
#pragma unroll
                    for (int m = 0; m < 3; ++m) F[i * 3 + m] = S[i][0] * Ji[m * 3] + S[i][1] * Ji[m * 3 + 1] + S[i][2] * Ji[m * 3 + 2];
            }
        }
        __syncthreads();

        // phase 2: test-function sums
        for (int wi = threadIdx.x; wi < ne * N; wi += THREADS) {
            const int el = wi / N, a = wi % N;
            T *re = r + (e0 + el) * (long long)ncomp * N;
            if constexpr (KIND == FK_MASS) {
                T acc[3] = {0, 0, 0};
                for (int q = 0; q < Q; ++q) {
                    const T pa = sB[q * N + a];
                    const T *F = sF + (el * Q + q) * NC * 3;
                    for (int i = 0; i < ncomp; ++i) acc[i] = fma(pa, F[i], acc[i]);
                }
                for (int i = 0; i < ncomp; ++i) re[i * N + a] = acc[i];
            } else {
                T acc[NC];
#pragma unroll
                for (int i = 0; i < NC; ++i) acc[i] = 0;
#pragma unroll 3
                for (int q = 0; q < Q; ++q) {
                    const T d0 = sB[(q * 3 + 0) * N + a], d1 = sB[(q * 3 + 1) * N + a], d2 = sB[(q * 3 + 2) * N + a];
                    const T *F = sF + (el * Q + q) * NC * 3;
#pragma unroll
                    for (int i = 0; i < NC; ++i) acc[i] = fma(F[i * 3], d0, fma(F[i * 3 + 1], d1, fma(F[i * 3 + 2], d2, acc[i])));
                }
#pragma unroll
                for (int i = 0; i < NC; ++i) re[i * N + a] = acc[i];
            }
        }
    }
}

template <typename T, int N, int Q, int KIND, int EPB>
cudaError_t launch_res(const fe_geometry_h *g, const fe_form_h *f, fe_material_args mat, const void *u, void *r,
                       unsigned long long *st, cudaStream_t s)
{
    constexpr int THREADS = 256;
    constexpr bool GRAD = KIND != FK_MASS;
    constexpr int NC = KIND == FK_LAPLACE ? 1 : 3;
    const size_t smem = sizeof(T) * ((GRAD ? (size_t)Q * 3 * N : (size_t)Q * N) + (size_t)EPB * Q * 9 +
                                     (size_t)EPB * Q + (size_t)EPB * NC * N + (size_t)EPB * Q * NC * 3 + EPB * 36);
    auto kern = k_residual<T, N, Q, KIND, EPB, THREADS>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long E = g->mesh.n_elems;
    long long blocks = (E + EPB - 1) / EPB;
    const long long cap = (long long)per_sm * sms * 4;
    if (blocks > cap) blocks = cap;
    const bool f64 = sizeof(T) == 8;
    kern<<<(unsigned)blocks, THREADS, smem, s>>>(
        f64 ? (const T *)g->d_jinv64 : (const T *)g->d_jinv32, f64 ? (const T *)g->d_wdetj64 : (const T *)g->d_wdetj32,
        f64 ? (const T *)g->d_dphi64 : (const T *)g->d_dphi32, f64 ? (const T *)g->d_phi64 : (const T *)g->d_phi32,
        g->mesh.conn, E, f->ncomp, mat.kind, mat.data, mat.transposed, (const T *)u, (T *)r, g->mesh.n_nodes, st);
    return cudaGetLastError();
}

template <typename T>
cudaError_t dispatch(const fe_geometry_h *g, const fe_form_h *f, fe_material_args mat, const void *u, void *r,
                     unsigned long long *st, cudaStream_t s)
{
    const int N = g->N, Q = g->Q;
#define FE_CASE(NN, QQ, EPB_)                                                                   \
    if (N == NN && Q == QQ) {                                                                   \
        switch (f->kind) {                                                                      \
        case FK_LAPLACE: return launch_res<T, NN, QQ, FK_LAPLACE, EPB_>(g, f, mat, u, r, st, s);       \
        case FK_MASS: return launch_res<T, NN, QQ, FK_MASS, EPB_>(g, f, mat, u, r, st, s);             \
        case FK_ELASTICITY: return launch_res<T, NN, QQ, FK_ELASTICITY, EPB_>(g, f, mat, u, r, st, s); \
        }                                                                                       \
    }
    FE_CASE(8, 8, 16)
    FE_CASE(8, 27, 8)
    FE_CASE(27, 27, 8)
    FE_CASE(27, 64, 4)
    FE_CASE(64, 64, 2)
#undef FE_CASE
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t fe_launch_residual(const fe_geometry_h *g, const fe_form_h *f, fe_material_args mat, bool f64,
                               const void *u, void *r, unsigned long long *st, cudaStream_t s)
{
    if (g->mesh.n_elems == 0) return cudaSuccess;
    return f64 ? dispatch<double>(g, f, mat, u, r, st, s) : dispatch<float>(g, f, mat, u, r, st, s);
}
