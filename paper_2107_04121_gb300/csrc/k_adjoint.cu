// Adjoint (vector-Jacobian product) of the isotropic elasticity residual
// 'IK,s(i:j)->I,s(k:l)->K' (Algorithm 1 of Cimrman, arXiv 2107.04121) with
// respect to the per-element Lame parameters and the node coordinates, on
// tensor-product hexahedra by sum factorisation.
//
// Given an adjoint DOF vector rbar (for an objective of the assembled residual
// R, rbar = dObjective/dR), the derivative of rbar . R is, element by element,
//   d/d lambda_e = sum_q w det J div(u_h) div(rbar_h)
//   d/d mu_e     = sum_q w det J 2 eps(u_h) : eps(rbar_h)
//   d/d x_(a,m)  = sum_q w det J sum_j [ f delta_mj - M_mj ] G[j][a]
//     f = sigma(u_h) : eps(rbar_h),  M = (grad rbar_h)^T sigma(u_h) + (grad u_h)^T sigma(rbar_h)
// (d det J = det J sum_a G_a . dx_a, d grad v = -(grad v)(grad dV)).  With
// G[j][a] = sum_k (J^-1)_kj dphi_a/dxi_k the coordinate term is a transposed
// gradient contraction of the fluxes F[m][k] = sum_j S_mj (J^-1)_kj,
// S = w det J (f I - M): the same z, y, x stages as the residual kernel.
//
// Per element: stages x, y, z give the reference gradients of u and rbar at the
// points; one thread per point forms the physical gradients, the stresses, the
// two material integrands and the fluxes; the Lame terms are summed over the
// points per element and the fluxes contracted back to the nodes.
#include "fe_device.cuh"

namespace {

template <typename T, int N1, int NQ>
struct AdPlan {
    static constexpr int N = N1 * N1 * N1, Q = NQ * NQ * NQ;
    static constexpr int LX = N1 * N1 * NQ, LY = N1 * NQ * NQ;
    static constexpr int U = 0;                       // [6][N]: u, rbar
    static constexpr int JI = U + 6 * N;              // [Q][9]
    static constexpr int WD = JI + 9 * Q;             // [Q]
    static constexpr int FL = WD + Q;                 // [3][3][Q] fluxes F[m][k]
    static constexpr int RED = FL + 9 * Q;            // [2][Q] material integrands
    static constexpr int R1 = RED + 2 * Q;            // stages x, y | transposed stages
    static constexpr int R1N = 6 * 2 * LX + 6 * 3 * LY;
    static constexpr int R2 = R1 + R1N;               // reference gradients [6][3][Q]
    static constexpr int PER_EL = R2 + 6 * 3 * Q;
};

template <typename T, int N1, int NQ, int EPB, int THREADS>
__global__ void __launch_bounds__(THREADS) k_adjoint_sf(const T *__restrict__ jinv, const T *__restrict__ wdetj,
                                                        const T *__restrict__ b1d, const T *__restrict__ d1d,
                                                        const int32_t *__restrict__ conn, long long E,
                                                        const double *__restrict__ lame, const T *__restrict__ u,
                                                        const T *__restrict__ rbar, T *__restrict__ dmat,
                                                        T *__restrict__ dxe, long long n_nodes,
                                                        unsigned long long *__restrict__ status)
{
    using P = AdPlan<T, N1, NQ>;
    constexpr int N = P::N, Q = P::Q, LX = P::LX, LY = P::LY, PE = P::PER_EL;
    extern __shared__ __align__(16) unsigned char ad_smem[];
    T *sm = reinterpret_cast<T *>(ad_smem);
    T B[NQ][N1], D[NQ][N1];
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int i = 0; i < N1; ++i) {
            B[q][i] = b1d[q * N1 + i];
            D[q][i] = d1d[q * N1 + i];
        }
    for (long long e0 = (long long)blockIdx.x * EPB; e0 < E; e0 += (long long)gridDim.x * EPB) {
        const int ne = (int)((E - e0) < EPB ? (E - e0) : EPB);
        __syncthreads();
        for (int t = threadIdx.x; t < ne * Q * 9; t += THREADS)
            sm[(t / (Q * 9)) * PE + P::JI + t % (Q * 9)] = jinv[e0 * Q * 9 + t];
        for (int t = threadIdx.x; t < ne * Q; t += THREADS) sm[(t / Q) * PE + P::WD + t % Q] = wdetj[e0 * Q + t];
        for (int t = threadIdx.x; t < ne * N; t += THREADS) {
            const int el = t / N, a = t % N;
            const long long node = conn[(e0 + el) * N + a];
            const bool ok = (unsigned long long)node < (unsigned long long)n_nodes;  // never read outside u, rbar
            if (!ok) fe_report(status, FE_ERR_SHAPE, e0 + el);
            T *U = sm + el * PE + P::U;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                U[c * N + a] = ok ? u[node * 3 + c] : (T)0;
                U[(3 + c) * N + a] = ok ? rbar[node * 3 + c] : (T)0;
            }
        }
        __syncthreads();
        // ---- x: line (el, c, k, j) -> X[c][0] = B_x U, X[c][1] = D_x U
        for (int t = threadIdx.x; t < ne * 6 * N1 * N1; t += THREADS) {
            const int kj = t % (N1 * N1), c = (t / (N1 * N1)) % 6, el = t / (N1 * N1 * 6);
            const T *U = sm + el * PE + P::U + c * N + kj * N1;
            T *X = sm + el * PE + P::R1 + c * 2 * LX + kj * NQ;
            T x[N1];
#pragma unroll
            for (int i = 0; i < N1; ++i) x[i] = U[i];
#pragma unroll
            for (int qx = 0; qx < NQ; ++qx) {
                T v0 = 0, v1 = 0;
#pragma unroll
                for (int i = 0; i < N1; ++i) {
                    v0 = fma(B[qx][i], x[i], v0);
                    v1 = fma(D[qx][i], x[i], v1);
                }
                X[qx] = v0;
                X[LX + qx] = v1;
            }
        }
        __syncthreads();
        // ---- y: line (el, c, k, qx) -> Y[c][0] = B_y B_x, [1] = D_y B_x, [2] = B_y D_x
        for (int t = threadIdx.x; t < ne * 6 * N1 * NQ; t += THREADS) {
            const int qx = t % NQ, k = (t / NQ) % N1, c = (t / (NQ * N1)) % 6, el = t / (NQ * N1 * 6);
            const T *X = sm + el * PE + P::R1 + c * 2 * LX;
            T *Y = sm + el * PE + P::R1 + 12 * LX + c * 3 * LY;
            T a0[N1], a1[N1];
#pragma unroll
            for (int j = 0; j < N1; ++j) {
                a0[j] = X[(k * N1 + j) * NQ + qx];
                a1[j] = X[LX + (k * N1 + j) * NQ + qx];
            }
#pragma unroll
            for (int qy = 0; qy < NQ; ++qy) {
                T v0 = 0, v1 = 0, v2 = 0;
#pragma unroll
                for (int j = 0; j < N1; ++j) {
                    v0 = fma(B[qy][j], a0[j], v0);
                    v1 = fma(D[qy][j], a0[j], v1);
                    v2 = fma(B[qy][j], a1[j], v2);
                }
                const int o = (k * NQ + qy) * NQ + qx;
                Y[o] = v0;
                Y[LY + o] = v1;
                Y[2 * LY + o] = v2;
            }
        }
        __syncthreads();
        // ---- z: line (el, c, qy, qx) -> PV[c][m][q] = d/dxi_m of component c
        for (int t = threadIdx.x; t < ne * 6 * NQ * NQ; t += THREADS) {
            const int qx = t % NQ, qy = (t / NQ) % NQ, c = (t / (NQ * NQ)) % 6, el = t / (NQ * NQ * 6);
            const T *Y = sm + el * PE + P::R1 + 12 * LX + c * 3 * LY;
            T *PV = sm + el * PE + P::R2 + c * 3 * Q;
            T y0[N1], y1[N1], y2[N1];
#pragma unroll
            for (int k = 0; k < N1; ++k) {
                const int o = (k * NQ + qy) * NQ + qx;
                y0[k] = Y[o];
                y1[k] = Y[LY + o];
                y2[k] = Y[2 * LY + o];
            }
#pragma unroll
            for (int qz = 0; qz < NQ; ++qz) {
                const int q = (qz * NQ + qy) * NQ + qx;
                T gx = 0, gy = 0, gz = 0;
#pragma unroll
                for (int k = 0; k < N1; ++k) {
                    gx = fma(B[qz][k], y2[k], gx);
                    gy = fma(B[qz][k], y1[k], gy);
                    gz = fma(D[qz][k], y0[k], gz);
                }
                PV[q] = gx;
                PV[Q + q] = gy;
                PV[2 * Q + q] = gz;
            }
        }
        __syncthreads();
        // ---- pointwise: gradients, stresses, material integrands, fluxes
        for (int t = threadIdx.x; t < ne * Q; t += THREADS) {
            const int el = t / Q, q = t % Q;
            T *S = sm + el * PE;
            const T *Ji = S + P::JI + q * 9;
            const T wd = S[P::WD + q];
            const T lam = (T)lame[2 * (e0 + el)], mu = (T)lame[2 * (e0 + el) + 1];
            T gu[3][3], gb[3][3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const T *pu = S + P::R2 + c * 3 * Q + q, *pb = S + P::R2 + (3 + c) * 3 * Q + q;
                const T u0 = pu[0], u1 = pu[Q], u2 = pu[2 * Q], b0 = pb[0], b1 = pb[Q], b2 = pb[2 * Q];
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    gu[c][j] = u0 * Ji[j] + u1 * Ji[3 + j] + u2 * Ji[6 + j];
                    gb[c][j] = b0 * Ji[j] + b1 * Ji[3 + j] + b2 * Ji[6 + j];
                }
            }
            const T divu = gu[0][0] + gu[1][1] + gu[2][2], divb = gb[0][0] + gb[1][1] + gb[2][2];
            T ee = 0;  // eps(u) : eps(rbar)
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) ee = fma((T)0.25 * (gu[i][j] + gu[j][i]), gb[i][j] + gb[j][i], ee);
            S[P::RED + q] = wd * divu * divb;
            S[P::RED + Q + q] = wd * (T)2 * ee;
            if (dxe) {
                T su[3][3], sb[3][3];
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        su[i][j] = mu * (gu[i][j] + gu[j][i]) + (i == j ? lam * divu : (T)0);
                        sb[i][j] = mu * (gb[i][j] + gb[j][i]) + (i == j ? lam * divb : (T)0);
                    }
                const T f = lam * divu * divb + (T)2 * mu * ee;
                T Sm[3][3];
#pragma unroll
                for (int m = 0; m < 3; ++m)
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        T s = m == j ? f : (T)0;
#pragma unroll
                        for (int i = 0; i < 3; ++i) s -= gb[i][m] * su[i][j] + gu[i][m] * sb[i][j];
                        Sm[m][j] = wd * s;
                    }
#pragma unroll
                for (int m = 0; m < 3; ++m)
#pragma unroll
                    for (int k = 0; k < 3; ++k)
                        S[P::FL + (m * 3 + k) * Q + q] =
                            Sm[m][0] * Ji[k * 3] + Sm[m][1] * Ji[k * 3 + 1] + Sm[m][2] * Ji[k * 3 + 2];
            }
        }
        __syncthreads();
        // ---- material terms: sums over the points, one thread per (element, term)
        for (int t = threadIdx.x; t < ne * 2; t += THREADS) {
            const int el = t / 2, which = t % 2;
            const T *R = sm + el * PE + P::RED + which * Q;
            T s = 0;
            for (int q = 0; q < Q; ++q) s += R[q];
            if (dmat) dmat[2 * (e0 + el) + which] = s;  // (lambda, mu) pairs, the material layout
        }
        if (!dxe) continue;
        // ---- coordinate term: dX[m][a] = sum_q sum_k F[m][k] dphi_a/dxi_k, stages z^T, y^T, x^T
        for (int t = threadIdx.x; t < ne * 3 * NQ * NQ; t += THREADS) {  // z^T: [0] B_z F_x, [1] B_z F_y, [2] D_z F_z
            const int qx = t % NQ, qy = (t / NQ) % NQ, m = (t / (NQ * NQ)) % 3, el = t / (NQ * NQ * 3);
            const T *F = sm + el * PE + P::FL + m * 3 * Q;
            T *Zt = sm + el * PE + P::R1 + m * 3 * LY;
            T f0[NQ], f1[NQ], f2[NQ];
#pragma unroll
            for (int qz = 0; qz < NQ; ++qz) {
                const int q = (qz * NQ + qy) * NQ + qx;
                f0[qz] = F[q];
                f1[qz] = F[Q + q];
                f2[qz] = F[2 * Q + q];
            }
#pragma unroll
            for (int k = 0; k < N1; ++k) {
                T v0 = 0, v1 = 0, v2 = 0;
#pragma unroll
                for (int qz = 0; qz < NQ; ++qz) {
                    v0 = fma(B[qz][k], f0[qz], v0);
                    v1 = fma(B[qz][k], f1[qz], v1);
                    v2 = fma(D[qz][k], f2[qz], v2);
                }
                const int o = (k * NQ + qy) * NQ + qx;
                Zt[o] = v0;
                Zt[LY + o] = v1;
                Zt[2 * LY + o] = v2;
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < ne * 3 * N1 * NQ; t += THREADS) {  // y^T: [0] B_y [0], [1] D_y [1] + B_y [2]
            const int qx = t % NQ, k = (t / NQ) % N1, m = (t / (NQ * N1)) % 3, el = t / (NQ * N1 * 3);
            const T *Zt = sm + el * PE + P::R1 + m * 3 * LY;
            T *Yt = sm + el * PE + P::R1 + 9 * LY + m * 2 * LX;
            T y0[NQ], y1[NQ], y2[NQ];
#pragma unroll
            for (int qy = 0; qy < NQ; ++qy) {
                const int o = (k * NQ + qy) * NQ + qx;
                y0[qy] = Zt[o];
                y1[qy] = Zt[LY + o];
                y2[qy] = Zt[2 * LY + o];
            }
#pragma unroll
            for (int j = 0; j < N1; ++j) {
                T v0 = 0, v1 = 0;
#pragma unroll
                for (int qy = 0; qy < NQ; ++qy) {
                    v0 = fma(B[qy][j], y0[qy], v0);
                    v1 = fma(D[qy][j], y1[qy], fma(B[qy][j], y2[qy], v1));
                }
                Yt[(k * N1 + j) * NQ + qx] = v0;
                Yt[LX + (k * N1 + j) * NQ + qx] = v1;
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < ne * 3 * N1 * N1; t += THREADS) {  // x^T: D_x [0] + B_x [1]
            const int kj = t % (N1 * N1), m = (t / (N1 * N1)) % 3, el = t / (N1 * N1 * 3);
            const T *Yt = sm + el * PE + P::R1 + 9 * LY + m * 2 * LX + kj * NQ;
            T x0[NQ], x1[NQ];
#pragma unroll
            for (int qx = 0; qx < NQ; ++qx) {
                x0[qx] = Yt[qx];
                x1[qx] = Yt[LX + qx];
            }
            T *o = dxe + (e0 + el) * (long long)(3 * N) + m * N + kj * N1;
#pragma unroll
            for (int i = 0; i < N1; ++i) {
                T v = 0;
#pragma unroll
                for (int qx = 0; qx < NQ; ++qx) v = fma(D[qx][i], x0[qx], fma(B[qx][i], x1[qx], v));
                o[i] = v;
            }
        }
    }
}

template <typename T, int N1, int NQ, int EPB>
cudaError_t launch_ad(const fe_geometry_h *g, const double *lame, const void *u, const void *rbar, void *dmat,
                      void *dxe, unsigned long long *st, cudaStream_t s)
{
    using P = AdPlan<T, N1, NQ>;
    constexpr int THREADS = 256;
    constexpr size_t SMEM = sizeof(T) * (size_t)P::PER_EL * EPB;
    static_assert(SMEM <= 227 * 1024, "shared memory plan too large");
    static_assert(6 * 2 * P::LX + 6 * 3 * P::LY >= 9 * P::LY + 6 * P::LX, "transposed stages must fit");
    auto kern = k_adjoint_sf<T, N1, NQ, EPB, THREADS>;
    static FeLaunchCache cache;
    long long cap = 0;
    cudaError_t err = fe_cached_grid(
        cache,
        [&](int dev, long long *v) {
            cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
            if (e2 != cudaSuccess) return e2;
            int sms = 0, per_sm = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, SMEM);
            if (e2 != cudaSuccess) return e2;
            if (per_sm < 1) return cudaErrorInvalidConfiguration;
            *v = (long long)per_sm * sms * 4;
            return cudaSuccess;
        },
        &cap);
    if (err != cudaSuccess) return err;
    const long long E = g->mesh.n_elems;
    long long blocks = (E + EPB - 1) / EPB;
    if (blocks > cap) blocks = cap;
    constexpr bool f64 = sizeof(T) == 8;
    kern<<<(unsigned)blocks, THREADS, SMEM, s>>>(
        f64 ? (const T *)g->d_jinv64 : (const T *)g->d_jinv32, f64 ? (const T *)g->d_wdetj64 : (const T *)g->d_wdetj32,
        f64 ? (const T *)g->d_b1d : (const T *)g->d_b1d32, f64 ? (const T *)g->d_d1d : (const T *)g->d_d1d32,
        g->mesh.conn, E, lame, (const T *)u, (const T *)rbar, (T *)dmat, (T *)dxe, g->mesh.n_nodes, st);
    return cudaGetLastError();
}

template <typename T>
cudaError_t dispatch_ad(const fe_geometry_h *g, const double *lame, const void *u, const void *rbar, void *dmat,
                        void *dxe, unsigned long long *st, cudaStream_t s)
{
    const int n1 = g->n1d, nq = g->nq1d;
    constexpr bool D = sizeof(T) == 8;
    if (n1 == 2 && nq == 2) return launch_ad<T, 2, 2, 8>(g, lame, u, rbar, dmat, dxe, st, s);
    if (n1 == 2 && nq == 3) return launch_ad<T, 2, 3, 4>(g, lame, u, rbar, dmat, dxe, st, s);
    if (n1 == 3 && nq == 3) return launch_ad<T, 3, 3, (D ? 4 : 8)>(g, lame, u, rbar, dmat, dxe, st, s);
    if (n1 == 3 && nq == 4) return launch_ad<T, 3, 4, (D ? 2 : 4)>(g, lame, u, rbar, dmat, dxe, st, s);
    if (n1 == 4 && nq == 4) return launch_ad<T, 4, 4, (D ? 1 : 2)>(g, lame, u, rbar, dmat, dxe, st, s);
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t fe_launch_adjoint(const fe_geometry_h *g, bool f64, const double *lame, const void *u,
                              const void *rbar, void *dmat, void *dxe, unsigned long long *status, cudaStream_t s)
{
    if (g->mesh.n_elems == 0) return cudaSuccess;
    return f64 ? dispatch_ad<double>(g, lame, u, rbar, dmat, dxe, status, s)
               : dispatch_ad<float>(g, lame, u, rbar, dmat, dxe, status, s);
}
