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
#include "geometry_body.cuh"

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

// Sum-factorised residual for tensor-product hexahedra (n1 nodes, nq points per
// axis; B/D the 1-D basis values/derivatives at the points, (nq, n1)).  Per
// element and component c with nodal values U[k][j][i]:
//   phase 1  u_h or grad_xi u_h at the points by three 1-D contractions
//            (x: B, D; y: B, D; z: B, D), as in the geometry kernel
//   point    the flux F (mass: c wdetJ u_h; Laplace: c wdetJ J^-1 J^-T g;
//            elasticity: wdetJ J^-1 sigma with sigma = D e(u_h))
//   phase 2  r[a] = sum_q sum_m F_m(q) d phi_a / d xi_m (q) by the transposed
//            contractions (z, y, x)
// Each thread computes one whole 1-D line of a stage (n1 or nq outputs) with
// the 1-D tables in registers; EPB elements per CTA, barriers between stages.
// Per-element material of ne elements into shared memory: the 6x6 D (Voigt,
// MATK 2), (lambda, mu) (MATK 1) or a scalar coefficient (1 without one).
template <typename T, int MATK, int THREADS>
__device__ __forceinline__ void load_material(int ne, long long e0, const double *__restrict__ mat, int mat_t,
                                              T (*__restrict__ sM)[36])
{
    if constexpr (MATK == 2) {
        for (int t = threadIdx.x; t < ne * 36; t += THREADS) {
            const int el = t / 36, I = (t % 36) / 6, Kv = t % 6;
            const long long e = e0 + el;
            sM[el][t % 36] = (T)(mat_t ? mat[e * 36 + Kv * 6 + I] : mat[e * 36 + I * 6 + Kv]);
        }
    } else if constexpr (MATK == 1) {
        for (int t = threadIdx.x; t < ne * 2; t += THREADS) sM[t / 2][t % 2] = (T)mat[e0 * 2 + t];
    } else {
        for (int t = threadIdx.x; t < ne; t += THREADS) sM[t][0] = mat ? (T)mat[e0 + t] : (T)1;
    }
}

// The stages of k_residual_sf after the loads, for ne elements starting at e0
// whose DOFs (sU), J^-1 (sJ), w det J (sW) and material (sM) are in shared
// memory; B, D = 1-D tables (nq, n1) in registers.  Ends with r written.
template <typename T, int N1, int NQ, int KIND, int MATK, int EPB, int THREADS, bool WARP = false>
__device__ __forceinline__ void residual_sf_stages(
    int ne, int nc_rt, long long e0, T (*__restrict__ sU)[KIND == FK_LAPLACE ? 1 : 3][N1 * N1 * N1],
    T (*__restrict__ sX)[KIND == FK_LAPLACE ? 1 : 3][KIND != FK_MASS ? 2 : 1][N1 * N1 * NQ],
    T (*__restrict__ sY)[KIND == FK_LAPLACE ? 1 : 3][KIND != FK_MASS ? 3 : 1][N1 * NQ * NQ],
    T (*__restrict__ sQ)[KIND == FK_LAPLACE ? 1 : 3][KIND != FK_MASS ? 3 : 1][NQ * NQ * NQ],
    T (*__restrict__ sJ)[NQ * NQ * NQ][9], T (*__restrict__ sW)[NQ * NQ * NQ], T (*__restrict__ sM)[36],
    const T (&B)[NQ][N1], const T (&D)[NQ][N1], T *__restrict__ r)
{
    constexpr int N = N1 * N1 * N1, Q = NQ * NQ * NQ;
    constexpr bool GRAD = KIND != FK_MASS;
    constexpr int NC = KIND == FK_LAPLACE ? 1 : 3;
    constexpr int NM = GRAD ? 3 : 1;
    (void)NM;
    // components: known at compile time except for the mass form (scalar or
    // vector), so that the stage index arithmetic divides by constants
    const int nc = KIND == FK_MASS ? nc_rt : NC;
    // WARP: one warp works through the stages of its own element (lanes = lines
    // or points), with warp-level instead of block-level synchronisation
    const int tid0 = WARP ? (int)(threadIdx.x & 31) : (int)threadIdx.x;
    constexpr int STRIDE = WARP ? 32 : THREADS;
    auto stage_sync = [] {
        if constexpr (WARP) __syncwarp();
        else __syncthreads();
    };
    // ---- phase 1, x: line (el, c, k, j) -> sX[0] = B_x U, sX[1] = D_x U at qx = 0..nq-1
    for (int t = tid0; t < ne * nc * N1 * N1; t += STRIDE) {
        const int kj = t % (N1 * N1), c = (t / (N1 * N1)) % nc, el = t / (N1 * N1 * nc);
        T x[N1];
#pragma unroll
        for (int i = 0; i < N1; ++i) x[i] = sU[el][c][kj * N1 + i];
#pragma unroll
        for (int qx = 0; qx < NQ; ++qx) {
            T v0 = 0, v1 = 0;
#pragma unroll
            for (int i = 0; i < N1; ++i) {
                v0 = fma(B[qx][i], x[i], v0);
                if constexpr (GRAD) v1 = fma(D[qx][i], x[i], v1);
            }
            sX[el][c][0][kj * NQ + qx] = v0;
            if constexpr (GRAD) sX[el][c][1][kj * NQ + qx] = v1;
        }
    }
    stage_sync();
    // ---- phase 1, y: line (el, c, k, qx) -> at qy: [0] B_y B_x, [1] D_y B_x, [2] B_y D_x
    for (int t = tid0; t < ne * nc * N1 * NQ; t += STRIDE) {
        const int qx = t % NQ, k = (t / NQ) % N1, c = (t / (NQ * N1)) % nc, el = t / (NQ * N1 * nc);
        T a0[N1], a1[N1];
#pragma unroll
        for (int j = 0; j < N1; ++j) {
            a0[j] = sX[el][c][0][(k * N1 + j) * NQ + qx];
            if constexpr (GRAD) a1[j] = sX[el][c][1][(k * N1 + j) * NQ + qx];
        }
#pragma unroll
        for (int qy = 0; qy < NQ; ++qy) {
            T v0 = 0, v1 = 0, v2 = 0;
#pragma unroll
            for (int j = 0; j < N1; ++j) {
                v0 = fma(B[qy][j], a0[j], v0);
                if constexpr (GRAD) {
                    v1 = fma(D[qy][j], a0[j], v1);
                    v2 = fma(B[qy][j], a1[j], v2);
                }
            }
            const int o = (k * NQ + qy) * NQ + qx;
            sY[el][c][0][o] = v0;
            if constexpr (GRAD) {
                sY[el][c][1][o] = v1;
                sY[el][c][2][o] = v2;
            }
        }
    }
    stage_sync();
    // ---- phase 1, z: line (el, c, qy, qx) -> sQ[m] at qz = d u_c / d xi_m (or u_c)
    for (int t = tid0; t < ne * nc * NQ * NQ; t += STRIDE) {
        const int qx = t % NQ, qy = (t / NQ) % NQ, c = (t / (NQ * NQ)) % nc, el = t / (NQ * NQ * nc);
        T y0[N1], y1[N1], y2[N1];
#pragma unroll
        for (int k = 0; k < N1; ++k) {
            const int o = (k * NQ + qy) * NQ + qx;
            y0[k] = sY[el][c][0][o];
            if constexpr (GRAD) {
                y1[k] = sY[el][c][1][o];
                y2[k] = sY[el][c][2][o];
            }
        }
#pragma unroll
        for (int qz = 0; qz < NQ; ++qz) {
            const int q = (qz * NQ + qy) * NQ + qx;
            T gx = 0, gy = 0, gz = 0;
#pragma unroll
            for (int k = 0; k < N1; ++k) {
                if constexpr (GRAD) {
                    gx = fma(B[qz][k], y2[k], gx);
                    gy = fma(B[qz][k], y1[k], gy);
                    gz = fma(D[qz][k], y0[k], gz);
                } else {
                    gx = fma(B[qz][k], y0[k], gx);
                }
            }
            sQ[el][c][0][q] = gx;
            if constexpr (GRAD) {
                sQ[el][c][1][q] = gy;
                sQ[el][c][2][q] = gz;
            }
        }
    }
    stage_sync();
    // ---- pointwise flux, in place: F_c,m(q) with r = sum_q sum_m F_c,m dphi_a/dxi_m
    for (int t = tid0; t < ne * Q; t += STRIDE) {
        const int el = t / Q, q = t % Q;
        const T wd = sW[el][q];
        if constexpr (KIND == FK_MASS) {
            const T cw = sM[el][0] * wd;
            for (int c = 0; c < nc; ++c) sQ[el][c][0][q] *= cw;
        } else {
            T Ji[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) Ji[k] = sJ[el][q][k];
            T H[NC][3];  // physical gradient H[c][j] = sum_m g[c][m] Jinv[m][j]
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const T g0 = sQ[el][c][0][q], g1 = sQ[el][c][1][q], g2 = sQ[el][c][2][q];
#pragma unroll
                for (int j = 0; j < 3; ++j) H[c][j] = g0 * Ji[j] + g1 * Ji[3 + j] + g2 * Ji[6 + j];
            }
            T S[NC][3];
            if constexpr (KIND == FK_LAPLACE) {
                const T cw = sM[el][0] * wd;
#pragma unroll
                for (int j = 0; j < 3; ++j) S[0][j] = cw * H[0][j];
            } else if constexpr (MATK == 1) {
                // isotropic: sigma = lambda tr(e) I + 2 mu e
                const T lam = sM[el][0] * wd, mu = sM[el][1] * wd;
                const T tr = lam * (H[0][0] + H[1][1] + H[2][2]);
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) S[i][j] = mu * (H[i][j] + H[j][i]) + (i == j ? tr : (T)0);
            } else {
                const T *Dm = sM[el];
                const T eps[6] = {H[0][0], H[1][1], H[2][2], H[0][1] + H[1][0], H[0][2] + H[2][0],
                                  H[1][2] + H[2][1]};
                T sig[6];
#pragma unroll
                for (int I = 0; I < 6; ++I) {
                    T acc = 0;
#pragma unroll
                    for (int Kv = 0; Kv < 6; ++Kv) acc = fma(Dm[I * 6 + Kv], eps[Kv], acc);
                    sig[I] = wd * acc;
                }
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) S[i][j] = sig[fe_voigt(i, j)];
            }
#pragma unroll
            for (int c = 0; c < NC; ++c)
#pragma unroll
                for (int m = 0; m < 3; ++m)
                    sQ[el][c][m][q] = S[c][0] * Ji[m * 3] + S[c][1] * Ji[m * 3 + 1] + S[c][2] * Ji[m * 3 + 2];
        }
    }
    stage_sync();
    // ---- phase 2, z^T: line (el, c, qy, qx) -> at k: [0] B_z F_x, [1] B_z F_y, [2] D_z F_z
    for (int t = tid0; t < ne * nc * NQ * NQ; t += STRIDE) {
        const int qx = t % NQ, qy = (t / NQ) % NQ, c = (t / (NQ * NQ)) % nc, el = t / (NQ * NQ * nc);
        T f0[NQ], f1[NQ], f2[NQ];
#pragma unroll
        for (int qz = 0; qz < NQ; ++qz) {
            const int q = (qz * NQ + qy) * NQ + qx;
            f0[qz] = sQ[el][c][0][q];
            if constexpr (GRAD) {
                f1[qz] = sQ[el][c][1][q];
                f2[qz] = sQ[el][c][2][q];
            }
        }
#pragma unroll
        for (int k = 0; k < N1; ++k) {
            T v0 = 0, v1 = 0, v2 = 0;
#pragma unroll
            for (int qz = 0; qz < NQ; ++qz) {
                v0 = fma(B[qz][k], f0[qz], v0);
                if constexpr (GRAD) {
                    v1 = fma(B[qz][k], f1[qz], v1);
                    v2 = fma(D[qz][k], f2[qz], v2);
                }
            }
            const int o = (k * NQ + qy) * NQ + qx;
            sY[el][c][0][o] = v0;
            if constexpr (GRAD) {
                sY[el][c][1][o] = v1;
                sY[el][c][2][o] = v2;
            }
        }
    }
    stage_sync();
    // ---- phase 2, y^T: line (el, c, k, qx) -> at j: [0] B_y [0], [1] D_y [1] + B_y [2]
    for (int t = tid0; t < ne * nc * N1 * NQ; t += STRIDE) {
        const int qx = t % NQ, k = (t / NQ) % N1, c = (t / (NQ * N1)) % nc, el = t / (NQ * N1 * nc);
        T y0[NQ], y1[NQ], y2[NQ];
#pragma unroll
        for (int qy = 0; qy < NQ; ++qy) {
            const int o = (k * NQ + qy) * NQ + qx;
            y0[qy] = sY[el][c][0][o];
            if constexpr (GRAD) {
                y1[qy] = sY[el][c][1][o];
                y2[qy] = sY[el][c][2][o];
            }
        }
#pragma unroll
        for (int j = 0; j < N1; ++j) {
            T v0 = 0, v1 = 0;
#pragma unroll
            for (int qy = 0; qy < NQ; ++qy) {
                v0 = fma(B[qy][j], y0[qy], v0);
                if constexpr (GRAD) v1 = fma(D[qy][j], y1[qy], fma(B[qy][j], y2[qy], v1));
            }
            sX[el][c][0][(k * N1 + j) * NQ + qx] = v0;
            if constexpr (GRAD) sX[el][c][1][(k * N1 + j) * NQ + qx] = v1;
        }
    }
    stage_sync();
    // ---- phase 2, x^T: line (el, c, k, j) -> r at i = D_x [0] + B_x [1] (mass: B_x [0])
    for (int t = tid0; t < ne * nc * N1 * N1; t += STRIDE) {
        const int kj = t % (N1 * N1), c = (t / (N1 * N1)) % nc, el = t / (N1 * N1 * nc);
        T x0[NQ], x1[NQ];
#pragma unroll
        for (int qx = 0; qx < NQ; ++qx) {
            x0[qx] = sX[el][c][0][kj * NQ + qx];
            if constexpr (GRAD) x1[qx] = sX[el][c][1][kj * NQ + qx];
        }
        T *ro = r + (e0 + el) * (long long)nc * N + c * N + kj * N1;
#pragma unroll
        for (int i = 0; i < N1; ++i) {
            T v = 0;
#pragma unroll
            for (int qx = 0; qx < NQ; ++qx) {
                if constexpr (GRAD)
                    v = fma(D[qx][i], x0[qx], fma(B[qx][i], x1[qx], v));
                else
                    v = fma(B[qx][i], x0[qx], v);
            }
            ro[i] = v;
        }
    }
}

template <typename T, int N1, int NQ, int KIND, int MATK, int EPB, int THREADS>
__global__ void __launch_bounds__(THREADS) k_residual_sf(const T *__restrict__ jinv, const T *__restrict__ wdetj,
                                                         const T *__restrict__ b1d, const T *__restrict__ d1d,
                                                         const int32_t *__restrict__ conn, long long E, int ncomp,
                                                         const double *__restrict__ mat, int mat_t,
                                                         const T *__restrict__ u, T *__restrict__ r,
                                                         long long n_nodes, unsigned long long *__restrict__ status)
{
    constexpr int N = N1 * N1 * N1, Q = NQ * NQ * NQ;
    constexpr bool GRAD = KIND != FK_MASS;
    constexpr int NC = KIND == FK_LAPLACE ? 1 : 3;  // max components
    constexpr int NM = GRAD ? 3 : 1;                // derivative directions carried
    constexpr int LX = N1 * N1 * NQ, LY = N1 * NQ * NQ;
    __shared__ T sU[EPB][NC][N];
    __shared__ T sX[EPB][NC][GRAD ? 2 : 1][LX];  // stage x (phase 1) / stage y^T (phase 2)
    __shared__ T sY[EPB][NC][NM][LY];            // stage y (phase 1) / stage z^T (phase 2)
    __shared__ T sQ[EPB][NC][NM][Q];             // point values: gradients, then fluxes
    __shared__ T sJ[EPB][Q][9];
    __shared__ T sW[EPB][Q];
    __shared__ T sM[EPB][36];
    T B[NQ][N1], D[NQ][N1];
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int i = 0; i < N1; ++i) {
            B[q][i] = b1d[q * N1 + i];
            D[q][i] = d1d[q * N1 + i];
        }
    const int nc = ncomp;
    for (long long e0 = (long long)blockIdx.x * EPB; e0 < E; e0 += (long long)gridDim.x * EPB) {
        const int ne = (int)((E - e0) < EPB ? (E - e0) : EPB);
        __syncthreads();
        if constexpr (GRAD)
            for (int t = threadIdx.x; t < ne * Q * 9; t += THREADS) (&sJ[0][0][0])[t] = jinv[e0 * Q * 9 + t];
        for (int t = threadIdx.x; t < ne * Q; t += THREADS) (&sW[0][0])[t] = wdetj[e0 * Q + t];
        for (int t = threadIdx.x; t < ne * N; t += THREADS) {
            const int el = t / N, a = t % N;
            const long long node = conn[(e0 + el) * N + a];
            const bool ok = (unsigned long long)node < (unsigned long long)n_nodes;  // never read outside u
            if (!ok) fe_report(status, FE_ERR_SHAPE, e0 + el);
            for (int c = 0; c < nc; ++c) sU[el][c][a] = ok ? u[node * nc + c] : (T)0;
        }
        load_material<T, MATK, THREADS>(ne, e0, mat, mat_t, sM);
        __syncthreads();
        residual_sf_stages<T, N1, NQ, KIND, MATK, EPB, THREADS>(ne, nc, e0, sU, sX, sY, sQ, sJ, sW, sM, B, D, r);
    }
}

// Float32 residual of Q2 hexahedra with 3 x 3 x 3 points, one element per warp:
// the same stages as k_residual_sf (lanes = the 27 lines or points of the
// element; Laplace uses 9 lines), synchronised within the warp only, with the
// inputs of the warp's next element (J^-1, w det J, the gathered DOFs, the
// material) loaded into registers while the stages of the current one run, and
// the connectivity two elements ahead.  Each warp has its own stage buffers.
template <int KIND, int MATK, int WPC>
__global__ void __launch_bounds__(WPC * 32) k_residual_sfw(const float *__restrict__ jinv,
                                                         const float *__restrict__ wdetj,
                                                         const float *__restrict__ b1d, const float *__restrict__ d1d,
                                                         const int32_t *__restrict__ conn, long long E, int ncomp,
                                                         const double *__restrict__ mat, int mat_t,
                                                         const float *__restrict__ u, float *__restrict__ r,
                                                         long long n_nodes, unsigned long long *__restrict__ status)
{
    constexpr int N1 = 3, NQ = 3, N = 27, Q = 27;
    constexpr bool GRAD = KIND != FK_MASS;
    constexpr int NC = KIND == FK_LAPLACE ? 1 : 3;  // max components
    constexpr int NM = GRAD ? 3 : 1;
    constexpr int LX = N1 * N1 * NQ, LY = N1 * NQ * NQ;
    constexpr int NJ = (Q * 9 + 31) / 32;  // J^-1 loads per lane
    __shared__ float sU[WPC][1][NC][N];
    __shared__ float sX[WPC][1][NC][GRAD ? 2 : 1][LX];
    __shared__ float sY[WPC][1][NC][NM][LY];
    __shared__ float sQ[WPC][1][NC][NM][Q];
    __shared__ float sJ[WPC][1][Q][9];
    __shared__ float sW[WPC][1][Q];
    __shared__ float sM[WPC][1][36];
    float B[NQ][N1], D[NQ][N1];
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int i = 0; i < N1; ++i) {
            B[q][i] = b1d[q * N1 + i];
            D[q][i] = d1d[q * N1 + i];
        }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nc = ncomp;
    const long long gstride = (long long)gridDim.x * WPC;
    float pj[NJ], pw = 0.0f, pu[NC], pm[2] = {0.0f, 0.0f};
    int pnode = 0;
    auto fetch_node = [&](long long e) {
        if (e < E && lane < N) pnode = conn[e * N + lane];
    };
    auto fetch = [&](long long e) {  // with pnode = the lane's node of element e
        if (e >= E) return;
#pragma unroll
        for (int i = 0; i < NJ; ++i) {
            const int t = lane + 32 * i;
            if (GRAD && t < Q * 9) pj[i] = jinv[e * (Q * 9) + t];
        }
        if (lane < Q) pw = wdetj[e * Q + lane];
        if (lane < N) {
            const bool ok = (unsigned)pnode < (unsigned long long)n_nodes;  // never read outside u
            if (!ok) fe_report(status, FE_ERR_SHAPE, e);
            const long long nd = ok ? pnode : 0;
#pragma unroll
            for (int c = 0; c < NC; ++c)
                if (c < nc) pu[c] = ok ? u[nd * nc + c] : 0.0f;
        }
        if constexpr (MATK == 2) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int t = lane + 32 * h;
                if (t < 36) {
                    const int I = t / 6, Kv = t % 6;
                    pm[h] = (float)(mat_t ? mat[e * 36 + Kv * 6 + I] : mat[e * 36 + I * 6 + Kv]);
                }
            }
        } else if constexpr (MATK == 1) {
            if (lane < 2) pm[0] = (float)mat[e * 2 + lane];
        } else {
            if (lane == 0) pm[0] = mat ? (float)mat[e] : 1.0f;
        }
    };
    long long e = (long long)blockIdx.x * WPC + w;
    fetch_node(e);
    fetch(e);
    fetch_node(e + gstride);
    for (; e < E; e += gstride) {
        __syncwarp();  // the stages of the previous element are done with the buffers
#pragma unroll
        for (int i = 0; i < NJ; ++i) {
            const int t = lane + 32 * i;
            if (GRAD && t < Q * 9) (&sJ[w][0][0][0])[t] = pj[i];
        }
        if (lane < Q) sW[w][0][lane] = pw;
        if (lane < N) {
#pragma unroll
            for (int c = 0; c < NC; ++c)
                if (c < nc) sU[w][0][c][lane] = pu[c];
        }
        if constexpr (MATK == 2) {
#pragma unroll
            for (int h = 0; h < 2; ++h)
                if (lane + 32 * h < 36) sM[w][0][lane + 32 * h] = pm[h];
        } else if constexpr (MATK == 1) {
            if (lane < 2) sM[w][0][lane] = pm[0];
        } else {
            if (lane == 0) sM[w][0][0] = pm[0];
        }
        fetch(e + gstride);
        fetch_node(e + 2 * gstride);
        __syncwarp();
        residual_sf_stages<float, N1, NQ, KIND, MATK, 1, 32, true>(1, nc, e, sU[w], sX[w], sY[w], sQ[w], sJ[w], sW[w],
                                                                   sM[w], B, D, r);
    }
}

// Residual of a float32-only geometry that is stale, with the geometry computed
// here (n1 == nq tensor-product bases): per group of EPB elements the FP64
// collocation stages of the geometry kernel (same roundings), whose float32
// J^-1 and w det J are stored in the handle and kept in shared memory for the
// stages of k_residual_sf.  The FP64 work of one group overlaps the float32
// stages of the other CTAs on the SM.  The FP64 work buffers share the space
// of the stage buffers, which are dead until the geometry is done.
template <int N1, int KIND, int MATK, int EPB, int THREADS>
struct ResGeoSmem {
    static constexpr int N = N1 * N1 * N1, NQ = N1, Q = N;
    static constexpr bool GRAD = KIND != FK_MASS;
    static constexpr int NC = KIND == FK_LAPLACE ? 1 : 3, NM = GRAD ? 3 : 1;
    static constexpr int LX = N1 * N1 * NQ, LY = N1 * NQ * NQ;
    static constexpr int U = 0;                                   // float [EPB][NC][N]
    static constexpr int X = U + EPB * NC * N * 4;                // float [EPB][NC][GRAD?2:1][LX]
    static constexpr int Y = X + EPB * NC * (GRAD ? 2 : 1) * LX * 4;  // float [EPB][NC][NM][LY]
    static constexpr int QV = Y + EPB * NC * NM * LY * 4;         // float [EPB][NC][NM][Q]
    static constexpr int STAGE_END = QV + EPB * NC * NM * Q * 4;
    static constexpr int G = (X + 7) / 8 * 8;                     // double [EPB][4][3 N], over the stage buffers
    static constexpr int G_END = G + EPB * 12 * N * 8;
    static constexpr int J = ((STAGE_END > G_END ? STAGE_END : G_END) + 15) / 16 * 16;  // float [EPB][Q][9]
    static constexpr int W = J + EPB * Q * 9 * 4;                 // float [EPB][Q]
    static constexpr int M = W + EPB * Q * 4;                     // float [EPB][36]
    static constexpr int T64 = (M + EPB * 36 * 4 + 7) / 8 * 8;   // double B[N1][N1], Dq[N1][N1] + extra, w[Q]
    static constexpr int BYTES = T64 + (2 * N1 * N1 + GEO_DQ_EXTRA + Q) * 8;
};

template <int N1, int KIND, int MATK, int EPB, int THREADS, bool CENTER>
__global__ void __launch_bounds__(THREADS, N1 == 3 ? 7 : 4) k_residual_geo(const double *__restrict__ coords,
                                                          const int32_t *__restrict__ conn, long long E,
                                                          long long n_nodes, const double *__restrict__ b1d64,
                                                          const double *__restrict__ dq64,
                                                          const double *__restrict__ w64,
                                                          const float *__restrict__ b1d, const float *__restrict__ d1d,
                                                          float *__restrict__ jinv_out, float *__restrict__ wdetj_out,
                                                          int ncomp, const double *__restrict__ mat, int mat_t,
                                                          const float *__restrict__ u, float *__restrict__ r,
                                                          unsigned long long *__restrict__ status)
{
    using L = ResGeoSmem<N1, KIND, MATK, EPB, THREADS>;
    using T = float;
    constexpr int N = L::N, NQ = L::NQ, Q = L::Q, NC = L::NC, NM = L::NM, LX = L::LX, LY = L::LY;
    constexpr bool GRAD = L::GRAD;
    static_assert(L::BYTES <= 48 * 1024, "static shared memory above 48 KB");
    __shared__ __align__(16) unsigned char raw[L::BYTES];
    T(*sU)[NC][N] = reinterpret_cast<T(*)[NC][N]>(raw + L::U);
    T(*sX)[NC][GRAD ? 2 : 1][LX] = reinterpret_cast<T(*)[NC][GRAD ? 2 : 1][LX]>(raw + L::X);
    T(*sY)[NC][NM][LY] = reinterpret_cast<T(*)[NC][NM][LY]>(raw + L::Y);
    T(*sQ)[NC][NM][Q] = reinterpret_cast<T(*)[NC][NM][Q]>(raw + L::QV);
    T(*sJ)[Q][9] = reinterpret_cast<T(*)[Q][9]>(raw + L::J);
    T(*sW)[Q] = reinterpret_cast<T(*)[Q]>(raw + L::W);
    T(*sM)[36] = reinterpret_cast<T(*)[36]>(raw + L::M);
    // per element: X (then P), U, V, and J (9 N doubles over U, V and a fourth block)
    double(*gG)[4][3 * N] = reinterpret_cast<double(*)[4][3 * N]>(raw + L::G);
    constexpr int LL = N1 * N1;
    double *gB = reinterpret_cast<double *>(raw + L::T64);
    double *gDq = gB + N1 * N1;
    double *gw = gDq + N1 * N1 + GEO_DQ_EXTRA;
    constexpr int LDQ = N1 * N1 + GEO_DQ_EXTRA;
    for (int i = threadIdx.x; i < N1 * N1 + LDQ + Q; i += THREADS)
        gB[i] = i < N1 * N1 ? b1d64[i] : (i < N1 * N1 + LDQ ? dq64[i - N1 * N1] : w64[i - N1 * N1 - LDQ]);
    T B[NQ][N1], D[NQ][N1];
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int i = 0; i < N1; ++i) {
            B[q][i] = b1d[q * N1 + i];
            D[q][i] = d1d[q * N1 + i];
        }
    const int nc = ncomp;
    for (long long e0 = (long long)blockIdx.x * EPB; e0 < E; e0 += (long long)gridDim.x * EPB) {
        const int ne = (int)((E - e0) < EPB ? (E - e0) : EPB);
        __syncthreads();
        for (int t = threadIdx.x; t < ne * N; t += THREADS) {
            const int el = t / N, a = t % N;
            const long long node = conn[(e0 + el) * N + a];
            const bool ok = (unsigned long long)node < (unsigned long long)n_nodes;  // never read outside
            if (!ok) fe_report(status, FE_ERR_SHAPE, e0 + el);
            const long long nd = ok ? node : 0;
#pragma unroll
            for (int c = 0; c < 3; ++c) gG[el][0][c * N + a] = coords[3 * nd + c];
            for (int c = 0; c < nc; ++c) sU[el][c][a] = ok ? u[node * nc + c] : (T)0;
        }
        load_material<T, MATK, THREADS>(ne, e0, mat, mat_t, sM);
        __syncthreads();
        for (int t = threadIdx.x; t < ne * 3 * LL; t += THREADS)  // geometry: contract i
            geo_lines_x<N1, CENTER>(t % (3 * LL), gG[t / (3 * LL)][0], gG[t / (3 * LL)][1], gB);
        __syncthreads();
        for (int t = threadIdx.x; t < ne * 3 * LL; t += THREADS)  // contract j
            geo_lines_y<N1, CENTER>(t % (3 * LL), gG[t / (3 * LL)][1], gG[t / (3 * LL)][2], gB);
        __syncthreads();
        for (int t = threadIdx.x; t < ne * 3 * LL; t += THREADS)  // contract k: x at the points
            geo_lines_z<N1, CENTER>(t % (3 * LL), gG[t / (3 * LL)][2], gG[t / (3 * LL)][0], gB);
        __syncthreads();
        for (int t = threadIdx.x; t < ne * 9 * LL; t += THREADS)  // J on the points
            geo_lines_jacobian<N1, CENTER>(t % (9 * LL), gG[t / (9 * LL)][0], gG[t / (9 * LL)][1], gDq);
        __syncthreads();
        for (int t = threadIdx.x; t < ne * Q; t += THREADS) {
            const int el = t / Q, q = t % Q;
            const double *J = gG[el][1] + q * 9;
            float o[9], wd;
            const double det = geo_point_f32(J, gw[q], o, wd);
            const int bad = geo_det_status(det);
            if (bad) fe_report(status, bad, e0 + el);
            const long long idx = (e0 + el) * Q + q;
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                jinv_out[idx * 9 + k] = o[k];
                sJ[el][q][k] = o[k];
            }
            wdetj_out[idx] = wd;
            sW[el][q] = wd;
        }
        __syncthreads();
        residual_sf_stages<T, N1, NQ, KIND, MATK, EPB, THREADS>(ne, nc, e0, sU, sX, sY, sQ, sJ, sW, sM, B, D, r);
    }
}

template <typename T, int N1, int NQ, int KIND, int MATK, int EPB>
cudaError_t launch_res_sf(const fe_geometry_h *g, const fe_form_h *f, fe_material_args mat, const void *u, void *r,
                          unsigned long long *st, cudaStream_t s)
{
    constexpr int THREADS = 256;
    auto kern = k_residual_sf<T, N1, NQ, KIND, MATK, EPB, THREADS>;
    static FeLaunchCache cache;
    long long cap = 0;
    cudaError_t err = fe_cached_grid(
        cache,
        [&](int dev, long long *v) {
            int sms = 0, per_sm = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaError_t e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, 0);
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
    const bool f64 = sizeof(T) == 8;
    kern<<<(unsigned)blocks, THREADS, 0, s>>>(
        f64 ? (const T *)g->d_jinv64 : (const T *)g->d_jinv32, f64 ? (const T *)g->d_wdetj64 : (const T *)g->d_wdetj32,
        f64 ? (const T *)g->d_b1d : (const T *)g->d_b1d32, f64 ? (const T *)g->d_d1d : (const T *)g->d_d1d32,
        g->mesh.conn, E, f->ncomp, mat.data, mat.transposed, (const T *)u, (T *)r, g->mesh.n_nodes, st);
    return cudaGetLastError();
}

template <int KIND, int MATK>
cudaError_t launch_res_sfw(const fe_geometry_h *g, const fe_form_h *f, fe_material_args mat, const void *u, void *r,
                           unsigned long long *st, cudaStream_t s)
{
    constexpr int WPC = 8;
    auto kern = k_residual_sfw<KIND, MATK, WPC>;
    static FeLaunchCache cache;
    long long cap = 0;
    cudaError_t err = fe_cached_grid(
        cache,
        [&](int dev, long long *v) {
            int sms = 0, per_sm = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaError_t e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WPC * 32, 0);
            if (e2 != cudaSuccess) return e2;
            if (per_sm < 1) return cudaErrorInvalidConfiguration;
            *v = (long long)per_sm * sms;  // one resident wave; warps stride over the elements
            return cudaSuccess;
        },
        &cap);
    if (err != cudaSuccess) return err;
    const long long E = g->mesh.n_elems;
    long long blocks = (E + WPC - 1) / WPC;
    if (blocks > cap) blocks = cap;
    kern<<<(unsigned)blocks, WPC * 32, 0, s>>>(g->d_jinv32, g->d_wdetj32, g->d_b1d32, g->d_d1d32, g->mesh.conn, E,
                                                f->ncomp, mat.data, mat.transposed, (const float *)u, (float *)r,
                                                g->mesh.n_nodes, st);
    return cudaGetLastError();
}

cudaError_t dispatch_sfw(const fe_geometry_h *g, const fe_form_h *f, fe_material_args mat, const void *u, void *r,
                         unsigned long long *st, cudaStream_t s)
{
    switch (f->kind) {
    case FK_LAPLACE: return launch_res_sfw<FK_LAPLACE, 0>(g, f, mat, u, r, st, s);
    case FK_MASS: return launch_res_sfw<FK_MASS, 0>(g, f, mat, u, r, st, s);
    case FK_ELASTICITY:
        if (mat.kind == FE_MAT_LAME) return launch_res_sfw<FK_ELASTICITY, 1>(g, f, mat, u, r, st, s);
        return launch_res_sfw<FK_ELASTICITY, 2>(g, f, mat, u, r, st, s);
    }
    return cudaErrorInvalidValue;
}

template <typename T, int N1, int NQ, int EPB_S, int EPB_V>
cudaError_t dispatch_sf_kind(const fe_geometry_h *g, const fe_form_h *f, fe_material_args mat, const void *u, void *r,
                             unsigned long long *st, cudaStream_t s)
{
    switch (f->kind) {
    case FK_LAPLACE: return launch_res_sf<T, N1, NQ, FK_LAPLACE, 0, EPB_S>(g, f, mat, u, r, st, s);
    case FK_MASS: return launch_res_sf<T, N1, NQ, FK_MASS, 0, EPB_S>(g, f, mat, u, r, st, s);
    case FK_ELASTICITY:
        if (mat.kind == FE_MAT_LAME) return launch_res_sf<T, N1, NQ, FK_ELASTICITY, 1, EPB_V>(g, f, mat, u, r, st, s);
        return launch_res_sf<T, N1, NQ, FK_ELASTICITY, 2, EPB_V>(g, f, mat, u, r, st, s);
    }
    return cudaErrorInvalidValue;
}

// Tensor-product bases with their 1-D factors: sum-factorised kernel; element
// counts per CTA keep the static shared memory under 48 KB.
template <typename T>
cudaError_t dispatch_sf(const fe_geometry_h *g, const fe_form_h *f, fe_material_args mat, const void *u, void *r,
                        unsigned long long *st, cudaStream_t s)
{
    const int n1 = g->n1d, nq = g->nq1d;
    constexpr bool D = sizeof(T) == 8;
    if (n1 == 2 && nq == 2) return dispatch_sf_kind<T, 2, 2, 16, 8>(g, f, mat, u, r, st, s);
    if (n1 == 2 && nq == 3) return dispatch_sf_kind<T, 2, 3, 8, 4>(g, f, mat, u, r, st, s);
    if (n1 == 3 && nq == 3) {
        if constexpr (!D) return dispatch_sfw(g, f, mat, u, r, st, s);  // float32: one element per warp
        return dispatch_sf_kind<T, 3, 3, 4, 2>(g, f, mat, u, r, st, s);
    }
    if (n1 == 3 && nq == 4) return dispatch_sf_kind<T, 3, 4, (D ? 2 : 4), (D ? 1 : 2)>(g, f, mat, u, r, st, s);
    if (n1 == 4 && nq == 4) return dispatch_sf_kind<T, 4, 4, (D ? 2 : 4), 1>(g, f, mat, u, r, st, s);
    return cudaErrorInvalidValue;
}

template <int N1, int KIND, int MATK, int EPB, bool CENTER>
cudaError_t launch_res_geo(fe_geometry_h *g, const fe_form_h *f, fe_material_args mat, const void *u, void *r,
                           unsigned long long *st, cudaStream_t s)
{
    constexpr int THREADS = N1 == 3 ? 192 : 256;  // Q2: 7 elements in 6 warps, 7 CTAs per SM
    auto kern = k_residual_geo<N1, KIND, MATK, EPB, THREADS, CENTER>;
    static FeLaunchCache cache;
    long long cap = 0;
    cudaError_t err = fe_cached_grid(
        cache,
        [&](int dev, long long *v) {
            int sms = 0, per_sm = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaError_t e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, 0);
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
    kern<<<(unsigned)blocks, THREADS, 0, s>>>(g->mesh.coords, g->mesh.conn, E, g->mesh.n_nodes, g->d_b1d, g->d_dq,
                                               g->d_w64, g->d_b1d32, g->d_d1d32, g->d_jinv32, g->d_wdetj32, f->ncomp,
                                               mat.data, mat.transposed, (const float *)u, (float *)r, st);
    return cudaGetLastError();
}

template <int N1, int EPB, bool CENTER>
cudaError_t dispatch_res_geo(fe_geometry_h *g, const fe_form_h *f, fe_material_args mat, const void *u, void *r,
                             unsigned long long *st, cudaStream_t s)
{
    switch (f->kind) {
    case FK_LAPLACE: return launch_res_geo<N1, FK_LAPLACE, 0, EPB, CENTER>(g, f, mat, u, r, st, s);
    case FK_MASS: return launch_res_geo<N1, FK_MASS, 0, EPB, CENTER>(g, f, mat, u, r, st, s);
    case FK_ELASTICITY:
        if (mat.kind == FE_MAT_LAME) return launch_res_geo<N1, FK_ELASTICITY, 1, EPB, CENTER>(g, f, mat, u, r, st, s);
        return launch_res_geo<N1, FK_ELASTICITY, 2, EPB, CENTER>(g, f, mat, u, r, st, s);
    }
    return cudaErrorNotSupported;
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
    static FeLaunchCache cache;
    long long cap = 0;
    cudaError_t err = fe_cached_grid(
        cache,
        [&](int dev, long long *v) {
            cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e2 != cudaSuccess) return e2;
            int sms = 0, per_sm = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, smem);
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
    FE_CASE(4, 5, 32)
    FE_CASE(10, 15, 16)
    FE_CASE(20, 35, 8)
#undef FE_CASE
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t fe_launch_residual(const fe_geometry_h *g, const fe_form_h *f, fe_material_args mat, bool f64,
                               const void *u, void *r, unsigned long long *st, cudaStream_t s)
{
    if (g->mesh.n_elems == 0) return cudaSuccess;
    if (g->d_b1d)
        return f64 ? dispatch_sf<double>(g, f, mat, u, r, st, s) : dispatch_sf<float>(g, f, mat, u, r, st, s);
    return f64 ? dispatch<double>(g, f, mat, u, r, st, s) : dispatch<float>(g, f, mat, u, r, st, s);
}

bool fe_residual_geometry_fusable(const fe_geometry_h *g, const fe_form_h *f)
{
    if (!g->d_dq || g->n1d != g->nq1d || g->n1d < 2 || g->n1d > 4 || !g->d_jinv32 || g->is_view) return false;
    if (!(g->flags & FE_GEOM_STORE_F32) || (g->flags & FE_GEOM_STORE_F64)) return false;
    return f->kind == FK_LAPLACE || f->kind == FK_MASS || f->kind == FK_ELASTICITY;
}

cudaError_t fe_launch_residual_geometry(fe_geometry_h *g, const fe_form_h *f, fe_material_args mat, const void *u,
                                        void *r, unsigned long long *st, cudaStream_t s)
{
    if (!fe_residual_geometry_fusable(g, f)) return cudaErrorNotSupported;
    if (g->mesh.n_elems == 0) return cudaSuccess;
    switch (g->n1d) {
    case 2: return dispatch_res_geo<2, 16, false>(g, f, mat, u, r, st, s);
    case 3:
        return g->geo_center ? dispatch_res_geo<3, 7, true>(g, f, mat, u, r, st, s)
                             : dispatch_res_geo<3, 7, false>(g, f, mat, u, r, st, s);
    case 4: return dispatch_res_geo<4, 2, false>(g, f, mat, u, r, st, s);
    }
    return cudaErrorNotSupported;
}
