// Navier-Stokes convective term 'i,i.j,j' (Eq. fe2 of Cimrman, arXiv
// 2107.04121, Tab. ewfd),
//   c(v, u, w) = int v_i (du_i/dx_j) w_j,
// in residual mode and in matrix mode (the derivative of Eq. fe4), on
// tensor-product hexahedra by sum factorisation.  u is the gradient operand
// and w the advection operand; the non-linear term has w = u.
//
// Per element (n = n1d nodes and m = nq1d points per axis, N = n^3, Q = m^3):
//   1. interpolation: the reference gradients of u and the values of w at the
//      points, by the 1-D contractions x, y, z (B = 1-D basis, D = its
//      derivative at the 1-D points);
//   2. pointwise: H_ab = w det J du_a/dx_b (physical gradient, J^-1 applied),
//      contravariant advection c_m = w det J sum_j (J^-1)_mj w_j;
//   3a. residual: F_a = sum_b H_ab w_b, r[(a,k)] = sum_q phi_k F_a by the
//       transposed contractions z, y, x;
//   3b. matrix: K[(a,k),(b,l)] = sum_q phi_k [ wrt_adv H_ab phi_l
//                                            + wrt_grad delta_ab sum_m c_m dphi_l/dxi_m ]
//       is a sum of weighted "mass-like" matrices sum_q W(q) phi_k(q) psi_l(q)
//       whose both factors are tensor products.  With twelve weight fields
//       (nine H_ab, three c_m) the point sums are contracted axis by axis:
//         T1[f][qx][qy][kz][lz] = sum_qz B[qz][kz] R_f,z[qz][lz] W_f(q)
//         T2[f][qx][ky][ly][kz][lz] = sum_qy B[qy][ky] R_f,y[qy][ly] T1[f][qx][qy][kz][lz]
//         K = sum_qx B[qx][kx] R_f,x[qx][lx] T2[f][qx][ky][ly][kz][lz]
//       where R_f,axis = D on axis m of field c_m and B otherwise.  The last
//       contraction runs with one thread per column (b, l) of the element
//       matrix, so each row of K is written by consecutive threads (coalesced).
// About 48 k FMA per Q2 element instead of the ~110 k of the point-by-point
// sums; FP64 is compute-bound, FP32 is bound by shared memory and the barriers
// between the stages (the K write alone would take about 60% of its time).  A stale
// float32-only deferred handle is computed by the FP32 residual or matrix kernel
// that reads it first: the geometry stages run at the start of each element group.
#include "geometry_body.cuh"

namespace {

template <typename T, int N1, int NQ, bool MAT>
struct CvPlan {
    static constexpr int N = N1 * N1 * N1, Q = NQ * NQ * NQ;
    static constexpr int LX = N1 * N1 * NQ, LY = N1 * NQ * NQ;
    static constexpr int NF = 12;                               // weight fields of the matrix
    static constexpr int T1N = NQ * NQ * N1 * N1, T2N = NQ * N1 * N1 * N1 * N1;
    // per-element layout in T units
    static constexpr int U = 0;                                 // [6][N]: u, then w
    static constexpr int JI = U + 6 * N;                        // [Q][9] J^-1
    static constexpr int WD = JI + 9 * Q;                       // [Q] w det J
    static constexpr int WT = WD + Q;                           // [NF][Q] weights / [3][Q] fluxes
    static constexpr int R1 = WT + NF * Q;                      // stages x, y | T1 | transposed stages
    static constexpr int R1N_I = 6 * 2 * LX + 6 * 3 * LY;
    static constexpr int R1N = MAT && NF * T1N > R1N_I ? NF * T1N : R1N_I;
    static constexpr int R2 = R1 + R1N;                         // point values [6][4][Q] | T2
    static constexpr int R2N_P = 6 * 4 * Q;
    // T2 keeps 11 fields (the nine H_ab, c_x, and c_y + c_z, which the last contraction
    // only uses summed) at a field stride of 3 mod 32 words, so that the lanes of one
    // warp reading three fields (the column blocks b) fall on disjoint banks
    static constexpr int NF2 = 11;
    static constexpr int FS = T2N + ((3 - T2N % 32) % 32 + 32) % 32;
    static constexpr int R2N = MAT && NF2 * FS > R2N_P ? NF2 * FS : R2N_P;
    static constexpr int PER_EL = (R2 + R2N + 1) / 2 * 2;  // even: the FP64 geometry area of each element
};

// Geometry computed in the FP32 residual or matrix kernel (a stale float32-only deferred
// handle, n1 == nq): the mesh, the FP64 1-D tables and where the float32 copy goes.
struct CvGeoArgs {
    const double *coords;
    const double *b1d, *dq, *w;  // (n1, n1) values at the points, derivative on the points, weights
    float *jinv_out, *wdetj_out;
};

template <typename T, int N1, int NQ, bool MAT, int EPB, int THREADS, int GEO>
__global__ void __launch_bounds__(THREADS) k_convect_sf(const T *__restrict__ jinv, const T *__restrict__ wdetj,
                                                        const T *__restrict__ b1d, const T *__restrict__ d1d,
                                                        const int32_t *__restrict__ conn, long long E,
                                                        const T *__restrict__ u, const T *__restrict__ w, int same,
                                                        int wrt_grad, int wrt_adv, T *__restrict__ K,
                                                        T *__restrict__ r, long long n_nodes,
                                                        unsigned long long *__restrict__ status, const CvGeoArgs geo)
{
    // GEO: 0 = geometry read from the handle, 1 = computed here, 2 = computed here
    // with the middle point on the middle node (three points per axis)
    using P = CvPlan<T, N1, NQ, MAT>;
    static_assert(!GEO || (N1 == NQ && sizeof(T) == 4), "in-kernel geometry: float32 kernels, n1 == nq");
    static_assert(!GEO || 12 * N1 * N1 * N1 * 2 <= P::R1N + P::R2N, "FP64 geometry fits the stage buffers");
    constexpr int N = P::N, Q = P::Q, LX = P::LX, LY = P::LY, PE = P::PER_EL;
    extern __shared__ __align__(16) unsigned char cv_smem[];
    T *sm = reinterpret_cast<T *>(cv_smem);
    T B[NQ][N1], D[NQ][N1];
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int i = 0; i < N1; ++i) {
            B[q][i] = b1d[q * N1 + i];
            D[q][i] = d1d[q * N1 + i];
        }
    const int nf = same ? 3 : 6;  // interpolated vector fields: u, and w when it differs
    // GEO tables after the per-element blocks: B, Dq (n1 x n1 + extra), w (Q), FP64
    double *gT = reinterpret_cast<double *>(sm + ((EPB * PE + 1) / 2) * 2);
    if constexpr (GEO != 0)
        for (int i = threadIdx.x; i < 2 * N1 * N1 + GEO_DQ_EXTRA + Q; i += THREADS)
            gT[i] = i < N1 * N1 ? geo.b1d[i]
                                : (i < 2 * N1 * N1 + GEO_DQ_EXTRA ? geo.dq[i - N1 * N1]
                                                                  : geo.w[i - 2 * N1 * N1 - GEO_DQ_EXTRA]);
    for (long long e0 = (long long)blockIdx.x * EPB; e0 < E; e0 += (long long)gridDim.x * EPB) {
        const int ne = (int)((E - e0) < EPB ? (E - e0) : EPB);
        __syncthreads();
        if constexpr (GEO == 0) {
            for (int t = threadIdx.x; t < ne * Q * 9; t += THREADS)
                sm[(t / (Q * 9)) * PE + P::JI + t % (Q * 9)] = jinv[e0 * Q * 9 + t];
            for (int t = threadIdx.x; t < ne * Q; t += THREADS) sm[(t / Q) * PE + P::WD + t % Q] = wdetj[e0 * Q + t];
        }
        for (int t = threadIdx.x; t < ne * N; t += THREADS) {
            const int el = t / N, a = t % N;
            const long long node = conn[(e0 + el) * N + a];
            const bool ok = (unsigned long long)node < (unsigned long long)n_nodes;  // never read outside u, w
            if (!ok) fe_report(status, FE_ERR_SHAPE, e0 + el);
            T *U = sm + el * PE + P::U;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                U[c * N + a] = ok ? u[node * 3 + c] : (T)0;
                if (!same) U[(3 + c) * N + a] = ok ? w[node * 3 + c] : (T)0;
            }
            if constexpr (GEO != 0) {
                // nodal x into the FP64 work area over the stage buffers: [X | U | V | -]
                double *G = reinterpret_cast<double *>(sm + el * PE + P::R1);
                const long long nd = ok ? node : 0;
#pragma unroll
                for (int c = 0; c < 3; ++c) G[c * N + a] = geo.coords[3 * nd + c];
            }
        }
        if constexpr (GEO != 0) {
            // FP64 geometry of the group (the stages and roundings of the geometry kernel)
            constexpr bool CENTER = GEO == 2;
            constexpr int L = N1 * N1;
            auto gbuf = [&](int el) { return reinterpret_cast<double *>(sm + el * PE + P::R1); };
            __syncthreads();
            for (int t = threadIdx.x; t < ne * 3 * L; t += THREADS)
                geo_lines_x<N1, CENTER>(t % (3 * L), gbuf(t / (3 * L)), gbuf(t / (3 * L)) + 3 * N, gT);
            __syncthreads();
            for (int t = threadIdx.x; t < ne * 3 * L; t += THREADS)
                geo_lines_y<N1, CENTER>(t % (3 * L), gbuf(t / (3 * L)) + 3 * N, gbuf(t / (3 * L)) + 6 * N, gT);
            __syncthreads();
            for (int t = threadIdx.x; t < ne * 3 * L; t += THREADS)
                geo_lines_z<N1, CENTER>(t % (3 * L), gbuf(t / (3 * L)) + 6 * N, gbuf(t / (3 * L)), gT);
            __syncthreads();
            for (int t = threadIdx.x; t < ne * 9 * L; t += THREADS)
                geo_lines_jacobian<N1, CENTER>(t % (9 * L), gbuf(t / (9 * L)), gbuf(t / (9 * L)) + 3 * N,
                                               gT + N1 * N1);
            __syncthreads();
            for (int t = threadIdx.x; t < ne * Q; t += THREADS) {
                const int el = t / Q, q = t % Q;
                float o[9], wdq;
                const double det =
                    geo_point_f32(gbuf(el) + 3 * N + q * 9, gT[2 * N1 * N1 + GEO_DQ_EXTRA + q], o, wdq);
                const int bad = geo_det_status(det);
                if (bad) fe_report(status, bad, e0 + el);
                const long long idx = (e0 + el) * Q + q;
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    geo.jinv_out[idx * 9 + k] = o[k];
                    sm[el * PE + P::JI + q * 9 + k] = o[k];
                }
                geo.wdetj_out[idx] = wdq;
                sm[el * PE + P::WD + q] = wdq;
            }
        }
        __syncthreads();
        // ---- 1x: line (el, c, k, j) -> X[c][0] = B_x U, X[c][1] = D_x U
        for (int t = threadIdx.x; t < ne * nf * N1 * N1; t += THREADS) {
            const int kj = t % (N1 * N1), c = (t / (N1 * N1)) % nf, el = t / (N1 * N1 * nf);
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
        // ---- 1y: line (el, c, k, qx) -> Y[c][0] = B_y B_x, Y[c][1] = D_y B_x, Y[c][2] = B_y D_x
        for (int t = threadIdx.x; t < ne * nf * N1 * NQ; t += THREADS) {
            const int qx = t % NQ, k = (t / NQ) % N1, c = (t / (NQ * N1)) % nf, el = t / (NQ * N1 * nf);
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
        // ---- 1z: line (el, c, qy, qx) -> PV[c][m][q]: d/dxi, d/deta, d/dzeta, value
        for (int t = threadIdx.x; t < ne * nf * NQ * NQ; t += THREADS) {
            const int qx = t % NQ, qy = (t / NQ) % NQ, c = (t / (NQ * NQ)) % nf, el = t / (NQ * NQ * nf);
            const T *Y = sm + el * PE + P::R1 + 12 * LX + c * 3 * LY;
            T *PV = sm + el * PE + P::R2 + c * 4 * Q;
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
                T gx = 0, gy = 0, gz = 0, v = 0;
#pragma unroll
                for (int k = 0; k < N1; ++k) {
                    gx = fma(B[qz][k], y2[k], gx);
                    gy = fma(B[qz][k], y1[k], gy);
                    gz = fma(D[qz][k], y0[k], gz);
                    v = fma(B[qz][k], y0[k], v);
                }
                PV[q] = gx;
                PV[Q + q] = gy;
                PV[2 * Q + q] = gz;
                PV[3 * Q + q] = v;
            }
        }
        __syncthreads();
        // ---- 2: pointwise physical gradient, advection and weights
        for (int t = threadIdx.x; t < ne * Q; t += THREADS) {
            const int el = t / Q, q = t % Q;
            const T *S = sm + el * PE;
            const T *Ji = S + P::JI + q * 9;
            const T wd = S[P::WD + q];
            const T *PV = S + P::R2;
            const int cw = same ? 0 : 3;
            T wv[3], H[3][3];
#pragma unroll
            for (int j = 0; j < 3; ++j) wv[j] = PV[((cw + j) * 4 + 3) * Q + q];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const T g0 = PV[(c * 4 + 0) * Q + q], g1 = PV[(c * 4 + 1) * Q + q], g2 = PV[(c * 4 + 2) * Q + q];
#pragma unroll
                for (int b = 0; b < 3; ++b) H[c][b] = wd * (g0 * Ji[b] + g1 * Ji[3 + b] + g2 * Ji[6 + b]);
            }
            T *W = sm + el * PE + P::WT;
            if constexpr (MAT) {
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int b = 0; b < 3; ++b) W[(c * 3 + b) * Q + q] = H[c][b];
#pragma unroll
                for (int m = 0; m < 3; ++m)
                    W[(9 + m) * Q + q] = wd * (Ji[m * 3] * wv[0] + Ji[m * 3 + 1] * wv[1] + Ji[m * 3 + 2] * wv[2]);
            } else {
#pragma unroll
                for (int c = 0; c < 3; ++c) W[c * Q + q] = H[c][0] * wv[0] + H[c][1] * wv[1] + H[c][2] * wv[2];
            }
        }
        __syncthreads();
        if constexpr (!MAT) {
            // ---- 3a: r[(c,k)] = sum_q phi_k F_c by the transposed contractions
            for (int t = threadIdx.x; t < ne * 3 * NQ * NQ; t += THREADS) {  // z^T
                const int qx = t % NQ, qy = (t / NQ) % NQ, c = (t / (NQ * NQ)) % 3, el = t / (NQ * NQ * 3);
                const T *F = sm + el * PE + P::WT + c * Q;
                T *Z = sm + el * PE + P::R1 + c * LY;
                T f[NQ];
#pragma unroll
                for (int qz = 0; qz < NQ; ++qz) f[qz] = F[(qz * NQ + qy) * NQ + qx];
#pragma unroll
                for (int kz = 0; kz < N1; ++kz) {
                    T v = 0;
#pragma unroll
                    for (int qz = 0; qz < NQ; ++qz) v = fma(B[qz][kz], f[qz], v);
                    Z[(kz * NQ + qy) * NQ + qx] = v;
                }
            }
            __syncthreads();
            for (int t = threadIdx.x; t < ne * 3 * N1 * NQ; t += THREADS) {  // y^T
                const int qx = t % NQ, kz = (t / NQ) % N1, c = (t / (NQ * N1)) % 3, el = t / (NQ * N1 * 3);
                const T *Z = sm + el * PE + P::R1 + c * LY;
                T *Yt = sm + el * PE + P::R1 + 3 * LY + c * LX;
                T z[NQ];
#pragma unroll
                for (int qy = 0; qy < NQ; ++qy) z[qy] = Z[(kz * NQ + qy) * NQ + qx];
#pragma unroll
                for (int ky = 0; ky < N1; ++ky) {
                    T v = 0;
#pragma unroll
                    for (int qy = 0; qy < NQ; ++qy) v = fma(B[qy][ky], z[qy], v);
                    Yt[(kz * N1 + ky) * NQ + qx] = v;
                }
            }
            __syncthreads();
            for (int t = threadIdx.x; t < ne * 3 * N1 * N1; t += THREADS) {  // x^T
                const int kzy = t % (N1 * N1), c = (t / (N1 * N1)) % 3, el = t / (N1 * N1 * 3);
                const T *Yt = sm + el * PE + P::R1 + 3 * LY + c * LX + kzy * NQ;
                T y[NQ];
#pragma unroll
                for (int qx = 0; qx < NQ; ++qx) y[qx] = Yt[qx];
                T *re = r + (e0 + el) * 3 * N + c * N + kzy * N1;
#pragma unroll
                for (int kx = 0; kx < N1; ++kx) {
                    T v = 0;
#pragma unroll
                    for (int qx = 0; qx < NQ; ++qx) v = fma(B[qx][kx], y[qx], v);
                    re[kx] = v;
                }
            }
        } else {
            // fields that enter the matrix: H_ab when differentiating w.r.t. w,
            // c_m when differentiating w.r.t. u
            const int f0 = wrt_adv ? 0 : 9, f1 = wrt_grad ? 12 : 9, nfl = f1 - f0;
            // ---- 3b step 1: T1[f][qx][qy][kz][lz] = sum_qz B[qz][kz] R[qz][lz] W_f
            for (int t = threadIdx.x; t < ne * nfl * NQ * NQ; t += THREADS) {
                const int qx = t % NQ, qy = (t / NQ) % NQ, f = f0 + (t / (NQ * NQ)) % nfl,
                          el = t / (NQ * NQ * nfl);
                const T *W = sm + el * PE + P::WT + f * Q;
                T *T1 = sm + el * PE + P::R1 + ((f * NQ + qx) * NQ + qy) * N1 * N1;
                const bool dz = f == 11;
                T bw[NQ][N1];
#pragma unroll
                for (int qz = 0; qz < NQ; ++qz) {
                    const T wq = W[(qz * NQ + qy) * NQ + qx];
#pragma unroll
                    for (int kz = 0; kz < N1; ++kz) bw[qz][kz] = B[qz][kz] * wq;
                }
#pragma unroll
                for (int kz = 0; kz < N1; ++kz)
#pragma unroll
                    for (int lz = 0; lz < N1; ++lz) {
                        T v = 0;
#pragma unroll
                        for (int qz = 0; qz < NQ; ++qz) v = fma(bw[qz][kz], dz ? D[qz][lz] : B[qz][lz], v);
                        T1[kz * N1 + lz] = v;
                    }
            }
            __syncthreads();
            // ---- step 2: T2[f][qx][ky][ly][kz][lz] = sum_qy B[qy][ky] R[qy][ly] T1[f][qx][qy][kz][lz];
            // output field 10 holds the sum of the fields 10 and 11 (each contracted, then added)
            const int fo1 = f1 == 12 ? 11 : f1, nfo = fo1 - f0;
            for (int t = threadIdx.x; t < ne * nfo * NQ * N1 * N1; t += THREADS) {
                const int kzlz = t % (N1 * N1), qx = (t / (N1 * N1)) % NQ, fo = f0 + (t / (N1 * N1 * NQ)) % nfo,
                          el = t / (N1 * N1 * NQ * nfo);
                T *T2 = sm + el * PE + P::R2 + fo * P::FS + qx * N1 * N1 * N1 * N1 + kzlz;
                T res[N1][N1];
                auto contract = [&](int f, bool first) {
                    const T *T1 = sm + el * PE + P::R1 + (f * NQ + qx) * NQ * N1 * N1 + kzlz;
                    const bool dy = f == 10;
                    T bt[NQ][N1];
#pragma unroll
                    for (int qy = 0; qy < NQ; ++qy) {
                        const T tq = T1[qy * N1 * N1];
#pragma unroll
                        for (int ky = 0; ky < N1; ++ky) bt[qy][ky] = B[qy][ky] * tq;
                    }
#pragma unroll
                    for (int ky = 0; ky < N1; ++ky)
#pragma unroll
                        for (int ly = 0; ly < N1; ++ly) {
                            T v = 0;
#pragma unroll
                            for (int qy = 0; qy < NQ; ++qy) v = fma(bt[qy][ky], dy ? D[qy][ly] : B[qy][ly], v);
                            res[ky][ly] = first ? v : res[ky][ly] + v;
                        }
                };
                contract(fo, true);
                if (fo == 10) contract(11, false);
#pragma unroll
                for (int ky = 0; ky < N1; ++ky)
#pragma unroll
                    for (int ly = 0; ly < N1; ++ly) T2[(ky * N1 + ly) * N1 * N1] = res[ky][ly];
            }
            __syncthreads();
            // ---- step 3: one thread per column (b, l); rows (a, k) in order
            for (int t = threadIdx.x; t < ne * 3 * N; t += THREADS) {
                const int col = t % (3 * N), el = t / (3 * N);
                const int b = col / N, l = col % N;
                const int lx = l % N1, ly = (l / N1) % N1, lz = l / (N1 * N1);
                T Bl[NQ], Dl[NQ];
#pragma unroll
                for (int qx = 0; qx < NQ; ++qx) {
                    Bl[qx] = B[qx][0];
                    Dl[qx] = D[qx][0];
#pragma unroll
                    for (int i = 1; i < N1; ++i)
                        if (lx == i) {
                            Bl[qx] = B[qx][i];
                            Dl[qx] = D[qx][i];
                        }
                }
                const T *T2 = sm + el * PE + P::R2 + ly * N1 * N1 + lz;
                constexpr int FS = P::FS;                   // field stride
                constexpr int QS = N1 * N1 * N1 * N1;       // qx stride
                T *Ke = K + (e0 + el) * (long long)(9 * N * N) + col;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const int f = a * 3 + b;
                    const bool diag = a == b && wrt_grad;
#pragma unroll
                    for (int kz = 0; kz < N1; ++kz)
#pragma unroll
                        for (int ky = 0; ky < N1; ++ky) {
                            T mv[NQ];
#pragma unroll
                            for (int qx = 0; qx < NQ; ++qx) {
                                const int o = qx * QS + ky * N1 * N1 * N1 + kz * N1;
                                T v = 0;
                                if (wrt_adv) v = Bl[qx] * T2[f * FS + o];
                                if (diag) v += Bl[qx] * T2[10 * FS + o] + Dl[qx] * T2[9 * FS + o];  // c_y + c_z, c_x
                                mv[qx] = v;
                            }
#pragma unroll
                            for (int kx = 0; kx < N1; ++kx) {
                                T v = 0;
#pragma unroll
                                for (int qx = 0; qx < NQ; ++qx) v = fma(B[qx][kx], mv[qx], v);
                                Ke[(long long)(a * N + (kz * N1 + ky) * N1 + kx) * (3 * N)] = v;
                            }
                        }
                }
            }
        }
    }
}

template <typename T, int N1, int NQ, bool MAT, int EPB, int GEO = 0>
cudaError_t launch_cv(const fe_geometry_h *g, const void *u, const void *w, int wrt_grad, int wrt_adv, void *K,
                      void *r, unsigned long long *st, cudaStream_t s)
{
    using P = CvPlan<T, N1, NQ, MAT>;
    // residual computing the Q2 geometry: 7 elements in 6 warps (measured faster than 8 in 8 or 7)
    constexpr int THREADS = MAT ? ((EPB * 3 * P::N + 31) / 32) * 32 : (GEO > 0 && N1 == 3 ? 192 : 256);
    // per-element blocks, then (GEO) the FP64 tables 8-byte aligned
    constexpr size_t SMEM = sizeof(T) * (size_t)((P::PER_EL * EPB + 1) / 2 * 2) +
                            (GEO ? sizeof(double) * (2 * N1 * N1 + GEO_DQ_EXTRA + P::Q) : 0);
    static_assert(SMEM <= 227 * 1024, "shared memory plan too large");
    auto kern = k_convect_sf<T, N1, NQ, MAT, EPB, THREADS, GEO>;
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
    const int same = u == w;
    CvGeoArgs geo{};
    if (GEO) geo = CvGeoArgs{g->mesh.coords, g->d_b1d, g->d_dq, g->d_w64, g->d_jinv32, g->d_wdetj32};
    kern<<<(unsigned)blocks, THREADS, SMEM, s>>>(
        f64 ? (const T *)g->d_jinv64 : (const T *)g->d_jinv32, f64 ? (const T *)g->d_wdetj64 : (const T *)g->d_wdetj32,
        f64 ? (const T *)g->d_b1d : (const T *)g->d_b1d32, f64 ? (const T *)g->d_d1d : (const T *)g->d_d1d32,
        g->mesh.conn, E, (const T *)u, (const T *)w, same, wrt_grad, wrt_adv, (T *)K, (T *)r, g->mesh.n_nodes, st,
        geo);
    return cudaGetLastError();
}

// Elements per CTA: the matrix kernel keeps one thread per column of an element
// matrix; both plans keep a few CTAs resident per SM.
template <typename T>
cudaError_t dispatch_cv(const fe_geometry_h *g, const void *u, const void *w, int wg, int wa, void *K, void *r,
                        unsigned long long *st, cudaStream_t s)
{
    const int n1 = g->n1d, nq = g->nq1d;
    constexpr bool D = sizeof(T) == 8;
    if (K) {
        if (n1 == 2 && nq == 2) return launch_cv<T, 2, 2, true, 8>(g, u, w, wg, wa, K, r, st, s);
        if (n1 == 2 && nq == 3) return launch_cv<T, 2, 3, true, (D ? 4 : 6)>(g, u, w, wg, wa, K, r, st, s);
        if (n1 == 3 && nq == 3) return launch_cv<T, 3, 3, true, (D ? 2 : 3)>(g, u, w, wg, wa, K, r, st, s);
        if (n1 == 3 && nq == 4) return launch_cv<T, 3, 4, true, (D ? 1 : 2)>(g, u, w, wg, wa, K, r, st, s);
        if (n1 == 4 && nq == 4) return launch_cv<T, 4, 4, true, 1>(g, u, w, wg, wa, K, r, st, s);
    } else {
        if (n1 == 2 && nq == 2) return launch_cv<T, 2, 2, false, 8>(g, u, w, wg, wa, K, r, st, s);
        if (n1 == 2 && nq == 3) return launch_cv<T, 2, 3, false, 4>(g, u, w, wg, wa, K, r, st, s);
        if (n1 == 3 && nq == 3) return launch_cv<T, 3, 3, false, (D ? 4 : 8)>(g, u, w, wg, wa, K, r, st, s);
        if (n1 == 3 && nq == 4) return launch_cv<T, 3, 4, false, (D ? 2 : 4)>(g, u, w, wg, wa, K, r, st, s);
        if (n1 == 4 && nq == 4) return launch_cv<T, 4, 4, false, (D ? 1 : 2)>(g, u, w, wg, wa, K, r, st, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

bool fe_convect_supported(const fe_geometry_h *g)
{
    if (!g->d_b1d) return false;
    const int n1 = g->n1d, nq = g->nq1d;
    return (n1 == 2 && (nq == 2 || nq == 3)) || (n1 == 3 && (nq == 3 || nq == 4)) || (n1 == 4 && nq == 4);
}

cudaError_t fe_launch_convect(const fe_geometry_h *g, bool f64, const void *u, const void *w, int wrt_grad,
                              int wrt_adv, void *K, void *r, unsigned long long *status, cudaStream_t s)
{
    if (g->mesh.n_elems == 0) return cudaSuccess;
    return f64 ? dispatch_cv<double>(g, u, w, wrt_grad, wrt_adv, K, r, status, s)
               : dispatch_cv<float>(g, u, w, wrt_grad, wrt_adv, K, r, status, s);
}

bool fe_convect_geometry_fusable(const fe_geometry_h *g)
{
    return g->d_dq && g->d_jinv32 && !g->is_view && (g->flags & FE_GEOM_STORE_F32) &&
           !(g->flags & FE_GEOM_STORE_F64) && g->n1d == g->nq1d && g->n1d >= 2 && g->n1d <= 4;
}

cudaError_t fe_launch_convect_residual_geometry(const fe_geometry_h *g, const void *u, const void *w, void *r,
                                                unsigned long long *status, cudaStream_t s)
{
    if (!fe_convect_geometry_fusable(g)) return cudaErrorNotSupported;
    if (g->mesh.n_elems == 0) return cudaSuccess;
    switch (g->n1d) {
    case 2: return launch_cv<float, 2, 2, false, 8, 1>(g, u, w, 0, 0, nullptr, r, status, s);
    case 3:
        return g->geo_center ? launch_cv<float, 3, 3, false, 7, 2>(g, u, w, 0, 0, nullptr, r, status, s)
                             : launch_cv<float, 3, 3, false, 7, 1>(g, u, w, 0, 0, nullptr, r, status, s);
    case 4: return launch_cv<float, 4, 4, false, 2, 1>(g, u, w, 0, 0, nullptr, r, status, s);
    }
    return cudaErrorNotSupported;
}

cudaError_t fe_launch_convect_matrix_geometry(const fe_geometry_h *g, const void *u, const void *w, int wrt_grad,
                                              int wrt_adv, void *K, unsigned long long *status, cudaStream_t s)
{
    if (!fe_convect_geometry_fusable(g)) return cudaErrorNotSupported;
    if (g->mesh.n_elems == 0) return cudaSuccess;
    switch (g->n1d) {
    case 2: return launch_cv<float, 2, 2, true, 8, 1>(g, u, w, wrt_grad, wrt_adv, K, nullptr, status, s);
    case 3:  // two elements per CTA, six CTAs per SM (measured 2.22 against 2.25 ms with three at 64^3)
        return g->geo_center ? launch_cv<float, 3, 3, true, 2, 2>(g, u, w, wrt_grad, wrt_adv, K, nullptr, status, s)
                             : launch_cv<float, 3, 3, true, 2, 1>(g, u, w, wrt_grad, wrt_adv, K, nullptr, status, s);
    case 4: return launch_cv<float, 4, 4, true, 1, 1>(g, u, w, wrt_grad, wrt_adv, K, nullptr, status, s);
    }
    return cudaErrorNotSupported;
}
