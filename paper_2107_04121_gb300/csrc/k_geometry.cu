// Geometry of the isoparametric reference mapping (Sec. 4.1 of Cimrman,
// arXiv 2107.04121): J_ik = sum_a x_a,i d phi_a / d xi_k, det J, J^-1 and
// w_q det J for every element and quadrature point, in FP64.
//
// The kernels are FP64-pipe bound on GB300 (FP64 runs at 1/61 of the FP32
// rate there), so what matters is the FP64 operation count:
//  - k_geometry_co (tensor-product bases with n1 == nq): x interpolated to
//    the points, then the collocation derivative on the points (1,134 DFMA
//    per Q2 element with 3x3x3 Gauss points, instead of 6,561 directly);
//  - k_geometry_sf (tensor-product bases with n1 != nq, or when the collocation
//    derivative cannot be formed): three 1-D contractions per coordinate and
//    derivative direction;
//  - k_geometry (any tabulated basis, e.g. tetrahedra): one thread per
//    (element, quadrature point), J = sum_a x_a (x) grad phi_a directly (9N
//    DFMA per point);
//  - k_geometry_simplex (the library's tetrahedron basis, float32-only
//    handles): J of a straight-sided element from its vertices, once.
// All finish each point with the same cofactor inverse (9 cofactors and det J:
// 21 FP64 operations), whose float32 rounding uses integer operations
// (geometry_body.cuh).
#include "geometry_body.cuh"

namespace {

constexpr int kGeomThreads = 256;

// det J, J^-1 = adj(J) / det J and w det J at one quadrature point; stores the
// float64 and/or float32 copies.  J[c][m] = d x_c / d xi_m.
__device__ __forceinline__ void finish_point(const double J[3][3], double wq, long long e, long long idx,
                                             double *__restrict__ jinv64, double *__restrict__ wdetj64,
                                             float *__restrict__ jinv32, float *__restrict__ wdetj32,
                                             unsigned long long *__restrict__ status)
{
    const double *Jf = &J[0][0];
    if (!jinv64) {
        // only the float32 copy is kept: J, det J and the cofactors are FP64 (they
        // carry the cancellation of distorted elements), the quotient that is
        // stored in float32 is formed in float32 (a few float32 ulps instead of
        // one; it saves the FP64 reciprocal and 10 FP64 multiplies per point)
        float o[9], wd;
        const double det = geo_point_f32(Jf, wq, o, wd);
        const int bad = geo_det_status(det);
        if (bad) fe_report(status, bad, e);
#pragma unroll
        for (int k = 0; k < 9; ++k) jinv32[idx * 9 + k] = o[k];
        wdetj32[idx] = wd;
        return;
    }
    double C[9];  // C[r][k]: J^-1[k][r] = C[r][k] / det J
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) C[r * 3 + k] = geo_cofactor(Jf, r, k);
    const double det = geo_det(Jf, C[0], C[1], C[2]);
    const int bad = geo_det_status(det);
    if (bad) fe_report(status, bad, e);
    const double rr = 1.0 / det;
    double inv[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) inv[k * 3 + r] = __dmul_rn(C[r * 3 + k], rr);
    const double wd = __dmul_rn(wq, det);
    double *o = jinv64 + idx * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k) o[k] = inv[k];
    wdetj64[idx] = wd;
    if (jinv32) {
        float *o32 = jinv32 + idx * 9;
#pragma unroll
        for (int k = 0; k < 9; ++k) o32[k] = (float)inv[k];
        wdetj32[idx] = (float)wd;
    }
}

// Sum-factorised geometry of tensor-product hexahedra: n1 nodes and nq points
// per axis, b1d/d1d the 1-D basis values and derivatives (nq, n1).  Per element
// and coordinate c, with X[k][j][i] the nodal values:
//   U0 = B_x X, U1 = D_x X                          (contract i)
//   V_DB = B_y U1, V_BD = D_y U0, V_BB = B_y U0     (contract j)
//   J[c][0] = B_z V_DB, J[c][1] = B_z V_BD, J[c][2] = D_z V_BB   (contract k)
template <int N1, int NQ, int EPB>
__global__ void __launch_bounds__(kGeomThreads) k_geometry_sf(const double *__restrict__ coords,
                                                              const int32_t *__restrict__ conn, long long E,
                                                              long long n_nodes, const double *__restrict__ b1d,
                                                              const double *__restrict__ d1d,
                                                              const double *__restrict__ w,
                                                              double *__restrict__ jinv64, double *__restrict__ wdetj64,
                                                              float *__restrict__ jinv32, float *__restrict__ wdetj32,
                                                              unsigned long long *__restrict__ status)
{
    constexpr int N = N1 * N1 * N1, Q = NQ * NQ * NQ;
    static_assert(8 * (2 * NQ * N1 + EPB * (3 * N + 6 * N1 * N1 * NQ + 9 * N1 * NQ * NQ + 9 * Q)) <= 48 * 1024,
                  "static shared memory above 48 KB");
    __shared__ double sB[NQ][N1], sD[NQ][N1];
    __shared__ double sX[EPB][3][N];              // [k][j][i]
    __shared__ double sU[EPB][2][3][N1][N1][NQ];  // [k][j][qx]
    __shared__ double sV[EPB][3][3][N1][NQ][NQ];  // [which][c][k][qy][qx]
    __shared__ double sJ[EPB][Q][9];
    for (int i = threadIdx.x; i < NQ * N1; i += blockDim.x) {
        sB[i / N1][i % N1] = b1d[i];
        sD[i / N1][i % N1] = d1d[i];
    }
    for (long long e0 = (long long)blockIdx.x * EPB; e0 < E; e0 += (long long)gridDim.x * EPB) {
        const int ne = (int)((E - e0) < EPB ? (E - e0) : EPB);
        __syncthreads();
        for (int t = threadIdx.x; t < ne * N; t += blockDim.x) {
            const int el = t / N, a = t % N;
            long long node = conn[(e0 + el) * N + a];
            if ((unsigned long long)node >= (unsigned long long)n_nodes) {  // never read outside coords
                fe_report(status, FE_ERR_SHAPE, e0 + el);
                node = 0;
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) sX[el][c][a] = coords[3 * node + c];
        }
        __syncthreads();
        for (int t = threadIdx.x; t < ne * 3 * N1 * N1 * NQ; t += blockDim.x) {
            const int qx = t % NQ, j = (t / NQ) % N1, k = (t / (NQ * N1)) % N1, c = (t / (NQ * N1 * N1)) % 3,
                      el = t / (NQ * N1 * N1 * 3);
            const double *x = &sX[el][c][(k * N1 + j) * N1];
            double u0 = 0.0, u1 = 0.0;
#pragma unroll
            for (int i = 0; i < N1; ++i) {
                u0 = fma(sB[qx][i], x[i], u0);
                u1 = fma(sD[qx][i], x[i], u1);
            }
            sU[el][0][c][k][j][qx] = u0;
            sU[el][1][c][k][j][qx] = u1;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < ne * 3 * N1 * NQ * NQ; t += blockDim.x) {
            const int qx = t % NQ, qy = (t / NQ) % NQ, k = (t / (NQ * NQ)) % N1, c = (t / (NQ * NQ * N1)) % 3,
                      el = t / (NQ * NQ * N1 * 3);
            double vdb = 0.0, vbd = 0.0, vbb = 0.0;
#pragma unroll
            for (int j = 0; j < N1; ++j) {
                const double u0 = sU[el][0][c][k][j][qx], u1 = sU[el][1][c][k][j][qx];
                vdb = fma(sB[qy][j], u1, vdb);
                vbd = fma(sD[qy][j], u0, vbd);
                vbb = fma(sB[qy][j], u0, vbb);
            }
            sV[el][0][c][k][qy][qx] = vdb;
            sV[el][1][c][k][qy][qx] = vbd;
            sV[el][2][c][k][qy][qx] = vbb;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < ne * 3 * Q; t += blockDim.x) {
            const int qx = t % NQ, qy = (t / NQ) % NQ, qz = (t / (NQ * NQ)) % NQ, c = (t / Q) % 3, el = t / (3 * Q);
            double j0 = 0.0, j1 = 0.0, j2 = 0.0;
#pragma unroll
            for (int k = 0; k < N1; ++k) {
                j0 = fma(sB[qz][k], sV[el][0][c][k][qy][qx], j0);
                j1 = fma(sB[qz][k], sV[el][1][c][k][qy][qx], j1);
                j2 = fma(sD[qz][k], sV[el][2][c][k][qy][qx], j2);
            }
            double *Jo = sJ[el][qx + NQ * (qy + NQ * qz)] + c * 3;
            Jo[0] = j0;
            Jo[1] = j1;
            Jo[2] = j2;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < ne * Q; t += blockDim.x) {
            const int el = t / Q, q = t % Q;
            double J[3][3];
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int m = 0; m < 3; ++m) J[c][m] = sJ[el][q][c * 3 + m];
            finish_point(J, w[q], e0 + el, (e0 + el) * Q + q, jinv64, wdetj64, jinv32, wdetj32, status);
        }
    }
}

// Collocation form of the sum-factorised geometry, for n1 == nq: along one
// axis the nq Gauss points fix a polynomial of degree n1 - 1, so the derivative
// at the points is Dq (point values), Dq = D B^-1 (nq x nq).  Per element:
//   P = B_z B_y B_x X       (x at the points: three 1-D contractions)
//   J[c][m] = Dq along axis m of P[c]
// one 1-D line per item (geometry_body.cuh); for Q2 1,458 DFMA per element, or
// 1,134 when the middle Gauss point is the middle node (CENTER).  Per element
// the shared buffer holds X (then P), U, V and J (9 N doubles over U, V and a
// fourth block).
template <int N1, int EPB, bool CENTER>
__global__ void __launch_bounds__(kGeomThreads) k_geometry_co(const double *__restrict__ coords,
                                                              const int32_t *__restrict__ conn, long long E,
                                                              long long n_nodes, const double *__restrict__ b1d,
                                                              const double *__restrict__ dq,
                                                              const double *__restrict__ w,
                                                              double *__restrict__ jinv64, double *__restrict__ wdetj64,
                                                              float *__restrict__ jinv32, float *__restrict__ wdetj32,
                                                              unsigned long long *__restrict__ status)
{
    constexpr int N = N1 * N1 * N1, L = N1 * N1;
    static_assert(8 * (2 * N1 * N1 + GEO_DQ_EXTRA + EPB * 12 * N) <= 48 * 1024, "static shared memory above 48 KB");
    __shared__ double sB[N1 * N1], sDq[N1 * N1 + GEO_DQ_EXTRA];
    __shared__ double sG[EPB][4][3 * N];
    for (int i = threadIdx.x; i < N1 * N1 + GEO_DQ_EXTRA; i += blockDim.x) {
        if (i < N1 * N1) sB[i] = b1d[i];
        sDq[i] = dq[i];
    }
    for (long long e0 = (long long)blockIdx.x * EPB; e0 < E; e0 += (long long)gridDim.x * EPB) {
        const int ne = (int)((E - e0) < EPB ? (E - e0) : EPB);
        __syncthreads();
        for (int t = threadIdx.x; t < ne * N; t += blockDim.x) {
            const int el = t / N, a = t % N;
            long long node = conn[(e0 + el) * N + a];
            if ((unsigned long long)node >= (unsigned long long)n_nodes) {  // never read outside coords
                fe_report(status, FE_ERR_SHAPE, e0 + el);
                node = 0;
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) sG[el][0][c * N + a] = coords[3 * node + c];
        }
        __syncthreads();
        for (int t = threadIdx.x; t < ne * 3 * L; t += blockDim.x)  // contract i
            geo_lines_x<N1, CENTER>(t % (3 * L), sG[t / (3 * L)][0], sG[t / (3 * L)][1], sB);
        __syncthreads();
        for (int t = threadIdx.x; t < ne * 3 * L; t += blockDim.x)  // contract j
            geo_lines_y<N1, CENTER>(t % (3 * L), sG[t / (3 * L)][1], sG[t / (3 * L)][2], sB);
        __syncthreads();
        for (int t = threadIdx.x; t < ne * 3 * L; t += blockDim.x)  // contract k: x at the points
            geo_lines_z<N1, CENTER>(t % (3 * L), sG[t / (3 * L)][2], sG[t / (3 * L)][0], sB);
        __syncthreads();
        for (int t = threadIdx.x; t < ne * 9 * L; t += blockDim.x)  // J on the points
            geo_lines_jacobian<N1, CENTER>(t % (9 * L), sG[t / (9 * L)][0], sG[t / (9 * L)][1], sDq);
        __syncthreads();
        for (int t = threadIdx.x; t < ne * N; t += blockDim.x) {
            const int el = t / N, q = t % N;
            finish_point(reinterpret_cast<const double(*)[3]>(sG[el][1] + q * 9), w[q], e0 + el, (e0 + el) * N + q,
                         jinv64, wdetj64, jinv32, wdetj32, status);
        }
    }
}

template <int N>
__global__ void __launch_bounds__(kGeomThreads) k_geometry(const double *__restrict__ coords,
                                                           const int32_t *__restrict__ conn, long long E,
                                                           long long n_nodes, int Q,
                                                           const double *__restrict__ dphi,
                                                           const double *__restrict__ w, double *__restrict__ jinv64,
                                                           double *__restrict__ wdetj64, float *__restrict__ jinv32,
                                                           float *__restrict__ wdetj32,
                                                           unsigned long long *__restrict__ status)
{
    extern __shared__ double s_dphi[];  // (Q, 3, N)
    for (int i = threadIdx.x; i < Q * 3 * N; i += blockDim.x) s_dphi[i] = dphi[i];
    __syncthreads();
    const long long total = E * Q;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long e = idx / Q;
        const int q = (int)(idx - e * Q);
        const int32_t *ce = conn + e * N;
        const double *d0 = s_dphi + (q * 3 + 0) * N;
        const double *d1 = d0 + N;
        const double *d2 = d1 + N;
        double J00 = 0, J01 = 0, J02 = 0, J10 = 0, J11 = 0, J12 = 0, J20 = 0, J21 = 0, J22 = 0;
#pragma unroll 9
        for (int a = 0; a < N; ++a) {
            long long node = __ldg(ce + a);
            if ((unsigned long long)node >= (unsigned long long)n_nodes) {  // never read outside coords
                fe_report(status, FE_ERR_SHAPE, e);
                node = 0;
            }
            const double x0 = __ldg(coords + 3 * node), x1 = __ldg(coords + 3 * node + 1),
                         x2 = __ldg(coords + 3 * node + 2);
            const double g0 = d0[a], g1 = d1[a], g2 = d2[a];
            J00 = fma(x0, g0, J00);
            J01 = fma(x0, g1, J01);
            J02 = fma(x0, g2, J02);
            J10 = fma(x1, g0, J10);
            J11 = fma(x1, g1, J11);
            J12 = fma(x1, g2, J12);
            J20 = fma(x2, g0, J20);
            J21 = fma(x2, g1, J21);
            J22 = fma(x2, g2, J22);
        }
        const double J[3][3] = {{J00, J01, J02}, {J10, J11, J12}, {J20, J21, J22}};
        finish_point(J, w[q], e, idx, jinv64, wdetj64, jinv32, wdetj32, status);
    }
}

// Tetrahedra of the library's order-p basis, float32-only handles: one thread
// per element.  When every node lies on the affine image of its lattice point
// (x_a = x_0 + J xi_a to 1e-12 of the element's size: straight edges and faces)
// J is the constant [x_1 - x_0, x_2 - x_0, x_3 - x_0] of the vertices and the
// inverse is formed once (21 FP64 operations per element instead of 9N + 21 per
// point); the warp then writes the Q copies of such elements together, one
// element at a time, with consecutive lanes on consecutive floats.  Elements
// with bent edges take the point loop of k_geometry.  Same float32 roundings.
template <int N>
__global__ void __launch_bounds__(kGeomThreads) k_geometry_simplex(
    const double *__restrict__ coords, const int32_t *__restrict__ conn, long long E, long long n_nodes, int Q,
    const double *__restrict__ dphi, const double *__restrict__ w, const double *__restrict__ xi, int p,
    float *__restrict__ jinv32, float *__restrict__ wdetj32, unsigned long long *__restrict__ status)
{
    // local indices of the vertices (0,0,0), (p,0,0), (0,p,0), (0,0,p) in the lattice order
    const int v1 = p, v2 = (p + 1) * (p + 2) / 2 - 1, v3 = N - 1;
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    // warp-uniform loop: the 32 lanes take 32 consecutive elements
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < E; base += stride) {
        const long long e = base + lane;
        const bool live = e < E;
        bool straight = false;
        float o[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, df = 0.f;
        if (live) {
            const int32_t *ce = conn + e * N;
            auto node_xyz = [&](int a, double x[3]) {
                long long node = __ldg(ce + a);
                if ((unsigned long long)node >= (unsigned long long)n_nodes) {  // never read outside coords
                    fe_report(status, FE_ERR_SHAPE, e);
                    node = 0;
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) x[c] = __ldg(coords + 3 * node + c);
            };
            double x0[3], xv[3][3];
            node_xyz(0, x0);
            node_xyz(v1, xv[0]);
            node_xyz(v2, xv[1]);
            node_xyz(v3, xv[2]);
            double J[3][3];
            double size = 0.0;
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    J[c][m] = __dsub_rn(xv[m][c], x0[c]);
                    size = fmax(size, fabs(J[c][m]));
                }
            // every node checked (no early exit), so that the node loads of all edges and
            // faces are in flight together
            straight = true;
#pragma unroll
            for (int a = 1; a < N; ++a) {
                if (a == v1 || a == v2 || a == v3) continue;
                double x[3];
                node_xyz(a, x);
                const double *xa = xi + 3 * a;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const double pred =
                        fma(J[c][2], __ldg(xa + 2), fma(J[c][1], __ldg(xa + 1), fma(J[c][0], __ldg(xa), x0[c])));
                    if (!(fabs(x[c] - pred) <= 1e-12 * size)) straight = false;
                }
            }
            if (straight) {
                float wd0;
                const double det = geo_point_f32(&J[0][0], __ldg(w), o, wd0);
                const int bad = geo_det_status(det);
                if (bad) fe_report(status, bad, e);
                df = geo_to_f32(det);
            } else {
                for (int q = 0; q < Q; ++q) {
                    const double *d0 = dphi + (size_t)(q * 3) * N;
                    double Jq[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
                    for (int a = 0; a < N; ++a) {
                        double x[3];
                        node_xyz(a, x);
                        const double g0 = __ldg(d0 + a), g1 = __ldg(d0 + N + a), g2 = __ldg(d0 + 2 * N + a);
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            Jq[c][0] = fma(x[c], g0, Jq[c][0]);
                            Jq[c][1] = fma(x[c], g1, Jq[c][1]);
                            Jq[c][2] = fma(x[c], g2, Jq[c][2]);
                        }
                    }
                    finish_point(Jq, __ldg(w + q), e, e * Q + q, nullptr, nullptr, jinv32, wdetj32, status);
                }
            }
        }
        // the straight elements' Q copies of J^-1 and w det J = fl(w_q) fl(det J), written
        // by the whole warp element by element (each element's block is contiguous)
        unsigned todo = __ballot_sync(0xffffffffu, live && straight);
        while (todo) {
            const int l = __ffs(todo) - 1;
            todo &= todo - 1;
            float ol[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) ol[k] = __shfl_sync(0xffffffffu, o[k], l);
            const float dl = __shfl_sync(0xffffffffu, df, l);
            const long long el = base + l;
            float *jo = jinv32 + el * Q * 9;
            for (int i = lane; i < Q * 9; i += 32) jo[i] = ol[i % 9];
            for (int i = lane; i < Q; i += 32) wdetj32[el * Q + i] = __fmul_rn(geo_to_f32(__ldg(w + i)), dl);
        }
    }
}

// G[e][q][j][a] = sum_k dphi[q][k][a] (J^-1)_kj from a stored J^-1 copy.
template <typename T>
__global__ void k_expand_G(const T *__restrict__ jinv, const T *__restrict__ dphi, long long E, int Q, int N,
                           T *__restrict__ G)
{
    const long long total = E * Q * 3 * N;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(idx % N);
        const int j = (int)((idx / N) % 3);
        const long long eq = idx / (3 * N);
        const int q = (int)(eq % Q);
        const T *Ji = jinv + eq * 9;
        T s = 0;
        for (int k = 0; k < 3; ++k) s += dphi[(q * 3 + k) * N + a] * Ji[k * 3 + j];
        G[idx] = s;
    }
}

template <int N>
cudaError_t launch_geom(const fe_geometry_h *g, unsigned long long *st, cudaStream_t s)
{
    const size_t smem = (size_t)g->Q * 3 * N * sizeof(double);
    if (smem > 48 * 1024) {
        static FeLaunchCache cache;
        long long unused = 0;
        cudaError_t err = fe_cached_grid(
            cache,
            [&](int, long long *v) {
                *v = 1;
                // the largest table any (N, Q) pair of this instantiation needs
                return cudaFuncSetAttribute(k_geometry<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            64 * 3 * N * (int)sizeof(double));
            },
            &unused);
        if (err != cudaSuccess) return err;
    }
    const long long total = g->mesh.n_elems * g->Q;
    long long blocks = (total + kGeomThreads - 1) / kGeomThreads;
    if (blocks > (1ll << 30)) blocks = 1ll << 30;
    if (blocks < 1) blocks = 1;
    const bool f64 = g->flags & FE_GEOM_STORE_F64, f32 = g->flags & FE_GEOM_STORE_F32;
    k_geometry<N><<<(unsigned)blocks, kGeomThreads, smem, s>>>(
        g->mesh.coords, g->mesh.conn, g->mesh.n_elems, g->mesh.n_nodes, g->Q, g->d_dphi64, g->d_w64, f64 ? g->d_jinv64 : nullptr,
        f64 ? g->d_wdetj64 : nullptr, f32 ? g->d_jinv32 : nullptr, f32 ? g->d_wdetj32 : nullptr, st);
    return cudaGetLastError();
}

template <int N>
cudaError_t launch_geom_simplex(const fe_geometry_h *g, unsigned long long *st, cudaStream_t s)
{
    long long blocks = (g->mesh.n_elems + kGeomThreads - 1) / kGeomThreads;
    if (blocks > (1ll << 30)) blocks = 1ll << 30;
    k_geometry_simplex<N><<<(unsigned)blocks, kGeomThreads, 0, s>>>(
        g->mesh.coords, g->mesh.conn, g->mesh.n_elems, g->mesh.n_nodes, g->Q, g->d_dphi64, g->d_w64, g->d_xi,
        g->simplex_p, g->d_jinv32, g->d_wdetj32, st);
    return cudaGetLastError();
}

template <int N1, int NQ, int EPB>
cudaError_t launch_geom_sf(const fe_geometry_h *g, unsigned long long *st, cudaStream_t s)
{
    static FeLaunchCache cache;
    long long cap = 0;
    cudaError_t err = fe_cached_grid(
        cache,
        [&](int dev, long long *v) {
            int sms = 0, per_sm = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaError_t e2 =
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_geometry_sf<N1, NQ, EPB>, kGeomThreads, 0);
            if (e2 != cudaSuccess) return e2;
            if (per_sm < 1) return cudaErrorInvalidConfiguration;
            *v = (long long)per_sm * sms * 8;
            return cudaSuccess;
        },
        &cap);
    if (err != cudaSuccess) return err;
    long long blocks = (g->mesh.n_elems + EPB - 1) / EPB;
    if (blocks > cap) blocks = cap;
    const bool f64 = g->flags & FE_GEOM_STORE_F64, f32 = g->flags & FE_GEOM_STORE_F32;
    k_geometry_sf<N1, NQ, EPB><<<(unsigned)blocks, kGeomThreads, 0, s>>>(
        g->mesh.coords, g->mesh.conn, g->mesh.n_elems, g->mesh.n_nodes, g->d_b1d, g->d_d1d, g->d_w64,
        f64 ? g->d_jinv64 : nullptr, f64 ? g->d_wdetj64 : nullptr, f32 ? g->d_jinv32 : nullptr,
        f32 ? g->d_wdetj32 : nullptr, st);
    return cudaGetLastError();
}

template <int N1, int EPB, bool CENTER = false>
cudaError_t launch_geom_co(const fe_geometry_h *g, unsigned long long *st, cudaStream_t s)
{
    // Q2: 7 elements in 6 warps (measured faster than 9 in 8, 8 in 7 and 4 in 4)
    constexpr int threads = N1 == 3 ? 192 : kGeomThreads;
    static FeLaunchCache cache;
    long long cap = 0;
    cudaError_t err = fe_cached_grid(
        cache,
        [&](int dev, long long *v) {
            int sms = 0, per_sm = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaError_t e2 =
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_geometry_co<N1, EPB, CENTER>, threads, 0);
            if (e2 != cudaSuccess) return e2;
            if (per_sm < 1) return cudaErrorInvalidConfiguration;
            *v = (long long)per_sm * sms * 8;
            return cudaSuccess;
        },
        &cap);
    if (err != cudaSuccess) return err;
    long long blocks = (g->mesh.n_elems + EPB - 1) / EPB;
    if (blocks > cap) blocks = cap;
    const bool f64 = g->flags & FE_GEOM_STORE_F64, f32 = g->flags & FE_GEOM_STORE_F32;
    k_geometry_co<N1, EPB, CENTER><<<(unsigned)blocks, threads, 0, s>>>(
        g->mesh.coords, g->mesh.conn, g->mesh.n_elems, g->mesh.n_nodes, g->d_b1d, g->d_dq, g->d_w64,
        f64 ? g->d_jinv64 : nullptr, f64 ? g->d_wdetj64 : nullptr, f32 ? g->d_jinv32 : nullptr,
        f32 ? g->d_wdetj32 : nullptr, st);
    return cudaGetLastError();
}

__global__ void k_round_f32(const double *__restrict__ in, float *__restrict__ out, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = geo_to_f32(in[i]);
}

}  // namespace

cudaError_t fe_launch_geometry(const fe_geometry_h *g, unsigned long long *st, cudaStream_t s)
{
    if (g->mesh.n_elems == 0) return cudaSuccess;
    if (g->d_b1d) {
        const int n1 = g->n1d, nq = g->nq1d;
        if (g->d_dq && n1 == nq) {
            if (n1 == 2) return launch_geom_co<2, 32>(g, st, s);
            if (n1 == 3) return g->geo_center ? launch_geom_co<3, 7, true>(g, st, s) : launch_geom_co<3, 7>(g, st, s);
            if (n1 == 4) return launch_geom_co<4, 4>(g, st, s);
        }
        if (n1 == 2 && nq == 2) return launch_geom_sf<2, 2, 16>(g, st, s);
        if (n1 == 2 && nq == 3) return launch_geom_sf<2, 3, 8>(g, st, s);
        if (n1 == 3 && nq == 3) return launch_geom_sf<3, 3, 8>(g, st, s);
        if (n1 == 3 && nq == 4) return launch_geom_sf<3, 4, 4>(g, st, s);
        if (n1 == 4 && nq == 4) return launch_geom_sf<4, 4, 2>(g, st, s);
    }
    if (g->simplex_p && g->d_xi && g->d_jinv32 && !g->d_jinv64) {
        switch (g->N) {
        case 4: return launch_geom_simplex<4>(g, st, s);
        case 10: return launch_geom_simplex<10>(g, st, s);
        case 20: return launch_geom_simplex<20>(g, st, s);
        default: break;
        }
    }
    switch (g->N) {
    case 8: return launch_geom<8>(g, st, s);
    case 27: return launch_geom<27>(g, st, s);
    case 64: return launch_geom<64>(g, st, s);
    case 4: return launch_geom<4>(g, st, s);
    case 10: return launch_geom<10>(g, st, s);
    case 20: return launch_geom<20>(g, st, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t fe_launch_geometry_G(const fe_geometry_h *g, bool f64, void *out, cudaStream_t s)
{
    const long long total = g->mesh.n_elems * g->Q * 3 * g->N;
    if (total == 0) return cudaSuccess;
    long long blocks = (total + 255) / 256;
    if (blocks > 1048576) blocks = 1048576;
    if (f64)
        k_expand_G<double><<<(unsigned)blocks, 256, 0, s>>>(g->d_jinv64, g->d_dphi64, g->mesh.n_elems, g->Q, g->N,
                                                            (double *)out);
    else
        k_expand_G<float><<<(unsigned)blocks, 256, 0, s>>>(g->d_jinv32, g->d_dphi32, g->mesh.n_elems, g->Q, g->N,
                                                           (float *)out);
    return cudaGetLastError();
}

cudaError_t fe_launch_round_f32(const double *in, float *out, long long n, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > 65536) blocks = 65536;
    k_round_f32<<<(unsigned)blocks, 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}
