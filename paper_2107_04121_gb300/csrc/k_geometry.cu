// Geometry of the isoparametric reference mapping (Sec. 4.1 of Cimrman,
// arXiv 2107.04121): J_ik = sum_a x_a,i d phi_a / d xi_k, det J, J^-1 and
// w_q det J for every element and quadrature point, in FP64.
//
// One thread per (element, quadrature point); consecutive threads share an
// element, so the gathered nodal coordinates are broadcast within a warp and
// served from L1.  The reference gradients (Q, 3, N) sit in shared memory.
// The kernel is FP64-pipe bound on GB300 (about 9N + 40 FP64 operations per
// thread against 80 bytes written).
#include "fe_device.cuh"

namespace {

constexpr int kGeomThreads = 256;

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
        // cofactors and determinant (expansion along the first row)
        const double c00 = J11 * J22 - J12 * J21;
        const double c01 = J12 * J20 - J10 * J22;
        const double c02 = J10 * J21 - J11 * J20;
        const double det = J00 * c00 + J01 * c01 + J02 * c02;
        if (!(det > 0.0) || !isfinite(det)) fe_report(status, isfinite(det) ? FE_ERR_NONPOSITIVE_DETJ : FE_ERR_NONFINITE, e);
        const double r = 1.0 / det;
        // J^-1 = adj(J) / det, adj = cof^T
        double inv[9];
        inv[0] = c00 * r;
        inv[3] = c01 * r;
        inv[6] = c02 * r;
        inv[1] = (J02 * J21 - J01 * J22) * r;
        inv[4] = (J00 * J22 - J02 * J20) * r;
        inv[7] = (J01 * J20 - J00 * J21) * r;
        inv[2] = (J01 * J12 - J02 * J11) * r;
        inv[5] = (J02 * J10 - J00 * J12) * r;
        inv[8] = (J00 * J11 - J01 * J10) * r;
        const double wd = w[q] * det;
        if (jinv64) {
            double *o = jinv64 + idx * 9;
#pragma unroll
            for (int k = 0; k < 9; ++k) o[k] = inv[k];
            wdetj64[idx] = wd;
        }
        if (jinv32) {
            float *o = jinv32 + idx * 9;
#pragma unroll
            for (int k = 0; k < 9; ++k) o[k] = (float)inv[k];
            wdetj32[idx] = (float)wd;
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
        cudaError_t err = cudaFuncSetAttribute(k_geometry<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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

}  // namespace

cudaError_t fe_launch_geometry(const fe_geometry_h *g, unsigned long long *st, cudaStream_t s)
{
    if (g->mesh.n_elems == 0) return cudaSuccess;
    switch (g->N) {
    case 8: return launch_geom<8>(g, st, s);
    case 27: return launch_geom<27>(g, st, s);
    case 64: return launch_geom<64>(g, st, s);
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
