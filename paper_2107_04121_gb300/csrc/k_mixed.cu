// Stokes coupling 'i.i,0' of Tab. ewfd (Cimrman, arXiv 2107.04121) between
// fields of different orders over the same elements: the vector field on the
// geometry's basis (N nodes, physical gradients G = J^-T grad_xi phi) and a
// scalar field on a second basis (Np nodes, values psi at the same quadrature
// points, its own connectivity), e.g. a Q2 velocity with a Q1 pressure or P2
// with P1 (Taylor-Hood pairs).  For the coupling div(v) p (test field vector):
//   matrix    K[(i,a)][b] = sum_q w det J G_q[i][a] psi_q[b]          (E, 3N, Np)
//   residual  r[(i,a)]    = sum_q w det J G_q[i][a] p_h(q)            (E, 3N)
// and for the transposed coupling q div(u) (test field scalar):
//   matrix    K[b][(i,a)] = the same sums                              (E, Np, 3N)
//   residual  r[b]        = sum_q w det J psi_q[b] div u_h(q)          (E, Np)
// Per element group a CTA stages J^-1, w det J and the gathered DOFs of the
// field the residual needs; residuals first form the point values p_h(q) or
// div u_h(q), then one thread per output row sums over the points.  The
// reference tables are read through the read-only cache.
#include "fe_device.cuh"

namespace {

constexpr int MX_THREADS = 128;

template <typename T>
struct MixArgs {
    int transposed;  // 0: test field vector (div(v) p), 1: test field scalar (q div(u))
    int mode;        // 0 residual, 1 matrix
    int N, Np, Q, epb;
    long long E, n_nodes, n_nodes_p;
    const T *jinv, *wdetj, *dphi, *psi;
    const int32_t *conn, *conn_p;
    const T *field;  // residual: the scalar DOFs (p) or the vector DOFs (u, 3 per node)
    T *out;
    unsigned long long *status;
};

// shared memory of one element, in T units: J^-1, w det J, the point values, the
// gathered DOFs (3N for u, Np for p)
__host__ __device__ inline int mix_per_elem(int N, int Np, int Q) { return 11 * Q + (3 * N > Np ? 3 * N : Np); }

// G_q[i][a] from the reference gradients of the geometry's basis and J^-1 (row-major,
// Ji[k * 3 + i] = (J^-1)_ki)
template <typename T>
__device__ __forceinline__ T grad_at(const T *__restrict__ dp, int N, const T *Ji, int i, int a)
{
    return __ldg(dp + a) * Ji[i] + __ldg(dp + N + a) * Ji[3 + i] + __ldg(dp + 2 * N + a) * Ji[6 + i];
}

template <typename T>
__global__ void __launch_bounds__(MX_THREADS) k_stokes_mixed(MixArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char mx_smem[];
    T *sm = reinterpret_cast<T *>(mx_smem);
    const int N = a.N, Np = a.Np, Q = a.Q, PE = mix_per_elem(N, Np, Q);
    const int O_JI = 0, O_WD = 9 * Q, O_PV = 10 * Q, O_F = 11 * Q;
    const int nrow = a.transposed ? Np : 3 * N, ncol = a.transposed ? 3 * N : Np;
    for (long long e0 = (long long)blockIdx.x * a.epb; e0 < a.E; e0 += (long long)gridDim.x * a.epb) {
        const int ne = (int)((a.E - e0) < a.epb ? (a.E - e0) : a.epb);
        __syncthreads();
        for (int t = threadIdx.x; t < ne * Q * 9; t += MX_THREADS)
            sm[(t / (Q * 9)) * PE + O_JI + t % (Q * 9)] = a.jinv[e0 * Q * 9 + t];
        for (int t = threadIdx.x; t < ne * Q; t += MX_THREADS) sm[(t / Q) * PE + O_WD + t % Q] = a.wdetj[e0 * Q + t];
        if (a.mode == 0) {
            // the residual's field: p on the scalar field's nodes, or u on the geometry's
            const int nf = a.transposed ? N : Np;
            const int32_t *cn = a.transposed ? a.conn : a.conn_p;
            const long long nn = a.transposed ? a.n_nodes : a.n_nodes_p;
            for (int t = threadIdx.x; t < ne * nf; t += MX_THREADS) {
                const int el = t / nf, b = t % nf;
                const long long node = cn[(e0 + el) * nf + b];
                const bool ok = (unsigned long long)node < (unsigned long long)nn;  // never read outside the field
                if (!ok) fe_report(a.status, FE_ERR_SHAPE, e0 + el);
                T *S = sm + el * PE + O_F;
                if (a.transposed) {
                    for (int c = 0; c < 3; ++c) S[c * N + b] = ok ? a.field[node * 3 + c] : (T)0;
                } else {
                    S[b] = ok ? a.field[node] : (T)0;
                }
            }
        }
        __syncthreads();
        if (a.mode == 0) {
            // point values: p_h(q) = sum_b psi_q[b] p_b, or div u_h(q) = sum_(i,a) u[i][a] G_q[i][a]
            for (int t = threadIdx.x; t < ne * Q; t += MX_THREADS) {
                const int el = t / Q, q = t % Q;
                T *S = sm + el * PE;
                T v = 0;
                if (a.transposed) {
                    const T *Ji = S + O_JI + q * 9;
                    const T *dp = a.dphi + (size_t)q * 3 * N;
                    for (int i = 0; i < 3; ++i)
                        for (int b = 0; b < N; ++b) v = fma(S[O_F + i * N + b], grad_at(dp, N, Ji, i, b), v);
                } else {
                    for (int b = 0; b < Np; ++b) v = fma(__ldg(a.psi + (size_t)q * Np + b), S[O_F + b], v);
                }
                S[O_PV + q] = S[O_WD + q] * v;
            }
            __syncthreads();
            for (int t = threadIdx.x; t < ne * nrow; t += MX_THREADS) {
                const int el = t / nrow, row = t % nrow;
                const T *S = sm + el * PE;
                T r = 0;
                if (a.transposed) {
                    for (int q = 0; q < Q; ++q) r = fma(__ldg(a.psi + (size_t)q * Np + row), S[O_PV + q], r);
                } else {
                    const int i = row / N, ra = row % N;
                    for (int q = 0; q < Q; ++q)
                        r = fma(grad_at(a.dphi + (size_t)q * 3 * N, N, S + O_JI + q * 9, i, ra), S[O_PV + q], r);
                }
                a.out[(e0 + el) * nrow + row] = r;
            }
        } else {
            // matrix: one thread per (element, vector row (i, a)); the scalar index b
            // runs along the row, or down the column of the transposed coupling
            for (int t = threadIdx.x; t < ne * 3 * N; t += MX_THREADS) {
                const int el = t / (3 * N), vr = t % (3 * N), i = vr / N, ra = vr % N;
                const T *S = sm + el * PE;
                T *Ke = a.out + (e0 + el) * (long long)nrow * ncol;
                for (int b = 0; b < Np; ++b) {
                    T s = 0;
                    for (int q = 0; q < Q; ++q) {
                        const T G = grad_at(a.dphi + (size_t)q * 3 * N, N, S + O_JI + q * 9, i, ra);
                        s = fma(S[O_WD + q] * G, __ldg(a.psi + (size_t)q * Np + b), s);
                    }
                    if (a.transposed)
                        Ke[(long long)b * ncol + vr] = s;
                    else
                        Ke[(long long)vr * ncol + b] = s;
                }
            }
        }
    }
}

template <typename T>
cudaError_t launch_mixed(const fe_geometry_h *g, const fe_field_h *f, bool transposed, int mode, const void *field,
                         void *out, unsigned long long *st, cudaStream_t s)
{
    constexpr bool D = sizeof(T) == 8;
    MixArgs<T> a{};
    a.transposed = transposed;
    a.mode = mode;
    a.N = g->N;
    a.Np = f->n_basis;
    a.Q = g->Q;
    const int per = mix_per_elem(a.N, a.Np, a.Q);
    int epb = (int)((32 * 1024) / ((size_t)per * sizeof(T)));
    if (epb > 16) epb = 16;
    if (epb < 1) epb = 1;
    a.epb = epb;
    a.E = g->mesh.n_elems;
    a.n_nodes = g->mesh.n_nodes;
    a.n_nodes_p = f->n_nodes;
    a.jinv = D ? (const T *)g->d_jinv64 : (const T *)g->d_jinv32;
    a.wdetj = D ? (const T *)g->d_wdetj64 : (const T *)g->d_wdetj32;
    a.dphi = D ? (const T *)g->d_dphi64 : (const T *)g->d_dphi32;
    a.psi = D ? (const T *)f->d_psi64 : (const T *)f->d_psi32;
    a.conn = g->mesh.conn;
    a.conn_p = f->conn;
    a.field = (const T *)field;
    a.out = (T *)out;
    a.status = st;
    const size_t smem = (size_t)per * epb * sizeof(T);
    static FeLaunchCache cache;
    long long cap = 0;
    cudaError_t err = fe_cached_grid(
        cache,
        [&](int dev, long long *v) {
            int sms = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            *v = (long long)sms * 8;
            return cudaSuccess;
        },
        &cap);
    if (err != cudaSuccess) return err;
    long long blocks = (a.E + epb - 1) / epb;
    if (blocks > cap) blocks = cap;
    k_stokes_mixed<T><<<(unsigned)blocks, MX_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t fe_launch_stokes_mixed(const fe_geometry_h *g, const fe_field_h *f, bool f64, bool transposed, int mode,
                                   const void *field, void *out, unsigned long long *status, cudaStream_t s)
{
    if (g->mesh.n_elems == 0) return cudaSuccess;
    return f64 ? launch_mixed<double>(g, f, transposed, mode, field, out, status, s)
               : launch_mixed<float>(g, f, transposed, mode, field, out, status, s);
}
