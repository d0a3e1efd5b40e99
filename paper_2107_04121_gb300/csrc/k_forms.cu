// The remaining weak forms of Tab. ewfd (Cimrman, arXiv 2107.04121) and the
// 'eval' mode of every form (Sec. 5.1), for any element of the library
// (runtime N nodes and Q points; FP64 or FP32):
//   weighted dot   'ij,i,j'   v_i M_ij u_j            residual, matrix, eval
//   Stokes         'i.i,0'    div(v) p                residual, matrix, eval
//   transposed     'i.i,0'    q div(u)                residual, matrix, eval
//   divergence     'i.i'      div(v)                  residual (linear form), eval
//   Cauchy stress  'IK,s(k:l)->K'   D e(u)            eval only (6 values)
//   and the eval integrals of the Laplacian, dot/mass, elasticity and
//   convective forms.
// Per element group a CTA stages J^-1, w det J, the gathered DOFs of the
// form's fields and the material; one thread per (element, point) forms the
// field values and physical gradients and the point contributions, then one
// thread per output row (or value) sums them over the points:
//   residual  r[(i,a)] = sum_q [ C_i(q) phi_a(q) + sum_k F_ik(q) dphi_a/dxi_k(q) ]
//   eval      out[m]   = sum_q V_m(q)
//   matrix    rows formed from the tables and the staged J^-1 directly.
// The reference tables are read through the read-only cache.
#include "fe_device.cuh"

namespace {

constexpr int GEN_THREADS = 128;

template <typename T>
struct GenArgs {
    int kind, mode, N, Q, epb;
    int nca, ncb, ncc;  // components of the fields a (test slot), b, c
    int mat_kind, mat_t, n_out, nrow, ncol;
    long long E, n_nodes;
    const T *jinv, *wdetj, *phi, *dphi;
    const int32_t *conn;
    const T *fa, *fb, *fc;
    const double *mat;
    T *out;
    unsigned long long *status;
};

// shared memory of one element, in T units
__host__ __device__ inline int gen_per_elem(int N, int Q) { return 22 * Q + 9 * N + 36; }

template <typename T>
__device__ inline void field_at(const T *__restrict__ U, int nc, int N, const T *__restrict__ ph,
                                const T *__restrict__ dp, const T *Ji, T v[3], T g[3][3])
{
    for (int c = 0; c < 3; ++c) {
        v[c] = 0;
        for (int j = 0; j < 3; ++j) g[c][j] = 0;
    }
    for (int c = 0; c < nc; ++c) {
        T r0 = 0, r1 = 0, r2 = 0, vv = 0;
        for (int b = 0; b < N; ++b) {
            const T x = U[c * N + b];
            vv = fma(__ldg(ph + b), x, vv);
            r0 = fma(__ldg(dp + b), x, r0);
            r1 = fma(__ldg(dp + N + b), x, r1);
            r2 = fma(__ldg(dp + 2 * N + b), x, r2);
        }
        v[c] = vv;
        for (int j = 0; j < 3; ++j) g[c][j] = r0 * Ji[j] + r1 * Ji[3 + j] + r2 * Ji[6 + j];
    }
}

template <typename T>
__device__ inline void voigt_strain(const T g[3][3], T e[6])
{
    e[0] = g[0][0];
    e[1] = g[1][1];
    e[2] = g[2][2];
    e[3] = g[0][1] + g[1][0];
    e[4] = g[0][2] + g[2][0];
    e[5] = g[1][2] + g[2][1];
}

template <typename T>
__global__ void __launch_bounds__(GEN_THREADS) k_generic(GenArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char gen_smem[];
    T *sm = reinterpret_cast<T *>(gen_smem);
    const int N = a.N, Q = a.Q, PE = gen_per_elem(N, Q);
    // per-element layout
    const int O_JI = 0, O_WD = 9 * Q, O_UA = 10 * Q, O_UB = O_UA + 3 * N, O_UC = O_UB + 3 * N, O_M = O_UC + 3 * N,
              O_PT = O_M + 36;
    for (long long e0 = (long long)blockIdx.x * a.epb; e0 < a.E; e0 += (long long)gridDim.x * a.epb) {
        const int ne = (int)((a.E - e0) < a.epb ? (a.E - e0) : a.epb);
        __syncthreads();
        for (int t = threadIdx.x; t < ne * Q * 9; t += GEN_THREADS)
            sm[(t / (Q * 9)) * PE + O_JI + t % (Q * 9)] = a.jinv[e0 * Q * 9 + t];
        for (int t = threadIdx.x; t < ne * Q; t += GEN_THREADS) sm[(t / Q) * PE + O_WD + t % Q] = a.wdetj[e0 * Q + t];
        for (int t = threadIdx.x; t < ne * N; t += GEN_THREADS) {
            const int el = t / N, b = t % N;
            const long long node = a.conn[(e0 + el) * N + b];
            const bool ok = (unsigned long long)node < (unsigned long long)a.n_nodes;  // never read outside a field
            if (!ok) fe_report(a.status, FE_ERR_SHAPE, e0 + el);
            T *S = sm + el * PE;
            for (int c = 0; c < a.nca; ++c) S[O_UA + c * N + b] = ok && a.fa ? a.fa[node * a.nca + c] : (T)0;
            for (int c = 0; c < a.ncb; ++c) S[O_UB + c * N + b] = ok && a.fb ? a.fb[node * a.ncb + c] : (T)0;
            for (int c = 0; c < a.ncc; ++c) S[O_UC + c * N + b] = ok && a.fc ? a.fc[node * a.ncc + c] : (T)0;
        }
        // material: scalar c, the 6x6 D (from a Lame pair or as given), or the 3x3 M
        for (int t = threadIdx.x; t < ne * 36; t += GEN_THREADS) {
            const int el = t / 36, x = t % 36;
            const long long e = e0 + el;
            T v = 0;
            if (a.mat_kind == FE_MAT_SCALAR) {
                v = x == 0 ? (a.mat ? (T)a.mat[e] : (T)1) : (T)0;
            } else if (a.mat_kind == FE_MAT_LAME) {
                const int I = x / 6, K = x % 6;
                const double lam = a.mat[2 * e], mu = a.mat[2 * e + 1];
                v = (T)((I < 3 && K < 3 ? lam : 0.0) + (I == K ? (I < 3 ? 2.0 * mu : mu) : 0.0));
            } else if (a.mat_kind == FE_MAT_D66) {
                const int I = x / 6, K = x % 6;
                v = (T)(a.mat_t ? a.mat[e * 36 + K * 6 + I] : a.mat[e * 36 + x]);
            } else if (a.mat_kind == FE_MAT_M33) {
                if (x < 9) v = (T)(a.mat_t ? a.mat[e * 9 + (x % 3) * 3 + x / 3] : a.mat[e * 9 + x]);
            } else {
                v = x == 0 ? (T)1 : (T)0;
            }
            sm[el * PE + O_M + x] = v;
        }
        __syncthreads();
        if (a.mode != 1) {
            // ---- point contributions
            for (int t = threadIdx.x; t < ne * Q; t += GEN_THREADS) {
                const int el = t / Q, q = t % Q;
                T *S = sm + el * PE;
                const T *Ji = S + O_JI + q * 9;
                const T wd = S[O_WD + q];
                const T *ph = a.phi + (size_t)q * N, *dp = a.dphi + (size_t)q * 3 * N;
                const T *Mm = S + O_M;
                T *P = S + O_PT + q * 12;
                for (int x = 0; x < 12; ++x) P[x] = 0;
                T va[3], ga[3][3], vb[3], gb[3][3], vc[3], gc[3][3];
                field_at(S + O_UA, a.nca, N, ph, dp, Ji, va, ga);
                field_at(S + O_UB, a.ncb, N, ph, dp, Ji, vb, gb);
                field_at(S + O_UC, a.ncc, N, ph, dp, Ji, vc, gc);
                if (a.mode == 0) {  // residual: P[i] = C_i, P[3 + 3 i + k] = F_ik
                    switch (a.kind) {
                    case FK_WDOT:
                        for (int i = 0; i < 3; ++i) P[i] = wd * (Mm[i * 3] * vb[0] + Mm[i * 3 + 1] * vb[1] + Mm[i * 3 + 2] * vb[2]);
                        break;
                    case FK_STOKES:
                    case FK_DIV: {
                        const T s = a.kind == FK_STOKES ? wd * vb[0] : wd;
                        for (int i = 0; i < 3; ++i)
                            for (int k = 0; k < 3; ++k) P[3 + 3 * i + k] = s * Ji[k * 3 + i];
                        break;
                    }
                    case FK_STOKES_T: P[0] = wd * (gb[0][0] + gb[1][1] + gb[2][2]); break;
                    default: break;
                    }
                } else {  // eval: P[m] = V_m
                    switch (a.kind) {
                    case FK_LAPLACE:
                        P[0] = wd * Mm[0] * (ga[0][0] * gb[0][0] + ga[0][1] * gb[0][1] + ga[0][2] * gb[0][2]);
                        break;
                    case FK_MASS: {
                        T s = 0;
                        for (int c = 0; c < a.nca; ++c) s += va[c] * vb[c];
                        P[0] = wd * Mm[0] * s;
                        break;
                    }
                    case FK_ELASTICITY: {
                        T ea[6], eb[6], s = 0;
                        voigt_strain(ga, ea);
                        voigt_strain(gb, eb);
                        for (int I = 0; I < 6; ++I)
                            for (int K = 0; K < 6; ++K) s += ea[I] * Mm[I * 6 + K] * eb[K];
                        P[0] = wd * s;
                        break;
                    }
                    case FK_WDOT: {
                        T s = 0;
                        for (int i = 0; i < 3; ++i)
                            for (int j = 0; j < 3; ++j) s += va[i] * Mm[i * 3 + j] * vb[j];
                        P[0] = wd * s;
                        break;
                    }
                    case FK_STOKES: P[0] = wd * (ga[0][0] + ga[1][1] + ga[2][2]) * vb[0]; break;
                    case FK_STOKES_T: P[0] = wd * va[0] * (gb[0][0] + gb[1][1] + gb[2][2]); break;
                    case FK_DIV: P[0] = wd * (ga[0][0] + ga[1][1] + ga[2][2]); break;
                    case FK_CAUCHY: {
                        T ea[6];
                        voigt_strain(ga, ea);
                        for (int I = 0; I < 6; ++I) {
                            T s = 0;
                            for (int K = 0; K < 6; ++K) s += Mm[I * 6 + K] * ea[K];
                            P[I] = wd * s;
                        }
                        break;
                    }
                    case FK_CONVECT: {  // a: test slot (i), b: gradient (i.j), c: advection (j)
                        T s = 0;
                        for (int i = 0; i < 3; ++i)
                            for (int j = 0; j < 3; ++j) s += va[i] * gb[i][j] * vc[j];
                        P[0] = wd * s;
                        break;
                    }
                    default: break;
                    }
                }
            }
            __syncthreads();
            if (a.mode == 0) {
                for (int t = threadIdx.x; t < ne * a.nrow; t += GEN_THREADS) {
                    const int el = t / a.nrow, row = t % a.nrow, i = row / N, b = row % N;
                    const T *S = sm + el * PE;
                    T r = 0;
                    for (int q = 0; q < Q; ++q) {
                        const T *P = S + O_PT + q * 12;
                        const T *dp = a.dphi + (size_t)q * 3 * N;
                        r += P[i] * __ldg(a.phi + (size_t)q * N + b) + P[3 + 3 * i] * __ldg(dp + b) +
                             P[4 + 3 * i] * __ldg(dp + N + b) + P[5 + 3 * i] * __ldg(dp + 2 * N + b);
                    }
                    a.out[(e0 + el) * a.nrow + row] = r;
                }
            } else {
                for (int t = threadIdx.x; t < ne * a.n_out; t += GEN_THREADS) {
                    const int el = t / a.n_out, m = t % a.n_out;
                    const T *S = sm + el * PE;
                    T s = 0;
                    for (int q = 0; q < Q; ++q) s += S[O_PT + q * 12 + m];
                    a.out[(e0 + el) * a.n_out + m] = s;
                }
            }
        } else {
            // ---- matrix rows
            for (int t = threadIdx.x; t < ne * a.nrow; t += GEN_THREADS) {
                const int el = t / a.nrow, row = t % a.nrow;
                const T *S = sm + el * PE;
                T *Ko = a.out + ((e0 + el) * a.nrow + row) * (long long)a.ncol;
                if (a.kind == FK_WDOT) {  // row (i, a): M_ij sum_q wd phi_a phi_b
                    const int i = row / N, ra = row % N;
                    const T *Mm = S + O_M;
                    for (int b = 0; b < N; ++b) {
                        T s = 0;
                        for (int q = 0; q < Q; ++q)
                            s += S[O_WD + q] * __ldg(a.phi + (size_t)q * N + ra) * __ldg(a.phi + (size_t)q * N + b);
                        for (int j = 0; j < 3; ++j) Ko[j * N + b] = Mm[i * 3 + j] * s;
                    }
                } else if (a.kind == FK_STOKES) {  // row (i, a): sum_q wd G[i][a] phi_b
                    const int i = row / N, ra = row % N;
                    for (int b = 0; b < N; ++b) {
                        T s = 0;
                        for (int q = 0; q < Q; ++q) {
                            const T *Ji = S + O_JI + q * 9;
                            const T *dp = a.dphi + (size_t)q * 3 * N;
                            const T G = __ldg(dp + ra) * Ji[i] + __ldg(dp + N + ra) * Ji[3 + i] +
                                        __ldg(dp + 2 * N + ra) * Ji[6 + i];
                            s += S[O_WD + q] * G * __ldg(a.phi + (size_t)q * N + b);
                        }
                        Ko[b] = s;
                    }
                } else {  // FK_STOKES_T, row a: sum_q wd phi_a G[i][b]
                    const int ra = row;
                    for (int i = 0; i < 3; ++i)
                        for (int b = 0; b < N; ++b) {
                            T s = 0;
                            for (int q = 0; q < Q; ++q) {
                                const T *Ji = S + O_JI + q * 9;
                                const T *dp = a.dphi + (size_t)q * 3 * N;
                                const T G = __ldg(dp + b) * Ji[i] + __ldg(dp + N + b) * Ji[3 + i] +
                                            __ldg(dp + 2 * N + b) * Ji[6 + i];
                                s += S[O_WD + q] * __ldg(a.phi + (size_t)q * N + ra) * G;
                            }
                            Ko[i * N + b] = s;
                        }
                }
            }
        }
    }
}

template <typename T>
cudaError_t launch_generic(const fe_geometry_h *g, const fe_form_h *f, fe_material_args mat, int mode, const void *f0,
                           const void *f1, const void *f2, void *out, unsigned long long *st, cudaStream_t s)
{
    constexpr bool D = sizeof(T) == 8;
    GenArgs<T> a{};
    a.kind = f->kind;
    a.mode = mode;
    a.N = g->N;
    a.Q = g->Q;
    const int per = gen_per_elem(a.N, a.Q);
    int epb = (int)((48 * 1024) / ((size_t)per * sizeof(T)));
    if (epb > 16) epb = 16;
    if (epb < 1) epb = 1;
    a.epb = epb;
    // the fields of the form, in its slots: a = test slot (eval: first field),
    // b = unknown or second field, c = third field (convection); for the
    // convective form b is the gradient operand and c the advection operand
    a.fa = (const T *)f0;
    a.fb = (const T *)f1;
    a.fc = (const T *)f2;
    a.nca = f0 ? f->ncomp_test : 0;
    a.ncb = f1 ? (f->kind == FK_CONVECT ? 3 : f->ncomp_trial) : 0;
    a.ncc = f2 ? 3 : 0;
    a.mat_kind = mat.kind;
    a.mat_t = mat.transposed;
    a.mat = mat.data;
    a.n_out = f->n_out;
    a.nrow = f->ncomp_test * a.N;
    a.ncol = f->kind == FK_DIV ? 0 : f->ncomp_trial * a.N;
    a.E = g->mesh.n_elems;
    a.n_nodes = g->mesh.n_nodes;
    a.jinv = D ? (const T *)g->d_jinv64 : (const T *)g->d_jinv32;
    a.wdetj = D ? (const T *)g->d_wdetj64 : (const T *)g->d_wdetj32;
    a.phi = D ? (const T *)g->d_phi64 : (const T *)g->d_phi32;
    a.dphi = D ? (const T *)g->d_dphi64 : (const T *)g->d_dphi32;
    a.conn = g->mesh.conn;
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
    k_generic<T><<<(unsigned)blocks, GEN_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t fe_launch_generic(const fe_geometry_h *g, const fe_form_h *f, fe_material_args mat, bool f64, int mode,
                              const void *f0, const void *f1, const void *f2, void *out, unsigned long long *status,
                              cudaStream_t s)
{
    if (g->mesh.n_elems == 0) return cudaSuccess;
    return f64 ? launch_generic<double>(g, f, mat, mode, f0, f1, f2, out, status, s)
               : launch_generic<float>(g, f, mat, mode, f0, f1, f2, out, status, s);
}
