// C ABI of libfe (declarations and argument contracts in include/fe.h).
// Host-side argument validation, handle management and kernel dispatch.
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "fe_internal.h"


// A deferred handle whose geometry is stale gets it computed before any use.
static cudaError_t settle_geometry(fe_geometry_h *g, unsigned long long *status, cudaStream_t s)
{
    if (!g->pending) return cudaSuccess;
    g->pending = 0;
    return fe_launch_geometry(g, status, s);
}

cudaError_t fe_settle_geometry(fe_geometry_h *g, unsigned long long *status, cudaStream_t s)
{
    return settle_geometry(g, status, s);
}

namespace {

thread_local char g_last_error[256] = "";

fe_status from_cuda(cudaError_t e, const char *where)
{
    if (e == cudaSuccess) return FE_OK;
    std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s", where, cudaGetErrorString(e));
    cudaGetLastError();  // clear a non-sticky error
    return e == cudaErrorMemoryAllocation ? FE_ERR_OOM : FE_ERR_CUDA;
}

inline cudaStream_t to_cuda(fe_stream_t s) { return reinterpret_cast<cudaStream_t>(s); }

template <typename T>
cudaError_t dev_alloc(T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void **)p, sizeof(T) * count);
}

bool valid_mesh(const fe_mesh *m)
{
    // an empty mesh may come with null arrays (zero-size device tensors)
    return m && (m->n_elems == 0 || (m->coords && m->conn)) && m->n_nodes >= 0 && m->n_elems >= 0 &&
           m->nodes_per_elem > 0 && m->n_nodes <= INT_MAX && m->n_elems * (long long)m->nodes_per_elem <= INT_MAX;
}

void free_geometry(fe_geometry_h *g)
{
    if (!g) return;
    if (g->is_view) {
        delete g;
        return;
    }
    cudaFree(g->d_phi64);
    cudaFree(g->d_dphi64);
    cudaFree(g->d_w64);
    cudaFree(g->d_b1d);
    cudaFree(g->d_d1d);
    cudaFree(g->d_b1d32);
    cudaFree(g->d_d1d32);
    cudaFree(g->d_dq);
    cudaFree(g->d_phi32);
    cudaFree(g->d_dphi32);
    cudaFree(g->d_jinv64);
    cudaFree(g->d_wdetj64);
    cudaFree(g->d_jinv32);
    cudaFree(g->d_wdetj32);
    cudaFree(g->d_xi);
    delete g;
}

}  // namespace

fe_status fe_status_from_cuda(cudaError_t e, const char *where) { return from_cuda(e, where); }

void fe_clear_last_error() { g_last_error[0] = 0; }

extern "C" {

int fe_version(void) { return 100; }

const char *fe_last_error_message(void) { return g_last_error; }

const char *fe_status_str(fe_status s)
{
    switch (s) {
    case FE_OK: return "FE_OK";
    case FE_ERR_INVALID_ARG: return "FE_ERR_INVALID_ARG";
    case FE_ERR_SHAPE: return "FE_ERR_SHAPE";
    case FE_ERR_UNSUPPORTED_SPEC: return "FE_ERR_UNSUPPORTED_SPEC";
    case FE_ERR_NONPOSITIVE_DETJ: return "FE_ERR_NONPOSITIVE_DETJ";
    case FE_ERR_NONFINITE: return "FE_ERR_NONFINITE";
    case FE_ERR_OOM: return "FE_ERR_OOM";
    case FE_ERR_CUDA: return "FE_ERR_CUDA";
    case FE_ERR_TIMEOUT: return "FE_ERR_TIMEOUT";
    }
    return "FE_ERR_UNKNOWN";
}

fe_status fe_create(int device, fe_ctx **out)
{
    fe_clear_last_error();
    if (!out) return FE_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        std::snprintf(g_last_error, sizeof(g_last_error), "fe_create: no CUDA device %d", device);
        return FE_ERR_CUDA;
    }
    fe_status st = from_cuda(cudaSetDevice(device), "cudaSetDevice");
    if (st) return st;
    fe_ctx *c = new (std::nothrow) fe_ctx();
    if (!c) return FE_ERR_OOM;
    c->device = device;
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    st = from_cuda(dev_alloc(&c->d_status, 2), "cudaMalloc(status)");
    if (st) {
        delete c;
        return st;
    }
    const unsigned long long init[2] = {0ull, ULLONG_MAX};
    st = from_cuda(cudaMemcpy(c->d_status, init, sizeof(init), cudaMemcpyHostToDevice), "status init");
    if (st) {
        cudaFree(c->d_status);
        delete c;
        return st;
    }
    *out = c;
    return FE_OK;
}

fe_status fe_destroy(fe_ctx *ctx)
{
    fe_clear_last_error();
    if (!ctx) return FE_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    cudaFree(ctx->d_status);
    cudaFree(ctx->d_hold);
    delete ctx;
    return FE_OK;
}

fe_status fe_get_status(fe_ctx *ctx, fe_stream_t stream, long long *bad_elem)
{
    fe_clear_last_error();
    if (!ctx) return FE_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    fe_status st = from_cuda(cudaStreamSynchronize(to_cuda(stream)), "fe_get_status sync");
    if (st) return st;
    unsigned long long h[2];
    st = from_cuda(cudaMemcpy(h, ctx->d_status, sizeof(h), cudaMemcpyDeviceToHost), "fe_get_status read");
    if (st) return st;
    const unsigned long long init[2] = {0ull, ULLONG_MAX};
    st = from_cuda(cudaMemcpy(ctx->d_status, init, sizeof(init), cudaMemcpyHostToDevice), "fe_get_status reset");
    if (st) return st;
    if (bad_elem) *bad_elem = h[1] == ULLONG_MAX ? -1 : (long long)h[1];
    return (fe_status)h[0];
}

// ---- geometry -----------------------------------------------------------------

fe_status fe_geometry(fe_ctx *ctx, const fe_mesh *mesh, const fe_refbasis *basis, const fe_quadrature *quad,
                      unsigned flags, fe_geometry_h **out, fe_stream_t stream)
{
    fe_clear_last_error();
    if (!ctx || !out || !valid_mesh(mesh) || !basis || !quad || !basis->phi || !basis->dphi || !quad->weights)
        return FE_ERR_INVALID_ARG;
    *out = nullptr;
    if (flags & ~(FE_GEOM_STORE_F64 | FE_GEOM_STORE_F32 | FE_GEOM_DEFERRED)) return FE_ERR_INVALID_ARG;
    if ((flags & ~FE_GEOM_DEFERRED) == 0) flags |= FE_GEOM_STORE_F64 | FE_GEOM_STORE_F32;
    const int N = basis->n_basis, Q = basis->n_qp;
    if (N != mesh->nodes_per_elem || quad->n_qp != Q || !fe_supported_nq(N, Q)) return FE_ERR_SHAPE;
    const bool tensor = basis->b1d || basis->d1d;
    if (tensor && (!basis->b1d || !basis->d1d || !fe_host_check_tensor_basis(basis))) {
        std::snprintf(g_last_error, sizeof(g_last_error), "fe_geometry: 1-D factors do not reproduce phi/dphi");
        return FE_ERR_INVALID_ARG;
    }
    cudaSetDevice(ctx->device);
    cudaStream_t s = to_cuda(stream);
    fe_geometry_h *g = new (std::nothrow) fe_geometry_h();
    if (!g) return FE_ERR_OOM;
    g->device = ctx->device;
    g->mesh = *mesh;
    g->N = N;
    g->Q = Q;
    g->flags = flags;
    const long long E = mesh->n_elems;
    std::vector<float> phi32((size_t)Q * N), dphi32((size_t)Q * 3 * N);
    for (size_t i = 0; i < phi32.size(); ++i) phi32[i] = (float)basis->phi[i];
    for (size_t i = 0; i < dphi32.size(); ++i) dphi32[i] = (float)basis->dphi[i];
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = dev_alloc(&g->d_phi64, (size_t)Q * N);
    if (e == cudaSuccess) e = dev_alloc(&g->d_dphi64, (size_t)Q * 3 * N);
    if (e == cudaSuccess) e = dev_alloc(&g->d_w64, (size_t)Q);
    {
        // points by weight sign, each group padded to a multiple of 8 slots
        int np = 0, nn = 0;
        for (int q = 0; q < Q; ++q) (quad->weights[q] >= 0.0 ? np : nn)++;
        g->n_wpos = np;
        g->n_wneg = nn;
        const int p8 = (np + 7) / 8 * 8, n8 = (nn + 7) / 8 * 8;
        for (int k = 0; k < 64; ++k) g->slot_q[k] = -1;
        if (p8 + n8 <= 64) {
            int ip = 0, in = p8;
            for (int q = 0; q < Q; ++q) g->slot_q[quad->weights[q] >= 0.0 ? ip++ : in++] = (signed char)q;
        }
    }
    if (e == cudaSuccess) e = dev_alloc(&g->d_phi32, (size_t)Q * N);
    if (e == cudaSuccess) e = dev_alloc(&g->d_dphi32, (size_t)Q * 3 * N);
    if (e == cudaSuccess && tensor) {
        g->n1d = basis->n1d;
        g->nq1d = basis->nq1d;
        const size_t n = (size_t)basis->n1d * basis->nq1d;
        e = dev_alloc(&g->d_b1d, n);
        if (e == cudaSuccess) e = dev_alloc(&g->d_d1d, n);
        if (e == cudaSuccess) e = cudaMemcpy(g->d_b1d, basis->b1d, sizeof(double) * n, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(g->d_d1d, basis->d1d, sizeof(double) * n, cudaMemcpyHostToDevice);
        std::vector<float> b32(n), d32(n);
        for (size_t t = 0; t < n; ++t) {
            b32[t] = (float)basis->b1d[t];
            d32[t] = (float)basis->d1d[t];
        }
        if (e == cudaSuccess) e = dev_alloc(&g->d_b1d32, n);
        if (e == cudaSuccess) e = dev_alloc(&g->d_d1d32, n);
        if (e == cudaSuccess) e = cudaMemcpy(g->d_b1d32, b32.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(g->d_d1d32, d32.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
        double dq[64];
        if (e == cudaSuccess && basis->n1d == basis->nq1d &&
            fe_host_collocation_derivative(basis->n1d, basis->b1d, basis->d1d, dq)) {
            // three points with the middle one on the middle node (B's middle row
            // exactly (0, 1, 0)): the middle row of Dq is (-d, 0, d) up to rounding;
            // made exact, the kernels use it to skip the trivial products
            // and symmetric points make the first and last rows antisymmetric
            // ((d0, d1, d2), (-d2, -d1, -d0)); made exact too, with the constants of
            // their even-odd form after the table (geometry_body.cuh)
            const double *B = basis->b1d;
            for (int i = 0; i < 4; ++i) dq[n + i] = 0.0;
            if (basis->n1d == 3 && B[3] == 0.0 && B[4] == 1.0 && B[5] == 0.0) {
                double sc = 0.0;
                for (int i = 0; i < 9; ++i) sc = std::fmax(sc, std::fabs(dq[i]));
                const double tol = 1e-13 * sc;
                if (std::fabs(dq[4]) <= tol && std::fabs(dq[3] + dq[5]) <= tol && std::fabs(dq[6] + dq[2]) <= tol &&
                    std::fabs(dq[7] + dq[1]) <= tol && std::fabs(dq[8] + dq[0]) <= tol) {
                    const double d = 0.5 * (dq[5] - dq[3]);
                    dq[3] = -d;
                    dq[4] = 0.0;
                    dq[5] = d;
                    dq[6] = -dq[2];
                    dq[7] = -dq[1];
                    dq[8] = -dq[0];
                    dq[9] = 0.5 * (dq[0] + dq[2]);
                    dq[10] = 0.5 * (dq[0] - dq[2]);
                    dq[11] = dq[1];
                    g->geo_center = 1;
                }
            }
            e = dev_alloc(&g->d_dq, n + 4);
            if (e == cudaSuccess) e = cudaMemcpy(g->d_dq, dq, sizeof(double) * (n + 4), cudaMemcpyHostToDevice);
        }
    }
    if (e == cudaSuccess && (flags & FE_GEOM_STORE_F64)) {
        e = dev_alloc(&g->d_jinv64, (size_t)E * Q * 9);
        if (e == cudaSuccess) e = dev_alloc(&g->d_wdetj64, (size_t)E * Q);
    }
    if (e == cudaSuccess && (flags & FE_GEOM_STORE_F32)) {
        e = dev_alloc(&g->d_jinv32, (size_t)E * Q * 9);
        if (e == cudaSuccess) e = dev_alloc(&g->d_wdetj32, (size_t)E * Q);
    }
    if (e == cudaSuccess && !tensor && (flags & FE_GEOM_STORE_F32) && !(flags & FE_GEOM_STORE_F64)) {
        // the library's tetrahedron basis in a float32-only handle: straight-sided
        // elements get J from their vertices (the float64 copy, when kept, follows
        // the isoparametric sum at every point)
        double xi[64 * 3];
        g->simplex_p = fe_host_simplex_order(N, Q, basis->phi, xi);
        if (g->simplex_p) {
            e = dev_alloc(&g->d_xi, (size_t)N * 3);
            if (e == cudaSuccess) e = cudaMemcpy(g->d_xi, xi, sizeof(double) * N * 3, cudaMemcpyHostToDevice);
        }
    }
    // the tables are tiny; synchronous copies keep the host buffers' lifetime simple
    if (e == cudaSuccess) e = cudaMemcpy(g->d_phi64, basis->phi, sizeof(double) * Q * N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_dphi64, basis->dphi, sizeof(double) * Q * 3 * N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_w64, quad->weights, sizeof(double) * Q, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_phi32, phi32.data(), sizeof(float) * Q * N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(g->d_dphi32, dphi32.data(), sizeof(float) * Q * 3 * N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        if (flags & FE_GEOM_DEFERRED)
            g->pending = 1;
        else
            e = fe_launch_geometry(g, ctx->d_status, s);
    }
    if (e != cudaSuccess) {
        fe_status st = from_cuda(e, "fe_geometry");
        free_geometry(g);
        return st;
    }
    *out = g;
    return FE_OK;
}

fe_status fe_geometry_view(fe_ctx *ctx, const fe_geometry_h *parent, long long e_begin, long long e_count,
                           fe_geometry_h **out)
{
    fe_clear_last_error();
    if (!ctx || !parent || !out || e_begin < 0 || e_count < 0 || e_begin + e_count > parent->mesh.n_elems)
        return FE_ERR_INVALID_ARG;
    if (parent->flags & FE_GEOM_DEFERRED) return FE_ERR_INVALID_ARG;  // views share computed storage
    *out = nullptr;
    fe_geometry_h *v = new (std::nothrow) fe_geometry_h(*parent);
    if (!v) return FE_ERR_OOM;
    const int N = parent->N, Q = parent->Q;
    v->is_view = 1;
    v->pending = 0;
    v->mesh.conn = parent->mesh.conn ? parent->mesh.conn + e_begin * N : nullptr;
    v->mesh.n_elems = e_count;
    if (v->d_jinv64) v->d_jinv64 += e_begin * Q * 9;
    if (v->d_wdetj64) v->d_wdetj64 += e_begin * Q;
    if (v->d_jinv32) v->d_jinv32 += e_begin * Q * 9;
    if (v->d_wdetj32) v->d_wdetj32 += e_begin * Q;
    *out = v;
    return FE_OK;
}

fe_status fe_geometry_update(fe_ctx *ctx, fe_geometry_h *geom, fe_stream_t stream)
{
    fe_clear_last_error();
    if (!ctx || !geom) return FE_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    if (geom->flags & FE_GEOM_DEFERRED) {
        geom->pending = 1;
        return FE_OK;
    }
    return from_cuda(fe_launch_geometry(geom, ctx->d_status, to_cuda(stream)), "fe_geometry_update");
}

fe_status fe_geometry_free(fe_geometry_h *geom)
{
    fe_clear_last_error();
    if (!geom) return FE_ERR_INVALID_ARG;
    cudaSetDevice(geom->device);
    free_geometry(geom);
    return FE_OK;
}

fe_status fe_geometry_get(fe_ctx *ctx, const fe_geometry_h *g, fe_geom_field field, fe_precision prec, void *out,
                          fe_stream_t stream)
{
    fe_clear_last_error();
    if (!ctx || !g || (!out && g->mesh.n_elems > 0)) return FE_ERR_INVALID_ARG;
    const bool f64 = prec == FE_F64;
    if (f64 ? !g->d_jinv64 : !g->d_jinv32) return FE_ERR_INVALID_ARG;
    if (g->mesh.n_elems == 0) return FE_OK;
    cudaSetDevice(ctx->device);
    cudaStream_t s = to_cuda(stream);
    fe_status st0 = from_cuda(settle_geometry(const_cast<fe_geometry_h *>(g), ctx->d_status, s), "fe_geometry_get");
    if (st0) return st0;
    const size_t es = f64 ? 8 : 4;
    const long long E = g->mesh.n_elems;
    cudaError_t e;
    switch (field) {
    case FE_GEOM_WDETJ:
        e = cudaMemcpyAsync(out, f64 ? (const void *)g->d_wdetj64 : (const void *)g->d_wdetj32, es * E * g->Q,
                            cudaMemcpyDeviceToDevice, s);
        break;
    case FE_GEOM_JINV:
        e = cudaMemcpyAsync(out, f64 ? (const void *)g->d_jinv64 : (const void *)g->d_jinv32, es * E * g->Q * 9,
                            cudaMemcpyDeviceToDevice, s);
        break;
    case FE_GEOM_G: e = fe_launch_geometry_G(g, f64, out, s); break;
    default: return FE_ERR_INVALID_ARG;
    }
    return from_cuda(e, "fe_geometry_get");
}

// ---- evaluation ------------------------------------------------------------------

static fe_status eval_common(fe_ctx *ctx, const fe_form_h *form, const fe_geometry_h *g, const void *const *args,
                             fe_precision prec, void *out, fe_material_args *mat)
{
    const bool empty = g && g->mesh.n_elems == 0;
    if (!ctx || !form || !g || (!out && !empty)) return FE_ERR_INVALID_ARG;
    if (prec < FE_F64 || prec > FE_BF16) return FE_ERR_INVALID_ARG;
    if (form->mat_op >= 0) {
        if (!args || (!args[form->mat_op] && !empty)) return FE_ERR_INVALID_ARG;
        mat->kind = form->mat;
        mat->data = (const double *)args[form->mat_op];
        mat->transposed = form->mat_transposed;
    } else {
        mat->kind = FE_MAT_NONE;
        mat->data = nullptr;
        mat->transposed = 0;
    }
    const bool f64 = prec == FE_F64;
    if (f64 ? !g->d_jinv64 : !g->d_jinv32) return FE_ERR_INVALID_ARG;  // geometry copy not stored
    cudaSetDevice(ctx->device);
    return FE_OK;
}

fe_status fe_eval_matrix(fe_ctx *ctx, const fe_form_h *form, const fe_geometry_h *g, const void *const *args,
                         int diff_op, fe_precision prec, void *K_out, fe_stream_t stream)
{
    fe_clear_last_error();
    fe_material_args mat{};
    fe_status st = eval_common(ctx, form, g, args, prec, K_out, &mat);
    if (st) return st;
    cudaError_t e;
    fe_geometry_h *gm = const_cast<fe_geometry_h *>(g);
    cudaStream_t s = to_cuda(stream);
    if (form->kind == FK_CONVECT) {
        // derivative with respect to the unknown: every FE_STATE operand (Eq. fe4)
        const bool ok_diff = (diff_op == form->grad_op && form->wrt_grad) || (diff_op == form->adv_op && form->wrt_adv);
        if (!ok_diff) return FE_ERR_INVALID_ARG;
        if (prec != FE_F64 && prec != FE_F32) return FE_ERR_UNSUPPORTED_SPEC;
        if (!fe_convect_supported(g)) return FE_ERR_UNSUPPORTED_SPEC;
        const bool empty = g->mesh.n_elems == 0;
        if (!args || (!empty && (!args[form->grad_op] || !args[form->adv_op]))) return FE_ERR_INVALID_ARG;
        if (gm->pending && prec != FE_F64 && fe_convect_geometry_fusable(gm)) {
            // stale float32-only deferred handle: the matrix kernel computes it
            e = fe_launch_convect_matrix_geometry(gm, args[form->grad_op], args[form->adv_op], form->wrt_grad,
                                                  form->wrt_adv, K_out, ctx->d_status, s);
            if (e == cudaSuccess) gm->pending = 0;
            return from_cuda(e, "fe_eval_matrix");
        }
        e = settle_geometry(gm, ctx->d_status, s);
        if (e == cudaSuccess)
            e = fe_launch_convect(g, prec == FE_F64, args[form->grad_op], args[form->adv_op], form->wrt_grad,
                                  form->wrt_adv, K_out, nullptr, ctx->d_status, s);
        return from_cuda(e, "fe_eval_matrix");
    }
    if (form->eval || form->kind == FK_DIV || form->kind == FK_CAUCHY) return FE_ERR_INVALID_ARG;  // no unknown
    if (diff_op != form->state_op) return FE_ERR_INVALID_ARG;
    if (form->kind == FK_WDOT || form->kind == FK_STOKES || form->kind == FK_STOKES_T) {
        if (prec != FE_F64 && prec != FE_F32) return FE_ERR_UNSUPPORTED_SPEC;
        e = settle_geometry(gm, ctx->d_status, s);
        if (e == cudaSuccess)
            e = fe_launch_generic(g, form, mat, prec == FE_F64, 1, nullptr, nullptr, nullptr, K_out, ctx->d_status,
                                  s);
        return from_cuda(e, "fe_eval_matrix");
    }
    if (prec == FE_F64 || prec == FE_F32) {
        e = settle_geometry(gm, ctx->d_status, s);
        if (e == cudaSuccess) e = fe_launch_matrix_simt(g, form, mat, prec == FE_F64, K_out, ctx->sm_count, s);
    } else {
        // tensor-core kernels: 27-node hexahedra with 27 points (Lame elasticity, the
        // scalar Laplacian); 64-node hexahedra with 64 points (TF32x3: Lame elasticity,
        // the scalar Laplacian, the scalar mass matrix); 20-node tetrahedra with the
        // 35-point rule (TF32x3: Lame elasticity, the scalar Laplacian)
        if (!fe_matrix_tc_supported(g, form, prec)) return FE_ERR_UNSUPPORTED_SPEC;
        // elasticity on a stale float32-only deferred handle: the tensor-core kernel
        // computes the FP64 geometry of its elements itself and stores the float32 copy
        const bool fused = form->kind == FK_ELASTICITY && fe_matrix_tc_geometry_fusable(gm);
        e = fused ? cudaSuccess : settle_geometry(gm, ctx->d_status, s);
        // the wait test hook acts on the 27-node kernel; it stays armed across the others
        const bool holdable = g->N == 27;
        const int *hold = holdable && ctx->hold_next_matrix ? ctx->d_hold : nullptr;
        if (holdable) ctx->hold_next_matrix = 0;
        if (e == cudaSuccess)
            e = fe_launch_matrix_tc(g, form, mat, prec, K_out, ctx->sm_count, ctx->d_status, hold, fused, s);
        if (fused && e == cudaSuccess) gm->pending = 0;
    }
    return from_cuda(e, "fe_eval_matrix");
}

fe_status fe_eval_residual(fe_ctx *ctx, const fe_form_h *form, const fe_geometry_h *g, const void *const *args,
                           fe_precision prec, void *r_out, fe_stream_t stream)
{
    fe_clear_last_error();
    fe_material_args mat{};
    fe_status st = eval_common(ctx, form, g, args, prec, r_out, &mat);
    if (st) return st;
    if (form->eval || form->kind == FK_CAUCHY) return FE_ERR_INVALID_ARG;  // no test function
    if (form->kind == FK_WDOT || form->kind == FK_STOKES || form->kind == FK_STOKES_T || form->kind == FK_DIV) {
        const bool empty = g->mesh.n_elems == 0;
        const void *u = form->op_b >= 0 && args ? args[form->op_b] : nullptr;
        if (form->kind != FK_DIV && !empty && !u) return FE_ERR_INVALID_ARG;
        cudaStream_t s = to_cuda(stream);
        cudaError_t e = settle_geometry(const_cast<fe_geometry_h *>(g), ctx->d_status, s);
        if (e == cudaSuccess)
            e = fe_launch_generic(g, form, mat, prec == FE_F64, 0, nullptr, u, nullptr, r_out, ctx->d_status, s);
        return from_cuda(e, "fe_eval_residual");
    }
    if (form->kind == FK_CONVECT) {
        if (!fe_convect_supported(g)) return FE_ERR_UNSUPPORTED_SPEC;
        const bool empty = g->mesh.n_elems == 0;
        if (!args || (!empty && (!args[form->grad_op] || !args[form->adv_op]))) return FE_ERR_INVALID_ARG;
        cudaStream_t s = to_cuda(stream);
        fe_geometry_h *gm = const_cast<fe_geometry_h *>(g);
        if (gm->pending && prec != FE_F64 && fe_convect_geometry_fusable(gm)) {
            // stale float32-only deferred handle: the residual kernel computes it
            cudaError_t e = fe_launch_convect_residual_geometry(gm, args[form->grad_op], args[form->adv_op], r_out,
                                                                ctx->d_status, s);
            if (e == cudaSuccess) gm->pending = 0;
            return from_cuda(e, "fe_eval_residual");
        }
        cudaError_t e = settle_geometry(gm, ctx->d_status, s);
        if (e == cudaSuccess)
            e = fe_launch_convect(g, prec == FE_F64, args[form->grad_op], args[form->adv_op], 0, 0, nullptr, r_out,
                                  ctx->d_status, s);
        return from_cuda(e, "fe_eval_residual");
    }
    if (!args || (!args[form->state_op] && g->mesh.n_elems > 0)) return FE_ERR_INVALID_ARG;
    fe_geometry_h *gm = const_cast<fe_geometry_h *>(g);
    cudaError_t e;
    if (gm->pending && prec != FE_F64 && fe_residual_geometry_fusable(gm, form)) {  // float32 residual kernels
        // a stale deferred handle that keeps only the float32 copy: the residual
        // kernel computes the FP64 geometry of its elements and stores the copy
        e = fe_launch_residual_geometry(gm, form, mat, args[form->state_op], r_out, ctx->d_status, to_cuda(stream));
        if (e == cudaSuccess) gm->pending = 0;
        return from_cuda(e, "fe_eval_residual");
    }
    e = settle_geometry(gm, ctx->d_status, to_cuda(stream));
    if (e == cudaSuccess) e = fe_launch_residual(g, form, mat, prec == FE_F64, args[form->state_op], r_out, ctx->d_status,
                                       to_cuda(stream));
    return from_cuda(e, "fe_eval_residual");
}

fe_status fe_field_create(fe_ctx *ctx, const fe_geometry_h *g, const double *psi, int n_basis, const int32_t *conn,
                          long long n_nodes, fe_field_h **out)
{
    fe_clear_last_error();
    if (!ctx || !g || !psi || !out || (!conn && g->mesh.n_elems > 0)) return FE_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_basis < 1 || n_basis > 64 || n_nodes < 0 || n_nodes > INT_MAX ||
        g->mesh.n_elems * (long long)n_basis > INT_MAX)
        return FE_ERR_SHAPE;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return from_cuda(e, "fe_field_create");
    fe_field_h *f = new (std::nothrow) fe_field_h();
    if (!f) return FE_ERR_OOM;
    f->device = ctx->device;
    f->n_elems = g->mesh.n_elems;
    f->n_basis = n_basis;
    f->Q = g->Q;
    f->n_nodes = n_nodes;
    f->conn = conn;
    const size_t n = (size_t)g->Q * n_basis;
    std::vector<float> psi32(n);
    for (size_t k = 0; k < n; ++k) psi32[k] = (float)psi[k];
    e = dev_alloc(&f->d_psi64, n);
    if (e == cudaSuccess) e = dev_alloc(&f->d_psi32, n);
    if (e == cudaSuccess) e = cudaMemcpy(f->d_psi64, psi, sizeof(double) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(f->d_psi32, psi32.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(f->d_psi64);
        cudaFree(f->d_psi32);
        delete f;
        return from_cuda(e, "fe_field_create");
    }
    *out = f;
    return FE_OK;
}

fe_status fe_field_free(fe_field_h *f)
{
    fe_clear_last_error();
    if (!f) return FE_ERR_INVALID_ARG;
    cudaSetDevice(f->device);
    cudaFree(f->d_psi64);
    cudaFree(f->d_psi32);
    delete f;
    return FE_OK;
}

// The Stokes coupling with its scalar operand on a second field: checks shared by
// matrix and residual mode.
static fe_status mixed_common(fe_ctx *ctx, const fe_form_h *form, const fe_geometry_h *g, const fe_field_h *f,
                              fe_precision prec, void *out)
{
    fe_material_args mat{};
    fe_status st = eval_common(ctx, form, g, nullptr, prec, out, &mat);
    if (st) return st;
    if (!f) return FE_ERR_INVALID_ARG;
    if (form->kind != FK_STOKES && form->kind != FK_STOKES_T) return FE_ERR_UNSUPPORTED_SPEC;
    if (form->eval) return FE_ERR_INVALID_ARG;
    if (f->n_elems != g->mesh.n_elems || f->Q != g->Q) return FE_ERR_SHAPE;
    return FE_OK;
}

fe_status fe_eval_matrix_mixed(fe_ctx *ctx, const fe_form_h *form, const fe_geometry_h *g, const fe_field_h *f,
                               const void *const *args, int diff_op, fe_precision prec, void *K_out,
                               fe_stream_t stream)
{
    fe_clear_last_error();
    (void)args;
    fe_status st = mixed_common(ctx, form, g, f, prec, K_out);
    if (st) return st;
    if (diff_op != form->state_op) return FE_ERR_INVALID_ARG;
    if (prec != FE_F64 && prec != FE_F32) return FE_ERR_UNSUPPORTED_SPEC;
    cudaStream_t s = to_cuda(stream);
    cudaError_t e = settle_geometry(const_cast<fe_geometry_h *>(g), ctx->d_status, s);
    if (e == cudaSuccess)
        e = fe_launch_stokes_mixed(g, f, prec == FE_F64, form->kind == FK_STOKES_T, 1, nullptr, K_out, ctx->d_status,
                                   s);
    return from_cuda(e, "fe_eval_matrix_mixed");
}

fe_status fe_eval_residual_mixed(fe_ctx *ctx, const fe_form_h *form, const fe_geometry_h *g, const fe_field_h *f,
                                 const void *const *args, fe_precision prec, void *r_out, fe_stream_t stream)
{
    fe_clear_last_error();
    fe_status st = mixed_common(ctx, form, g, f, prec, r_out);
    if (st) return st;
    if (!args || (!args[form->state_op] && g->mesh.n_elems > 0)) return FE_ERR_INVALID_ARG;
    cudaStream_t s = to_cuda(stream);
    cudaError_t e = settle_geometry(const_cast<fe_geometry_h *>(g), ctx->d_status, s);
    if (e == cudaSuccess)
        e = fe_launch_stokes_mixed(g, f, prec == FE_F64, form->kind == FK_STOKES_T, 0, args[form->state_op], r_out,
                                   ctx->d_status, s);
    return from_cuda(e, "fe_eval_residual_mixed");
}

fe_status fe_eval_integral(fe_ctx *ctx, const fe_form_h *form, const fe_geometry_h *g, const void *const *args,
                           fe_precision prec, void *out, fe_stream_t stream)
{
    fe_clear_last_error();
    fe_material_args mat{};
    fe_status st = eval_common(ctx, form, g, args, prec, out, &mat);
    if (st) return st;
    if (!form->eval) return FE_ERR_INVALID_ARG;
    const bool empty = g->mesh.n_elems == 0;
    // fields in the kernel's slots; for the convective form the gradient and
    // the advection operands
    const int ob = form->kind == FK_CONVECT ? form->grad_op : form->op_b;
    const int oc = form->kind == FK_CONVECT ? form->adv_op : form->op_c;
    const void *f0 = args ? args[form->op_a] : nullptr;
    const void *f1 = ob >= 0 && args ? args[ob] : nullptr;
    const void *f2 = oc >= 0 && args ? args[oc] : nullptr;
    if (!empty && (!f0 || (ob >= 0 && !f1) || (oc >= 0 && !f2))) return FE_ERR_INVALID_ARG;
    cudaStream_t s = to_cuda(stream);
    cudaError_t e = settle_geometry(const_cast<fe_geometry_h *>(g), ctx->d_status, s);
    if (e == cudaSuccess) e = fe_launch_generic(g, form, mat, prec == FE_F64, 2, f0, f1, f2, out, ctx->d_status, s);
    return from_cuda(e, "fe_eval_integral");
}

fe_status fe_eval_residual_adjoint(fe_ctx *ctx, const fe_form_h *form, const fe_geometry_h *g,
                                   const void *const *args, const void *rbar, fe_precision prec, void *d_mat,
                                   void *d_x_e, fe_stream_t stream)
{
    fe_clear_last_error();
    fe_material_args mat{};
    const bool empty = g && g->mesh.n_elems == 0;
    if (!d_mat && !d_x_e && !empty) return FE_ERR_INVALID_ARG;
    fe_status st = eval_common(ctx, form, g, args, prec, d_mat ? d_mat : d_x_e, &mat);
    if (st) return st;
    if (form->kind != FK_ELASTICITY || form->mat != FE_MAT_LAME || form->mat_transposed)
        return FE_ERR_UNSUPPORTED_SPEC;
    if (prec != FE_F64 && prec != FE_F32) return FE_ERR_UNSUPPORTED_SPEC;
    if (!fe_convect_supported(g)) return FE_ERR_UNSUPPORTED_SPEC;  // same sum-factorised (n1d, nq1d) set
    if (!empty && (!args[form->state_op] || !rbar)) return FE_ERR_INVALID_ARG;
    cudaStream_t s = to_cuda(stream);
    cudaError_t e = settle_geometry(const_cast<fe_geometry_h *>(g), ctx->d_status, s);
    if (e == cudaSuccess)
        e = fe_launch_adjoint(g, prec == FE_F64, mat.data, args[form->state_op], rbar, d_mat, d_x_e, ctx->d_status,
                              s);
    return from_cuda(e, "fe_eval_residual_adjoint");
}

// ---- assembly -----------------------------------------------------------------------

fe_status fe_assembly_create(fe_ctx *ctx, const fe_mesh *mesh, fe_assembly_h **out, fe_stream_t stream)
{
    fe_clear_last_error();
    if (!ctx || !out || !valid_mesh(mesh)) return FE_ERR_INVALID_ARG;
    *out = nullptr;
    cudaSetDevice(ctx->device);
    cudaStream_t s = to_cuda(stream);
    fe_assembly_h *a = new (std::nothrow) fe_assembly_h();
    if (!a) return FE_ERR_OOM;
    a->device = ctx->device;
    a->mesh = *mesh;
    int *d_flag = nullptr;
    cudaError_t e = dev_alloc(&a->d_offsets, (size_t)mesh->n_nodes + 1);
    if (e == cudaSuccess) e = dev_alloc(&a->d_entries, (size_t)(mesh->n_elems * mesh->nodes_per_elem));
    if (e == cudaSuccess) e = dev_alloc(&d_flag, 1);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_flag, 0, sizeof(int), s);
    if (e == cudaSuccess) e = fe_launch_assembly_build(a, d_flag, s);
    int flag = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_flag);
    if (e != cudaSuccess || flag) {
        fe_status st = e != cudaSuccess ? from_cuda(e, "fe_assembly_create") : FE_ERR_SHAPE;
        if (flag) std::snprintf(g_last_error, sizeof(g_last_error), "fe_assembly_create: node index out of range");
        cudaFree(a->d_offsets);
        cudaFree(a->d_entries);
        delete a;
        return st;
    }
    *out = a;
    return FE_OK;
}

fe_status fe_assembly_free(fe_assembly_h *a)
{
    fe_clear_last_error();
    if (!a) return FE_ERR_INVALID_ARG;
    cudaSetDevice(a->device);
    cudaFree(a->d_offsets);
    cudaFree(a->d_entries);
    delete a;
    return FE_OK;
}

fe_status fe_assemble_vector(fe_ctx *ctx, const fe_assembly_h *a, int ncomp, const void *r_e, fe_precision prec,
                             void *global_out, unsigned flags, fe_stream_t stream)
{
    fe_clear_last_error();
    if (!ctx || !a || (ncomp != 1 && ncomp != 3)) return FE_ERR_INVALID_ARG;
    if ((!r_e && a->mesh.n_elems > 0) || (!global_out && a->mesh.n_nodes > 0)) return FE_ERR_INVALID_ARG;
    if (flags & ~(FE_ASSEMBLE_ACCUMULATE | FE_ASSEMBLE_COMPENSATED)) return FE_ERR_INVALID_ARG;
    if (prec < FE_F64 || prec > FE_BF16) return FE_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    return from_cuda(fe_launch_assemble(a, ncomp, prec == FE_F64, r_e, global_out, flags, to_cuda(stream)),
                     "fe_assemble_vector");
}

fe_status fe_debug_hold_next_matrix(fe_ctx *ctx)
{
    fe_clear_last_error();
    if (!ctx) return FE_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    if (!ctx->d_hold) {
        cudaError_t e = dev_alloc(&ctx->d_hold, 1);
        if (e == cudaSuccess) e = cudaMemset(ctx->d_hold, 0, sizeof(int));
        if (e != cudaSuccess) return from_cuda(e, "fe_debug_hold_next_matrix");
    }
    ctx->hold_next_matrix = 1;
    return FE_OK;
}

fe_status fe_diag_fp64(fe_ctx *ctx, int kind, int warps, int ilp, int steps, double *out, fe_stream_t stream)
{
    fe_clear_last_error();
    if (!ctx || !out || (kind != 0 && kind != 1) || warps < 1 || warps > 32 || steps < 1 ||
        (ilp != 1 && ilp != 2 && ilp != 4))
        return FE_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) e = fe_launch_diag_fp64(kind, ctx->sm_count, warps, ilp, steps, out, to_cuda(stream));
    return from_cuda(e, "fe_diag_fp64");
}

fe_status fe_round_f32(fe_ctx *ctx, const double *in, float *out, long long n, fe_stream_t stream)
{
    fe_clear_last_error();
    if (!ctx || n < 0 || (n > 0 && (!in || !out))) return FE_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    return from_cuda(fe_launch_round_f32(in, out, n, to_cuda(stream)), "fe_round_f32");
}

fe_status fe_assemble_vector_noalloc(fe_ctx *ctx, const fe_mesh *mesh, int ncomp, const void *r_e,
                                     fe_precision prec, void *global_out, unsigned flags, fe_stream_t stream)
{
    fe_clear_last_error();
    if (!ctx || !valid_mesh(mesh) || (ncomp != 1 && ncomp != 3)) return FE_ERR_INVALID_ARG;
    if ((!r_e && mesh->n_elems > 0) || (!global_out && mesh->n_nodes > 0)) return FE_ERR_INVALID_ARG;
    if (flags & ~(FE_ASSEMBLE_ACCUMULATE | FE_ASSEMBLE_COMPENSATED)) return FE_ERR_INVALID_ARG;
    if (prec < FE_F64 || prec > FE_BF16) return FE_ERR_INVALID_ARG;
    if (fe_noalloc_limits(mesh->n_nodes, mesh->n_elems * (long long)mesh->nodes_per_elem) != cudaSuccess) {
        std::snprintf(g_last_error, sizeof(g_last_error),
                      "fe_assemble_vector_noalloc: at most %d nodes and %d element-node incidences", 1 << 19,
                      1 << 21);
        return FE_ERR_SHAPE;
    }
    cudaError_t dev_err = cudaSetDevice(ctx->device);
    if (dev_err != cudaSuccess) return from_cuda(dev_err, "fe_assemble_vector_noalloc");
    return from_cuda(fe_launch_assemble_noalloc(ctx->device, mesh, ncomp, prec == FE_F64, r_e, global_out, flags,
                                                ctx->d_status, to_cuda(stream)),
                     "fe_assemble_vector_noalloc");
}

}  // extern "C"
