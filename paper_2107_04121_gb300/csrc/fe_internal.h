// Internal declarations of libfe: handle layouts, kernel launchers, status word.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fe.h"

// ---------------------------------------------------------------------------
// Device status word: [0] first error code (0 = none), [1] smallest offending
// element index (ULLONG_MAX = none).  Kernels only ever atomically lower or
// set it; fe_get_status reads and resets it.
struct fe_ctx {
    int device;
    int sm_count;
    unsigned long long *d_status;  // 2 words
    int *d_hold;                   // test hook: a device flag that nothing sets (fe_debug_hold_next_matrix)
    int hold_next_matrix;          // the next tensor-core matrix launch waits on d_hold
};

// Geometry handle: FP64-derived reference-mapping data, element-outermost so
// that a CTA working on consecutive elements reads one contiguous block.
struct fe_geometry_h {
    int device;
    fe_mesh mesh;  // borrowed device pointers
    int N, Q;
    unsigned flags;
    double *d_phi64, *d_dphi64, *d_w64;  // (Q,N), (Q,3,N), (Q)
    int n1d, nq1d;                       // tensor-product factors (sum-factorised geometry)
    double *d_b1d, *d_d1d;               // (nq1d, n1d) each, or null
    float *d_b1d32, *d_d1d32;
    double *d_dq;  // (nq1d, nq1d) collocation derivative on the points when n1d == nq1d, or null
    int geo_center;  // n1d == nq1d == 3 with the middle point on the middle node (see geometry_body.cuh)
    float *d_phi32, *d_dphi32;
    double *d_jinv64, *d_wdetj64;  // (E,Q,3,3), (E,Q)
    float *d_jinv32, *d_wdetj32;
    int pending;  // deferred handle: the stored geometry is stale (host-side, stream-ordered use)
    // float32-only handle whose basis is the library's order-p tetrahedron basis:
    // straight-sided elements take J from their vertices (k_geometry_simplex)
    int simplex_p;
    double *d_xi;  // (N, 3) reference positions of the nodes (lattice points / p)
    int is_view;  // aliases a parent's storage for a range of its elements (owns nothing)
    // quadrature points ordered by the sign of their weight (positive first), for the
    // tensor-core kernels of rules with negative weights: counts and the point of each
    // slot of a K dimension padded to 8 per sign group (-1: padding)
    int n_wpos, n_wneg;
    signed char slot_q[64];
};

enum fe_form_kind {
    FK_LAPLACE = 0,
    FK_MASS = 1,
    FK_ELASTICITY = 2,
    FK_CONVECT = 3,
    FK_WDOT = 4,      // 'ij,i,j'
    FK_STOKES = 5,    // 'i.i,0' with the vector test function
    FK_STOKES_T = 6,  // 'i.i,0' with the scalar test function
    FK_DIV = 7,       // 'i.i'
    FK_CAUCHY = 8     // 'IK,s(k:l)->K', eval only
};

struct fe_form_h {
    fe_form_kind kind;
    int ncomp;       // components of the field operands
    int n_ops;
    int virtual_op;  // operand index of the test function
    int state_op;    // operand index of the unknown
    int mat_op;      // operand index of the material, -1 if none
    fe_material_kind mat;
    int mat_transposed;  // elasticity: material indices given as (u-index, v-index)
    // convective term 'i,i.j,j': operand of the gradient (u) and of the advection
    // velocity (w); the matrix is the derivative with respect to every FE_STATE
    // operand among them (both for the non-linear term, Eq. fe4)
    int grad_op, adv_op;
    int wrt_grad, wrt_adv;
    // 'eval' form (no test function): the first field plays the test slot;
    // field operand indices in expression order (test slot, unknown, third)
    int eval;
    int op_a, op_b, op_c;
    int ncomp_test, ncomp_trial;  // rows / columns of one element matrix per node
    int n_out;                    // values per element in eval mode
};

// A scalar field on a second basis over the elements of a geometry (the second
// field of a mixed-order pair): its reference values at the geometry's points
// and its borrowed connectivity.
struct fe_field_h {
    int device;
    long long n_elems;
    int n_basis, Q;
    long long n_nodes;
    const int32_t *conn;  // (n_elems, n_basis), borrowed
    double *d_psi64;      // (Q, n_basis)
    float *d_psi32;
};

struct fe_assembly_h {
    int device;
    fe_mesh mesh;
    int *d_offsets;  // (n_nodes + 1)
    int *d_entries;  // (n_elems * N): e * N + a, ascending per node
};

// Materials handed to the kernels: always float64 device arrays.
struct fe_material_args {
    fe_material_kind kind;
    const double *data;
    int transposed;
};

// ---------------------------------------------------------------------------
// Launchers (return cudaError_t of the launch; argument checks done by the API).
cudaError_t fe_launch_geometry(const fe_geometry_h *g, unsigned long long *d_status, cudaStream_t s);
cudaError_t fe_launch_geometry_G(const fe_geometry_h *g, bool f64, void *out, cudaStream_t s);
// Matrix mode on the CUDA cores (FP32 or FP64) for the (N, Q) pairs of fe_supported_nq.
cudaError_t fe_launch_matrix_simt(const fe_geometry_h *g, const fe_form_h *f, fe_material_args mat, bool f64,
                                  void *K, int sm_count, cudaStream_t s);
// Lame elasticity (lame: lambda, mu per element) and the weighted scalar Laplacian
// (coef per element, 1 where NULL) of the same FP32 geometry from one set of Gram
// blocks on the CUDA cores: K (E, 3N, 3N) and K2 (E, N, N), float32.
bool fe_matrix_pair_supported(const fe_geometry_h *g);
cudaError_t fe_launch_matrix_pair(const fe_geometry_h *g, const double *lame, void *K, const double *coef, void *K2,
                                  int sm_count, cudaStream_t s);
// The same pair on the tensor cores (TF32x3; 27-node hexahedra with 27 points in
// k_matrix_tc.cu, 64-node hexahedra with 64 points in k_matrix_tc64.cu).
bool fe_matrix_tc_pair_supported(const fe_geometry_h *g);
cudaError_t fe_launch_matrix_tc_pair(const fe_geometry_h *g, const double *lame, void *K, const double *coef,
                                     void *K2, int sm_count, unsigned long long *status, cudaStream_t s);
bool fe_matrix_tc64_pair_supported(const fe_geometry_h *g);
cudaError_t fe_launch_matrix_tc64_pair(const fe_geometry_h *g, const double *lame, void *K, const double *coef,
                                       void *K2, int sm_count, unsigned long long *status, cudaStream_t s);
cudaError_t fe_launch_matrix(const fe_geometry_h *g, const fe_form_h *f, fe_material_args mat, fe_precision prec,
                             void *K, int sm_count, cudaStream_t s);
// Matrix mode on the tensor cores (k_matrix_tc.cu): Lame elasticity, 27 nodes, 27
// points; with_geometry: a stale float32-only deferred handle computed in the launch.
cudaError_t fe_launch_matrix_tc(const fe_geometry_h *g, const fe_form_h *f, fe_material_args mat, fe_precision prec,
                                void *K, int sm_count, unsigned long long *status, const int *hold,
                                bool with_geometry, cudaStream_t s);
// Whether a tensor-core matrix kernel covers the form on these elements in this
// precision (27-node hexahedra with 27 points: Lame elasticity, the scalar
// Laplacian; 64-node hexahedra with 64 points, TF32x3: Lame elasticity, the
// scalar Laplacian and the scalar mass matrix; P3 tetrahedra with 35 points,
// TF32x3: Lame elasticity and the scalar Laplacian).
bool fe_matrix_tc_supported(const fe_geometry_h *g, const fe_form_h *f, fe_precision prec);
cudaError_t fe_launch_matrix_tcs(const fe_geometry_h *g, const fe_form_h *f, fe_material_args mat,
                                 fe_precision prec, void *K, int sm_count, unsigned long long *status,
                                 cudaStream_t s);
bool fe_matrix_tcs_supported(const fe_geometry_h *g, const fe_form_h *f, fe_precision prec);
cudaError_t fe_launch_matrix_tc64(const fe_geometry_h *g, const fe_form_h *f, fe_material_args mat,
                                  fe_precision prec, void *K, int sm_count, unsigned long long *status,
                                  cudaStream_t s);
bool fe_matrix_tc_geometry_fusable(const fe_geometry_h *g);
cudaError_t fe_launch_residual(const fe_geometry_h *g, const fe_form_h *f, fe_material_args mat, bool f64,
                               const void *u, void *r, unsigned long long *status, cudaStream_t s);
// Residual of a stale float32-only deferred geometry with the geometry computed
// in the same kernel (tensor-product bases with n1 == nq); stores the float32
// copy of the handle.
bool fe_residual_geometry_fusable(const fe_geometry_h *g, const fe_form_h *f);
cudaError_t fe_launch_residual_geometry(fe_geometry_h *g, const fe_form_h *f, fe_material_args mat, const void *u,
                                        void *r, unsigned long long *st, cudaStream_t s);
// Convective term on tensor-product hexahedra (sum factorisation): residual
// (K == nullptr) or matrix (r == nullptr) of 'i,i.j,j' with gradient operand u
// and advection operand w (global DOF vectors, 3 per node).
cudaError_t fe_launch_convect(const fe_geometry_h *g, bool f64, const void *u, const void *w, int wrt_grad,
                              int wrt_adv, void *K, void *r, unsigned long long *status, cudaStream_t s);
bool fe_convect_supported(const fe_geometry_h *g);
// Convective residual of a stale float32-only deferred geometry with the
// geometry computed in the same kernel (n1 == nq); stores the float32 copy.
bool fe_convect_geometry_fusable(const fe_geometry_h *g);
cudaError_t fe_launch_convect_residual_geometry(const fe_geometry_h *g, const void *u, const void *w, void *r,
                                                unsigned long long *status, cudaStream_t s);
// The same for the convective matrix (Eq. fe4): the FP32 matrix kernel of a stale
// float32-only deferred geometry computes it first and stores the float32 copy.
cudaError_t fe_launch_convect_matrix_geometry(const fe_geometry_h *g, const void *u, const void *w, int wrt_grad,
                                              int wrt_adv, void *K, unsigned long long *status, cudaStream_t s);
// Generic kernels (runtime N, Q) of the remaining forms and of eval mode:
// mode 0 residual (out (E, ncomp_test N)), 1 matrix (out (E, rows, cols)),
// 2 eval (out (E, n_out)).  f0, f1, f2: the DOF vectors of the form's field
// operands op_a, op_b, op_c (null where absent).
cudaError_t fe_launch_generic(const fe_geometry_h *g, const fe_form_h *f, fe_material_args mat, bool f64, int mode,
                              const void *f0, const void *f1, const void *f2, void *out, unsigned long long *status,
                              cudaStream_t s);
// Adjoint of the isotropic elasticity residual (sum factorisation, same (n1d,
// nq1d) pairs as the convective kernels): d(rbar . R)/d(lambda_e, mu_e) into
// dmat (E, 2) and per-element coordinate derivatives into dxe (E, 3 N); either
// may be null.
cudaError_t fe_launch_adjoint(const fe_geometry_h *g, bool f64, const double *lame, const void *u,
                              const void *rbar, void *dmat, void *dxe, unsigned long long *status, cudaStream_t s);
// Stokes coupling with its scalar operand on `f` (k_mixed.cu): transposed = the
// scalar field is the test field; mode 0 residual (field = p, or u for the
// transposed coupling), 1 matrix.
cudaError_t fe_launch_stokes_mixed(const fe_geometry_h *g, const fe_field_h *f, bool f64, bool transposed, int mode,
                                   const void *field, void *out, unsigned long long *status, cudaStream_t s);
cudaError_t fe_launch_assembly_build(fe_assembly_h *a, int *d_flag, cudaStream_t s);
cudaError_t fe_launch_assemble(const fe_assembly_h *a, int ncomp, bool f64, const void *r, void *out,
                               unsigned flags, cudaStream_t s);

cudaError_t fe_noalloc_limits(long long n_nodes, long long n_incidences);
cudaError_t fe_launch_assemble_noalloc(int device, const fe_mesh *mesh, int ncomp, bool f64, const void *r,
                                       void *out, unsigned flags, unsigned long long *status, cudaStream_t s);

// Status of a CUDA error, recorded as the thread's last error message (api.cu).
fe_status fe_status_from_cuda(cudaError_t e, const char *where);
// FP64 rate diagnostic (k_diag.cu): kind 0 DFMA chains, 1 FP64 MMA chains.
cudaError_t fe_launch_diag_fp64(int kind, int sms, int warps, int ilp, int steps, double *out, cudaStream_t s);
// The float64 -> float32 rounding of the geometry kernels over an array (k_geometry.cu).
cudaError_t fe_launch_round_f32(const double *in, float *out, long long n, cudaStream_t s);

// Every fe_status entry point starts with this: the message of
// fe_last_error_message then always belongs to the latest call (api.cu).
void fe_clear_last_error();
// Settle a deferred geometry (api.cu): compute it now if it is stale.
cudaError_t fe_settle_geometry(fe_geometry_h *g, unsigned long long *status, cudaStream_t s);

// The order p (1..3) when phi (Q, N) is the library's order-p tetrahedron basis at
// a Grundmann-Moller rule (fe_refbasis_tet), else 0 (refelem.cpp); xi (N, 3)
// receives its node positions.
int fe_host_simplex_order(int N, int Q, const double *phi, double *xi);
// Which (N, Q) pairs have kernels.
bool fe_supported_nq(int N, int Q);

// Host reference element (refelem.cpp).
int fe_host_gauss_legendre01(int n, double *x, double *w);
bool fe_host_check_tensor_basis(const fe_refbasis *b);
bool fe_host_collocation_derivative(int n, const double *b1d, const double *d1d, double *dq);
