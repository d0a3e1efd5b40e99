/*
 * fe.h - C ABI of the GB300 finite element weak-form evaluator (libfe.so).
 *
 * The library evaluates multilinear finite element weak forms element by
 * element on one GPU, following Cimrman, "Fast Evaluation of Finite Element
 * Weak Forms Using Python Tensor Contraction Packages" (arXiv 2107.04121):
 *
 *   fe_geometry         reference mapping J, det J, J^-1 per element and
 *                       quadrature point (Sec. 4.1; operand "v.det" and the
 *                       gradients "bfg" of Tab. suee)
 *   fe_form_compile     a weak form written in the generalized einsum notation
 *                       (Tab. wfc, examples in Tab. ewfd) compiled to a kernel
 *                       plan, cached in a handle (Algorithm 3, "transpile")
 *   fe_eval_matrix      element matrices M[c, :, :] (Algorithm 2, "matrix" mode)
 *   fe_eval_residual    element residuals r[c, :] (Algorithm 1, "residual" mode)
 *   fe_assemble_vector  optional scatter-add of element vectors into a global
 *                       vector (the assembly step that Sec. 6 leaves untimed)
 *
 * General conventions
 *  - Every array argument is caller-owned memory; the library never frees it.
 *    "device" arrays must be CUDA device memory of the context's device;
 *    "host" arrays are ordinary host memory.  All arrays are C row-major and
 *    contiguous.
 *  - Handles returned through an out-pointer are owned by the caller and are
 *    released with the matching *_free / fe_destroy call.
 *  - Calls that take a cudaStream_t are asynchronous on that stream (0 = the
 *    legacy default stream).  Argument, shape and expression errors are
 *    detected on the host and returned synchronously; nothing is launched then.
 *  - Problems found on the device (det J <= 0, a non-finite geometry value)
 *    are recorded in a device status word of the context and reported by
 *    fe_get_status.  No call aborts, traps or throws across the ABI.
 *  - Reference hexahedron [0,1]^3.  Order-p Lagrange nodes are equispaced and
 *    numbered lexicographically with x fastest: node (i,j,k) is
 *    i + (p+1) j + (p+1)^2 k.  Quadrature points use the same order.
 *  - Vector element DOFs are component-major: local row/column index
 *    comp * n_basis + node (the "cresf" output order of Sec. 5.3.3, eq. fe1b).
 *    Global DOF vectors are node-major: index ncomp * node + comp.
 *  - Symmetric tensors use Voigt order (11, 22, 33, 12, 13, 23) with
 *    engineering shear strains (the "s(i:j)->I" storage of Tab. wfc).
 */
#ifndef FE_H
#define FE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* cudaStream_t without pulling in the CUDA headers. */
typedef struct CUstream_st *fe_stream_t;

typedef enum {
    FE_OK = 0,
    FE_ERR_INVALID_ARG = 1,      /* null pointer, negative size, bad flag */
    FE_ERR_SHAPE = 2,            /* sizes that do not fit together or are not supported */
    FE_ERR_UNSUPPORTED_SPEC = 3, /* expression outside the implemented set of forms */
    FE_ERR_NONPOSITIVE_DETJ = 4, /* device: det J <= 0 in some element */
    FE_ERR_NONFINITE = 5,        /* device: a non-finite geometry value */
    FE_ERR_OOM = 6,              /* device allocation failed */
    FE_ERR_CUDA = 7,             /* other CUDA runtime error */
    FE_ERR_TIMEOUT = 8           /* a bounded device wait gave up */
} fe_status;

/* Arithmetic of the contraction.  The geometry (J, det J, J^-1) is always
 * computed in FP64.  FE_F64 takes and returns float64 arrays; every other
 * precision takes float32 DOF vectors and returns float32 element arrays.
 *   FE_F64    FP64 throughout
 *   FE_F32    FP32 FMA contraction of FP64-derived geometry
 *   FE_TF32X3 tensor cores, TF32 operands split hi + lo, three products, FP32 accumulation
 *   FE_BF16X3 tensor cores, BF16 operands split hi + lo, three products, FP32 accumulation
 *   FE_BF16   tensor cores, plain BF16 operands, FP32 accumulation (reported, not recovered) */
typedef enum { FE_F64 = 0, FE_F32 = 1, FE_TF32X3 = 2, FE_BF16X3 = 3, FE_BF16 = 4 } fe_precision;

/* Operand roles of a weak form (Sec. 5.1): test function, unknown field,
 * known field, material data. */
typedef enum { FE_VIRTUAL = 0, FE_STATE = 1, FE_PARAMETER = 2, FE_MATERIAL = 3 } fe_role;

/* Layout of a material operand (device float64 array, "cq0" layout of Tab. mls
 * with a constant q axis):
 *   FE_MAT_SCALAR  (n_elems)       one coefficient per element
 *   FE_MAT_LAME    (n_elems, 2)    Lame pair (lambda, mu) per element; the elastic
 *                                  matrix is D = lambda m m^T + mu diag(2,2,2,1,1,1),
 *                                  m = (1,1,1,0,0,0)
 *   FE_MAT_D66     (n_elems, 6, 6) elastic matrix D per element, Voigt order
 *   FE_MAT_M33     (n_elems, 3, 3) matrix M per element, row-major (weighted dot product) */
typedef enum { FE_MAT_NONE = 0, FE_MAT_SCALAR = 1, FE_MAT_LAME = 2, FE_MAT_D66 = 3, FE_MAT_M33 = 4 } fe_material_kind;

typedef struct {
    fe_role role;
    int ncomp;                 /* components of a field operand (1 or 3); ignored for materials */
    fe_material_kind material; /* layout of a material operand; FE_MAT_NONE for fields */
} fe_operand;

/* Mesh: device arrays, caller-owned, valid for as long as any handle made from
 * them is used.  coords (n_nodes, 3) float64; conn (n_elems, nodes_per_elem)
 * int32 indices into coords.  Node indices and the (element, local node)
 * incidences are 32-bit: every call that takes a mesh returns
 * FE_ERR_INVALID_ARG, before any launch, when n_nodes or n_elems *
 * nodes_per_elem exceeds 2^31 - 1.  Element outputs (K, r) are indexed with
 * 64 bits and may hold more than 2^31 entries. */
typedef struct {
    const double *coords;
    long long n_nodes;
    const int32_t *conn;
    long long n_elems;
    int nodes_per_elem;
} fe_mesh;

/* Reference basis tabulated at the quadrature points: host arrays.
 * phi (n_qp, n_basis), dphi (n_qp, 3, n_basis) with dphi[q][k][a] = d phi_a / d xi_k.
 * The same basis maps the geometry and approximates the fields (isoparametric
 * elements, Sec. 4.1 footnote).
 * Optional tensor-product factors (set b1d = d1d = NULL if the basis is not a
 * tensor product): b1d (nq1d, n1d) and d1d (nq1d, n1d) hold the 1-D basis
 * values and derivatives at the 1-D points, with phi[q][a] = b1d[qx][i]
 * b1d[qy][j] b1d[qz][k] for a = i + n1d (j + n1d k), q = qx + nq1d (qy + nq1d qz).
 * When given (and consistent with phi and dphi, which fe_geometry checks), the
 * geometry kernel uses sum factorisation: about 3x fewer FP64 operations for Q2. */
typedef struct {
    int n_basis;
    int n_qp;
    const double *phi;
    const double *dphi;
    int n1d;
    int nq1d;
    const double *b1d;
    const double *d1d;
} fe_refbasis;

/* Quadrature rule on the reference element: host arrays points (n_qp, 3), weights (n_qp). */
typedef struct {
    int n_qp;
    const double *points;
    const double *weights;
} fe_quadrature;

typedef struct fe_ctx fe_ctx;
typedef struct fe_geometry_h fe_geometry_h;
typedef struct fe_form_h fe_form_h;
typedef struct fe_assembly_h fe_assembly_h;
typedef struct fe_batch_h fe_batch_h;
typedef struct fe_field_h fe_field_h;

/* ---- context ------------------------------------------------------------- */

/* Create a context on CUDA device `device` (makes it current for the calling
 * thread).  The context owns a device status word.  Errors: FE_ERR_INVALID_ARG
 * (null out), FE_ERR_CUDA (no such device), FE_ERR_OOM. */
fe_status fe_create(int device, fe_ctx **out);
fe_status fe_destroy(fe_ctx *ctx);

/* Static string naming a status code; never NULL. */
const char *fe_status_str(fe_status s);

/* Wait for `stream`, read and clear the device status word.  Returns FE_OK or
 * the first device-detected error since the last call; *bad_elem (optional)
 * receives the smallest offending element index, or -1. */
fe_status fe_get_status(fe_ctx *ctx, fe_stream_t stream, long long *bad_elem);

/* Diagnostic with no counterpart in the paper: the FP64 rates that decide where
 * the library computes in FP64.  Launches one CTA of `warps` warps (1..32) on
 * every SM of the context's device; each lane runs `ilp` (1, 2 or 4)
 * independent chains of `steps` (>= 1) dependent operations: kind 0 a DFMA
 * (one lane-FMA per lane and step), kind 1 the FP64 tensor-core MMA
 * mma.sync.m8n8k4 (256 FMAs per warp and step).  `out` is a caller-owned
 * device array of (SM count x warps x 32) doubles that keeps the chains alive.
 * The caller times the launch on `stream`.  Errors: FE_ERR_INVALID_ARG. */
fe_status fe_diag_fp64(fe_ctx *ctx, int kind, int warps, int ilp, int steps, double *out, fe_stream_t stream);

/* Library version as major*10000 + minor*100 + patch. */
int fe_version(void);

/* Text that describes the failure of the latest fe_status call on the calling
 * thread: the CUDA error, or the argument or shape problem where the call
 * names one; empty after a call that succeeded or failed without a text.
 * Static thread-local storage; never NULL. */
const char *fe_last_error_message(void);

/* ---- reference element (host) ----------------------------------------------- */

/* Tabulate the order-p Lagrange basis of the reference hexahedron and the
 * tensor-product Gauss-Legendre rule with nq points per axis (Tab. cdc uses
 * nq = p + 1).  Host arrays of sizes points (nq^3, 3), weights (nq^3),
 * phi (nq^3, (p+1)^3), dphi (nq^3, 3, (p+1)^3).  Any output pointer may be
 * NULL.  Supports 1 <= p <= 4, 1 <= nq <= 10; otherwise FE_ERR_SHAPE. */
fe_status fe_refbasis_hex(int p, int nq, double *points, double *weights, double *phi, double *dphi);

/* The 1-D factors of fe_refbasis_hex: host arrays b1d (nq, p+1) with the
 * Lagrange basis values at the Gauss points on [0,1], d1d (nq, p+1) with their
 * derivatives.  Same limits as fe_refbasis_hex. */
fe_status fe_refbasis_hex_1d(int p, int nq, double *b1d, double *d1d);

/* Lagrange basis of order p (1..3) on the reference tetrahedron
 * {x, y, z >= 0, x + y + z <= 1} at the points of the Grundmann-Moller rule of
 * index s (0..6, exact for degree 2s + 1; negative weights occur for s >= 1).
 * Nodes are the lattice points (i, j, k) / p with i + j + k <= p, numbered with
 * x fastest: N = (p+1)(p+2)(p+3)/6 (4, 10, 20).  The basis is the barycentric
 * product prod_m prod_{t < a_m} (p l_m - t) / (t + 1) (l = barycentric
 * coordinates, a = the node's barycentric multi-index).  The rule's points are
 * listed by GM level i and then by composition; its weights sum to the volume
 * 1/6.  Output arrays as fe_refbasis_hex with Q = fe_gm_rule_size(s) points;
 * any may be NULL.  Errors: FE_ERR_SHAPE.  (The rule of index p is the one of
 * "order 2p" for the P_p mixed-mesh workload: 5, 15, 35 points.) */
fe_status fe_refbasis_tet(int p, int s, double *points, double *weights, double *phi, double *dphi);
/* Number of points of the Grundmann-Moller rule of index s (0..6), -1 otherwise. */
int fe_gm_rule_size(int s);

/* ---- geometry ----------------------------------------------------------------- */

/* Storage flags of fe_geometry. */
#define FE_GEOM_STORE_F64 1u /* keep float64 J^-1 and w det J (needed by FE_F64 evaluation) */
#define FE_GEOM_STORE_F32 2u /* keep float32 copies (needed by the other precisions) */
#define FE_GEOM_DEFERRED 4u  /* compute lazily: fe_geometry / fe_geometry_update only mark the
                                geometry stale; the next call that reads it (evaluation or
                                fe_geometry_get) computes it first, on its own stream.  A
                                handle that keeps only the float32 copy (FE_GEOM_STORE_F32)
                                of a tensor-product hexahedron with n1d == nq1d is computed
                                by fe_eval_residual itself (Laplace, mass, elasticity or the
                                convective form, any precision but FE_F64): one kernel for the
                                FP64 geometry, the stored float32 copy and the residual, with
                                the same bits as the separate geometry kernel.  Such a handle of
                                27-node hexahedra with 3 x 3 x 3 Gauss points is also computed
                                by fe_eval_matrix itself in the tensor-core precisions (Lame
                                elasticity): warps of the tensor-core kernel compute the FP64
                                geometry beside the K_e stream and store the float32 copy, same
                                bits again; and by fe_eval_matrix of the convective form in
                                FE_F32 (the matrix kernel runs the geometry stages first, same
                                bits).  A call that reports an error (e.g. FE_ERR_TIMEOUT)
                                leaves the geometry it was computing undefined until the next
                                fe_geometry_update.  The stale mark is host state: use a
                                deferred handle from one stream. */

/* Geometry of the reference mapping (Sec. 4.1): for every element e and
 * quadrature point q, J = sum_a x_a (x) grad_xi phi_a(q), det J, J^-1 and
 * w_q det J, computed in FP64 on the device.  The handle keeps J^-1 (E, Q, 3, 3)
 * and w det J (E, Q) in the precisions `flags` asks for (0 means both) together
 * with device copies of the reference tables; the physical gradients
 * G[e][q][j][a] = sum_k dphi[q][k][a] (J^-1)_kj are formed inside the
 * evaluation kernels.  The mesh arrays are borrowed: they must stay valid while
 * the handle is used.  Supported: hexahedra with n_basis in {8, 27, 64} and
 * n_qp <= 64.  det J <= 0 is recorded in the status word (fe_get_status).
 * Errors: FE_ERR_INVALID_ARG, FE_ERR_SHAPE, FE_ERR_OOM, FE_ERR_CUDA. */
fe_status fe_geometry(fe_ctx *ctx, const fe_mesh *mesh, const fe_refbasis *basis, const fe_quadrature *quad,
                      unsigned flags, fe_geometry_h **out, fe_stream_t stream);
fe_status fe_geometry_free(fe_geometry_h *geom);

/* A handle for the elements [e_begin, e_begin + e_count) of `parent` that
 * aliases its stored geometry (no copy, no allocation of device memory): every
 * evaluation call takes it like any geometry, and fe_geometry_update on it
 * recomputes only its range.  Useful to evaluate a mesh in chunks, e.g. to
 * overlap the transfer of one chunk's element matrices with the evaluation of
 * the next.  The parent must outlive the view and must not be deferred; free
 * the view with fe_geometry_free (which then frees nothing else).  Errors:
 * FE_ERR_INVALID_ARG (range outside the parent, deferred parent), FE_ERR_OOM. */
fe_status fe_geometry_view(fe_ctx *ctx, const fe_geometry_h *parent, long long e_begin, long long e_count,
                           fe_geometry_h **out);

/* Recompute the geometry of `geom` in place from the current contents of its
 * (borrowed) mesh arrays, e.g. after the nodal coordinates moved; no device
 * memory is allocated.  Same kernel and status reporting as fe_geometry.
 * Errors: FE_ERR_INVALID_ARG, FE_ERR_CUDA. */
fe_status fe_geometry_update(fe_ctx *ctx, fe_geometry_h *geom, fe_stream_t stream);

/* What fe_geometry_get copies out. */
typedef enum { FE_GEOM_WDETJ = 0, FE_GEOM_JINV = 1, FE_GEOM_G = 2 } fe_geom_field;

/* Copy a geometry field into the caller's device array: w det J (E, Q),
 * J^-1 (E, Q, 3, 3) or the physical gradients G (E, Q, 3, N), as float64
 * (prec FE_F64) or float32 (any other prec), from the stored copy of that
 * precision.  Errors: FE_ERR_INVALID_ARG (copy not stored, null pointers). */
fe_status fe_geometry_get(fe_ctx *ctx, const fe_geometry_h *geom, fe_geom_field field, fe_precision prec,
                          void *out, fe_stream_t stream);

/* ---- forms ---------------------------------------------------------------------- */

/* Compile a weak form given in the generalized einsum notation of Tab. wfc
 * (symbols 0, i, i.j, i:j, s(i:j)->I), one comma-separated subscript per
 * operand, with the operands' roles and layouts.  Recognised forms (Tab. ewfd;
 * index letters are free, operands may come in any order):
 *   weak Laplacian        "0.i,0.i"                    (VIRTUAL, STATE), ncomp 1
 *   weighted Laplacian    "0,0.i,0.i"                  (MATERIAL SCALAR, VIRTUAL, STATE)
 *   dot product / mass    "i,i" (ncomp 1 or 3), "0,0"  (VIRTUAL, STATE)
 *   weighted mass         "0,i,i", "0,0,0"             (MATERIAL SCALAR, VIRTUAL, STATE)
 *   linear elasticity     "IK,s(i:j)->I,s(k:l)->K"     (MATERIAL LAME or D66, VIRTUAL, STATE), ncomp 3
 *   weighted dot product  "ij,i,j"                     (MATERIAL M33, VIRTUAL, STATE), ncomp 3
 *   Stokes coupling       "i.i,0"                      (VIRTUAL vector, STATE scalar): int div(v) p
 *   transposed coupling   "i.i,0"                      (STATE vector, VIRTUAL scalar): int q div(u)
 *   divergence            "i.i"                        (VIRTUAL vector): int div(v), residual only
 *   Cauchy stress         "IK,s(k:l)->K"               (MATERIAL LAME or D66, field): eval only
 *   Navier-Stokes         "i,i.j,j"                    (VIRTUAL, u, w), ncomp 3: int v_i (du_i/dx_j) w_j
 *   convection (Eq. fe2)  u and w each STATE or PARAMETER (at least one STATE);
 *                         (VIRTUAL, STATE, STATE) is the non-linear term with
 *                         w = u, whose matrix is the two-term derivative of
 *                         Eq. fe4; tensor-product hexahedra only (the basis
 *                         must carry its 1-D factors)
 * Every form may also be compiled with no VIRTUAL operand, all its fields
 * being FE_STATE or FE_PARAMETER: it is then an 'eval' form (Sec. 5.1,
 * evaluation modes) for fe_eval_integral, the first field taking the test
 * function's place.  Stokes coupling and its transpose use one basis for both
 * fields (equal order).
 * `ctx` may be NULL: compilation is host-only.  The handle caches the plan
 * (Sec. 5.1: transpilation results are cached).  Errors: FE_ERR_INVALID_ARG
 * (syntax, roles, sizes), FE_ERR_UNSUPPORTED_SPEC (a valid expression with no
 * kernel). */
fe_status fe_form_compile(fe_ctx *ctx, const char *expr, const fe_operand *ops, int n_ops, fe_form_h **out);
fe_status fe_form_free(fe_form_h *form);

/* Rows and columns of one element matrix (rows: residual length) of `form`
 * for elements of n_basis nodes: the test field's components times n_basis,
 * the unknown's components times n_basis (0 for the divergence form, which
 * has no unknown).  For an eval form: n_rows = values per element (1, or 6 for
 * the Cauchy stress), n_cols = 0. */
fe_status fe_form_shape(const fe_form_h *form, int n_basis, int *n_rows, int *n_cols);

/* args[k] is the device array of operand k of the compiled expression:
 *   FE_VIRTUAL            NULL (the test function is what the rows enumerate)
 *   FE_STATE, FE_PARAMETER global DOF vector (n_nodes * ncomp), float64 for
 *                         FE_F64 else float32; in matrix mode read only by
 *                         forms that are not linear in the state (convection)
 *   FE_MATERIAL           float64 array in the operand's fe_material_kind layout
 */

/* Matrix mode (Algorithm 2): K_out[e][r][c] = derivative of the form with
 * respect to the DOFs of operand `diff_op` (which must be an FE_STATE operand;
 * where several operands are FE_STATE they are one unknown and the derivative
 * sums over them, as Eq. fe4 does for the convective term),
 * integrated with the quadrature of `geom`; K_out is a device array
 * (n_elems, n_rows, n_cols), float64 for FE_F64 else float32.
 * FE_F64 and FE_F32 cover every form and element.  The tensor-core precisions
 * cover: on 27-node hexahedra with 27 points (FE_TF32X3, FE_BF16X3, FE_BF16)
 * linear elasticity with FE_MAT_LAME materials and the (weighted) scalar
 * Laplacian, for elasticity on a stale float32-only deferred handle computing its
 * geometry in the same launch (see FE_GEOM_DEFERRED); on 64-node hexahedra with
 * 64 points (FE_TF32X3) Lame elasticity, the scalar Laplacian and the scalar mass
 * matrix; on 20-node tetrahedra with the 35-point Grundmann-Moller rule
 * (FE_TF32X3) Lame elasticity and the scalar Laplacian.  A tensor-core wait that
 * times out is reported as FE_ERR_TIMEOUT through fe_get_status.
 * Errors: FE_ERR_INVALID_ARG, FE_ERR_SHAPE, FE_ERR_UNSUPPORTED_SPEC (e.g. a
 * precision without a kernel for this form), FE_ERR_CUDA. */
fe_status fe_eval_matrix(fe_ctx *ctx, const fe_form_h *form, const fe_geometry_h *geom, const void *const *args,
                         int diff_op, fe_precision prec, void *K_out, fe_stream_t stream);

/* Residual mode (Algorithm 1): r_out[e][r] = the form's action on the DOF
 * vectors of its FE_STATE and FE_PARAMETER operands, whose element values are gathered through
 * the mesh connectivity; r_out is a device array (n_elems, n_rows), float64
 * for FE_F64 else float32.  FE_TF32X3/FE_BF16X3/FE_BF16 evaluate residuals
 * with the FE_F32 kernels.  Errors as fe_eval_matrix. */
fe_status fe_eval_residual(fe_ctx *ctx, const fe_form_h *form, const fe_geometry_h *geom, const void *const *args,
                           fe_precision prec, void *r_out, fe_stream_t stream);

/* ---- fields of different orders (mixed-order pairs) ------------------------------ */

/* A scalar field on a second basis over the elements of `geom`, for the Stokes
 * coupling "i.i,0" (Tab. ewfd) between fields of different orders, e.g. a Q1
 * pressure beside a Q2 velocity or P1 beside P2 (Taylor-Hood pairs; the
 * coupling of two fields is the Stokes row of Tab. ewfd, and the paper's
 * SfePy setting lets each field carry its own order).
 *   psi      host array (Q, n_basis): the field's reference basis at the
 *            quadrature points of `geom`, in the point order of the rule given to
 *            fe_geometry (e.g. fe_refbasis_hex(1, 3, ...) beside a Q2 basis with
 *            3 x 3 x 3 points; fe_refbasis_tet(1, s, ...) beside P2 with rule s);
 *            copied
 *   conn     device int32 (n_elems of geom, n_basis): the field's DOF numbering
 *            per element, borrowed (must stay valid while the handle is used)
 *   n_nodes  number of the field's DOFs
 * Free with fe_field_free.  Errors: FE_ERR_INVALID_ARG (null arguments),
 * FE_ERR_SHAPE (n_basis outside 1..64, n_nodes out of range), FE_ERR_OOM. */
fe_status fe_field_create(fe_ctx *ctx, const fe_geometry_h *geom, const double *psi, int n_basis,
                          const int32_t *conn, long long n_nodes, fe_field_h **out);
fe_status fe_field_free(fe_field_h *field);

/* Matrix mode of the Stokes coupling "i.i,0" whose scalar operand lives on
 * `field` and whose vector operand on the basis of `geom`:
 *   (VIRTUAL vector, STATE scalar)  K[e][(i,a)][b] = sum_q w det J G_q[i][a] psi_q[b],
 *                                   K_out (n_elems, 3 N, n_basis of field)
 *   (STATE vector, VIRTUAL scalar)  the transposed element matrices,
 *                                   K_out (n_elems, n_basis of field, 3 N)
 * with G = J^-T grad_xi phi of the geometry's basis (rows component-major like
 * every vector element output).  diff_op must be the FE_STATE operand.
 * FE_F64 or FE_F32 (output dtype as fe_eval_matrix).  Errors:
 * FE_ERR_INVALID_ARG, FE_ERR_SHAPE (field of another mesh size or point count),
 * FE_ERR_UNSUPPORTED_SPEC (other forms or precisions), FE_ERR_CUDA. */
fe_status fe_eval_matrix_mixed(fe_ctx *ctx, const fe_form_h *form, const fe_geometry_h *geom, const fe_field_h *field,
                               const void *const *args, int diff_op, fe_precision prec, void *K_out,
                               fe_stream_t stream);

/* Residual mode of the same coupling: args[state operand] is the scalar field's
 * DOF vector (field n_nodes; the rows of r_out (n_elems, 3 N) are the vector
 * test function's) or, for the transposed coupling, the vector field's DOF
 * vector (3 * mesh n_nodes; r_out (n_elems, n_basis of field)); float64 for
 * FE_F64 else float32.  An out-of-range DOF index in either connectivity is
 * reported as FE_ERR_SHAPE through fe_get_status.  Errors as
 * fe_eval_matrix_mixed. */
fe_status fe_eval_residual_mixed(fe_ctx *ctx, const fe_form_h *form, const fe_geometry_h *geom,
                                 const fe_field_h *field, const void *const *args, fe_precision prec, void *r_out,
                                 fe_stream_t stream);

/* Adjoint of residual mode (a vector-Jacobian product).  For an adjoint DOF
 * vector rbar (n_nodes * 3, device array, float64 for FE_F64 else float32),
 * e.g. rbar = dObjective/dR for an objective of the assembled residual R, the
 * derivatives of rbar . R(u; lambda, mu, X), element by element:
 *   d_mat  (n_elems, 2): [d/d lambda_e, d/d mu_e], the layout of the
 *          FE_MAT_LAME material operand (NULL: not computed)
 *   d_x_e  (n_elems, 3 * N): d/d x of the element's nodes, component-major
 *          [m * N + a] like a vector element residual; fe_assemble_vector with
 *          ncomp 3 sums it into d/dX (n_nodes, 3) (NULL: not computed)
 * with d/d lambda_e = sum_q w det J div(u_h) div(rbar_h), d/d mu_e = sum_q
 * w det J 2 eps(u_h) : eps(rbar_h), and the coordinate term from d(det J) and
 * d(J^-1) (the shape derivative of sum_e int sigma(u_h) : eps(rbar_h)).
 * The paper has no counterpart: it differentiates forms with respect to DOFs
 * only (Eq. fe4); this is the reverse mode of its residual (Algorithm 1) in the
 * material and geometry inputs.  Supported: linear elasticity with FE_MAT_LAME
 * materials (material letters in (v, u) order) on tensor-product hexahedra
 * whose basis carries its 1-D factors, FE_F64 or FE_F32 (outputs of that
 * dtype).  args as fe_eval_residual.  Errors: FE_ERR_INVALID_ARG (both outputs
 * NULL, missing arrays), FE_ERR_UNSUPPORTED_SPEC (other forms, precisions or
 * elements), FE_ERR_CUDA. */
fe_status fe_eval_residual_adjoint(fe_ctx *ctx, const fe_form_h *form, const fe_geometry_h *geom,
                                   const void *const *args, const void *rbar, fe_precision prec, void *d_mat,
                                   void *d_x_e, fe_stream_t stream);

/* 'eval' mode (Sec. 5.1): the integral over every element of an eval form,
 * out (n_elems, n_rows of fe_form_shape) float64 for FE_F64 else float32,
 * computed in that precision (FE_TF32X3/FE_BF16X3/FE_BF16 evaluate as FE_F32).
 * args as fe_eval_residual (every field operand needs its DOF vector); the
 * total over the mesh is the sum of the element values.  Forms: the weighted
 * Laplacian, dot/mass, elasticity, weighted dot product, Stokes coupling,
 * divergence, Cauchy stress (6 values: int D e(u), Voigt order) and the
 * convective term.  Errors: FE_ERR_INVALID_ARG (a form with a test function,
 * missing arrays), FE_ERR_SHAPE, FE_ERR_CUDA. */
fe_status fe_eval_integral(fe_ctx *ctx, const fe_form_h *form, const fe_geometry_h *geom, const void *const *args,
                           fe_precision prec, void *out, fe_stream_t stream);

/* ---- batched matrix mode ---------------------------------------------------------- */

/* One item of a batch: the element matrices of `form` on the elements of
 * `geom`, written to K_out (n_elems, n_rows, n_cols) float32.  material is the
 * form's float64 material array (NULL when the form has none).  The arrays are
 * borrowed: they must stay allocated while the batch is used. */
typedef struct {
    const fe_geometry_h *geom;
    const fe_form_h *form;
    const void *material;
    void *K_out;
} fe_batch_item;

#define FE_BATCH_GEOMETRY 1u   /* every run recomputes the geometry of each item's handle first */
#define FE_BATCH_AUTOTUNE 2u   /* time every candidate configuration at creation, keep the fastest */
#define FE_BATCH_GRAPH 4u      /* capture the run (geometry and matrices) in a CUDA graph at creation */
#define FE_BATCH_PERSISTENT 8u /* schedule: the persistent class kernels (the default without AUTOTUNE) */
#define FE_BATCH_LAUNCHES 16u  /* schedule: one launch per item of the kernel fe_eval_matrix uses */
#define FE_BATCH_SHARED_GRAM 32u /* launches schedule: pair Lame elasticity with the scalar Laplacian (below) */

/* A batch evaluates matrix mode (Algorithm 2) for many items, e.g. the groups
 * of a mixed mesh of P1-P3 tetrahedra and Q1-Q3 hexahedra with the Laplace,
 * mass and elasticity forms, under one of two schedules:
 * - persistent: the items' elements are cut into chunks and resident CTAs
 *   stride over a work list, one persistent kernel per register class of the
 *   chosen configurations (at most three: light, heavy, and 4x4-tile Q3
 *   elasticity, 3, 2 and 1 CTAs per SM), the classes running concurrently on
 *   forked streams.  Every (element, form) pair has candidate configurations
 *   (node tile, elements per chunk, output staging); FE_BATCH_AUTOTUNE times
 *   each on the item's own elements (writing its K_out) and keeps the fastest,
 *   otherwise the first is used;
 * - launches: one launch per item of the kernel that fe_eval_matrix runs for
 *   it (compiled, and occupied, for that item alone), the items spread over the
 *   caller's stream and two forked streams, largest first, each to the least
 *   loaded stream.  A Lame elasticity item and a scalar Laplacian item on the
 *   same geometry may share one CUDA-core launch instead: its Gram blocks
 *   A_jl give the elasticity matrix and, as c sum_j A_jj, the Laplacian.
 *   FE_BATCH_AUTOTUNE times the shared launch (on the CUDA cores, and on the
 *   tensor cores for 27- and 64-node hexahedra) against the two items' own kernels and
 *   keeps it where it is faster; FE_BATCH_SHARED_GRAM pairs every such couple
 *   without timing (each elasticity item with the first unpaired Laplacian
 *   item of its geometry; on the tensor cores where that kernel exists).
 * FE_BATCH_PERSISTENT or FE_BATCH_LAUNCHES fixes the schedule (not both); with
 * neither, FE_BATCH_AUTOTUNE times both schedules' matrix launches at creation
 * and keeps the faster, and without it the persistent schedule is used.  Both
 * schedules compute every entry with the same sums, in an order that may
 * differ in the last float32 bits.  FE_F32 arithmetic from the FP32 copy of the FP64
 * geometry, so every geometry must store FE_GEOM_STORE_F32.  Supported: the
 * weighted Laplacian, the (vector) mass and Lame elasticity on the (N, Q)
 * pairs of fe_geometry.  The paper has no batched evaluator (it evaluates one
 * form on one element type at a time, Sec. 5.2); this is the GPU-resident
 * counterpart of looping over its calls.  The call synchronizes `stream`.
 * Errors: FE_ERR_INVALID_ARG, FE_ERR_UNSUPPORTED_SPEC (a form or element
 * without a batch configuration), FE_ERR_OOM, FE_ERR_CUDA. */
fe_status fe_batch_create(fe_ctx *ctx, const fe_batch_item *items, int n_items, unsigned flags, fe_batch_h **out,
                          fe_stream_t stream);
/* Run the batch on `stream` (one graph launch with FE_BATCH_GRAPH, otherwise
 * the geometry launches and the matrix launches of the schedule). */
fe_status fe_batch_run(fe_ctx *ctx, fe_batch_h *batch, fe_stream_t stream);
/* The persistent-schedule configuration of item `item`: node tile, elements
 * per chunk, staging (1: bulk-copied row blocks, 0: direct stores); any may be
 * NULL.  Under the launches schedule the item runs fe_eval_matrix's kernel. */
fe_status fe_batch_describe(const fe_batch_h *batch, int item, int *tile, int *elems_per_chunk, int *staging);
/* The contraction path of item `item` in the batch's schedule: *path = 0 for
 * the Gram blocks on the CUDA cores (FP32), 1 for the TF32x3 Gram on the tensor
 * cores (the items fe_eval_matrix covers with FE_TF32X3, chosen by
 * FE_BATCH_AUTOTUNE in the per-item schedule when it is faster; max element
 * error of Q2 elasticity 6.5e-7 against the FP64 oracle on the 48^3
 * workload), 2 (CUDA cores) or 3 (tensor cores, TF32x3, 27- and 64-node hexahedra)
 * for a Lame elasticity item and a scalar Laplacian item on the same geometry
 * computed by one launch from the same Gram blocks A_jl (the Laplacian is
 * c sum_j A_jj; both items report the pair's value).  Errors:
 * FE_ERR_INVALID_ARG. */
fe_status fe_batch_describe_path(const fe_batch_h *batch, int item, int *path);
/* The schedule of a batch: *per_item_launches = 1 for one launch per item,
 * 0 for the persistent class kernels.  Errors: FE_ERR_INVALID_ARG (NULL). */
fe_status fe_batch_schedule(const fe_batch_h *batch, int *per_item_launches);
fe_status fe_batch_free(fe_batch_h *batch);

/* ---- assembly ------------------------------------------------------------------- */

/* Build the node -> (element, local node) incidence lists of a mesh on the
 * device (CSR, each list in ascending element order) so that assembly is a
 * deterministic gather.  The mesh arrays are borrowed.  Errors:
 * FE_ERR_INVALID_ARG, FE_ERR_SHAPE (an index outside [0, n_nodes) is reported
 * here), FE_ERR_OOM, FE_ERR_CUDA.  This call synchronizes `stream`. */
fe_status fe_assembly_create(fe_ctx *ctx, const fe_mesh *mesh, fe_assembly_h **out, fe_stream_t stream);
fe_status fe_assembly_free(fe_assembly_h *asm_h);

#define FE_ASSEMBLE_ACCUMULATE 1u  /* add into global_out instead of overwriting it */
#define FE_ASSEMBLE_COMPENSATED 2u /* float32: Neumaier-compensated sums (ignored for FE_F64) */

/* global_out[ncomp * conn[e][a] + i] (+)= sum over incidences of r_e[e][i * N + a],
 * summed per node in ascending (e, a) order, so results are bit-reproducible.
 * r_e (n_elems, ncomp * N) and global_out (n_nodes * ncomp) are device arrays,
 * float64 for FE_F64 else float32.  ncomp in {1, 3}. */
fe_status fe_assemble_vector(fe_ctx *ctx, const fe_assembly_h *asm_h, int ncomp, const void *r_e, fe_precision prec,
                             void *global_out, unsigned flags, fe_stream_t stream);

/* Test hook for the bounded device waits: the next tensor-core matrix launch
 * on 27-node hexahedra (fe_eval_matrix with FE_TF32X3, FE_BF16X3 or FE_BF16;
 * launches on other elements leave the hook armed) on this context first
 * waits on a device flag that nothing sets.  Its bounded wait (about two
 * seconds) runs out, every CTA takes its abort path (the MMAs it issued are
 * drained, its tensor memory freed) and FE_ERR_TIMEOUT is reported through
 * fe_get_status; the context stays usable.  Errors: FE_ERR_INVALID_ARG,
 * FE_ERR_CUDA. */
fe_status fe_debug_hold_next_matrix(fe_ctx *ctx);

/* Diagnostic: rounds n float64 values (device array `in`) to float32 (device
 * array `out`) with the rounding that the geometry kernels apply to the
 * cofactors, det J and the weights of a float32 copy (nearest, ties to even:
 * the same bits as a hardware conversion; computed with integer operations
 * for normal results).  Errors: FE_ERR_INVALID_ARG (NULL arrays, n < 0),
 * FE_ERR_CUDA. */
fe_status fe_round_f32(fe_ctx *ctx, const double *in, float *out, long long n, fe_stream_t stream);

/* One-shot assembly for callers that cannot allocate device memory.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * must not call cudaMalloc/cudaFree (directly or through a library such as
 * torch), e.g. an application whose device memory is owned by its own
 * allocator or budget, a real-time loop in which an allocation's implicit
 * device synchronisation would stall other streams, or a callback run inside
 * a framework step that forbids allocation.  It computes exactly what
 * fe_assembly_create followed by fe_assemble_vector computes (same kernels,
 * same summation order, same results), without an assembly handle and
 * without allocating anything.
 *
 * Its workspace (node -> (element, local node) incidence lists, counters and
 * the scan workspace) is one fixed file-scope device array of about 13 MB
 * that every GPU loading libfe holds until the process exits.  Limits:
 * n_nodes <= 524,288 and n_elems * nodes_per_elem <= 2,097,152; larger meshes
 * get FE_ERR_SHAPE (with a message in fe_last_error_message) and nothing is
 * launched.  The first call on a device resolves the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  All calls on a device share the array and it
 * keeps the previous call's contents (the counters are cleared on every
 * call): calls that may overlap on the GPU (different streams, or different
 * host threads) race and must be serialised by the caller.
 *
 * Arguments as fe_assemble_vector, with the mesh given directly (device
 * arrays, borrowed for the duration of the call).  An out-of-range node index
 * is recorded in the context status word (FE_ERR_SHAPE, element index; see
 * fe_get_status) and that incidence is skipped.  Asynchronous on `stream`. */
fe_status fe_assemble_vector_noalloc(fe_ctx *ctx, const fe_mesh *mesh, int ncomp, const void *r_e,
                                     fe_precision prec, void *global_out, unsigned flags, fe_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* FE_H */
