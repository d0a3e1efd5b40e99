"""Thin ctypes binding of libfe (include/fe.h): argument marshalling only.

Device arrays are torch CUDA tensors (PyTorch supplies memory and streams);
every step of the evaluation runs in the library's CUDA kernels.  There is no
CPU fallback: if libfe.so is missing or no GPU is present, calls fail loudly.

The names follow the C ABI: geometry (fe_geometry), form_compile
(fe_form_compile), eval_matrix (fe_eval_matrix), eval_residual
(fe_eval_residual), assembly_create / assemble_vector (fe_assemble_vector).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfe.so")

# ---- enums (mirror include/fe.h) -------------------------------------------------
FE_OK, FE_ERR_INVALID_ARG, FE_ERR_SHAPE, FE_ERR_UNSUPPORTED_SPEC = 0, 1, 2, 3
FE_ERR_NONPOSITIVE_DETJ, FE_ERR_NONFINITE, FE_ERR_OOM, FE_ERR_CUDA, FE_ERR_TIMEOUT = 4, 5, 6, 7, 8
F64, F32, TF32X3, BF16X3, BF16 = 0, 1, 2, 3, 4
PRECISIONS = {"f64": F64, "f32": F32, "tf32x3": TF32X3, "bf16x3": BF16X3, "bf16": BF16}
VIRTUAL, STATE, PARAMETER, MATERIAL = 0, 1, 2, 3
MAT_NONE, MAT_SCALAR, MAT_LAME, MAT_D66, MAT_M33 = 0, 1, 2, 3, 4
GEOM_STORE_F64, GEOM_STORE_F32, GEOM_DEFERRED = 1, 2, 4
GEOM_WDETJ, GEOM_JINV, GEOM_G = 0, 1, 2
ASSEMBLE_ACCUMULATE, ASSEMBLE_COMPENSATED = 1, 2
BATCH_GEOMETRY, BATCH_AUTOTUNE, BATCH_GRAPH, BATCH_PERSISTENT, BATCH_LAUNCHES = 1, 2, 4, 8, 16
BATCH_SHARED_GRAM = 32

EXPORTED = [
    "fe_create", "fe_destroy", "fe_status_str", "fe_get_status", "fe_version", "fe_last_error_message",
    "fe_refbasis_hex", "fe_refbasis_hex_1d", "fe_refbasis_tet", "fe_gm_rule_size", "fe_geometry", "fe_geometry_view",
    "fe_geometry_update", "fe_geometry_free", "fe_geometry_get", "fe_form_compile", "fe_form_free",
    "fe_form_shape", "fe_eval_matrix", "fe_eval_residual", "fe_eval_integral", "fe_eval_residual_adjoint",
    "fe_assembly_create",
    "fe_assembly_free",
    "fe_assemble_vector", "fe_assemble_vector_noalloc", "fe_batch_create", "fe_batch_run", "fe_batch_describe",
    "fe_batch_schedule", "fe_batch_free", "fe_round_f32", "fe_debug_hold_next_matrix",
    "fe_field_create", "fe_field_free", "fe_eval_matrix_mixed", "fe_eval_residual_mixed", "fe_diag_fp64",
    "fe_batch_describe_path",
]


class FEError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        lib = _lib
        name = lib.fe_status_str(status).decode() if lib else str(status)
        msg = lib.fe_last_error_message().decode() if lib else ""
        super().__init__("%s failed: %s%s" % (where, name, (" (" + msg + ")") if msg else ""))


class _Mesh(ctypes.Structure):
    _fields_ = [("coords", ctypes.c_void_p), ("n_nodes", ctypes.c_longlong), ("conn", ctypes.c_void_p),
                ("n_elems", ctypes.c_longlong), ("nodes_per_elem", ctypes.c_int)]


class _RefBasis(ctypes.Structure):
    _fields_ = [("n_basis", ctypes.c_int), ("n_qp", ctypes.c_int), ("phi", ctypes.c_void_p),
                ("dphi", ctypes.c_void_p), ("n1d", ctypes.c_int), ("nq1d", ctypes.c_int), ("b1d", ctypes.c_void_p),
                ("d1d", ctypes.c_void_p)]


class _Quad(ctypes.Structure):
    _fields_ = [("n_qp", ctypes.c_int), ("points", ctypes.c_void_p), ("weights", ctypes.c_void_p)]


class _BatchItem(ctypes.Structure):
    _fields_ = [("geom", ctypes.c_void_p), ("form", ctypes.c_void_p), ("material", ctypes.c_void_p),
                ("K_out", ctypes.c_void_p)]


class _Operand(ctypes.Structure):
    _fields_ = [("role", ctypes.c_int), ("ncomp", ctypes.c_int), ("material", ctypes.c_int)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libfe.so (built by paper_2107_04121_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libfe.so not found at %s: run `python -m paper_2107_04121_gb300.build` "
                          "(there is no CPU fallback)" % path)
    L = ctypes.CDLL(path)
    vp, i, ll, st = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_int
    dp = ctypes.POINTER(ctypes.c_double)
    L.fe_create.argtypes = [i, ctypes.POINTER(vp)]
    L.fe_destroy.argtypes = [vp]
    L.fe_status_str.argtypes = [st]
    L.fe_status_str.restype = ctypes.c_char_p
    L.fe_last_error_message.restype = ctypes.c_char_p
    L.fe_get_status.argtypes = [vp, vp, ctypes.POINTER(ll)]
    L.fe_refbasis_hex.argtypes = [i, i, dp, dp, dp, dp]
    L.fe_refbasis_hex_1d.argtypes = [i, i, dp, dp]
    L.fe_refbasis_tet.argtypes = [i, i, dp, dp, dp, dp]
    L.fe_gm_rule_size.argtypes = [i]
    L.fe_geometry.argtypes = [vp, ctypes.POINTER(_Mesh), ctypes.POINTER(_RefBasis), ctypes.POINTER(_Quad),
                              ctypes.c_uint, ctypes.POINTER(vp), vp]
    L.fe_geometry_update.argtypes = [vp, vp, vp]
    L.fe_geometry_view.argtypes = [vp, vp, ctypes.c_longlong, ctypes.c_longlong, ctypes.POINTER(vp)]
    L.fe_geometry_free.argtypes = [vp]
    L.fe_geometry_get.argtypes = [vp, vp, i, i, vp, vp]
    L.fe_form_compile.argtypes = [vp, ctypes.c_char_p, ctypes.POINTER(_Operand), i, ctypes.POINTER(vp)]
    L.fe_form_free.argtypes = [vp]
    L.fe_form_shape.argtypes = [vp, i, ctypes.POINTER(i), ctypes.POINTER(i)]
    L.fe_eval_matrix.argtypes = [vp, vp, vp, ctypes.POINTER(vp), i, i, vp, vp]
    L.fe_eval_residual.argtypes = [vp, vp, vp, ctypes.POINTER(vp), i, vp, vp]
    L.fe_eval_residual_adjoint.argtypes = [vp, vp, vp, ctypes.POINTER(vp), vp, i, vp, vp, vp]
    L.fe_eval_integral.argtypes = [vp, vp, vp, ctypes.POINTER(vp), i, vp, vp]
    L.fe_field_create.argtypes = [vp, vp, dp, i, vp, ll, ctypes.POINTER(vp)]
    L.fe_field_free.argtypes = [vp]
    L.fe_diag_fp64.argtypes = [vp, i, i, i, i, vp, vp]
    L.fe_eval_matrix_mixed.argtypes = [vp, vp, vp, vp, ctypes.POINTER(vp), i, i, vp, vp]
    L.fe_eval_residual_mixed.argtypes = [vp, vp, vp, vp, ctypes.POINTER(vp), i, vp, vp]
    L.fe_batch_create.argtypes = [vp, ctypes.POINTER(_BatchItem), i, ctypes.c_uint, ctypes.POINTER(vp), vp]
    L.fe_batch_run.argtypes = [vp, vp, vp]
    L.fe_batch_describe.argtypes = [vp, i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]
    L.fe_batch_describe_path.argtypes = [vp, i, ctypes.POINTER(i)]
    L.fe_batch_schedule.argtypes = [vp, ctypes.POINTER(i)]
    L.fe_batch_free.argtypes = [vp]
    L.fe_assembly_create.argtypes = [vp, ctypes.POINTER(_Mesh), ctypes.POINTER(vp), vp]
    L.fe_assembly_free.argtypes = [vp]
    L.fe_assemble_vector.argtypes = [vp, vp, i, vp, i, vp, ctypes.c_uint, vp]
    L.fe_assemble_vector_noalloc.argtypes = [vp, ctypes.POINTER(_Mesh), i, vp, i, vp, ctypes.c_uint, vp]
    L.fe_round_f32.argtypes = [vp, vp, vp, ctypes.c_longlong, vp]
    L.fe_debug_hold_next_matrix.argtypes = [vp]
    for name in EXPORTED:
        if name not in ("fe_status_str", "fe_last_error_message", "fe_version"):
            getattr(L, name).restype = st
    L.fe_version.restype = i
    _lib = L
    return L


def _check(status, where):
    if status != FE_OK:
        raise FEError(status, where)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev(t, dtype, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must have dtype %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return ctypes.c_void_p(t.data_ptr())


def _prec(p):
    return PRECISIONS[p] if isinstance(p, str) else int(p)


# ---- reference element (host only) -----------------------------------------------

def refbasis_hex(p: int, nq: int):
    """Order-p hex Lagrange basis and nq^3 Gauss rule (fe_refbasis_hex):
    points (Q,3), weights (Q), phi (Q,N), dphi (Q,3,N), numpy float64."""
    L = load_library()
    Q, N = nq ** 3, (p + 1) ** 3
    pts, w, phi, dphi = np.zeros((Q, 3)), np.zeros(Q), np.zeros((Q, N)), np.zeros((Q, 3, N))
    dp = ctypes.POINTER(ctypes.c_double)
    _check(L.fe_refbasis_hex(p, nq, pts.ctypes.data_as(dp), w.ctypes.data_as(dp), phi.ctypes.data_as(dp),
                             dphi.ctypes.data_as(dp)), "fe_refbasis_hex")
    return pts, w, phi, dphi


def refbasis_hex_1d(p: int, nq: int):
    """1-D factors of refbasis_hex (fe_refbasis_hex_1d): b1d, d1d of shape (nq, p+1)."""
    L = load_library()
    b, d = np.zeros((nq, p + 1)), np.zeros((nq, p + 1))
    dp = ctypes.POINTER(ctypes.c_double)
    _check(L.fe_refbasis_hex_1d(p, nq, b.ctypes.data_as(dp), d.ctypes.data_as(dp)), "fe_refbasis_hex_1d")
    return b, d


def refbasis_tet(p: int, s: int):
    """Order-p tetrahedron Lagrange basis at the Grundmann-Moller rule of index s
    (fe_refbasis_tet): points (Q,3), weights (Q), phi (Q,N), dphi (Q,3,N)."""
    L = load_library()
    Q = L.fe_gm_rule_size(s)
    if Q < 0:
        raise ValueError("Grundmann-Moller index must be in 0..6")
    N = (p + 1) * (p + 2) * (p + 3) // 6
    pts, w, phi, dphi = np.zeros((Q, 3)), np.zeros(Q), np.zeros((Q, N)), np.zeros((Q, 3, N))
    dp = ctypes.POINTER(ctypes.c_double)
    _check(L.fe_refbasis_tet(p, s, pts.ctypes.data_as(dp), w.ctypes.data_as(dp), phi.ctypes.data_as(dp),
                             dphi.ctypes.data_as(dp)), "fe_refbasis_tet")
    return pts, w, phi, dphi


# ---- context -------------------------------------------------------------------------

class Context:
    def __init__(self, device: int = 0):
        L = load_library()
        self._h = ctypes.c_void_p()
        _check(L.fe_create(device, ctypes.byref(self._h)), "fe_create")
        self.device = device

    @property
    def handle(self):
        return self._h

    def status(self, stream=None):
        """(status code, smallest offending element or -1); synchronizes the stream."""
        bad = ctypes.c_longlong(-1)
        st = _lib.fe_get_status(self._h, _stream_ptr(stream), ctypes.byref(bad))
        return st, bad.value

    def check(self, stream=None):
        st, bad = self.status(stream)
        if st != FE_OK:
            raise FEError(st, "device check (element %d)" % bad)

    def close(self):
        if self._h:
            _lib.fe_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mesh:
    """Borrowed device mesh: coords (n_nodes,3) float64, conn (n_elems,N) int32."""

    def __init__(self, coords, conn):
        import torch
        self.coords, self.conn = coords, conn
        _dev(coords, torch.float64, "coords")
        _dev(conn, torch.int32, "conn")
        if coords.dim() != 2 or coords.shape[1] != 3 or conn.dim() != 2:
            raise ValueError("coords must be (n_nodes,3), conn (n_elems,N)")
        self.struct = _Mesh(coords.data_ptr(), coords.shape[0], conn.data_ptr(), conn.shape[0], conn.shape[1])

    @property
    def n_nodes(self):
        return self.coords.shape[0]

    @property
    def n_elems(self):
        return self.conn.shape[0]

    @property
    def nodes_per_elem(self):
        return self.conn.shape[1]


class Geometry:
    def __init__(self, ctx, mesh, handle, N, Q):
        self.ctx, self.mesh, self._h, self.N, self.Q = ctx, mesh, handle, N, Q

    def get(self, field: int, precision="f64", stream=None):
        import torch
        f64 = _prec(precision) == F64
        E = self.mesh.n_elems
        shape = {GEOM_WDETJ: (E, self.Q), GEOM_JINV: (E, self.Q, 3, 3), GEOM_G: (E, self.Q, 3, self.N)}[field]
        out = torch.empty(shape, dtype=torch.float64 if f64 else torch.float32, device=self.mesh.coords.device)
        _check(_lib.fe_geometry_get(self.ctx.handle, self._h, field, _prec(precision),
                                    ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)), "fe_geometry_get")
        return out

    def update(self, stream=None):
        """fe_geometry_update: recompute in place from the mesh's current coordinates."""
        _check(_lib.fe_geometry_update(self.ctx.handle, self._h, _stream_ptr(stream)), "fe_geometry_update")

    def view(self, e_begin: int, e_count: int) -> "Geometry":
        """fe_geometry_view: the elements [e_begin, e_begin + e_count), aliasing this
        handle's storage (keep this handle alive while the view is used)."""
        h = ctypes.c_void_p()
        _check(_lib.fe_geometry_view(self.ctx.handle, self._h, e_begin, e_count, ctypes.byref(h)),
               "fe_geometry_view")
        sub = Mesh(self.mesh.coords, self.mesh.conn[e_begin:e_begin + e_count])
        g = Geometry(self.ctx, sub, h, self.N, self.Q)
        g._parent = self
        return g

    def free(self):
        if self._h:
            _lib.fe_geometry_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def geometry(ctx: Context, mesh: Mesh, phi, dphi, weights, flags: int = 0, stream=None, b1d=None,
             d1d=None) -> Geometry:
    """fe_geometry: FP64 J, det J, J^-1, w det J for every element and qp.
    b1d/d1d (optional): tensor-product factors enabling the sum-factorised kernel."""
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    dphi = np.ascontiguousarray(dphi, dtype=np.float64)
    weights = np.ascontiguousarray(weights, dtype=np.float64)
    Q, N = phi.shape
    if b1d is not None:
        b1d = np.ascontiguousarray(b1d, dtype=np.float64)
        d1d = np.ascontiguousarray(d1d, dtype=np.float64)
        basis = _RefBasis(N, Q, phi.ctypes.data, dphi.ctypes.data, b1d.shape[1], b1d.shape[0], b1d.ctypes.data,
                          d1d.ctypes.data)
    else:
        basis = _RefBasis(N, Q, phi.ctypes.data, dphi.ctypes.data, 0, 0, None, None)
    quad = _Quad(Q, None, weights.ctypes.data)
    h = ctypes.c_void_p()
    _check(_lib.fe_geometry(ctx.handle, ctypes.byref(mesh.struct), ctypes.byref(basis), ctypes.byref(quad), flags,
                            ctypes.byref(h), _stream_ptr(stream)), "fe_geometry")
    return Geometry(ctx, mesh, h, N, Q)


def hex_geometry(ctx: Context, mesh: Mesh, p: int, nq: int, flags: int = 0, stream=None) -> Geometry:
    """fe_geometry with the library's order-p hex basis and nq^3 Gauss rule (tensor-product path)."""
    pts, w, phi, dphi = refbasis_hex(p, nq)
    b1d, d1d = refbasis_hex_1d(p, nq)
    return geometry(ctx, mesh, phi, dphi, w, flags, stream, b1d, d1d)


def tet_geometry(ctx: Context, mesh: Mesh, p: int, s: int = None, flags: int = 0, stream=None) -> Geometry:
    """fe_geometry with the library's order-p tetrahedron basis and the
    Grundmann-Moller rule of index s (default p: exact for degree 2p + 1)."""
    pts, w, phi, dphi = refbasis_tet(p, p if s is None else s)
    return geometry(ctx, mesh, phi, dphi, w, flags, stream)


class Form:
    def __init__(self, expr, operands, handle):
        self.expr, self.operands, self._h = expr, operands, handle
        states = [k for k, o in enumerate(operands) if o[0] == STATE]
        self.state_op = states[0] if states else None

    def shape(self, n_basis):
        r, c = ctypes.c_int(), ctypes.c_int()
        _check(_lib.fe_form_shape(self._h, n_basis, ctypes.byref(r), ctypes.byref(c)), "fe_form_shape")
        return r.value, c.value

    def free(self):
        if self._h:
            _lib.fe_form_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def form_compile(expr: str, operands, ctx: Context | None = None) -> Form:
    """fe_form_compile.  operands: list of (role, ncomp, material_kind)."""
    L = load_library()
    arr = (_Operand * len(operands))(*[_Operand(r, n, m) for r, n, m in operands])
    h = ctypes.c_void_p()
    _check(L.fe_form_compile(ctx.handle if ctx else None, expr.encode(), arr, len(operands), ctypes.byref(h)),
           "fe_form_compile(%r)" % expr)
    return Form(expr, list(operands), h)


_MAT_SIZE = {MAT_SCALAR: 1, MAT_LAME: 2, MAT_D66: 36, MAT_M33: 9}


def _args(form: Form, args, geom: Geometry, dtype=None):
    """Device pointers of the operands; checks materials (float64, one row per
    element) and, given their dtype, the DOF vectors of field operands."""
    import torch
    if len(args) != len(form.operands):
        raise ValueError("expected %d operands, got %d" % (len(form.operands), len(args)))
    ptrs = (ctypes.c_void_p * len(form.operands))()
    for k, (a, (role, ncomp, mk)) in enumerate(zip(args, form.operands)):
        if role == MATERIAL:
            _dev(a, torch.float64, "material operand %d" % k)
            if a.numel() != geom.mesh.n_elems * _MAT_SIZE[mk]:
                raise ValueError("material operand %d must have %d values per element" % (k, _MAT_SIZE[mk]))
        elif role in (STATE, PARAMETER) and a is not None and dtype is not None:
            _dev(a, dtype, "DOF vector of operand %d" % k)
            if a.numel() != geom.mesh.n_nodes * ncomp:
                raise ValueError("DOF vector of operand %d must have n_nodes * %d entries" % (k, ncomp))
        ptrs[k] = None if a is None else a.data_ptr()
    return ptrs


def _out_dtype(precision):
    import torch
    return torch.float64 if _prec(precision) == F64 else torch.float32


def eval_matrix(ctx: Context, form: Form, geom: Geometry, args, precision="f64", out=None, diff_op=None,
                stream=None):
    """fe_eval_matrix: element matrices (E, n_rows, n_cols)."""
    import torch
    nr, nc = form.shape(geom.N)
    E = geom.mesh.n_elems
    if out is None:
        out = torch.empty((E, nr, nc), dtype=_out_dtype(precision), device=geom.mesh.coords.device)
    _dev(out, _out_dtype(precision), "K_out")
    if tuple(out.shape) != (E, nr, nc):
        raise ValueError("K_out must have shape %s" % ((E, nr, nc),))
    d = form.state_op if diff_op is None else diff_op
    _check(_lib.fe_eval_matrix(ctx.handle, form._h, geom._h, _args(form, args, geom, _out_dtype(precision)), d,
                               _prec(precision),
                               ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)), "fe_eval_matrix")
    return out


def eval_residual(ctx: Context, form: Form, geom: Geometry, args, precision="f64", out=None, stream=None):
    """fe_eval_residual: element residuals (E, n_rows)."""
    import torch
    nr, _ = form.shape(geom.N)
    E = geom.mesh.n_elems
    if out is None:
        out = torch.empty((E, nr), dtype=_out_dtype(precision), device=geom.mesh.coords.device)
    _dev(out, _out_dtype(precision), "r_out")
    if tuple(out.shape) != (E, nr):
        raise ValueError("r_out must have shape %s" % ((E, nr),))
    for k, (role, _, _) in enumerate(form.operands):
        if role in (STATE, PARAMETER) and args[k] is None:
            raise ValueError("operand %d needs its DOF vector in residual mode" % k)
    _check(_lib.fe_eval_residual(ctx.handle, form._h, geom._h, _args(form, args, geom, _out_dtype(precision)),
                                 _prec(precision),
                                 ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)), "fe_eval_residual")
    return out


class Field:
    """fe_field_create: a scalar field on a second basis over the elements of a
    geometry (the second field of a mixed-order pair): psi (Q, n_basis) float64
    host array at the geometry's points, conn (n_elems, n_basis) int32 device
    tensor (borrowed), n_nodes DOFs."""

    def __init__(self, ctx: Context, geom: Geometry, psi, conn, n_nodes: int):
        import torch
        psi = np.ascontiguousarray(psi, dtype=np.float64)
        _dev(conn, torch.int32, "conn")
        if psi.ndim != 2 or psi.shape[0] != geom.Q or conn.dim() != 2 or conn.shape[1] != psi.shape[1] \
                or conn.shape[0] != geom.mesh.n_elems:
            raise ValueError("psi must be (Q, n_basis) and conn (n_elems, n_basis)")
        self.geom, self.conn, self.n_basis, self.n_nodes = geom, conn, psi.shape[1], int(n_nodes)
        self._h = ctypes.c_void_p()
        _check(_lib.fe_field_create(ctx.handle, geom._h, psi.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    self.n_basis, ctypes.c_void_p(conn.data_ptr()), self.n_nodes,
                                    ctypes.byref(self._h)), "fe_field_create")

    def free(self):
        if self._h:
            _lib.fe_field_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _mixed_args(form: Form, args, geom: Geometry, field: Field, dtype):
    """Operand pointers of a Stokes coupling whose scalar operand is on `field`."""
    if len(args) != len(form.operands):
        raise ValueError("expected %d operands, got %d" % (len(form.operands), len(args)))
    ptrs = (ctypes.c_void_p * len(form.operands))()
    for k, (a, (role, ncomp, mk)) in enumerate(zip(args, form.operands)):
        if a is not None:
            _dev(a, dtype, "DOF vector of operand %d" % k)
            want = field.n_nodes if ncomp == 1 else geom.mesh.n_nodes * ncomp
            if a.numel() != want:
                raise ValueError("DOF vector of operand %d must have %d entries" % (k, want))
        ptrs[k] = None if a is None else a.data_ptr()
    return ptrs


def eval_matrix_mixed(ctx: Context, form: Form, geom: Geometry, field: Field, args, precision="f64", out=None,
                      stream=None):
    """fe_eval_matrix_mixed: the Stokes coupling with its scalar operand on `field`:
    (E, 3 N, Np) with the vector test function, (E, Np, 3 N) with the scalar one."""
    import torch
    E, N, Np = geom.mesh.n_elems, geom.N, field.n_basis
    vec_test = form.operands[[r for r, _, _ in form.operands].index(VIRTUAL)][1] == 3
    shape = (E, 3 * N, Np) if vec_test else (E, Np, 3 * N)
    if out is None:
        out = torch.empty(shape, dtype=_out_dtype(precision), device=geom.mesh.coords.device)
    _dev(out, _out_dtype(precision), "K_out")
    if tuple(out.shape) != shape:
        raise ValueError("K_out must have shape %s" % (shape,))
    _check(_lib.fe_eval_matrix_mixed(ctx.handle, form._h, geom._h, field._h,
                                     _mixed_args(form, args, geom, field, _out_dtype(precision)), form.state_op,
                                     _prec(precision), ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)),
           "fe_eval_matrix_mixed")
    return out


def eval_residual_mixed(ctx: Context, form: Form, geom: Geometry, field: Field, args, precision="f64", out=None,
                        stream=None):
    """fe_eval_residual_mixed: residuals (E, 3 N) with the vector test function,
    (E, Np) with the scalar one; the unknown's DOF vector in its operand slot."""
    import torch
    E, N, Np = geom.mesh.n_elems, geom.N, field.n_basis
    vec_test = form.operands[[r for r, _, _ in form.operands].index(VIRTUAL)][1] == 3
    shape = (E, 3 * N) if vec_test else (E, Np)
    if out is None:
        out = torch.empty(shape, dtype=_out_dtype(precision), device=geom.mesh.coords.device)
    _dev(out, _out_dtype(precision), "r_out")
    if tuple(out.shape) != shape:
        raise ValueError("r_out must have shape %s" % (shape,))
    _check(_lib.fe_eval_residual_mixed(ctx.handle, form._h, geom._h, field._h,
                                       _mixed_args(form, args, geom, field, _out_dtype(precision)),
                                       _prec(precision), ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)),
           "fe_eval_residual_mixed")
    return out


def diag_fp64(ctx: Context, kind: int, warps: int, ilp: int, steps: int, out, stream=None):
    """fe_diag_fp64: launch the FP64 rate diagnostic (kind 0 DFMA, 1 FP64 MMA) with
    one CTA of `warps` warps per SM; `out` a float64 device tensor of
    SMs x warps x 32 entries.  Time it with CUDA events on `stream`."""
    import torch
    _dev(out, torch.float64, "out")
    _check(_lib.fe_diag_fp64(ctx.handle, kind, warps, ilp, steps, ctypes.c_void_p(out.data_ptr()),
                             _stream_ptr(stream)), "fe_diag_fp64")


def eval_integral(ctx: Context, form: Form, geom: Geometry, args, precision="f64", out=None, stream=None):
    """fe_eval_integral ('eval' mode): element integrals (E, n_values) of a form
    whose operands all carry DOFs."""
    import torch
    nv, _ = form.shape(geom.N)
    E = geom.mesh.n_elems
    if out is None:
        out = torch.empty((E, nv), dtype=_out_dtype(precision), device=geom.mesh.coords.device)
    _dev(out, _out_dtype(precision), "out")
    if tuple(out.shape) != (E, nv):
        raise ValueError("out must have shape %s" % ((E, nv),))
    _check(_lib.fe_eval_integral(ctx.handle, form._h, geom._h, _args(form, args, geom, _out_dtype(precision)),
                                 _prec(precision), ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)),
           "fe_eval_integral")
    return out


def eval_residual_adjoint(ctx: Context, form: Form, geom: Geometry, args, rbar, precision="f64", d_mat=None,
                          d_x_e=None, want_mat=True, want_x=True, stream=None):
    """fe_eval_residual_adjoint: derivatives of rbar . R with respect to the Lame
    pairs, d_mat (E, 2), and the element node coordinates, d_x_e (E, 3 N)
    component-major (assemble with assemble_vector(ncomp=3) for (n_nodes, 3))."""
    import torch
    dt = _out_dtype(precision)
    E, dev = geom.mesh.n_elems, geom.mesh.coords.device
    if want_mat and d_mat is None:
        d_mat = torch.empty((E, 2), dtype=dt, device=dev)
    if want_x and d_x_e is None:
        d_x_e = torch.empty((E, 3 * geom.N), dtype=dt, device=dev)
    for t, name in ((d_mat, "d_mat"), (d_x_e, "d_x_e"), (rbar, "rbar")):
        if t is not None:
            _dev(t, dt, name)
    if rbar.numel() != 3 * geom.mesh.n_nodes:
        raise ValueError("rbar must have n_nodes * 3 entries")
    ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
    _check(_lib.fe_eval_residual_adjoint(ctx.handle, form._h, geom._h, _args(form, args, geom, dt), ptr(rbar),
                                         _prec(precision), ptr(d_mat), ptr(d_x_e), _stream_ptr(stream)),
           "fe_eval_residual_adjoint")
    return d_mat, d_x_e


class Batch:
    """fe_batch_create / fe_batch_run: element matrices of many (geometry, form)
    items, by persistent class kernels or one launch per item (BATCH_PERSISTENT,
    BATCH_LAUNCHES, or timed with BATCH_AUTOTUNE).  items: list of (geometry,
    form, material tensor or None, K_out tensor or None); the tensors are kept
    alive here."""

    def __init__(self, ctx: Context, items, flags: int = 0, stream=None):
        import torch
        self.ctx, self._keep, self.outputs = ctx, [], []
        arr = (_BatchItem * len(items))()
        for k, (geom, form, mat, K) in enumerate(items):
            nr, nc = form.shape(geom.N)
            E = geom.mesh.n_elems
            if K is None:
                K = torch.empty((E, nr, nc), dtype=torch.float32, device=geom.mesh.coords.device)
            _dev(K, torch.float32, "K_out")
            if tuple(K.shape) != (E, nr, nc):
                raise ValueError("K_out of item %d must have shape %s" % (k, (E, nr, nc)))
            if mat is not None:
                _dev(mat, torch.float64, "material of item %d" % k)
            arr[k] = _BatchItem(geom._h.value, form._h.value, mat.data_ptr() if mat is not None else None,
                                K.data_ptr())
            self._keep += [geom, form, mat, K]
            self.outputs.append(K)
        self._h = ctypes.c_void_p()
        _check(_lib.fe_batch_create(ctx.handle, arr, len(items), flags, ctypes.byref(self._h), _stream_ptr(stream)),
               "fe_batch_create")

    def run(self, stream=None):
        _check(_lib.fe_batch_run(self.ctx.handle, self._h, _stream_ptr(stream)), "fe_batch_run")
        return self.outputs

    def describe(self, item: int):
        t, e, s = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(_lib.fe_batch_describe(self._h, item, ctypes.byref(t), ctypes.byref(e), ctypes.byref(s)),
               "fe_batch_describe")
        pth = ctypes.c_int()
        _check(_lib.fe_batch_describe_path(self._h, item, ctypes.byref(pth)), "fe_batch_describe_path")
        paths = {0: "cuda-core Gram blocks", 1: "tensor-core tf32x3 Gram",
                 2: "cuda-core Gram blocks shared by elasticity and Laplacian",
                 3: "tensor-core tf32x3 Gram shared by elasticity and Laplacian"}
        return {"tile": t.value, "elems_per_chunk": e.value, "staging": "bulk" if s.value else "direct",
                "path": paths[pth.value]}

    def schedule(self) -> str:
        """'launches' (one kernel launch per item) or 'persistent' (the class kernels)."""
        v = ctypes.c_int()
        _check(_lib.fe_batch_schedule(self._h, ctypes.byref(v)), "fe_batch_schedule")
        return "launches" if v.value else "persistent"

    def free(self):
        if self._h:
            _lib.fe_batch_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Assembly:
    def __init__(self, ctx, mesh, handle):
        self.ctx, self.mesh, self._h = ctx, mesh, handle

    def free(self):
        if self._h:
            _lib.fe_assembly_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def assembly_create(ctx: Context, mesh: Mesh, stream=None) -> Assembly:
    h = ctypes.c_void_p()
    _check(_lib.fe_assembly_create(ctx.handle, ctypes.byref(mesh.struct), ctypes.byref(h), _stream_ptr(stream)),
           "fe_assembly_create")
    return Assembly(ctx, mesh, h)


def assemble_vector(ctx: Context, asm: Assembly, ncomp: int, r_e, precision="f64", out=None, flags: int = 0,
                    stream=None):
    """fe_assemble_vector: deterministic gather of element vectors into (n_nodes*ncomp)."""
    import torch
    dt = _out_dtype(precision)
    _dev(r_e, dt, "r_e")
    if r_e.numel() != asm.mesh.n_elems * ncomp * asm.mesh.nodes_per_elem:
        raise ValueError("r_e must be (n_elems, ncomp * nodes_per_elem)")
    if out is None:
        out = torch.zeros(asm.mesh.n_nodes * ncomp, dtype=dt, device=r_e.device)
    _dev(out, dt, "global_out")
    if out.numel() != asm.mesh.n_nodes * ncomp:
        raise ValueError("global_out must have n_nodes * ncomp entries")
    _check(_lib.fe_assemble_vector(ctx.handle, asm._h, ncomp, ctypes.c_void_p(r_e.data_ptr()), _prec(precision),
                                   ctypes.c_void_p(out.data_ptr()), flags, _stream_ptr(stream)), "fe_assemble_vector")
    return out


def assemble_vector_noalloc(ctx: Context, mesh: Mesh, ncomp: int, r_e, out, precision="f64", flags: int = 0,
                            stream=None):
    """fe_assemble_vector_noalloc: the same assembly as assembly_create + assemble_vector
    for callers that cannot allocate device memory; the library allocates nothing and
    `out` must be preallocated (n_nodes * ncomp).  The library's fixed workspace is
    shared by all calls on a device: calls that overlap on the GPU race."""
    import torch
    dt = _out_dtype(precision)
    _dev(r_e, dt, "r_e")
    _dev(out, dt, "global_out")
    if r_e.numel() != mesh.n_elems * ncomp * mesh.nodes_per_elem or out.numel() != mesh.n_nodes * ncomp:
        raise ValueError("r_e must be (n_elems, ncomp * N) and global_out (n_nodes * ncomp)")
    _check(_lib.fe_assemble_vector_noalloc(ctx.handle, ctypes.byref(mesh.struct), ncomp,
                                           ctypes.c_void_p(r_e.data_ptr()), _prec(precision),
                                           ctypes.c_void_p(out.data_ptr()), flags, _stream_ptr(stream)),
           "fe_assemble_vector_noalloc")
    return out


# ---- named forms of Tab. ewfd ---------------------------------------------------------

def laplace_form(weighted: bool = False) -> Form:
    if weighted:
        return form_compile("0,0.i,0.i", [(MATERIAL, 1, MAT_SCALAR), (VIRTUAL, 1, MAT_NONE), (STATE, 1, MAT_NONE)])
    return form_compile("0.i,0.i", [(VIRTUAL, 1, MAT_NONE), (STATE, 1, MAT_NONE)])


def mass_form(ncomp: int = 1, weighted: bool = False) -> Form:
    ops = [(VIRTUAL, ncomp, MAT_NONE), (STATE, ncomp, MAT_NONE)]
    if weighted:
        return form_compile("0,i,i", [(MATERIAL, 1, MAT_SCALAR)] + ops)
    return form_compile("i,i", ops)


def convect_form(advection: int = STATE, gradient: int = STATE) -> Form:
    """Navier-Stokes convection 'i,i.j,j' with operands (v, u, w): the gradient
    operand u and the advection operand w are each STATE or PARAMETER; both
    STATE (the default) is the non-linear term, whose matrix is Eq. fe4."""
    return form_compile("i,i.j,j", [(VIRTUAL, 3, MAT_NONE), (gradient, 3, MAT_NONE), (advection, 3, MAT_NONE)])


def elasticity_form(material: int = MAT_LAME) -> Form:
    return form_compile("IK,s(i:j)->I,s(k:l)->K",
                        [(MATERIAL, 1, material), (VIRTUAL, 3, MAT_NONE), (STATE, 3, MAT_NONE)])


def round_f32(ctx: Context, x, stream=None):
    """fe_round_f32: float64 device tensor -> float32, with the rounding of the
    geometry kernels' float32 copy (diagnostic)."""
    import torch
    _dev(x, torch.float64, "in")
    out = torch.empty(x.shape, dtype=torch.float32, device=x.device)
    _check(_lib.fe_round_f32(ctx.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), x.numel(),
                             _stream_ptr(stream)), "fe_round_f32")
    return out


def debug_hold_next_matrix(ctx: Context):
    """fe_debug_hold_next_matrix: the next tensor-core matrix launch waits on a
    flag that nothing sets, times out and reports FE_ERR_TIMEOUT (test hook)."""
    _check(_lib.fe_debug_hold_next_matrix(ctx.handle), "fe_debug_hold_next_matrix")
