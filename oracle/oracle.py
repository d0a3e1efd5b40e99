"""ctypes wrapper of the FP64 nested-loop oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the benchmark's
CPU-baseline leg call it; the product path never does.  Every function is a
plain definition from Cimrman, arXiv 2107.04121 (Sec. 4.1 geometry and
Algorithms 1-2; Sec. 5.3 forms), see the comments in oracle.c.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (-O2, no fast-math, OpenMP over elements)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-fopenmp", "-fPIC", "-shared", "-Wall",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.oracle_gauss_1d.argtypes = [ctypes.c_int, _D, _D]
        L.oracle_hex_basis.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D]
        L.oracle_hex_quadrature.argtypes = [ctypes.c_int, _D, _D]
        L.oracle_gm_rule.argtypes = [ctypes.c_int, _D, _D]
        L.oracle_tet_basis.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D]
        L.oracle_geometry.restype = ctypes.c_longlong
        L.oracle_geometry.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.c_int, _D, _I, _D, _D, _D, _D, _D]
        L.oracle_matrix_laplace.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.c_int, _D, _D, _D, _D]
        L.oracle_matrix_mass.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, _D, _D]
        L.oracle_lame_to_D.argtypes = [ctypes.c_longlong, _D, _D, _D]
        L.oracle_matrix_elasticity.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.c_int, _D, _D, _D, _D]
        L.oracle_residual_laplace.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.c_int, _I, _D, _D, _D, _D, _D]
        L.oracle_residual_mass.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ctypes.c_int, _I, _D, _D,
                                           _D, _D, _D]
        L.oracle_residual_elasticity.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.c_int, _I, _D, _D, _D, _D,
                                                 _D]
        L.oracle_residual_convect.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.c_int, _I, _D, _D, _D, _D, _D,
                                              _D]
        L.oracle_matrix_convect.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.c_int, _I, _D, _D, _D, _D, _D,
                                            ctypes.c_int, ctypes.c_int, _D]
        L.oracle_adjoint_elasticity.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.c_int, _I, _D, _D, _D, _D,
                                                _D, _D, _D, _D, _D]
        L.oracle_matrix_wdot.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.c_int, _D, _D, _D, _D]
        L.oracle_residual_wdot.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.c_int, _I, _D, _D, _D, _D, _D]
        L.oracle_matrix_stokes.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.c_int, _D, _D, _D, _D]
        L.oracle_residual_stokes.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.c_int, _I, _D, _D, _D, _D, _D]
        L.oracle_residual_stokes_t.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.c_int, _I, _D, _D, _D, _D,
                                               _D]
        L.oracle_matrix_stokes_mixed.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D,
                                                 _D, _D]
        L.oracle_residual_stokes_mixed.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ctypes.c_int, _I,
                                                   _D, _D, _D, _D, _D]
        L.oracle_residual_stokes_t_mixed.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                     _I, _D, _D, _D, _D, _D]
        L.oracle_eval_form.argtypes = [ctypes.c_int, ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ctypes.c_int, _I,
                                       _D, _D, _D, _D, _D, _D, _D, _D, _D]
        L.oracle_assemble.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.c_int, _I, _D, ctypes.c_longlong,
                                      ctypes.c_int, _D]
        L.oracle_num_threads.restype = ctypes.c_int
        L.oracle_set_num_threads.argtypes = [ctypes.c_int]
        L.oracle_set_num_threads.restype = None
        _lib = L
    return _lib


def _d(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _i(a):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(_I)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _check(rc):
    if rc != 0:
        raise RuntimeError("oracle call failed with code %d" % rc)


def num_threads() -> int:
    return lib().oracle_num_threads()


def set_num_threads(n: int) -> None:
    """OpenMP threads of the following oracle calls (the arithmetic is the same)."""
    lib().oracle_set_num_threads(int(n))


def gauss_1d(n: int):
    """Gauss-Legendre points and weights on [0, 1], ascending."""
    x = np.zeros(n)
    w = np.zeros(n)
    _check(lib().oracle_gauss_1d(n, _d(x), _d(w)))
    return x, w


def hex_quadrature(nq: int):
    """Tensor Gauss rule on [0,1]^3, lexicographic x fastest: pts (nq^3, 3), w (nq^3)."""
    pts = np.zeros((nq ** 3, 3))
    w = np.zeros(nq ** 3)
    _check(lib().oracle_hex_quadrature(nq, _d(pts), _d(w)))
    return pts, w


def hex_basis(p: int, pts):
    """Order-p Lagrange basis on [0,1]^3 at pts: phi (n, N), dphi (n, 3, N)."""
    pts = _f64(pts).reshape(-1, 3)
    N = (p + 1) ** 3
    phi = np.zeros((pts.shape[0], N))
    dphi = np.zeros((pts.shape[0], 3, N))
    _check(lib().oracle_hex_basis(p, pts.shape[0], _d(pts), _d(phi), _d(dphi)))
    return phi, dphi


def gm_rule(s: int):
    """Grundmann-Moller rule of index s on the reference tetrahedron: points (Q,3), weights (Q)."""
    Q = lib().oracle_gm_rule(s, None, None)
    if Q < 0:
        raise ValueError("bad GM index")
    pts, w = np.zeros((Q, 3)), np.zeros(Q)
    lib().oracle_gm_rule(s, _d(pts), _d(w))
    return pts, w


def tet_basis(p: int, pts):
    pts = _f64(pts)
    Q = pts.shape[0]
    N = (p + 1) * (p + 2) * (p + 3) // 6
    phi, dphi = np.zeros((Q, N)), np.zeros((Q, 3, N))
    _check(lib().oracle_tet_basis(p, Q, _d(pts), _d(phi), _d(dphi)))
    return phi, dphi


class RefTet:
    """Reference tetrahedron of order p with the Grundmann-Moller rule of index s."""

    def __init__(self, p: int, s: int):
        self.p, self.s = p, s
        self.pts, self.w = gm_rule(s)
        self.phi, self.dphi = tet_basis(p, self.pts)
        self.N = (p + 1) * (p + 2) * (p + 3) // 6
        self.Q = self.pts.shape[0]


class RefElement:
    """Reference hexahedron of order p with an nq^3 Gauss rule."""

    def __init__(self, p: int, nq: int):
        self.p, self.nq = p, nq
        self.pts, self.w = hex_quadrature(nq)
        self.phi, self.dphi = hex_basis(p, self.pts)
        self.N = (p + 1) ** 3
        self.Q = nq ** 3


def geometry(coords, conn, ref: RefElement, want_G=True, want_Jinv=False):
    """wdetJ (E,Q), G (E,Q,3,N), Jinv (E,Q,3,3); raises on det J <= 0."""
    coords = _f64(coords)
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    E = conn.shape[0]
    wdetJ = np.zeros((E, ref.Q))
    G = np.zeros((E, ref.Q, 3, ref.N)) if want_G else None
    Jinv = np.zeros((E, ref.Q, 3, 3)) if want_Jinv else None
    bad = lib().oracle_geometry(E, ref.N, ref.Q, _d(coords), _i(conn), _d(ref.dphi), _d(ref.w), _d(wdetJ), _d(G),
                                _d(Jinv))
    if bad < 0:
        raise RuntimeError("oracle_geometry: bad argument")
    if bad > 0:
        raise ValueError("non-positive det J in element %d" % (bad - 1))
    return wdetJ, G, Jinv


def matrix_laplace(wdetJ, G, coef=None):
    E, Q, _, N = G.shape
    K = np.zeros((E, N, N))
    _check(lib().oracle_matrix_laplace(E, N, Q, _d(wdetJ), _d(G), _d(_f64(coef)), _d(K)))
    return K


def matrix_mass(wdetJ, phi, ncomp=1, coef=None):
    E, Q = wdetJ.shape
    N = phi.shape[1]
    n = ncomp * N
    K = np.zeros((E, n, n))
    _check(lib().oracle_matrix_mass(E, N, Q, ncomp, _d(wdetJ), _d(_f64(phi)), _d(_f64(coef)), _d(K)))
    return K


def lame_to_D(lam, mu):
    lam = _f64(lam)
    mu = _f64(mu)
    D = np.zeros((lam.shape[0], 6, 6))
    _check(lib().oracle_lame_to_D(lam.shape[0], _d(lam), _d(mu), _d(D)))
    return D


def matrix_elasticity(wdetJ, G, D):
    E, Q, _, N = G.shape
    K = np.zeros((E, 3 * N, 3 * N))
    _check(lib().oracle_matrix_elasticity(E, N, Q, _d(wdetJ), _d(G), _d(_f64(D)), _d(K)))
    return K


def residual_laplace(conn, wdetJ, G, u, coef=None):
    E, Q, _, N = G.shape
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    r = np.zeros((E, N))
    _check(lib().oracle_residual_laplace(E, N, Q, _i(conn), _d(wdetJ), _d(G), _d(_f64(coef)), _d(_f64(u)), _d(r)))
    return r


def residual_mass(conn, wdetJ, phi, u, ncomp=1, coef=None):
    E, Q = wdetJ.shape
    N = phi.shape[1]
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    r = np.zeros((E, ncomp * N))
    _check(lib().oracle_residual_mass(E, N, Q, ncomp, _i(conn), _d(wdetJ), _d(_f64(phi)), _d(_f64(coef)),
                                      _d(_f64(u)), _d(r)))
    return r


def residual_elasticity(conn, wdetJ, G, D, u):
    E, Q, _, N = G.shape
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    r = np.zeros((E, 3 * N))
    _check(lib().oracle_residual_elasticity(E, N, Q, _i(conn), _d(wdetJ), _d(G), _d(_f64(D)), _d(_f64(u)), _d(r)))
    return r


def residual_convect(conn, wdetJ, phi, G, u, w=None):
    """Convective term 'i,i.j,j' (Eq. fe2): r[e, i*N+a] = sum_q wdetJ phi_a (grad u_h)_ij w_h,j;
    w defaults to u (the non-linear term)."""
    E, Q, _, N = G.shape
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    u = _f64(u)
    w = u if w is None else _f64(w)
    r = np.zeros((E, 3 * N))
    _check(lib().oracle_residual_convect(E, N, Q, _i(conn), _d(wdetJ), _d(_f64(phi)), _d(G), _d(u), _d(w), _d(r)))
    return r


def matrix_convect(conn, wdetJ, phi, G, u, w=None, wrt_u=True, wrt_w=True):
    """Derivative of the convective term (Eq. fe4) with respect to the gradient
    operand u (wrt_u) and/or the advection operand w (wrt_w); w defaults to u."""
    E, Q, _, N = G.shape
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    u = _f64(u)
    w = u if w is None else _f64(w)
    K = np.zeros((E, 3 * N, 3 * N))
    _check(lib().oracle_matrix_convect(E, N, Q, _i(conn), _d(wdetJ), _d(_f64(phi)), _d(G), _d(u), _d(w),
                                       int(bool(wrt_u)), int(bool(wrt_w)), _d(K)))
    return K


def adjoint_elasticity_terms(conn, wdetJ, G, lam, mu, u, rbar):
    """Per-element derivatives of sum_e rbar_e . r_e for the isotropic elasticity
    residual: (dlam (E,), dmu (E,), dX_e (E, 3*N) component-major); see oracle.c."""
    E, Q, _, N = G.shape
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    dlam, dmu, dX = np.zeros(E), np.zeros(E), np.zeros((E, 3 * N))
    _check(lib().oracle_adjoint_elasticity(E, N, Q, _i(conn), _d(wdetJ), _d(G), _d(_f64(lam)), _d(_f64(mu)),
                                           _d(_f64(u)), _d(_f64(rbar)), _d(dlam), _d(dmu), _d(dX)))
    return dlam, dmu, dX


def elasticity_objective(coords, conn, ref: RefElement, lam, mu, u):
    """J = |R|^2 / 2 with R the assembled isotropic elasticity residual (3 per node)."""
    wdetJ, G, _ = geometry(coords, conn, ref)
    r = residual_elasticity(conn, wdetJ, G, lame_to_D(lam, mu), u)
    R = assemble(conn, r, np.asarray(coords).shape[0], 3)
    return 0.5 * float(R @ R), R


def elasticity_objective_gradient(coords, conn, ref: RefElement, lam, mu, u):
    """J and its gradient with respect to lambda_e, mu_e and the node coordinates
    (n_nodes, 3): rbar = R, per-element terms, dX_e assembled over the mesh."""
    J, R = elasticity_objective(coords, conn, ref, lam, mu, u)
    wdetJ, G, _ = geometry(coords, conn, ref)
    dlam, dmu, dXe = adjoint_elasticity_terms(conn, wdetJ, G, lam, mu, u, R)
    dX = assemble(conn, dXe, np.asarray(coords).shape[0], 3).reshape(-1, 3)
    return J, dlam, dmu, dX


def matrix_wdot(wdetJ, phi, M):
    """Weighted dot product 'ij,i,j': K[(i,a),(j,b)] = M_ij sum_q wdetJ phi_a phi_b."""
    E, Q = wdetJ.shape
    N = phi.shape[1]
    K = np.zeros((E, 3 * N, 3 * N))
    _check(lib().oracle_matrix_wdot(E, N, Q, _d(wdetJ), _d(_f64(phi)), _d(_f64(M)), _d(K)))
    return K


def residual_wdot(conn, wdetJ, phi, M, u):
    E, Q = wdetJ.shape
    N = phi.shape[1]
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    r = np.zeros((E, 3 * N))
    _check(lib().oracle_residual_wdot(E, N, Q, _i(conn), _d(wdetJ), _d(_f64(phi)), _d(_f64(M)), _d(_f64(u)), _d(r)))
    return r


def matrix_stokes(wdetJ, G, phi):
    """Stokes coupling 'i.i,0' (v, p): B[(i,a), b] = sum_q wdetJ G[i][a] phi_b; the
    transposed coupling (u, q) has B^T."""
    E, Q, _, N = G.shape
    B = np.zeros((E, 3 * N, N))
    _check(lib().oracle_matrix_stokes(E, N, Q, _d(wdetJ), _d(G), _d(_f64(phi)), _d(B)))
    return B


def residual_stokes(conn, wdetJ, G, phi, p=None):
    """r[(i,a)] = sum_q wdetJ G[i][a] p_h; p = None: the divergence form 'i.i'."""
    E, Q, _, N = G.shape
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    r = np.zeros((E, 3 * N))
    _check(lib().oracle_residual_stokes(E, N, Q, _i(conn), _d(wdetJ), _d(G), _d(_f64(phi)),
                                        _d(_f64(p) if p is not None else None), _d(r)))
    return r


def residual_stokes_t(conn, wdetJ, G, phi, u):
    """r[a] = sum_q wdetJ phi_a div(u_h)."""
    E, Q, _, N = G.shape
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    r = np.zeros((E, N))
    _check(lib().oracle_residual_stokes_t(E, N, Q, _i(conn), _d(wdetJ), _d(G), _d(_f64(phi)), _d(_f64(u)), _d(r)))
    return r


def matrix_stokes_mixed(wdetJ, G, psi):
    """Stokes coupling 'i.i,0' of a vector field on the geometry's basis (G: E, Q, 3, N)
    and a scalar field on a second basis (psi: Q, Np at the same points):
    B[(i,a), b] = sum_q wdetJ G[i][a] psi_b, shape (E, 3N, Np); the transposed
    coupling has B^T."""
    E, Q, _, N = G.shape
    psi = _f64(psi)
    Np = psi.shape[1]
    B = np.zeros((E, 3 * N, Np))
    _check(lib().oracle_matrix_stokes_mixed(E, N, Np, Q, _d(wdetJ), _d(G), _d(psi), _d(B)))
    return B


def residual_stokes_mixed(conn_p, wdetJ, G, psi, p):
    """r[(i,a)] = sum_q wdetJ G[i][a] p_h, p_h = sum_b psi_b p[conn_p[e][b]]."""
    E, Q, _, N = G.shape
    psi = _f64(psi)
    conn_p = np.ascontiguousarray(conn_p, dtype=np.int32)
    r = np.zeros((E, 3 * N))
    _check(lib().oracle_residual_stokes_mixed(E, N, psi.shape[1], Q, _i(conn_p), _d(wdetJ), _d(G), _d(psi),
                                              _d(_f64(p)), _d(r)))
    return r


def residual_stokes_t_mixed(conn, wdetJ, G, psi, u):
    """r[b] = sum_q wdetJ psi_b div(u_h), u_h on the geometry's basis via conn."""
    E, Q, _, N = G.shape
    psi = _f64(psi)
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    r = np.zeros((E, psi.shape[1]))
    _check(lib().oracle_residual_stokes_t_mixed(E, N, psi.shape[1], Q, _i(conn), _d(wdetJ), _d(G), _d(psi),
                                                _d(_f64(u)), _d(r)))
    return r


EVAL_KINDS = {"laplace": 0, "mass": 1, "elasticity": 2, "wdot": 3, "stokes": 4, "div": 5, "cauchy": 6,
              "convect": 7}


def eval_form(kind, conn, wdetJ, G, phi, u, w=None, z=None, coef=None, mat=None, ncomp=3):
    """'eval' mode integrals per element (E, 1) or (E, 6) for the Cauchy stress."""
    E, Q, _, N = G.shape
    k = EVAL_KINDS[kind]
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    out = np.zeros((E, 6 if kind == "cauchy" else 1))
    f = lambda a: _d(_f64(a)) if a is not None else _d(None)
    _check(lib().oracle_eval_form(k, E, N, Q, ncomp, _i(conn), _d(wdetJ), _d(G), _d(_f64(phi)), f(coef), f(mat),
                                  _d(_f64(u)), f(w), f(z), _d(out)))
    return out


def assemble(conn, r, n_nodes, ncomp, g=None):
    """g[ncomp*conn[e,a] + i] += r[e, i*N + a], ascending (e, a, i)."""
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    E, N = conn.shape
    r = _f64(r).reshape(E, ncomp * N)
    acc = 1 if g is not None else 0
    out = np.zeros(n_nodes * ncomp) if g is None else _f64(g).copy()
    _check(lib().oracle_assemble(E, N, ncomp, _i(conn), _d(r), n_nodes, acc, _d(out)))
    return out
