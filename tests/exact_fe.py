"""Exact rational 1-D Lagrange integrals, used to pin the oracle on undistorted boxes.

Everything here is exact (fractions.Fraction): polynomials are coefficient lists,
integrals over [0, 1] are sums of c_n / (n + 1).  Nothing is shared with the
oracle's C code or with the CUDA library.
"""
from fractions import Fraction

import numpy as np


def _pmul(a, b):
    out = [Fraction(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def _pder(a):
    return [a[n] * n for n in range(1, len(a))] or [Fraction(0)]


def _pint01(a):
    return sum((c / (n + 1) for n, c in enumerate(a)), Fraction(0))


def lagrange_polys(p):
    """Coefficients of L_k on equispaced nodes t_m = m/p, k = 0..p."""
    nodes = [Fraction(m, p) for m in range(p + 1)]
    polys = []
    for k in range(p + 1):
        poly = [Fraction(1)]
        for m in range(p + 1):
            if m == k:
                continue
            poly = _pmul(poly, [-nodes[m] / (nodes[k] - nodes[m]), 1 / (nodes[k] - nodes[m])])
        polys.append(poly)
    return polys


def matrices_1d(p):
    """Exact 1-D stiffness k_ab = int L_a' L_b', mass m_ab = int L_a L_b,
    and c_ab = int L_a' L_b over [0, 1], as float arrays."""
    L = lagrange_polys(p)
    dL = [_pder(x) for x in L]
    n = p + 1
    k = [[_pint01(_pmul(dL[a], dL[b])) for b in range(n)] for a in range(n)]
    m = [[_pint01(_pmul(L[a], L[b])) for b in range(n)] for a in range(n)]
    c = [[_pint01(_pmul(dL[a], L[b])) for b in range(n)] for a in range(n)]
    f = lambda M: np.array([[float(x) for x in row] for row in M])
    return f(k), f(m), f(c)


def _kron3(Mx, My, Mz):
    # node index i + n j + n^2 k (x fastest) -> kron(z, y, x)
    return np.kron(Mz, np.kron(My, Mx))


def box_gradient_blocks(p, h):
    """P[j][l][a][b] = int_box d_j phi_a d_l phi_b for the box [0,hx]x[0,hy]x[0,hz]."""
    k, m, c = matrices_1d(p)
    P = [[None] * 3 for _ in range(3)]
    for j in range(3):
        for l in range(3):
            fac = []
            for d in range(3):
                if d == j and d == l:
                    fac.append(k / h[d])
                elif d == j:
                    fac.append(c)
                elif d == l:
                    fac.append(c.T)
                else:
                    fac.append(m * h[d])
            P[j][l] = _kron3(*fac)
    return P


def box_laplace(p, h):
    P = box_gradient_blocks(p, h)
    return P[0][0] + P[1][1] + P[2][2]


def box_mass(p, h):
    k, m, c = matrices_1d(p)
    return _kron3(m * h[0], m * h[1], m * h[2])


def box_elasticity(p, h, lam, mu):
    """K[(i,a),(k,b)] = sum_{j,l} C_ijkl int d_j phi_a d_l phi_b with the isotropic
    stiffness C_ijkl = lam d_ij d_kl + mu (d_ik d_jl + d_il d_jk)."""
    P = box_gradient_blocks(p, h)
    N = (p + 1) ** 3
    K = np.zeros((3 * N, 3 * N))
    d = np.eye(3)
    for i in range(3):
        for kk in range(3):
            blk = np.zeros((N, N))
            for j in range(3):
                for l in range(3):
                    C = lam * d[i, j] * d[kk, l] + mu * (d[i, kk] * d[j, l] + d[i, l] * d[j, kk])
                    if C != 0.0:
                        blk += C * P[j][l]
            K[i * N:(i + 1) * N, kk * N:(kk + 1) * N] = blk
    return K


def moments_1d(p):
    """Exact 1-D integrals over [0, 1] with the test function L_a first:
    m_ab = int L_a L_b, d_ab = int L_a L_b', xm_ab = int t L_a L_b, xd_ab = int t L_a L_b'."""
    L = lagrange_polys(p)
    dL = [_pder(x) for x in L]
    t = [Fraction(0), Fraction(1)]
    n = p + 1
    m = [[_pint01(_pmul(L[a], L[b])) for b in range(n)] for a in range(n)]
    d = [[_pint01(_pmul(L[a], dL[b])) for b in range(n)] for a in range(n)]
    xm = [[_pint01(_pmul(t, _pmul(L[a], L[b]))) for b in range(n)] for a in range(n)]
    xd = [[_pint01(_pmul(t, _pmul(L[a], dL[b]))) for b in range(n)] for a in range(n)]
    f = lambda M: np.array([[float(x) for x in row] for row in M])
    return f(m), f(d), f(xm), f(xd)


def box_convection(p, h, x0, A, c):
    """C_ab = int_box phi_a (w . grad phi_b) for the linear field w(x) = A x + c on
    the box x0 + [0,h0]x[0,h1]x[0,h2], from separable 1-D integrals: on axis e the
    factor is m h_e, or d on the differentiated axis (the 1/h and h cancel), and
    x_d = x0_d + h_d t contributes x0_d (factor) + h_d (the t-moment factor)."""
    m, d, xm, xd = moments_1d(p)
    h = np.asarray(h, dtype=float)
    x0 = np.asarray(x0, dtype=float)

    def factors(j):
        return [d if e == j else m * h[e] for e in range(3)]

    N = (p + 1) ** 3
    C = np.zeros((N, N))
    for j in range(3):
        base = factors(j)
        Ij = _kron3(*base)
        C += (c[j] + sum(A[j, dd] * x0[dd] for dd in range(3))) * Ij
        for dd in range(3):
            if A[j, dd] == 0.0:
                continue
            fac = list(base)
            fac[dd] = xd if dd == j else xm * h[dd]
            C += A[j, dd] * h[dd] * _kron3(*fac)
    return C


def box_stokes_blocks(p, h):
    """B_i[a][b] = int_box (d phi_a / d x_i) phi_b, i = 0, 1, 2: on axis i the
    derivative factor int L_a' L_b (the 1/h and h cancel), m h elsewhere."""
    m, d, xm, xd = moments_1d(p)
    h = np.asarray(h, dtype=float)
    return [_kron3(*[d.T if e == i else m * h[e] for e in range(3)]) for i in range(3)]


def box_stokes_mixed_blocks(pu, pp, h):
    """B_i[a][b] = int_box (d phi_a / d x_i) psi_b with phi of order pu and psi of
    order pp (equispaced Lagrange, tensor products): on axis i the factor
    int L_a^(pu)' L_b^(pp) (the 1/h and h cancel), int L_a^(pu) L_b^(pp) h elsewhere."""
    Lu, Lp = lagrange_polys(pu), lagrange_polys(pp)
    dLu = [_pder(x) for x in Lu]
    f = lambda M: np.array([[float(x) for x in row] for row in M])
    mm = f([[_pint01(_pmul(Lu[a], Lp[b])) for b in range(pp + 1)] for a in range(pu + 1)])
    dm = f([[_pint01(_pmul(dLu[a], Lp[b])) for b in range(pp + 1)] for a in range(pu + 1)])
    h = np.asarray(h, dtype=float)
    return [_kron3(*[dm if e == i else mm * h[e] for e in range(3)]) for i in range(3)]
