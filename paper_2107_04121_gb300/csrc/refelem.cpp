// Reference hexahedron of libfe: order-p Lagrange basis and tensor Gauss rules,
// tabulated on the host (the isoparametric basis of Sec. 4.1 of Cimrman,
// arXiv 2107.04121; (p+1)^3 Gauss points per Tab. cdc).
//
// The Gauss-Legendre rule is computed by the Golub-Welsch method: the nodes are
// the eigenvalues of the symmetric tridiagonal Jacobi matrix of the Legendre
// recurrence (off-diagonal k / sqrt(4k^2 - 1)), the weights are 2 v_0^2 of the
// normalised eigenvectors.  The eigenproblem is solved with cyclic Jacobi
// rotations, which is plenty for n <= 10.
#include <cmath>
#include <utility>
#include <cstring>
#include <vector>

#include "fe_internal.h"

int fe_host_gauss_legendre01(int n, double *x, double *w)
{
    if (n < 1 || n > 16) return -1;
    double A[16][16] = {{0}}, V[16][16] = {{0}};
    for (int i = 0; i < n; ++i) V[i][i] = 1.0;
    for (int k = 1; k < n; ++k) {
        double b = k / std::sqrt(4.0 * k * k - 1.0);
        A[k - 1][k] = A[k][k - 1] = b;
    }
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) off += A[i][j] * A[i][j];
        if (off < 1e-34) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                if (A[p][q] == 0.0) continue;
                // rotation that annihilates A[p][q]
                double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {  // A <- A R
                    double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  // A <- R^T A
                    double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {  // V <- V R
                    double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
            }
    }
    // sort eigenpairs ascending
    int idx[16];
    for (int i = 0; i < n; ++i) idx[i] = i;
    for (int i = 1; i < n; ++i)
        for (int j = i; j > 0 && A[idx[j]][idx[j]] < A[idx[j - 1]][idx[j - 1]]; --j) {
            int t = idx[j];
            idx[j] = idx[j - 1];
            idx[j - 1] = t;
        }
    for (int i = 0; i < n; ++i) {
        int k = idx[i];
        double v0 = V[0][k];
        double nrm = 0.0;
        for (int r = 0; r < n; ++r) nrm += V[r][k] * V[r][k];
        x[i] = 0.5 * (A[k][k] + 1.0);
        w[i] = v0 * v0 / nrm;  // 2 v0^2 on [-1,1], halved on [0,1]
    }
    // symmetric rule: enforce exact symmetry of points and weights
    for (int i = 0; i < n / 2; ++i) {
        double xm = 0.5 * (x[i] + (1.0 - x[n - 1 - i]));
        double wm = 0.5 * (w[i] + w[n - 1 - i]);
        x[i] = xm;
        x[n - 1 - i] = 1.0 - xm;
        w[i] = w[n - 1 - i] = wm;
    }
    if (n % 2) x[n / 2] = 0.5;
    return 0;
}

// Lagrange polynomial k of the equispaced nodes {m/p} and its derivative at t.
static void lagrange1d(int p, int k, double t, double *val, double *der)
{
    double tk = (double)k / p;
    double v = 1.0, d = 0.0;
    for (int m = 0; m <= p; ++m) {
        if (m == k) continue;
        double f = (t - (double)m / p) / (tk - (double)m / p);
        double df = 1.0 / (tk - (double)m / p);
        d = d * f + v * df;  // (v f)' = v' f + v f'
        v = v * f;
    }
    *val = v;
    *der = d;
}

extern "C" fe_status fe_refbasis_hex(int p, int nq, double *points, double *weights, double *phi, double *dphi)
{
    fe_clear_last_error();
    if (p < 1 || p > 4 || nq < 1 || nq > 10) return FE_ERR_SHAPE;
    double g[16], gw[16];
    if (fe_host_gauss_legendre01(nq, g, gw)) return FE_ERR_SHAPE;
    const int n1 = p + 1, N = n1 * n1 * n1, Q = nq * nq * nq;
    double L[10][5], dL[10][5];
    for (int q = 0; q < nq; ++q)
        for (int k = 0; k < n1; ++k) lagrange1d(p, k, g[q], &L[q][k], &dL[q][k]);
    for (int qz = 0; qz < nq; ++qz)
        for (int qy = 0; qy < nq; ++qy)
            for (int qx = 0; qx < nq; ++qx) {
                const int q = qx + nq * (qy + nq * qz);
                if (points) {
                    points[3 * q + 0] = g[qx];
                    points[3 * q + 1] = g[qy];
                    points[3 * q + 2] = g[qz];
                }
                if (weights) weights[q] = gw[qx] * gw[qy] * gw[qz];
                for (int k = 0; k < n1; ++k)
                    for (int j = 0; j < n1; ++j)
                        for (int i = 0; i < n1; ++i) {
                            const int a = i + n1 * (j + n1 * k);
                            if (phi) phi[(size_t)q * N + a] = L[qx][i] * L[qy][j] * L[qz][k];
                            if (dphi) {
                                dphi[((size_t)q * 3 + 0) * N + a] = dL[qx][i] * L[qy][j] * L[qz][k];
                                dphi[((size_t)q * 3 + 1) * N + a] = L[qx][i] * dL[qy][j] * L[qz][k];
                                dphi[((size_t)q * 3 + 2) * N + a] = L[qx][i] * L[qy][j] * dL[qz][k];
                            }
                        }
            }
    (void)Q;
    return FE_OK;
}

extern "C" fe_status fe_refbasis_hex_1d(int p, int nq, double *b1d, double *d1d)
{
    fe_clear_last_error();
    if (p < 1 || p > 4 || nq < 1 || nq > 10 || !b1d || !d1d) return p < 1 || p > 4 || nq < 1 || nq > 10
                                                                          ? FE_ERR_SHAPE
                                                                          : FE_ERR_INVALID_ARG;
    double g[16], gw[16];
    if (fe_host_gauss_legendre01(nq, g, gw)) return FE_ERR_SHAPE;
    for (int q = 0; q < nq; ++q)
        for (int k = 0; k <= p; ++k) lagrange1d(p, k, g[q], &b1d[q * (p + 1) + k], &d1d[q * (p + 1) + k]);
    return FE_OK;
}

// Collocation derivative on the quadrature points of one axis, n1 == nq:
// the nq point values of a polynomial of degree n1 - 1 determine it, so its
// derivatives at the points are Dq (values at the points) with Dq = D B^-1
// (B, D: (nq, n1) values and derivatives of the 1-D nodal basis).  Gauss-Jordan
// with partial pivoting in FP64; false when B is (numerically) singular or the
// product does not reproduce D.
bool fe_host_collocation_derivative(int n, const double *b1d, const double *d1d, double *dq)
{
    if (n < 1 || n > 8) return false;
    double A[8][8], Ainv[8][8];
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) {
            A[r][c] = b1d[r * n + c];
            Ainv[r][c] = r == c ? 1.0 : 0.0;
        }
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
        if (!(std::fabs(A[piv][c]) > 1e-12)) return false;
        for (int k = 0; k < n; ++k) {
            std::swap(A[c][k], A[piv][k]);
            std::swap(Ainv[c][k], Ainv[piv][k]);
        }
        const double inv = 1.0 / A[c][c];
        for (int k = 0; k < n; ++k) {
            A[c][k] *= inv;
            Ainv[c][k] *= inv;
        }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double f = A[r][c];
            if (f == 0.0) continue;
            for (int k = 0; k < n; ++k) {
                A[r][k] -= f * A[c][k];
                Ainv[r][k] -= f * Ainv[c][k];
            }
        }
    }
    // B is (point, node); B^-1 maps point values to nodal values: dq = D B^-1
    double scale = 1.0;
    for (int i = 0; i < n * n; ++i) scale = std::fmax(scale, std::fabs(d1d[i]));
    for (int q = 0; q < n; ++q)
        for (int p = 0; p < n; ++p) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) s += d1d[q * n + k] * Ainv[k][p];
            dq[q * n + p] = s;
        }
    for (int q = 0; q < n; ++q)
        for (int k = 0; k < n; ++k) {
            double s = 0.0;
            for (int p = 0; p < n; ++p) s += dq[q * n + p] * b1d[p * n + k];
            if (std::fabs(s - d1d[q * n + k]) > 1e-12 * scale) return false;
        }
    return true;
}

// Does the tensor product of the 1-D factors reproduce the 3-D tables?
bool fe_host_check_tensor_basis(const fe_refbasis *b)
{
    const int n1 = b->n1d, nq = b->nq1d;
    if (n1 < 1 || nq < 1 || n1 * n1 * n1 != b->n_basis || nq * nq * nq != b->n_qp) return false;
    double scale = 0.0;
    for (int i = 0; i < b->n_qp * 3 * b->n_basis; ++i) scale = std::fmax(scale, std::fabs(b->dphi[i]));
    for (int i = 0; i < b->n_qp * b->n_basis; ++i) scale = std::fmax(scale, std::fabs(b->phi[i]));
    const double tol = 1e-13 * (scale > 1.0 ? scale : 1.0);
    for (int qz = 0; qz < nq; ++qz)
        for (int qy = 0; qy < nq; ++qy)
            for (int qx = 0; qx < nq; ++qx)
                for (int k = 0; k < n1; ++k)
                    for (int j = 0; j < n1; ++j)
                        for (int i = 0; i < n1; ++i) {
                            const int q = qx + nq * (qy + nq * qz), a = i + n1 * (j + n1 * k);
                            const double bx = b->b1d[qx * n1 + i], by = b->b1d[qy * n1 + j], bz = b->b1d[qz * n1 + k];
                            const double dx = b->d1d[qx * n1 + i], dy = b->d1d[qy * n1 + j], dz = b->d1d[qz * n1 + k];
                            const size_t N = b->n_basis;
                            if (std::fabs(b->phi[q * N + a] - bx * by * bz) > tol) return false;
                            if (std::fabs(b->dphi[(q * 3 + 0) * N + a] - dx * by * bz) > tol) return false;
                            if (std::fabs(b->dphi[(q * 3 + 1) * N + a] - bx * dy * bz) > tol) return false;
                            if (std::fabs(b->dphi[(q * 3 + 2) * N + a] - bx * by * dz) > tol) return false;
                        }
    return true;
}

// ---------------------------------------------------------------------------
// Reference tetrahedron {x, y, z >= 0, x + y + z <= 1} with barycentric
// coordinates l0 = 1 - x - y - z, l1 = x, l2 = y, l3 = z.
//
// Grundmann-Moller rule of index s (Grundmann & Moller, SIAM J. Numer. Anal.
// 15 (1978)), exact for polynomials of degree 2s + 1: with d = 2s + 1 and n = 3,
//   Q f = sum_{i=0}^{s} (-1)^i 2^{-2s} (d + n - 2i)^d / (i! (d + n - i)!)
//         sum_{|beta| = s - i} f( (2 beta + 1) / (d + n - 2i) ),
// beta running over the 4-part compositions of s - i (barycentric point
// coordinates); the weights integrate over the tetrahedron itself (sum 1/6).
// Points are listed by i, then by beta in lexicographic order (beta_0 slowest).
static int gm_points(int s, double *pts, double *wts)
{
    const int d = 2 * s + 1, n = 3;
    int np = 0;
    for (int i = 0; i <= s; ++i) {
        const int m = s - i, den = d + n - 2 * i;
        // (-1)^i 2^{-2s} den^d / (i! (d + n - i)!)
        double w = (i % 2 ? -1.0 : 1.0) * std::ldexp(1.0, -2 * s);
        for (int t = 0; t < d; ++t) w *= den;
        for (int t = 2; t <= i; ++t) w /= t;
        for (int t = 2; t <= d + n - i; ++t) w /= t;
        for (int b0 = m; b0 >= 0; --b0)
            for (int b1 = m - b0; b1 >= 0; --b1)
                for (int b2 = m - b0 - b1; b2 >= 0; --b2) {
                    const int b3 = m - b0 - b1 - b2;
                    if (pts) {
                        pts[3 * np + 0] = (2.0 * b1 + 1.0) / den;
                        pts[3 * np + 1] = (2.0 * b2 + 1.0) / den;
                        pts[3 * np + 2] = (2.0 * b3 + 1.0) / den;
                    }
                    if (wts) wts[np] = w;
                    ++np;
                }
    }
    return np;
}

// 1-D factor of the barycentric Lagrange basis: prod_{t < n} (p l - t) / (t + 1)
// and its derivative with respect to l.
static void bary_factor(int p, int n, double l, double *val, double *der)
{
    double v = 1.0, dv = 0.0;
    for (int t = 0; t < n; ++t) {
        const double f = (p * l - t) / (t + 1.0), df = p / (t + 1.0);
        dv = dv * f + v * df;
        v *= f;
    }
    *val = v;
    *der = dv;
}

extern "C" int fe_gm_rule_size(int s)
{
    if (s < 0 || s > 6) return -1;
    return gm_points(s, nullptr, nullptr);
}

extern "C" fe_status fe_refbasis_tet(int p, int s, double *points, double *weights, double *phi, double *dphi)
{
    fe_clear_last_error();
    if (p < 1 || p > 3 || s < 0 || s > 6) return FE_ERR_SHAPE;
    double qp[3 * 512], qw[512];
    const int Q = gm_points(s, qp, qw);
    const int N = (p + 1) * (p + 2) * (p + 3) / 6;
    int idx[20][4];  // barycentric multi-indices of the lattice nodes, x fastest
    int a = 0;
    for (int k = 0; k <= p; ++k)
        for (int j = 0; j <= p - k; ++j)
            for (int i = 0; i <= p - k - j; ++i) {
                idx[a][0] = p - i - j - k;
                idx[a][1] = i;
                idx[a][2] = j;
                idx[a][3] = k;
                ++a;
            }
    for (int q = 0; q < Q; ++q) {
        const double x = qp[3 * q], y = qp[3 * q + 1], z = qp[3 * q + 2];
        const double l[4] = {1.0 - x - y - z, x, y, z};
        if (points)
            for (int c = 0; c < 3; ++c) points[3 * q + c] = qp[3 * q + c];
        if (weights) weights[q] = qw[q];
        for (int b = 0; b < N; ++b) {
            double f[4], df[4];
            for (int m = 0; m < 4; ++m) bary_factor(p, idx[b][m], l[m], &f[m], &df[m]);
            if (phi) phi[(size_t)q * N + b] = f[0] * f[1] * f[2] * f[3];
            if (dphi)
                for (int c = 0; c < 3; ++c) {
                    // d l0 / dx_c = -1, d l_(c+1) / dx_c = 1
                    double g = -df[0] * f[1] * f[2] * f[3];
                    double t = df[c + 1];
                    for (int m = 1; m < 4; ++m)
                        if (m != c + 1) t *= f[m];
                    g += t * f[0];
                    dphi[((size_t)q * 3 + c) * N + b] = g;
                }
        }
    }
    return FE_OK;
}

int fe_host_simplex_order(int N, int Q, const double *phi, double *xi)
{
    for (int p = 1; p <= 3; ++p) {
        if (N != (p + 1) * (p + 2) * (p + 3) / 6) continue;
        for (int s = 0; s <= 6; ++s) {
            if (fe_gm_rule_size(s) != Q) continue;
            std::vector<double> ref((size_t)Q * N);
            if (fe_refbasis_tet(p, s, nullptr, nullptr, ref.data(), nullptr) != FE_OK) continue;
            bool same = true;
            for (size_t k = 0; k < ref.size() && same; ++k) same = std::fabs(ref[k] - phi[k]) <= 1e-13;
            if (!same) continue;
            // lattice points (i, j, k) / p, x fastest (the basis' node order)
            int a = 0;
            for (int k = 0; k <= p; ++k)
                for (int j = 0; j <= p - k; ++j)
                    for (int i = 0; i <= p - k - j; ++i, ++a) {
                        xi[3 * a] = (double)i / p;
                        xi[3 * a + 1] = (double)j / p;
                        xi[3 * a + 2] = (double)k / p;
                    }
            return p;
        }
    }
    return 0;
}
