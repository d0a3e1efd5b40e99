/*
 * Oracle for the finite element weak-form evaluator: plain, slow, FP64 CPU code.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the CPU-baseline leg of the benchmark load this library.  The product path
 * (the CUDA library and its binding) never calls it and shares no code with it:
 * the reference element, the quadrature rule, the geometry mapping, the forms
 * and the assembly are all written again here, independently, as the plain
 * definitions that Cimrman, "Fast Evaluation of Finite Element Weak Forms Using
 * Python Tensor Contraction Packages" (arXiv 2107.04121) states them.
 *
 * Every element loop is the nested cells x quadrature-points loop of
 * Algorithm 1 (residual mode) and Algorithm 2 (matrix mode) of the paper, Sec. 4.1.
 * The only parallelism is an OpenMP "parallel for" over elements; each element
 * is computed with the same sequential loops whatever the thread count.
 *
 * Conventions the paper leaves open, fixed here:
 *  - reference hexahedron [0,1]^3; order-p Lagrange nodes equispaced, numbered
 *    lexicographically with x fastest: node (i,j,k) -> i + (p+1) j + (p+1)^2 k;
 *  - Gauss-Legendre points on [0,1], same lexicographic order, weights sum to 1;
 *  - vector element DOFs component-major: local index = comp * N + a
 *    (the "cresf" output order of the elasticity expression, Sec. 5.3.3);
 *  - global vector DOF index = ncomp * node + comp;
 *  - Voigt order (11, 22, 33, 12, 13, 23) with engineering shear strains.
 *
 * Parity status: every function below is pinned by CPU tests against closed
 * forms, exact rational integrals, library routines or invariants (see the
 * pins in tests/test_oracle_pins.py).
 */
#define _USE_MATH_DEFINES
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846264338327950288
#endif

#define OR_OK 0
#define OR_BAD_ARG -1
/* A positive return value k means element k-1 had det J <= 0. */

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre rule (oracle_gauss_1d): Newton iteration on P_n evaluated with the three-term
 * recurrence (n+1) P_{n+1} = (2n+1) x P_n - n P_{n-1}, derivative from
 * (1-x^2) P_n' = n (P_{n-1} - x P_n).  Points mapped from [-1,1] to [0,1]. */
/* P_n(x) and P_{n-1}(x) by the three-term recurrence, starting at P_0 = 1, P_1 = x. */
static void legendre_pair(int n, double x, double *pn_out, double *pm_out)
{
    double pm = 1.0, pn = x;
    for (int k = 1; k < n; ++k) {
        double next = ((2.0 * k + 1.0) * x * pn - k * pm) / (k + 1.0);
        pm = pn;
        pn = next;
    }
    *pn_out = pn;
    *pm_out = pm;
}

int oracle_gauss_1d(int n, double *pts, double *wts)
{
    if (n < 1 || n > 64 || !pts || !wts) return OR_BAD_ARG;
    for (int i = 0; i < n; ++i) {
        /* initial guess for the i-th root, counted from the right end */
        double x = cos(M_PI * (i + 0.75) / (n + 0.5));
        double pn, pm, dp;
        for (int it = 0; it < 100; ++it) {
            legendre_pair(n, x, &pn, &pm);
            dp = n * (pm - x * pn) / (1.0 - x * x);
            double dx = pn / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        legendre_pair(n, x, &pn, &pm);
        dp = n * (pm - x * pn) / (1.0 - x * x);
        double w = 2.0 / ((1.0 - x * x) * dp * dp);
        /* ascending order on [0,1] */
        pts[n - 1 - i] = 0.5 * (x + 1.0);
        wts[n - 1 - i] = 0.5 * w;
    }
    return OR_OK;
}

/* 1-D Lagrange polynomial L_k on equispaced nodes t_m = m/p, m = 0..p:
 * L_k(t) = prod_{m != k} (t - t_m) / (t_k - t_m); derivative by the product rule. */
static double lagrange_1d(int p, int k, double t)
{
    double v = 1.0;
    for (int m = 0; m <= p; ++m) {
        if (m == k) continue;
        v *= (t - (double)m / p) / ((double)(k - m) / p);
    }
    return v;
}

static double lagrange_1d_deriv(int p, int k, double t)
{
    double s = 0.0;
    for (int l = 0; l <= p; ++l) {
        if (l == k) continue;
        double term = 1.0 / ((double)(k - l) / p);
        for (int m = 0; m <= p; ++m) {
            if (m == k || m == l) continue;
            term *= (t - (double)m / p) / ((double)(k - m) / p);
        }
        s += term;
    }
    return s;
}

/* Tensor-product Lagrange basis of order p on the reference hexahedron,
 * evaluated at n_pts points (n_pts, 3): phi (n_pts, N), dphi (n_pts, 3, N)
 * with dphi[q][k][a] = d phi_a / d xi_k (Sec. 4.1, isoparametric basis). */
int oracle_hex_basis(int p, int n_pts, const double *pts, double *phi, double *dphi)
{
    if (p < 1 || p > 8 || n_pts < 1 || !pts || !phi || !dphi) return OR_BAD_ARG;
    int n1 = p + 1, N = n1 * n1 * n1;
    for (int q = 0; q < n_pts; ++q) {
        double x = pts[3 * q], y = pts[3 * q + 1], z = pts[3 * q + 2];
        for (int k = 0; k < n1; ++k)
            for (int j = 0; j < n1; ++j)
                for (int i = 0; i < n1; ++i) {
                    int a = i + n1 * j + n1 * n1 * k;
                    double lx = lagrange_1d(p, i, x), ly = lagrange_1d(p, j, y), lz = lagrange_1d(p, k, z);
                    double dx = lagrange_1d_deriv(p, i, x), dy = lagrange_1d_deriv(p, j, y),
                           dz = lagrange_1d_deriv(p, k, z);
                    phi[(size_t)q * N + a] = lx * ly * lz;
                    dphi[((size_t)q * 3 + 0) * N + a] = dx * ly * lz;
                    dphi[((size_t)q * 3 + 1) * N + a] = lx * dy * lz;
                    dphi[((size_t)q * 3 + 2) * N + a] = lx * ly * dz;
                }
    }
    return OR_OK;
}

/* Tensor-product Gauss rule with nq points per axis on [0,1]^3, lexicographic
 * (x fastest): pts (nq^3, 3), w (nq^3). */
int oracle_hex_quadrature(int nq, double *pts, double *w)
{
    if (nq < 1 || nq > 16 || !pts || !w) return OR_BAD_ARG;
    double g[16], gw[16];
    int rc = oracle_gauss_1d(nq, g, gw);
    if (rc) return rc;
    for (int k = 0; k < nq; ++k)
        for (int j = 0; j < nq; ++j)
            for (int i = 0; i < nq; ++i) {
                int q = i + nq * j + nq * nq * k;
                pts[3 * q] = g[i];
                pts[3 * q + 1] = g[j];
                pts[3 * q + 2] = g[k];
                w[q] = gw[i] * gw[j] * gw[k];
            }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Geometry (Sec. 4.1): x(xi) = sum_a x^a phi_a(xi), J_ij = d x_i / d xi_j,
 * d/dx_j = d/dxi_k (J^-1)_kj.  Per element e and quadrature point q:
 *   wdetJ[e][q]     = w_q det J      (the "v.det" operand of Tab. suee)
 *   G[e][q][j][a]   = sum_k dphi[q][k][a] (J^-1)_kj   (physical gradients, "bfg")
 *   Jinv[e][q][k][j] (optional)
 * det J by cofactor expansion along the first row; J^-1 = adj(J) / det J.
 * Returns 0, or 1 + the first element index with det J <= 0. */
/* ------------------------------------------------------------------------ */
/* Reference tetrahedron T = {x, y, z >= 0, x + y + z <= 1}, barycentric
 * coordinates L = (1 - x - y - z, x, y, z).
 *
 * Grundmann-Moller rule of index s (Grundmann & Moller 1978), degree 2s + 1:
 * level i = 0..s carries the weight (-1)^i 2^(-2s) (2s + 4 - 2i)^(2s+1) /
 * (i! (2s + 4 - i)!) at the barycentric points (2 b + 1) / (2s + 4 - 2i) for
 * every b in N^4 with |b| = s - i.  Points are listed level by level, and within
 * a level with b_0 slowest and b_3 fastest, each b_k descending from its
 * largest possible value; Cartesian point = (L1, L2, L3). */
static double factorial(int n)
{
    double f = 1.0;
    for (int k = 2; k <= n; ++k) f *= k;
    return f;
}

int oracle_gm_rule(int s, double *pts, double *w)
{
    if (s < 0 || s > 6) return OR_BAD_ARG;
    int count = 0;
    for (int i = 0; i <= s; ++i) {
        const int m = s - i;
        const int den = 2 * s + 4 - 2 * i;
        const double wi = ((i & 1) ? -1.0 : 1.0) * pow(2.0, -2.0 * s) * pow((double)den, 2.0 * s + 1.0) /
                          (factorial(i) * factorial(2 * s + 4 - i));
        for (int b0 = m; b0 >= 0; --b0)
            for (int b1 = m - b0; b1 >= 0; --b1)
                for (int b2 = m - b0 - b1; b2 >= 0; --b2) {
                    const int b3 = m - b0 - b1 - b2;
                    if (pts) {
                        pts[3 * count + 0] = (2.0 * b1 + 1.0) / den;
                        pts[3 * count + 1] = (2.0 * b2 + 1.0) / den;
                        pts[3 * count + 2] = (2.0 * b3 + 1.0) / den;
                    }
                    if (w) w[count] = wi;
                    ++count;
                }
    }
    return count;
}

/* Order-p Lagrange basis on T: nodes at the lattice points (i, j, k)/p,
 * i + j + k <= p, x fastest (k slowest); the node with barycentric indices
 * a = (p - i - j - k, i, j, k) has phi_a = prod_m S_{a_m}(L_m) with the
 * Silvester factor S_n(L) = prod_{t=0}^{n-1} (p L - t) / (t + 1). */
static double silvester(int p, int n, double L)
{
    double v = 1.0;
    for (int t = 0; t < n; ++t) v *= (p * L - t) / (t + 1.0);
    return v;
}

static double silvester_deriv(int p, int n, double L)
{
    /* product rule over the n linear factors */
    double s = 0.0;
    for (int r = 0; r < n; ++r) {
        double v = p / (r + 1.0);
        for (int t = 0; t < n; ++t)
            if (t != r) v *= (p * L - t) / (t + 1.0);
        s += v;
    }
    return s;
}

int oracle_tet_basis(int p, int n_pts, const double *pts, double *phi, double *dphi)
{
    if (p < 1 || p > 3 || n_pts < 0 || !pts) return OR_BAD_ARG;
    const int N = (p + 1) * (p + 2) * (p + 3) / 6;
    for (int q = 0; q < n_pts; ++q) {
        const double x = pts[3 * q], y = pts[3 * q + 1], z = pts[3 * q + 2];
        const double L[4] = {1.0 - x - y - z, x, y, z};
        /* dL_m / dx_c */
        const double dL[4][3] = {{-1, -1, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
        int a = 0;
        for (int k = 0; k <= p; ++k)
            for (int j = 0; j <= p - k; ++j)
                for (int i = 0; i <= p - k - j; ++i, ++a) {
                    const int A[4] = {p - i - j - k, i, j, k};
                    double S[4], dS[4];
                    for (int m = 0; m < 4; ++m) {
                        S[m] = silvester(p, A[m], L[m]);
                        dS[m] = silvester_deriv(p, A[m], L[m]);
                    }
                    if (phi) phi[q * N + a] = S[0] * S[1] * S[2] * S[3];
                    if (dphi)
                        for (int c = 0; c < 3; ++c) {
                            double g = 0.0;
                            for (int m = 0; m < 4; ++m) {
                                double t = dS[m] * dL[m][c];
                                for (int o = 0; o < 4; ++o)
                                    if (o != m) t *= S[o];
                                g += t;
                            }
                            dphi[(q * 3 + c) * N + a] = g;
                        }
                }
    }
    return OR_OK;
}

long long oracle_geometry(long long n_elems, int N, int Q, const double *coords, const int32_t *conn,
                          const double *dphi, const double *w, double *wdetJ, double *G, double *Jinv)
{
    if (n_elems < 0 || N < 1 || Q < 1 || !coords || !conn || !dphi || !w || !wdetJ) return OR_BAD_ARG;
    long long first_bad = 0;
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < n_elems; ++e) {
        for (int q = 0; q < Q; ++q) {
            double J[3][3] = {{0}};
            for (int a = 0; a < N; ++a) {
                const double *X = coords + 3 * (size_t)conn[(size_t)e * N + a];
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) J[i][j] += X[i] * dphi[((size_t)q * 3 + j) * N + a];
            }
            double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
            double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
            double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
            double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
            if (!(det > 0.0)) {
#pragma omp critical
                {
                    if (first_bad == 0 || e + 1 < first_bad) first_bad = e + 1;
                }
            }
            /* adjugate: inv[i][j] = cofactor[j][i] / det */
            double cof[3][3];
            cof[0][0] = c00;
            cof[0][1] = c01;
            cof[0][2] = c02;
            cof[1][0] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
            cof[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
            cof[1][2] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
            cof[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
            cof[2][1] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
            cof[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
            double inv[3][3];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) inv[i][j] = cof[j][i] / det;
            wdetJ[(size_t)e * Q + q] = w[q] * det;
            if (Jinv)
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) Jinv[(((size_t)e * Q + q) * 3 + i) * 3 + j] = inv[i][j];
            if (G)
                for (int j = 0; j < 3; ++j)
                    for (int a = 0; a < N; ++a) {
                        double s = 0.0;
                        for (int k = 0; k < 3; ++k) s += dphi[((size_t)q * 3 + k) * N + a] * inv[k][j];
                        G[(((size_t)e * Q + q) * 3 + j) * N + a] = s;
                    }
        }
    }
    return first_bad;
}

/* ------------------------------------------------------------------------ */
/* Matrix mode (Algorithm 2), weak Laplacian ('0.i,0.i', v, u), Tab. ewfd:
 *   K[e][a][b] = c_e sum_q wdetJ[e][q] sum_j G[e][q][j][a] G[e][q][j][b]
 * (the einsum 'cq,cqjd,cqje->cde' of Sec. 5.3.1).  coef may be NULL (c = 1). */
int oracle_matrix_laplace(long long n_elems, int N, int Q, const double *wdetJ, const double *G,
                          const double *coef, double *K)
{
    if (n_elems < 0 || !wdetJ || !G || !K) return OR_BAD_ARG;
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < n_elems; ++e) {
        double *Ke = K + (size_t)e * N * N;
        for (int i = 0; i < N * N; ++i) Ke[i] = 0.0;
        double c = coef ? coef[e] : 1.0;
        for (int q = 0; q < Q; ++q) {
            const double *Gq = G + ((size_t)e * Q + q) * 3 * N;
            double wd = wdetJ[(size_t)e * Q + q];
            for (int a = 0; a < N; ++a)
                for (int b = 0; b < N; ++b) {
                    double s = 0.0;
                    for (int j = 0; j < 3; ++j) s += Gq[j * N + a] * Gq[j * N + b];
                    Ke[a * N + b] += wd * c * s;
                }
        }
    }
    return OR_OK;
}

/* Matrix mode, (vector) dot product / mass ('i,i', v, u), eq. (fe3c):
 *   M[e][(r,a)][(s,b)] = c_e sum_q wdetJ phi_q,a phi_q,b delta_rs
 * rows and columns component-major (comp * N + node).  ncomp = 1 is the scalar
 * mass matrix; ncomp = D gives D diagonal copies of it (Sec. 4.2). */
int oracle_matrix_mass(long long n_elems, int N, int Q, int ncomp, const double *wdetJ, const double *phi,
                       const double *coef, double *K)
{
    if (n_elems < 0 || ncomp < 1 || !wdetJ || !phi || !K) return OR_BAD_ARG;
    int n = ncomp * N;
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < n_elems; ++e) {
        double *Ke = K + (size_t)e * n * n;
        for (int i = 0; i < n * n; ++i) Ke[i] = 0.0;
        double c = coef ? coef[e] : 1.0;
        for (int q = 0; q < Q; ++q) {
            double wd = wdetJ[(size_t)e * Q + q];
            for (int r = 0; r < ncomp; ++r)
                for (int a = 0; a < N; ++a)
                    for (int s = 0; s < ncomp; ++s)
                        for (int b = 0; b < N; ++b) {
                            double delta = (r == s) ? 1.0 : 0.0;
                            Ke[(r * N + a) * n + s * N + b] += wd * c * phi[q * N + a] * phi[q * N + b] * delta;
                        }
        }
    }
    return OR_OK;
}

/* The 0/1 tensor Psg[i][j][I] of shape (3,3,6) that maps the displacement
 * gradient du_i/dx_j to the Voigt strain vector e_I (engineering shear),
 * order (11,22,33,12,13,23): e_I = sum_ij Psg[i][j][I] du_i/dx_j (Sec. 5.3.3). */
static void voigt_psg(double Psg[3][3][6])
{
    memset(Psg, 0, sizeof(double) * 54);
    Psg[0][0][0] = 1.0;
    Psg[1][1][1] = 1.0;
    Psg[2][2][2] = 1.0;
    Psg[0][1][3] = 1.0;
    Psg[1][0][3] = 1.0;
    Psg[0][2][4] = 1.0;
    Psg[2][0][4] = 1.0;
    Psg[1][2][5] = 1.0;
    Psg[2][1][5] = 1.0;
}

/* Isotropic elasticity matrix in the Voigt order above:
 * D = lambda m m^T + mu diag(2,2,2,1,1,1), m = (1,1,1,0,0,0).  D (E,6,6). */
int oracle_lame_to_D(long long n_elems, const double *lam, const double *mu, double *D)
{
    if (n_elems < 0 || !lam || !mu || !D) return OR_BAD_ARG;
    for (long long e = 0; e < n_elems; ++e) {
        double *De = D + (size_t)e * 36;
        for (int I = 0; I < 6; ++I)
            for (int K = 0; K < 6; ++K) {
                double v = 0.0;
                if (I < 3 && K < 3) v += lam[e];
                if (I == K) v += (I < 3) ? 2.0 * mu[e] : mu[e];
                De[I * 6 + K] = v;
            }
    }
    return OR_OK;
}

/* Strain-displacement matrix B (6, 3N) at one quadrature point:
 * B[I][(i,a)] = sum_j Psg[i][j][I] G[j][a]  (the "rjI,cqje" factor). */
static void strain_matrix(int N, const double *Gq, double *B)
{
    double Psg[3][3][6];
    voigt_psg(Psg);
    for (int I = 0; I < 6; ++I)
        for (int i = 0; i < 3; ++i)
            for (int a = 0; a < N; ++a) {
                double s = 0.0;
                for (int j = 0; j < 3; ++j) s += Psg[i][j][I] * Gq[j * N + a];
                B[(size_t)I * 3 * N + i * N + a] = s;
            }
}

/* Matrix mode, linear elasticity ('IK,s(i:j)->I,s(k:l)->K', D, v, u), Sec. 5.3.3:
 *   K[e][(i,a)][(k,b)] = sum_q wdetJ sum_{I,K} B[I][(i,a)] D[I][K] B[K][(k,b)]
 * with D per element (E,6,6) (material layout cq0 with a constant q axis). */
int oracle_matrix_elasticity(long long n_elems, int N, int Q, const double *wdetJ, const double *G,
                             const double *D, double *K)
{
    if (n_elems < 0 || N > 512 || !wdetJ || !G || !D || !K) return OR_BAD_ARG;
    int n = 3 * N;
    int rc = OR_OK;
#pragma omp parallel
    {
        double *B = (double *)malloc(sizeof(double) * 6 * n);
        double *DB = (double *)malloc(sizeof(double) * 6 * n);
        if (!B || !DB) {
#pragma omp critical
            rc = OR_BAD_ARG;
        }
#pragma omp for schedule(static)
        for (long long e = 0; e < n_elems; ++e) {
            if (!B || !DB) continue;
            double *Ke = K + (size_t)e * n * n;
            const double *De = D + (size_t)e * 36;
            for (int i = 0; i < n * n; ++i) Ke[i] = 0.0;
            for (int q = 0; q < Q; ++q) {
                strain_matrix(N, G + ((size_t)e * Q + q) * 3 * N, B);
                double wd = wdetJ[(size_t)e * Q + q];
                for (int I = 0; I < 6; ++I)
                    for (int c = 0; c < n; ++c) {
                        double s = 0.0;
                        for (int L = 0; L < 6; ++L) s += De[I * 6 + L] * B[(size_t)L * n + c];
                        DB[(size_t)I * n + c] = s;
                    }
                for (int r = 0; r < n; ++r)
                    for (int c = 0; c < n; ++c) {
                        double s = 0.0;
                        for (int I = 0; I < 6; ++I) s += B[(size_t)I * n + r] * DB[(size_t)I * n + c];
                        Ke[(size_t)r * n + c] += wd * s;
                    }
            }
        }
        free(B);
        free(DB);
    }
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Residual mode (Algorithm 1): the element DOFs are gathered from the global
 * DOF vector u (ncomp * node + comp) through the connectivity, the integrand
 * F is evaluated at each quadrature point and integrated with wdetJ. */

/* Weak Laplacian: r[e][a] = c_e sum_q wdetJ sum_j G[j][a] (grad u_h)_j,
 * (grad u_h)_j = sum_b G[j][b] u[conn[e][b]]. */
int oracle_residual_laplace(long long n_elems, int N, int Q, const int32_t *conn, const double *wdetJ,
                            const double *G, const double *coef, const double *u, double *r)
{
    if (n_elems < 0 || !conn || !wdetJ || !G || !u || !r) return OR_BAD_ARG;
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < n_elems; ++e) {
        double *re = r + (size_t)e * N;
        for (int a = 0; a < N; ++a) re[a] = 0.0;
        double c = coef ? coef[e] : 1.0;
        for (int q = 0; q < Q; ++q) {
            const double *Gq = G + ((size_t)e * Q + q) * 3 * N;
            double grad[3] = {0.0, 0.0, 0.0};
            for (int j = 0; j < 3; ++j)
                for (int b = 0; b < N; ++b) grad[j] += Gq[j * N + b] * u[conn[(size_t)e * N + b]];
            double wd = wdetJ[(size_t)e * Q + q];
            for (int a = 0; a < N; ++a) {
                double s = 0.0;
                for (int j = 0; j < 3; ++j) s += Gq[j * N + a] * grad[j];
                re[a] += wd * c * s;
            }
        }
    }
    return OR_OK;
}

/* (Vector) dot product: r[e][(i,a)] = c_e sum_q wdetJ phi_a u_h,i,
 * u_h,i = sum_b phi_b u[ncomp*conn[e][b] + i]. */
int oracle_residual_mass(long long n_elems, int N, int Q, int ncomp, const int32_t *conn, const double *wdetJ,
                         const double *phi, const double *coef, const double *u, double *r)
{
    if (n_elems < 0 || ncomp < 1 || ncomp > 3 || !conn || !wdetJ || !phi || !u || !r) return OR_BAD_ARG;
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < n_elems; ++e) {
        double *re = r + (size_t)e * ncomp * N;
        for (int a = 0; a < ncomp * N; ++a) re[a] = 0.0;
        double c = coef ? coef[e] : 1.0;
        for (int q = 0; q < Q; ++q) {
            double uh[3] = {0.0, 0.0, 0.0};
            for (int i = 0; i < ncomp; ++i)
                for (int b = 0; b < N; ++b)
                    uh[i] += phi[q * N + b] * u[(size_t)ncomp * conn[(size_t)e * N + b] + i];
            double wd = wdetJ[(size_t)e * Q + q];
            for (int i = 0; i < ncomp; ++i)
                for (int a = 0; a < N; ++a) re[i * N + a] += wd * c * phi[q * N + a] * uh[i];
        }
    }
    return OR_OK;
}

/* Linear elasticity: r[e][(i,a)] = sum_q wdetJ sum_I B[I][(i,a)] sigma_I,
 * sigma = D e(u_h), e(u_h)_K = sum_(k,b) B[K][(k,b)] u[3*conn[e][b] + k]. */
int oracle_residual_elasticity(long long n_elems, int N, int Q, const int32_t *conn, const double *wdetJ,
                               const double *G, const double *D, const double *u, double *r)
{
    if (n_elems < 0 || N > 512 || !conn || !wdetJ || !G || !D || !u || !r) return OR_BAD_ARG;
    int n = 3 * N;
    int rc = OR_OK;
#pragma omp parallel
    {
        double *B = (double *)malloc(sizeof(double) * 6 * n);
        double *ue = (double *)malloc(sizeof(double) * n);
        if (!B || !ue) {
#pragma omp critical
            rc = OR_BAD_ARG;
        }
#pragma omp for schedule(static)
        for (long long e = 0; e < n_elems; ++e) {
            if (!B || !ue) continue;
            double *re = r + (size_t)e * n;
            const double *De = D + (size_t)e * 36;
            for (int k = 0; k < 3; ++k)
                for (int b = 0; b < N; ++b) ue[k * N + b] = u[3 * (size_t)conn[(size_t)e * N + b] + k];
            for (int c = 0; c < n; ++c) re[c] = 0.0;
            for (int q = 0; q < Q; ++q) {
                strain_matrix(N, G + ((size_t)e * Q + q) * 3 * N, B);
                double eps[6], sig[6];
                for (int K = 0; K < 6; ++K) {
                    double s = 0.0;
                    for (int c = 0; c < n; ++c) s += B[(size_t)K * n + c] * ue[c];
                    eps[K] = s;
                }
                for (int I = 0; I < 6; ++I) {
                    double s = 0.0;
                    for (int K = 0; K < 6; ++K) s += De[I * 6 + K] * eps[K];
                    sig[I] = s;
                }
                double wd = wdetJ[(size_t)e * Q + q];
                for (int c = 0; c < n; ++c) {
                    double s = 0.0;
                    for (int I = 0; I < 6; ++I) s += B[(size_t)I * n + c] * sig[I];
                    re[c] += wd * s;
                }
            }
        }
        free(B);
        free(ue);
    }
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Navier-Stokes convective term 'i,i.j,j' (Eq. fe2, Tab. ewfd):
 *   c(v, u, w) = int v_i (du_i/dx_j) w_j,
 * with a gradient operand u and an advection operand w, both vector fields
 * gathered through conn (u[3*node + i]); for the non-linear term w = u.
 * At a point: u_h,i = sum_b phi_b u_(i,b), (grad u_h)_ij = sum_b u_(i,b) G[j][b]. */
static void convect_point(int N, const double *phi_q, const double *Gq, const double *ue, const double *we,
                          double gu[3][3], double wh[3])
{
    for (int i = 0; i < 3; ++i) {
        wh[i] = 0.0;
        for (int b = 0; b < N; ++b) wh[i] += phi_q[b] * we[i * N + b];
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int b = 0; b < N; ++b) s += ue[i * N + b] * Gq[j * N + b];
            gu[i][j] = s;
        }
    }
}

static void gather_vec(int N, const int32_t *conn_e, const double *u, double *ue)
{
    for (int i = 0; i < 3; ++i)
        for (int b = 0; b < N; ++b) ue[i * N + b] = u[3 * (size_t)conn_e[b] + i];
}

/* Residual mode: r[e][(i,a)] = sum_q wdetJ phi_a sum_j (grad u_h)_ij w_h,j. */
int oracle_residual_convect(long long n_elems, int N, int Q, const int32_t *conn, const double *wdetJ,
                            const double *phi, const double *G, const double *u, const double *w, double *r)
{
    if (n_elems < 0 || N < 1 || N > 512 || !conn || !wdetJ || !phi || !G || !u || !w || !r) return OR_BAD_ARG;
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < n_elems; ++e) {
        double ue[3 * 512], we[3 * 512];
        gather_vec(N, conn + (size_t)e * N, u, ue);
        gather_vec(N, conn + (size_t)e * N, w, we);
        double *re = r + (size_t)e * 3 * N;
        for (int c = 0; c < 3 * N; ++c) re[c] = 0.0;
        for (int q = 0; q < Q; ++q) {
            double gu[3][3], wh[3];
            convect_point(N, phi + (size_t)q * N, G + ((size_t)e * Q + q) * 3 * N, ue, we, gu, wh);
            const double wd = wdetJ[(size_t)e * Q + q];
            for (int i = 0; i < 3; ++i) {
                const double s = gu[i][0] * wh[0] + gu[i][1] * wh[1] + gu[i][2] * wh[2];
                for (int a = 0; a < N; ++a) re[i * N + a] += wd * phi[(size_t)q * N + a] * s;
            }
        }
    }
    return OR_OK;
}

/* Matrix mode, the two terms of Eq. fe4: the derivative with respect to the
 * gradient operand (wrt_u) and to the advection operand (wrt_w),
 *   K[e][(i,a),(k,b)] = sum_q wdetJ phi_a [ wrt_u delta_ik (w_h . grad phi_b)
 *                                          + wrt_w (du_h,i/dx_k) phi_b ];
 * with w = u and both flags set this is the Jacobian of the non-linear term. */
int oracle_matrix_convect(long long n_elems, int N, int Q, const int32_t *conn, const double *wdetJ,
                          const double *phi, const double *G, const double *u, const double *w, int wrt_u, int wrt_w,
                          double *K)
{
    if (n_elems < 0 || N < 1 || N > 512 || !conn || !wdetJ || !phi || !G || !u || !w || !K) return OR_BAD_ARG;
    const int n = 3 * N;
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < n_elems; ++e) {
        double ue[3 * 512], we[3 * 512];
        gather_vec(N, conn + (size_t)e * N, u, ue);
        gather_vec(N, conn + (size_t)e * N, w, we);
        double *Ke = K + (size_t)e * n * n;
        for (long long c = 0; c < (long long)n * n; ++c) Ke[c] = 0.0;
        for (int q = 0; q < Q; ++q) {
            const double *Gq = G + ((size_t)e * Q + q) * 3 * N;
            const double *ph = phi + (size_t)q * N;
            double gu[3][3], wh[3];
            convect_point(N, ph, Gq, ue, we, gu, wh);
            const double wd = wdetJ[(size_t)e * Q + q];
            for (int i = 0; i < 3; ++i)
                for (int a = 0; a < N; ++a)
                    for (int k = 0; k < 3; ++k)
                        for (int b = 0; b < N; ++b) {
                            double v = 0.0;
                            if (wrt_u && i == k) v += wh[0] * Gq[b] + wh[1] * Gq[N + b] + wh[2] * Gq[2 * N + b];
                            if (wrt_w) v += gu[i][k] * ph[b];
                            Ke[(size_t)(i * N + a) * n + k * N + b] += wd * ph[a] * v;
                        }
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* The remaining weak forms of Tab. ewfd, element by element at every point:
 *   weighted dot  'ij,i,j'  (M, v, u):  v_i M_ij u_j
 *   Stokes        'i.i,0'   (v, p):     div(v) p
 *   transposed    'i.i,0'   (u, q):     q div(u)
 *   divergence    'i.i'     (v):        div(v)
 * M is a 3x3 matrix per element (row-major).  Field DOFs are gathered through
 * conn: vector u[3*node + i], scalar p[node]. */
static void gather_scalar(int N, const int32_t *conn_e, const double *p, double *pe)
{
    for (int b = 0; b < N; ++b) pe[b] = p[conn_e[b]];
}

/* Matrix of the weighted dot product: K[(i,a),(j,b)] = M_ij sum_q wdetJ phi_a phi_b. */
int oracle_matrix_wdot(long long n_elems, int N, int Q, const double *wdetJ, const double *phi, const double *M,
                       double *K)
{
    if (n_elems < 0 || !wdetJ || !phi || !M || !K) return OR_BAD_ARG;
    const int n = 3 * N;
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < n_elems; ++e)
        for (int i = 0; i < 3; ++i)
            for (int a = 0; a < N; ++a)
                for (int j = 0; j < 3; ++j)
                    for (int b = 0; b < N; ++b) {
                        double s = 0.0;
                        for (int q = 0; q < Q; ++q)
                            s += wdetJ[(size_t)e * Q + q] * phi[(size_t)q * N + a] * phi[(size_t)q * N + b];
                        K[(size_t)e * n * n + (size_t)(i * N + a) * n + j * N + b] = M[(size_t)e * 9 + i * 3 + j] * s;
                    }
    return OR_OK;
}

/* Residual of the weighted dot product: r[(i,a)] = sum_q wdetJ phi_a sum_j M_ij u_h,j. */
int oracle_residual_wdot(long long n_elems, int N, int Q, const int32_t *conn, const double *wdetJ,
                         const double *phi, const double *M, const double *u, double *r)
{
    if (n_elems < 0 || N > 512 || !conn || !wdetJ || !phi || !M || !u || !r) return OR_BAD_ARG;
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < n_elems; ++e) {
        double ue[3 * 512];
        gather_vec(N, conn + (size_t)e * N, u, ue);
        double *re = r + (size_t)e * 3 * N;
        for (int c = 0; c < 3 * N; ++c) re[c] = 0.0;
        for (int q = 0; q < Q; ++q) {
            double uh[3] = {0, 0, 0};
            for (int j = 0; j < 3; ++j)
                for (int b = 0; b < N; ++b) uh[j] += phi[(size_t)q * N + b] * ue[j * N + b];
            const double wd = wdetJ[(size_t)e * Q + q];
            for (int i = 0; i < 3; ++i) {
                double mu = 0.0;
                for (int j = 0; j < 3; ++j) mu += M[(size_t)e * 9 + i * 3 + j] * uh[j];
                for (int a = 0; a < N; ++a) re[i * N + a] += wd * phi[(size_t)q * N + a] * mu;
            }
        }
    }
    return OR_OK;
}

/* Stokes coupling matrix: B[(i,a), b] = sum_q wdetJ G[i][a] phi_b (rows 3N, columns N);
 * the transposed coupling 'i.i,0' (u, q) has the matrix B^T. */
int oracle_matrix_stokes(long long n_elems, int N, int Q, const double *wdetJ, const double *G, const double *phi,
                         double *B)
{
    if (n_elems < 0 || !wdetJ || !G || !phi || !B) return OR_BAD_ARG;
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < n_elems; ++e)
        for (int i = 0; i < 3; ++i)
            for (int a = 0; a < N; ++a)
                for (int b = 0; b < N; ++b) {
                    double s = 0.0;
                    for (int q = 0; q < Q; ++q)
                        s += wdetJ[(size_t)e * Q + q] * G[(((size_t)e * Q + q) * 3 + i) * N + a] * phi[(size_t)q * N + b];
                    B[(size_t)e * 3 * N * N + (size_t)(i * N + a) * N + b] = s;
                }
    return OR_OK;
}

/* Stokes residual r[(i,a)] = sum_q wdetJ G[i][a] p_h with p_h = sum_b phi_b p_b;
 * with p = NULL the divergence form 'i.i' (v): r[(i,a)] = sum_q wdetJ G[i][a]. */
int oracle_residual_stokes(long long n_elems, int N, int Q, const int32_t *conn, const double *wdetJ,
                           const double *G, const double *phi, const double *p, double *r)
{
    if (n_elems < 0 || N > 512 || !conn || !wdetJ || !G || !phi || !r) return OR_BAD_ARG;
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < n_elems; ++e) {
        double pe[512];
        if (p) gather_scalar(N, conn + (size_t)e * N, p, pe);
        double *re = r + (size_t)e * 3 * N;
        for (int c = 0; c < 3 * N; ++c) re[c] = 0.0;
        for (int q = 0; q < Q; ++q) {
            double ph = 1.0;
            if (p) {
                ph = 0.0;
                for (int b = 0; b < N; ++b) ph += phi[(size_t)q * N + b] * pe[b];
            }
            const double wd = wdetJ[(size_t)e * Q + q];
            for (int i = 0; i < 3; ++i)
                for (int a = 0; a < N; ++a) re[i * N + a] += wd * G[(((size_t)e * Q + q) * 3 + i) * N + a] * ph;
        }
    }
    return OR_OK;
}

/* Transposed Stokes residual r[a] = sum_q wdetJ phi_a div(u_h). */
int oracle_residual_stokes_t(long long n_elems, int N, int Q, const int32_t *conn, const double *wdetJ,
                             const double *G, const double *phi, const double *u, double *r)
{
    if (n_elems < 0 || N > 512 || !conn || !wdetJ || !G || !phi || !u || !r) return OR_BAD_ARG;
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < n_elems; ++e) {
        double ue[3 * 512];
        gather_vec(N, conn + (size_t)e * N, u, ue);
        double *re = r + (size_t)e * N;
        for (int a = 0; a < N; ++a) re[a] = 0.0;
        for (int q = 0; q < Q; ++q) {
            double div = 0.0;
            for (int i = 0; i < 3; ++i)
                for (int b = 0; b < N; ++b) div += ue[i * N + b] * G[(((size_t)e * Q + q) * 3 + i) * N + b];
            const double wd = wdetJ[(size_t)e * Q + q];
            for (int a = 0; a < N; ++a) re[a] += wd * phi[(size_t)q * N + a] * div;
        }
    }
    return OR_OK;
}

/* Stokes coupling 'i.i,0' between fields of different orders (Tab. ewfd; Sec. 5
 * names the coupling of fields, which SfePy lets carry different orders): a
 * vector field on the geometry's basis (N nodes, physical gradients G) and a
 * scalar field on a second basis over the same elements (Np nodes, values psi
 * (Q, Np) at the same quadrature points, DOFs through its own connectivity),
 * e.g. a Q2 velocity with a Q1 pressure or P2 with P1:
 *   B[(i,a), b] = sum_q wdetJ G[i][a] psi_b                     (rows 3N, columns Np)
 *   r[(i,a)]    = sum_q wdetJ G[i][a] p_h,  p_h = sum_b psi_b p[conn_p[e][b]]
 *   rt[b]       = sum_q wdetJ psi_b div(u_h), u_h on the geometry's basis via conn
 * (the transposed coupling 'i.i,0' (u, q) has the matrix B^T). */
int oracle_matrix_stokes_mixed(long long n_elems, int N, int Np, int Q, const double *wdetJ, const double *G,
                               const double *psi, double *B)
{
    if (n_elems < 0 || !wdetJ || !G || !psi || !B) return OR_BAD_ARG;
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < n_elems; ++e)
        for (int i = 0; i < 3; ++i)
            for (int a = 0; a < N; ++a)
                for (int b = 0; b < Np; ++b) {
                    double s = 0.0;
                    for (int q = 0; q < Q; ++q)
                        s += wdetJ[(size_t)e * Q + q] * G[(((size_t)e * Q + q) * 3 + i) * N + a] *
                             psi[(size_t)q * Np + b];
                    B[(size_t)e * 3 * N * Np + (size_t)(i * N + a) * Np + b] = s;
                }
    return OR_OK;
}

int oracle_residual_stokes_mixed(long long n_elems, int N, int Np, int Q, const int32_t *conn_p,
                                 const double *wdetJ, const double *G, const double *psi, const double *p,
                                 double *r)
{
    if (n_elems < 0 || Np > 512 || !conn_p || !wdetJ || !G || !psi || !p || !r) return OR_BAD_ARG;
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < n_elems; ++e) {
        double pe[512];
        gather_scalar(Np, conn_p + (size_t)e * Np, p, pe);
        double *re = r + (size_t)e * 3 * N;
        for (int c = 0; c < 3 * N; ++c) re[c] = 0.0;
        for (int q = 0; q < Q; ++q) {
            double ph = 0.0;
            for (int b = 0; b < Np; ++b) ph += psi[(size_t)q * Np + b] * pe[b];
            const double wd = wdetJ[(size_t)e * Q + q];
            for (int i = 0; i < 3; ++i)
                for (int a = 0; a < N; ++a) re[i * N + a] += wd * G[(((size_t)e * Q + q) * 3 + i) * N + a] * ph;
        }
    }
    return OR_OK;
}

int oracle_residual_stokes_t_mixed(long long n_elems, int N, int Np, int Q, const int32_t *conn,
                                   const double *wdetJ, const double *G, const double *psi, const double *u,
                                   double *r)
{
    if (n_elems < 0 || N > 512 || !conn || !wdetJ || !G || !psi || !u || !r) return OR_BAD_ARG;
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < n_elems; ++e) {
        double ue[3 * 512];
        gather_vec(N, conn + (size_t)e * N, u, ue);
        double *re = r + (size_t)e * Np;
        for (int b = 0; b < Np; ++b) re[b] = 0.0;
        for (int q = 0; q < Q; ++q) {
            double div = 0.0;
            for (int i = 0; i < 3; ++i)
                for (int a = 0; a < N; ++a) div += ue[i * N + a] * G[(((size_t)e * Q + q) * 3 + i) * N + a];
            const double wd = wdetJ[(size_t)e * Q + q];
            for (int b = 0; b < Np; ++b) re[b] += wd * psi[(size_t)q * Np + b] * div;
        }
    }
    return OR_OK;
}

/* 'eval' mode: the integral over each element of a form whose operands all
 * carry DOFs (Sec. 5.1, evaluation modes), out (E, n_out):
 *   kind 0 Laplace      c sum_q wdetJ grad u . grad w           (scalar fields)
 *   kind 1 dot / mass   c sum_q wdetJ u . w                     (ncomp 1 or 3)
 *   kind 2 elasticity   sum_q wdetJ e(u)^T D e(w)               (Voigt, engineering shear)
 *   kind 3 weighted dot sum_q wdetJ u_i M_ij w_j
 *   kind 4 Stokes       sum_q wdetJ div(u) p                    (w = p scalar)
 *   kind 5 divergence   sum_q wdetJ div(u)
 *   kind 6 Cauchy stress sum_q wdetJ D e(u)                     (6 values)
 *   kind 7 convection   sum_q wdetJ u_i (d w_i / d x_j) z_j     (three vector fields)
 * coef: per-element scalar (kinds 0, 1; NULL = 1); mat: D (E,6,6) for 2, 6,
 * M (E,3,3) for 3. */
int oracle_eval_form(int kind, long long n_elems, int N, int Q, int ncomp, const int32_t *conn, const double *wdetJ,
                     const double *G, const double *phi, const double *coef, const double *mat, const double *u,
                     const double *w, const double *z, double *out)
{
    if (kind < 0 || kind > 7 || n_elems < 0 || N > 512 || !conn || !wdetJ || !G || !phi || !u || !out)
        return OR_BAD_ARG;
    const int n_out = kind == 6 ? 6 : 1;
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < n_elems; ++e) {
        double ue[3 * 512], we[3 * 512], ze[3 * 512];
        const int32_t *ce = conn + (size_t)e * N;
        const int cu = (kind == 0 || (kind == 1 && ncomp == 1)) ? 1 : 3;
        for (int i = 0; i < cu; ++i)
            for (int b = 0; b < N; ++b) ue[i * N + b] = u[(size_t)cu * ce[b] + i];
        if (w) {
            const int cw = (kind == 0 || kind == 4 || (kind == 1 && ncomp == 1)) ? 1 : 3;
            for (int i = 0; i < cw; ++i)
                for (int b = 0; b < N; ++b) we[i * N + b] = w[(size_t)cw * ce[b] + i];
        }
        if (z)
            for (int i = 0; i < 3; ++i)
                for (int b = 0; b < N; ++b) ze[i * N + b] = z[(size_t)3 * ce[b] + i];
        double acc[6] = {0, 0, 0, 0, 0, 0};
        for (int q = 0; q < Q; ++q) {
            const double *Gq = G + ((size_t)e * Q + q) * 3 * N;
            const double *pq = phi + (size_t)q * N;
            const double wd = wdetJ[(size_t)e * Q + q];
            double uv[3] = {0, 0, 0}, wv[3] = {0, 0, 0}, zv[3] = {0, 0, 0}, gu[3][3] = {{0}}, gw[3][3] = {{0}};
            for (int i = 0; i < 3; ++i)
                for (int b = 0; b < N; ++b) {
                    if (i < cu) {
                        uv[i] += pq[b] * ue[i * N + b];
                        for (int j = 0; j < 3; ++j) gu[i][j] += ue[i * N + b] * Gq[j * N + b];
                    }
                    if (w && (i < 3)) {
                        const int cw = (kind == 0 || kind == 4 || (kind == 1 && ncomp == 1)) ? 1 : 3;
                        if (i < cw) {
                            wv[i] += pq[b] * we[i * N + b];
                            for (int j = 0; j < 3; ++j) gw[i][j] += we[i * N + b] * Gq[j * N + b];
                        }
                    }
                    if (z) zv[i] += pq[b] * ze[i * N + b];
                }
            const double c = coef ? coef[e] : 1.0;
            const double *Me = mat ? mat + (size_t)e * (kind == 3 ? 9 : 36) : NULL;
            double eu[6] = {gu[0][0], gu[1][1], gu[2][2], gu[0][1] + gu[1][0], gu[0][2] + gu[2][0], gu[1][2] + gu[2][1]};
            double ew[6] = {gw[0][0], gw[1][1], gw[2][2], gw[0][1] + gw[1][0], gw[0][2] + gw[2][0], gw[1][2] + gw[2][1]};
            switch (kind) {
            case 0: acc[0] += wd * c * (gu[0][0] * gw[0][0] + gu[0][1] * gw[0][1] + gu[0][2] * gw[0][2]); break;
            case 1: {
                double s = 0.0;
                for (int i = 0; i < cu; ++i) s += uv[i] * wv[i];
                acc[0] += wd * c * s;
                break;
            }
            case 2: {
                double s = 0.0;
                for (int I = 0; I < 6; ++I)
                    for (int K = 0; K < 6; ++K) s += eu[I] * Me[I * 6 + K] * ew[K];
                acc[0] += wd * s;
                break;
            }
            case 3: {
                double s = 0.0;
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) s += uv[i] * Me[i * 3 + j] * wv[j];
                acc[0] += wd * s;
                break;
            }
            case 4: acc[0] += wd * (gu[0][0] + gu[1][1] + gu[2][2]) * wv[0]; break;
            case 5: acc[0] += wd * (gu[0][0] + gu[1][1] + gu[2][2]); break;
            case 6:
                for (int I = 0; I < 6; ++I) {
                    double s = 0.0;
                    for (int K = 0; K < 6; ++K) s += Me[I * 6 + K] * eu[K];
                    acc[I] += wd * s;
                }
                break;
            case 7: {
                double s = 0.0;
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) s += uv[i] * gw[i][j] * zv[j];
                acc[0] += wd * s;
                break;
            }
            }
        }
        for (int m = 0; m < n_out; ++m) out[(size_t)e * n_out + m] = acc[m];
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Adjoint of the assembled isotropic elasticity residual.  The paper states the
 * residual (Algorithm 1, form 'IK,s(i:j)->I,s(k:l)->K'); the derivatives below
 * are derived here.  For a scalar objective of the assembled residual R with
 * adjoint vector rbar = dObjective/dR (for J = |R|^2 / 2, rbar = R), the
 * objective's derivative is rbar . dR = sum_e int sigma(u) : eps(rbar) dx in
 * each parameter, with lambda_e, mu_e entering sigma = lambda tr(eps) I + 2 mu eps
 * and the node positions entering the integration domain (det J) and the
 * physical gradients.  Per element:
 *   d/d lambda_e = sum_q wdetJ div(u_h) div(rbar_h)
 *   d/d mu_e     = sum_q wdetJ 2 eps(u_h) : eps(rbar_h)
 *   d/d x_(a,m)  = sum_q wdetJ [ f G[m][a] - sum_j M_mj G[j][a] ],
 *       f = sigma(u_h) : eps(rbar_h),
 *       M = (grad rbar_h)^T sigma(u_h) + (grad u_h)^T sigma(rbar_h)
 * (from d(det J) = det J sum_a G_a . dx_a and d(grad v) = -(grad v)(grad dV) for a
 * node displacement field dV).  dX_e is written component-major, dX_e[e][m*N + a],
 * the layout of a vector element residual, so that it assembles like one. */
static void grad_at(int N, const double *Gq, const double *ve, double gv[3][3])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int b = 0; b < N; ++b) s += ve[i * N + b] * Gq[j * N + b];
            gv[i][j] = s;
        }
}

static void lame_stress(double lam, double mu, double g[3][3], double sig[3][3])
{
    const double tr = g[0][0] + g[1][1] + g[2][2];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) sig[i][j] = mu * (g[i][j] + g[j][i]) + (i == j ? lam * tr : 0.0);
}

int oracle_adjoint_elasticity(long long n_elems, int N, int Q, const int32_t *conn, const double *wdetJ,
                              const double *G, const double *lam, const double *mu, const double *u,
                              const double *rbar, double *dlam, double *dmu, double *dX)
{
    if (n_elems < 0 || N < 1 || N > 512 || !conn || !wdetJ || !G || !lam || !mu || !u || !rbar) return OR_BAD_ARG;
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < n_elems; ++e) {
        double ue[3 * 512], be[3 * 512];
        gather_vec(N, conn + (size_t)e * N, u, ue);
        gather_vec(N, conn + (size_t)e * N, rbar, be);
        double sl = 0.0, sm = 0.0;
        double *dxe = dX ? dX + (size_t)e * 3 * N : NULL;
        if (dxe)
            for (int c = 0; c < 3 * N; ++c) dxe[c] = 0.0;
        for (int q = 0; q < Q; ++q) {
            const double *Gq = G + ((size_t)e * Q + q) * 3 * N;
            const double wd = wdetJ[(size_t)e * Q + q];
            double gu[3][3], gb[3][3], su[3][3], sb[3][3];
            grad_at(N, Gq, ue, gu);
            grad_at(N, Gq, be, gb);
            const double divu = gu[0][0] + gu[1][1] + gu[2][2], divb = gb[0][0] + gb[1][1] + gb[2][2];
            double ee = 0.0; /* eps(u) : eps(rbar) */
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) ee += 0.25 * (gu[i][j] + gu[j][i]) * (gb[i][j] + gb[j][i]);
            sl += wd * divu * divb;
            sm += wd * 2.0 * ee;
            if (!dxe) continue;
            lame_stress(lam[e], mu[e], gu, su);
            lame_stress(lam[e], mu[e], gb, sb);
            const double f = lam[e] * divu * divb + 2.0 * mu[e] * ee;
            double M[3][3];
            for (int m = 0; m < 3; ++m)
                for (int j = 0; j < 3; ++j) {
                    double s = 0.0;
                    for (int i = 0; i < 3; ++i) s += gb[i][m] * su[i][j] + gu[i][m] * sb[i][j];
                    M[m][j] = s;
                }
            for (int m = 0; m < 3; ++m)
                for (int a = 0; a < N; ++a) {
                    double s = f * Gq[m * N + a];
                    for (int j = 0; j < 3; ++j) s -= M[m][j] * Gq[j * N + a];
                    dxe[m * N + a] += wd * s;
                }
        }
        if (dlam) dlam[e] = sl;
        if (dmu) dmu[e] = sm;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Assembly of element vectors into a global vector (outside the timed region
 * of the paper, Sec. 6): g[ncomp*conn[e][a] + i] += r[e][i*N + a], summed
 * sequentially in ascending (e, a, i) order.  accumulate = 0 zeroes g first. */
int oracle_assemble(long long n_elems, int N, int ncomp, const int32_t *conn, const double *r, long long n_nodes,
                    int accumulate, double *g)
{
    if (n_elems < 0 || ncomp < 1 || !conn || !r || !g) return OR_BAD_ARG;
    if (!accumulate)
        for (long long k = 0; k < n_nodes * ncomp; ++k) g[k] = 0.0;
    for (long long e = 0; e < n_elems; ++e)
        for (int a = 0; a < N; ++a)
            for (int i = 0; i < ncomp; ++i) {
                long long node = conn[(size_t)e * N + a];
                if (node < 0 || node >= n_nodes) return OR_BAD_ARG;
                g[ncomp * node + i] += r[(size_t)e * ncomp * N + i * N + a];
            }
    return OR_OK;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the following parallel loops (timing of the oracle on one core). */
void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}
