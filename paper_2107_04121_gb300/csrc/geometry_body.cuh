// Device pieces of the FP64 geometry of the reference mapping (Sec. 4.1 of
// Cimrman, arXiv 2107.04121) shared by the geometry kernels and by the residual
// kernel that computes the geometry of its elements itself.  Every rounding is
// explicit (__fma_rn, __dmul_rn, __fmul_rn, ...) so that each kernel that uses
// these functions produces the same bits for the same element.
#pragma once

#include "fe_device.cuh"

// Collocation stages for tensor-product bases with n1 nodes and n1 Gauss
// points per axis, one element: X, U, V, P are [3][N] (N = n1^3) with the
// fastest index along x; B = (point, node) 1-D values, row-major.
//   U[c][k][j][qx] = sum_i B[qx][i] X[c][k][j][i]
//   V[c][k][qy][qx] = sum_j B[qy][j] U[c][k][j][qx]
//   P[c][qz][qy][qx] = sum_k B[qz][k] V[c][k][qy][qx]       (x at the points)
// Item t of a stage lies in [0, 3N).
template <int N1>
__device__ __forceinline__ void geo_stage_x(int t, const double *__restrict__ X, double *__restrict__ U,
                                            const double *__restrict__ B)
{
    constexpr int N = N1 * N1 * N1;
    const int qx = t % N1, kj = (t / N1) % (N1 * N1), c = t / N;
    const double *x = X + c * N + kj * N1;
    double u = 0.0;
#pragma unroll
    for (int i = 0; i < N1; ++i) u = __fma_rn(B[qx * N1 + i], x[i], u);
    U[c * N + kj * N1 + qx] = u;
}

template <int N1>
__device__ __forceinline__ void geo_stage_y(int t, const double *__restrict__ U, double *__restrict__ V,
                                            const double *__restrict__ B)
{
    constexpr int N = N1 * N1 * N1;
    const int qx = t % N1, qy = (t / N1) % N1, k = (t / (N1 * N1)) % N1, c = t / N;
    const double *x = U + c * N + k * N1 * N1 + qx;
    double v = 0.0;
#pragma unroll
    for (int j = 0; j < N1; ++j) v = __fma_rn(B[qy * N1 + j], x[j * N1], v);
    V[c * N + (k * N1 + qy) * N1 + qx] = v;
}

template <int N1>
__device__ __forceinline__ void geo_stage_z(int t, const double *__restrict__ V, double *__restrict__ P,
                                            const double *__restrict__ B)
{
    constexpr int N = N1 * N1 * N1;
    const int qxy = t % (N1 * N1), qz = (t / (N1 * N1)) % N1, c = t / N;
    const double *x = V + c * N + qxy;
    double p = 0.0;
#pragma unroll
    for (int k = 0; k < N1; ++k) p = __fma_rn(B[qz * N1 + k], x[k * N1 * N1], p);
    P[c * N + qz * N1 * N1 + qxy] = p;
}

// Row c of J at point q = (qx, qy, qz): J[c][m] = derivative along axis m of
// the point values P[c], Dq = (point, point) collocation derivative.
template <int N1>
__device__ __forceinline__ void geo_jacobian_row(int q, int c, const double *__restrict__ P,
                                                 const double *__restrict__ Dq, double out[3])
{
    constexpr int N = N1 * N1 * N1;
    const int qx = q % N1, qy = (q / N1) % N1, qz = q / (N1 * N1);
    const double *Pc = P + c * N;
    double j0 = 0.0, j1 = 0.0, j2 = 0.0;
#pragma unroll
    for (int p = 0; p < N1; ++p) {
        j0 = __fma_rn(Dq[qx * N1 + p], Pc[(qz * N1 + qy) * N1 + p], j0);
        j1 = __fma_rn(Dq[qy * N1 + p], Pc[(qz * N1 + p) * N1 + qx], j1);
        j2 = __fma_rn(Dq[qz * N1 + p], Pc[(p * N1 + qy) * N1 + qx], j2);
    }
    out[0] = j0;
    out[1] = j1;
    out[2] = j2;
}

// Cofactor C[r][k] of J (row-major, J[c][m] = d x_c / d xi_m), so that
// J^-1[k][r] = C[r][k] / det J.  Rows and columns taken cyclically:
// C[r][k] = J[r+1][k+1] J[r+2][k+2] - J[r+1][k+2] J[r+2][k+1] (indices mod 3).
__device__ __forceinline__ double geo_cofactor(const double *J, int r, int k)
{
    const int r1 = r == 2 ? 0 : r + 1, r2 = r == 0 ? 2 : r - 1;
    const int k1 = k == 2 ? 0 : k + 1, k2 = k == 0 ? 2 : k - 1;
    return __fma_rn(J[r1 * 3 + k1], J[r2 * 3 + k2], -__dmul_rn(J[r1 * 3 + k2], J[r2 * 3 + k1]));
}

// det J by the first row: J00 C00 + J01 C01 + J02 C02.
__device__ __forceinline__ double geo_det(const double *J, double c00, double c01, double c02)
{
    return __fma_rn(J[2], c02, __fma_rn(J[1], c01, __dmul_rn(J[0], c00)));
}

// float32 part of the stored copy: 1 / det J and w det J, both formed in
// float32 from the rounded det J (the cofactors and det J carry the FP64
// cancellation of distorted elements).
__device__ __forceinline__ void geo_quotient_f32(double det, double wq, float &rf, float &wd)
{
    const float df = __double2float_rn(det);
    rf = __fdiv_rn(1.0f, df);
    wd = __fmul_rn(__double2float_rn(wq), df);
}

__device__ __forceinline__ float geo_inverse_entry(double c, float rf) { return __fmul_rn(__double2float_rn(c), rf); }

// One quadrature point of a float32-only geometry: det J (returned, FP64), the
// float32 J^-1 (row-major, o[m * 3 + j] = (J^-1)_mj) and w det J.
__device__ __forceinline__ double geo_point_f32(const double *J, double wq, float o[9], float &wd)
{
    double C[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) C[r * 3 + k] = geo_cofactor(J, r, k);
    const double det = geo_det(J, C[0], C[1], C[2]);
    float rf;
    geo_quotient_f32(det, wq, rf, wd);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) o[k * 3 + r] = geo_inverse_entry(C[r * 3 + k], rf);
    return det;
}

// Status of a point's det J: positive and finite, else the error to report.
__device__ __forceinline__ int geo_det_status(double det)
{
    if (det > 0.0 && isfinite(det)) return FE_OK;
    return isfinite(det) ? FE_ERR_NONPOSITIVE_DETJ : FE_ERR_NONFINITE;
}
