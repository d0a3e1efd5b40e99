// Device pieces of the FP64 geometry of the reference mapping (Sec. 4.1 of
// Cimrman, arXiv 2107.04121) shared by the geometry kernels and by the residual
// kernel that computes the geometry of its elements itself.  Every rounding is
// explicit (__fma_rn, __dmul_rn, __fmul_rn, ...) so that each kernel that uses
// these functions produces the same bits for the same element.
#pragma once

#include "fe_device.cuh"

// Collocation stages for tensor-product bases with n1 nodes and n1 Gauss
// points per axis, one element, one 1-D line per item: X, U, V, P are [3][N]
// (N = n1^3) with the fastest index along x; B = (point, node) 1-D values,
// Dq = (point, point) collocation derivative, both row-major.
//   U[c][k][j][qx] = sum_i B[qx][i] X[c][k][j][i]
//   V[c][k][qy][qx] = sum_j B[qy][j] U[c][k][j][qx]
//   P[c][qz][qy][qx] = sum_k B[qz][k] V[c][k][qy][qx]          (x at the points)
//   J[q][c * 3 + m] = sum_p Dq[q_m][p] P[c][.. p along axis m ..]
// CENTER (n1 = 3 only): the middle Gauss point is the middle node and the middle
// row of Dq is (-d, 0, d), so that point's value is the nodal value and its
// derivative d (x2 - x0): 6 instead of 9 FMA per interpolated line; with the first
// and last rows of Dq antisymmetric, 7 instead of 9 operations per differentiated
// line.  The host sets CENTER only when the middle row of B is exactly (0, 1, 0),
// where the copy equals the FMA chain.
template <int N1, bool CENTER>
__device__ __forceinline__ void geo_line_interp(const double *__restrict__ x, int sx, double *__restrict__ out,
                                                int so, const double *__restrict__ B)
{
    static_assert(!CENTER || N1 == 3, "the centre specialisation is for three points");
    double v[N1];
#pragma unroll
    for (int i = 0; i < N1; ++i) v[i] = x[i * sx];
#pragma unroll
    for (int q = 0; q < N1; ++q) {
        if (CENTER && q == 1) {
            out[q * so] = v[1];
            continue;
        }
        double acc = 0.0;
#pragma unroll
        for (int i = 0; i < N1; ++i) acc = __fma_rn(B[q * N1 + i], v[i], acc);
        out[q * so] = acc;
    }
}

// The device table of the collocation derivative: Dq (n1 x n1, row-major),
// then GEO_DQ_EXTRA values that CENTER uses: with the first and last rows
// (d0, d1, d2) and (-d2, -d1, -d0) (symmetric points, made exact on the host),
// [n1 n1] = (d0 + d2) / 2, [n1 n1 + 1] = (d0 - d2) / 2, [n1 n1 + 2] = d1.
constexpr int GEO_DQ_EXTRA = 4;

template <int N1, bool CENTER>
__device__ __forceinline__ void geo_line_deriv(const double *__restrict__ x, int sx, double *__restrict__ out,
                                               int so, const double *__restrict__ Dq)
{
    double v[N1];
#pragma unroll
    for (int i = 0; i < N1; ++i) v[i] = x[i * sx];
    if constexpr (CENTER) {
        // e = v0 + v2, o = v0 - v2, t = (d0 + d2)/2 e + d1 v1:
        // out0 = (d0 - d2)/2 o + t, out2 = (d0 - d2)/2 o - t, out1 = -c o
        // (7 operations instead of 9 + 2 + 9)
        const double o = __dsub_rn(v[0], v[2]), e = __dadd_rn(v[0], v[2]);
        const double t = __fma_rn(Dq[N1 * N1], e, __dmul_rn(Dq[N1 * N1 + 2], v[1]));
        out[0] = __fma_rn(Dq[N1 * N1 + 1], o, t);
        out[so] = __dmul_rn(-Dq[1 * N1 + 2], o);
        out[2 * so] = __fma_rn(Dq[N1 * N1 + 1], o, -t);
    } else {
#pragma unroll
        for (int q = 0; q < N1; ++q) {
            double acc = 0.0;
#pragma unroll
            for (int p = 0; p < N1; ++p) acc = __fma_rn(Dq[q * N1 + p], v[p], acc);
            out[q * so] = acc;
        }
    }
}

// Stage items: t in [0, 3 n1^2) lines for the interpolations, [0, 9 n1^2) for J.
template <int N1, bool CENTER>
__device__ __forceinline__ void geo_lines_x(int t, const double *__restrict__ X, double *__restrict__ U,
                                            const double *__restrict__ B)
{
    constexpr int N = N1 * N1 * N1;
    const int c = t / (N1 * N1), kj = t % (N1 * N1);
    geo_line_interp<N1, CENTER>(X + c * N + kj * N1, 1, U + c * N + kj * N1, 1, B);
}

template <int N1, bool CENTER>
__device__ __forceinline__ void geo_lines_y(int t, const double *__restrict__ U, double *__restrict__ V,
                                            const double *__restrict__ B)
{
    constexpr int N = N1 * N1 * N1;
    const int c = t / (N1 * N1), k = (t / N1) % N1, qx = t % N1;
    const int o = c * N + k * N1 * N1 + qx;
    geo_line_interp<N1, CENTER>(U + o, N1, V + o, N1, B);
}

template <int N1, bool CENTER>
__device__ __forceinline__ void geo_lines_z(int t, const double *__restrict__ V, double *__restrict__ P,
                                            const double *__restrict__ B)
{
    constexpr int N = N1 * N1 * N1;
    const int c = t / (N1 * N1), qxy = t % (N1 * N1);
    geo_line_interp<N1, CENTER>(V + c * N + qxy, N1 * N1, P + c * N + qxy, N1 * N1, B);
}

// J[q][c * 3 + m] (J row-major per point, 9 N doubles) from the point values P:
// item t -> coordinate c, axis m, and the line along m through the other two.
template <int N1, bool CENTER>
__device__ __forceinline__ void geo_lines_jacobian(int t, const double *__restrict__ P, double *__restrict__ J,
                                                   const double *__restrict__ Dq)
{
    constexpr int N = N1 * N1 * N1;
    const int c = t / (3 * N1 * N1), m = (t / (N1 * N1)) % 3, l = t % (N1 * N1);
    const int la = l / N1, lb = l % N1;  // the two other point indices, slower one first
    // first point of the line and the stride along axis m, in point numbering
    const int q0 = m == 0 ? (la * N1 + lb) * N1 : (m == 1 ? la * N1 * N1 + lb : la * N1 + lb);
    const int sq = m == 0 ? 1 : (m == 1 ? N1 : N1 * N1);
    geo_line_deriv<N1, CENTER>(P + c * N + q0, sq, J + q0 * 9 + c * 3 + m, sq * 9, Dq);
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

// Round an FP64 value to float32 (to nearest, ties to even) with integer
// operations, off the FP64 pipe that the geometry saturates.  When the result is
// a normal float32 (biased FP64 exponent 897 ... 1150): the top 23 mantissa bits
// with the exponent rebiased by 1023 - 127 = 896 (a funnel shift of the two
// words), plus one when the 29 dropped bits exceed half an ulp or equal it with
// an odd result (a carry into the exponent is the correct rounding, up to
// infinity).  Zero, subnormal results, infinities and NaN take the hardware
// conversion.  Same bits as __double2float_rn for every input.
__device__ __forceinline__ float geo_to_f32(double x)
{
    const unsigned lo = (unsigned)__double2loint(x), hi = (unsigned)__double2hiint(x);
    const unsigned e11 = (hi >> 20) & 0x7FFu;
    if (e11 - 897u <= 253u) {
        unsigned f = __funnelshift_l(lo, (hi & 0x7FFFFFFFu) - 0x38000000u, 3);
        const unsigned rem = lo & 0x1FFFFFFFu;
        f += (unsigned)(rem > 0x10000000u) | ((unsigned)(rem == 0x10000000u) & f);
        return __uint_as_float(f | (hi & 0x80000000u));
    }
    return __double2float_rn(x);
}

// float32 part of the stored copy: 1 / det J and w det J, both formed in
// float32 from the rounded det J (the cofactors and det J carry the FP64
// cancellation of distorted elements).
__device__ __forceinline__ void geo_quotient_f32(double det, double wq, float &rf, float &wd)
{
    const float df = geo_to_f32(det);
    rf = __fdiv_rn(1.0f, df);
    wd = __fmul_rn(geo_to_f32(wq), df);
}

__device__ __forceinline__ float geo_inverse_entry(double c, float rf) { return __fmul_rn(geo_to_f32(c), rf); }

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
// Read from the bits with integer operations (the FP64 pipe is the busy one):
// an all-ones exponent is infinite or NaN, a set sign bit or +0 is not positive.
__device__ __forceinline__ int geo_det_status(double det)
{
    const unsigned hi = (unsigned)__double2hiint(det), lo = (unsigned)__double2loint(det);
    if (((hi >> 20) & 0x7FFu) == 0x7FFu) return FE_ERR_NONFINITE;
    if ((hi >> 31) != 0u || (hi | lo) == 0u) return FE_ERR_NONPOSITIVE_DETJ;
    return FE_OK;
}
