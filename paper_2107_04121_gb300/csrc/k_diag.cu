// Diagnostic kernels behind fe_diag_fp64: the FP64 rates that decide where the
// library computes in FP64.  Each lane runs `ilp` independent chains of
// `steps` dependent operations, one CTA of `warps` warps per SM:
//   kind 0  DFMA (the FP64 pipe of the CUDA cores), 1 lane-FMA per lane per step
//   kind 1  mma.sync.m8n8k4 with FP64 operands and accumulators (the FP64
//           tensor-core path), 256 FMAs per warp per step
// The caller times the launch; the result only keeps the chains alive.
#include "fe_device.cuh"

namespace {

template <int ILP>
__global__ void k_diag_dfma(double *out, int steps, double a, double b)
{
    double x[ILP];
#pragma unroll
    for (int i = 0; i < ILP; ++i) x[i] = threadIdx.x * 1e-3 + i;
    for (int it = 0; it < steps; ++it) {
#pragma unroll
        for (int i = 0; i < ILP; ++i) x[i] = fma(x[i], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < ILP; ++i) s += x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int ILP>
__global__ void k_diag_dmma(double *out, int steps)
{
    const int lane = threadIdx.x & 31;
    const double a = 1.0 + lane * 1e-3, b = 1.0 - lane * 1e-3;
    double c[ILP][2];
#pragma unroll
    for (int i = 0; i < ILP; ++i) c[i][0] = c[i][1] = i;
    for (int it = 0; it < steps; ++it) {
#pragma unroll
        for (int i = 0; i < ILP; ++i)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                         : "+d"(c[i][0]), "+d"(c[i][1])
                         : "d"(a), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < ILP; ++i) s += c[i][0] + c[i][1];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int ILP>
cudaError_t launch_diag(int kind, int sms, int warps, int steps, double *out, cudaStream_t s)
{
    if (kind == 0)
        k_diag_dfma<ILP><<<sms, 32 * warps, 0, s>>>(out, steps, 0.999999, 1e-9);
    else
        k_diag_dmma<ILP><<<sms, 32 * warps, 0, s>>>(out, steps);
    return cudaGetLastError();
}

}  // namespace

cudaError_t fe_launch_diag_fp64(int kind, int sms, int warps, int ilp, int steps, double *out, cudaStream_t s)
{
    switch (ilp) {
    case 1: return launch_diag<1>(kind, sms, warps, steps, out, s);
    case 2: return launch_diag<2>(kind, sms, warps, steps, out, s);
    case 4: return launch_diag<4>(kind, sms, warps, steps, out, s);
    default: return cudaErrorInvalidValue;
    }
}
