// Tensor-core matrix mode: filled in by the split-precision kernels.
#include "fe_device.cuh"

cudaError_t fe_launch_matrix_tc(const fe_geometry_h *, const fe_form_h *, fe_material_args, fe_precision, void *,
                                int, cudaStream_t)
{
    return cudaErrorNotSupported;
}
