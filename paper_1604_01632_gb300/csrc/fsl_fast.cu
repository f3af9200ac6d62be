// fsl_fast.cu -- FP32-collide instantiations of the per-precision kernels:
// FP32 storage, and FP16 / BF16 storage of the shifted deviations f_a - w_a.
// Compiled with FMA contraction on (these forms are compared with the FP64
// oracle within stated tolerances, not bit for bit).
#include <cuda_runtime.h>

#include "fsl_device.cuh"
#include "fsl_internal.h"

namespace fsl {

FSL_INSTANTIATE_FORM(float)
FSL_INSTANTIATE_FORM(__half)
FSL_INSTANTIATE_FORM(__nv_bfloat16)

}  // namespace fsl
