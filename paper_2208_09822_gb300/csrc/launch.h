// Host-side declarations of the kernel launchers (defined in the .cu files).
#pragma once
#include <cuda_runtime.h>
#include "common.cuh"

namespace iaat {
cudaError_t prepare_fma(int dtype);
cudaError_t launch_fma(int dtype, const KParams &kp, int grid, cudaStream_t stream);
cudaError_t single_call_err_ptr(int32_t **p);
}  // namespace iaat
