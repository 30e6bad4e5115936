// Instantiations and launchers of the CUDA-core grouped kernel.
#include <cuda_runtime.h>
#include "grouped.cuh"
#include "launch.h"

namespace iaat {

// Error word of the single-call entry points (iaat_sgemm / iaat_dgemm),
// which own no device memory of their own.
__device__ int32_t g_single_call_err;

cudaError_t prepare_fma(int dtype)
{
    if (dtype == 0)
        return cudaFuncSetAttribute(grouped_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTotal);
    return cudaFuncSetAttribute(grouped_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTotal);
}

cudaError_t launch_fma(int dtype, const KParams &kp, int grid, cudaStream_t stream)
{
    if (grid <= 0)
        return cudaSuccess;
    if (dtype == 0)
        grouped_kernel<float><<<grid, kThreads, kSmemTotal, stream>>>(kp);
    else
        grouped_kernel<double><<<grid, kThreads, kSmemTotal, stream>>>(kp);
    return cudaGetLastError();
}

cudaError_t single_call_err_ptr(int32_t **p)
{
    return cudaGetSymbolAddress(reinterpret_cast<void **>(p), g_single_call_err);
}

}  // namespace iaat
