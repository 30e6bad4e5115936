// Instantiations and launchers of the warp-direct CUDA-core kernel (wd.cuh).
#include <cuda_runtime.h>

#include "wd.cuh"
#include "launch.h"

namespace iaat {

cudaError_t prepare_wd(int esz)
{
    const int bytes = kWdWarps * wd_warp_bytes(esz);
    return esz == 4 ? cudaFuncSetAttribute(wd_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)
                    : cudaFuncSetAttribute(wd_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_wd(int esz, const WdParams &p, int grid, cudaStream_t stream)
{
    if (grid <= 0)
        return cudaSuccess;
    const int bytes = kWdWarps * wd_warp_bytes(esz);
    if (esz == 4)
        wd_kernel<float><<<grid, kWdThreads, bytes, stream>>>(p);
    else
        wd_kernel<double><<<grid, kWdThreads, bytes, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace iaat
