// Launcher of the warp-stream FP32 grouped kernel (ws.cuh).
#include <cuda_runtime.h>

#include "ws.cuh"
#include "launch.h"

namespace iaat {

cudaError_t prepare_ws()
{
    return cudaFuncSetAttribute(ws_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kWsWarps * kWsRingBytes);
}

cudaError_t launch_ws(const WsParams &p, int grid, cudaStream_t stream)
{
    if (grid <= 0)
        return cudaSuccess;
    ws_kernel<<<grid, kWsThreads, kWsWarps * kWsRingBytes, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace iaat
