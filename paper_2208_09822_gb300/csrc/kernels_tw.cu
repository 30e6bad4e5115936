// Instantiations and launchers of the warp-tile tensor-core kernel (tw.cuh).
#include <cuda_runtime.h>

#include "tw.cuh"
#include "launch.h"

namespace iaat {

template <int P>
static cudaError_t prep()
{
    return cudaFuncSetAttribute(tw_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTotal);
}

cudaError_t prepare_tw(int precision)
{
    switch (precision) {
    case kTc3xBF16: return prep<kTc3xBF16>();
    case kTcTF32: return prep<kTcTF32>();
    case kTcFP16: return prep<kTcFP16>();
    case kTc6xBF16: return prep<kTc6xBF16>();
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_tw(int precision, const TwParams &p, int grid, cudaStream_t stream)
{
    if (grid <= 0)
        return cudaSuccess;
    switch (precision) {
    case kTc3xBF16: tw_kernel<kTc3xBF16><<<grid, kTwThreads, kSmemTotal, stream>>>(p); break;
    case kTcTF32: tw_kernel<kTcTF32><<<grid, kTwThreads, kSmemTotal, stream>>>(p); break;
    case kTcFP16: tw_kernel<kTcFP16><<<grid, kTwThreads, kSmemTotal, stream>>>(p); break;
    case kTc6xBF16: tw_kernel<kTc6xBF16><<<grid, kTwThreads, kSmemTotal, stream>>>(p); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int tw_ring_bytes(int precision)
{
    switch (precision) {
    case kTc3xBF16: return tw_ring<kTc3xBF16>();
    case kTcTF32: return tw_ring<kTcTF32>();
    case kTcFP16: return tw_ring<kTcFP16>();
    case kTc6xBF16: return tw_ring<kTc6xBF16>();
    default: return 0;
    }
}

}  // namespace iaat
