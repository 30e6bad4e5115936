// Instantiations and launchers of the pack-stream tensor-core kernel (tc2.cuh).
#include <cuda_runtime.h>

#include "tc2.cuh"
#include "launch.h"

namespace iaat {

template <int P>
static cudaError_t prep()
{
    return cudaFuncSetAttribute(tc2_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTotal);
}

cudaError_t prepare_tc2(int precision)
{
    switch (precision) {
    case kTc3xBF16: return prep<kTc3xBF16>();
    case kTcTF32: return prep<kTcTF32>();
    case kTcFP16: return prep<kTcFP16>();
    case kTc6xBF16: return prep<kTc6xBF16>();
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_tc2(int precision, const Tc2Params &p, int grid, cudaStream_t stream)
{
    if (grid <= 0)
        return cudaSuccess;
    switch (precision) {
    case kTc3xBF16: tc2_kernel<kTc3xBF16><<<grid, kT2Threads, kSmemTotal, stream>>>(p); break;
    case kTcTF32: tc2_kernel<kTcTF32><<<grid, kT2Threads, kSmemTotal, stream>>>(p); break;
    case kTcFP16: tc2_kernel<kTcFP16><<<grid, kT2Threads, kSmemTotal, stream>>>(p); break;
    case kTc6xBF16: tc2_kernel<kTc6xBF16><<<grid, kT2Threads, kSmemTotal, stream>>>(p); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int tc2_ring_bytes(int precision)
{
    switch (precision) {
    case kTc3xBF16: return t2_ring_bytes<kTc3xBF16>();
    case kTcTF32: return t2_ring_bytes<kTcTF32>();
    case kTcFP16: return t2_ring_bytes<kTcFP16>();
    case kTc6xBF16: return t2_ring_bytes<kTc6xBF16>();
    default: return 0;
    }
}

}  // namespace iaat
