// Instantiations and launchers of the tcgen05 grouped kernel.
#include <cuda_runtime.h>
#include "tc.cuh"
#include "launch.h"

namespace iaat {

cudaError_t prepare_tc(int precision)
{
    switch (precision) {
    case kTc3xBF16:
        return cudaFuncSetAttribute(grouped_tc_kernel<kTc3xBF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTotal);
    case kTcTF32:
        return cudaFuncSetAttribute(grouped_tc_kernel<kTcTF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTotal);
    case kTcFP16:
        return cudaFuncSetAttribute(grouped_tc_kernel<kTcFP16>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTotal);
    case kTc6xBF16:
        return cudaFuncSetAttribute(grouped_tc_kernel<kTc6xBF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTotal);
    default:
        return cudaErrorInvalidValue;
    }
}

cudaError_t launch_tc(int precision, const KParams &kp, int grid, cudaStream_t stream)
{
    if (grid <= 0)
        return cudaSuccess;
    switch (precision) {
    case kTc3xBF16:
        grouped_tc_kernel<kTc3xBF16><<<grid, kTcThreads, kSmemTotal, stream>>>(kp);
        break;
    case kTcTF32:
        grouped_tc_kernel<kTcTF32><<<grid, kTcThreads, kSmemTotal, stream>>>(kp);
        break;
    case kTcFP16:
        grouped_tc_kernel<kTcFP16><<<grid, kTcThreads, kSmemTotal, stream>>>(kp);
        break;
    case kTc6xBF16:
        grouped_tc_kernel<kTc6xBF16><<<grid, kTcThreads, kSmemTotal, stream>>>(kp);
        break;
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int tc_group_cap(int precision)
{
    switch (precision) {
    case kTc3xBF16:
        return tc_max_group_bytes<kTc3xBF16>();
    case kTcTF32:
        return tc_max_group_bytes<kTcTF32>();
    case kTcFP16:
        return tc_max_group_bytes<kTcFP16>();
    case kTc6xBF16:
        return tc_max_group_bytes<kTc6xBF16>();
    default:
        return 0;
    }
}

void tc_ring(int precision, uint32_t *off, uint32_t *bytes)
{
    switch (precision) {
    case kTc3xBF16:
        *off = tc_ring_offset<kTc3xBF16>(), *bytes = tc_ring_bytes<kTc3xBF16>();
        break;
    case kTcTF32:
        *off = tc_ring_offset<kTcTF32>(), *bytes = tc_ring_bytes<kTcTF32>();
        break;
    case kTcFP16:
        *off = tc_ring_offset<kTcFP16>(), *bytes = tc_ring_bytes<kTcFP16>();
        break;
    default:
        *off = tc_ring_offset<kTc6xBF16>(), *bytes = tc_ring_bytes<kTc6xBF16>();
        break;
    }
}

}  // namespace iaat
