// Instantiations and launchers of the complex grouped kernel (CGEMM / ZGEMM).
#include <cuda_runtime.h>

#include "complex.cuh"
#include "launch.h"

namespace iaat {

// dtype: IAAT_C32 (complex float) or IAAT_C64 (complex double)
cudaError_t prepare_cplx(int dtype)
{
    if (dtype == IAAT_C32)
        return cudaFuncSetAttribute(grouped_cplx_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    kSmemTotal);
    if (dtype == IAAT_C64)
        return cudaFuncSetAttribute(grouped_cplx_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    kSmemTotal);
    return cudaErrorInvalidValue;
}

cudaError_t launch_cplx(int dtype, const KParams &kp, int grid, cudaStream_t stream)
{
    if (grid <= 0)
        return cudaSuccess;
    if (dtype == IAAT_C32)
        grouped_cplx_kernel<float><<<grid, 32 * (kCplxWarps + 1), kSmemTotal, stream>>>(kp);
    else if (dtype == IAAT_C64)
        grouped_cplx_kernel<double><<<grid, 32 * (kCplxWarps + 1), kSmemTotal, stream>>>(kp);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

void cplx_ring(uint32_t *off, uint32_t *bytes)
{
    *off = (uint32_t)cplx_ring_offset();
    *bytes = (uint32_t)cplx_ring_bytes();
}

// Scratch of the single-call complex entry points (iaat_cgemm / iaat_zgemm):
// the call's scalars, stage-program offsets and stage programs, in a fixed
// array that every GPU loading this library holds (512 KB).
constexpr size_t kCplxSingleBytes = 512 * 1024;
static __device__ __align__(256) unsigned char g_cplx_single[kCplxSingleBytes];

cudaError_t cplx_single_scratch(char **p, size_t *bytes)
{
    *bytes = kCplxSingleBytes;
    return cudaGetSymbolAddress(reinterpret_cast<void **>(p), g_cplx_single);
}

}  // namespace iaat
