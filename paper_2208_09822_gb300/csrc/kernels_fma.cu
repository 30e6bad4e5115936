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

// FMA-pipe throughput probe: every thread runs 8 independent FMA chains of
// `iters` steps; the result is written so the work cannot be removed.
template <typename T>
__global__ void __launch_bounds__(256) fma_peak_kernel(T *out, int iters, T a, T b)
{
    T x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
        x[i] = (T)(threadIdx.x + i);
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int i = 0; i < 8; ++i)
                x[i] = fma(x[i], a, b);
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i)
        s += x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

cudaError_t measure_fma_peak(int dtype, double *gflops)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
        return e;
    const int blocks = sms * 8, threads = 256;
    const int iters = dtype == 0 ? 4096 : 256;
    void *buf = nullptr;
    if ((e = cudaMalloc(&buf, (size_t)blocks * threads * 8)) != cudaSuccess)
        return e;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int r = 0; r < 5 && e == cudaSuccess; ++r) {
        cudaEventRecord(e0);
        if (dtype == 0)
            fma_peak_kernel<float><<<blocks, threads>>>((float *)buf, iters, 0.999999f, 1e-7f);
        else
            fma_peak_kernel<double><<<blocks, threads>>>((double *)buf, iters, 0.999999, 1e-7);
        cudaEventRecord(e1);
        e = cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0 && ms < best)
            best = ms;
    }
    if (e == cudaSuccess)
        e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    const double flops = 2.0 * 16 * 8 * (double)iters * blocks * threads;
    *gflops = flops / (best * 1e-3) / 1e9;
    return e;
}

}  // namespace iaat
