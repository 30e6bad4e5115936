// Instantiations and launchers of the CUDA-core grouped kernel.
#include <cuda_runtime.h>

#include <mutex>

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
        grouped_kernel<float><<<grid, kernel_threads<4>(), kSmemTotal, stream>>>(kp);
    else
        grouped_kernel<double><<<grid, kernel_threads<8>(), kSmemTotal, stream>>>(kp);
    return cudaGetLastError();
}

void fma_ring(int esz, uint32_t *off, uint32_t *bytes)
{
    *off = esz == 4 ? smem_ring_offset<4>() : smem_ring_offset<8>();
    *bytes = esz == 4 ? ring_bytes<4>() : ring_bytes<8>();
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

// ------------------------------------------------ allocation-free entry
// Scratch of iaat_gemm_grouped_noalloc: the error word, the stage index and
// the task descriptors of one call, in a fixed array that every GPU loading
// this library holds until the process exits (about 545 KB).
namespace iaat {
constexpr int kNoAllocMaxTasks = 8192;
constexpr size_t kNoAllocGbegOff = 256;
constexpr size_t kNoAllocTasksOff = kNoAllocGbegOff + (((kNoAllocMaxTasks + 1) * sizeof(int32_t) + 255) & ~(size_t)255);
constexpr size_t kNoAllocBytes = kNoAllocTasksOff + (size_t)kNoAllocMaxTasks * sizeof(TaskDesc);
}  // namespace iaat

static __device__ __align__(256) unsigned char g_noalloc_scratch[iaat::kNoAllocBytes];

namespace {
std::mutex g_noalloc_mutex;          // guards the host staging arrays below
char *g_noalloc_dev[64];             // device address of the scratch, per device (set-up)
iaat::TaskDesc g_na_tasks[iaat::kNoAllocMaxTasks];
iaat::TaskDesc g_na_sorted[iaat::kNoAllocMaxTasks];
uint32_t g_na_bytes[iaat::kNoAllocMaxTasks];
double g_na_cost[iaat::kNoAllocMaxTasks];
int32_t g_na_order[iaat::kNoAllocMaxTasks];
int32_t g_na_gbeg[iaat::kNoAllocMaxTasks + 1];
}  // namespace

// See include/iaat.h.  Host planning goes into the static arrays above; the
// result is copied into g_noalloc_scratch on the caller's stream and the
// CUDA-core grouped kernel runs from there.
extern "C" iaat_status_t iaat_gemm_grouped_noalloc(const iaat_gemm_desc_t *descs, int64_t count, iaat_dtype_t dtype,
                                                   void *stream)
{
    using namespace iaat;
    if (count < 0 || (count > 0 && !descs))
        return noalloc_fail(IAAT_ERR_INVALID_VALUE, "bad descriptor array");
    if (dtype != IAAT_F32 && dtype != IAAT_F64)
        return noalloc_fail(IAAT_ERR_INVALID_VALUE, "unknown dtype");
    if (count > kNoAllocMaxTasks)
        return noalloc_fail(IAAT_ERR_INVALID_VALUE,
                            "more than 8192 instances: the allocation-free entry point holds at most 8192 tasks");
    const int esz = dtype == IAAT_F32 ? 4 : 8;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return noalloc_fail(IAAT_ERR_CUDA, "cudaGetDevice failed");
    {
        // the plan reaches the scratch through copies from host arrays that
        // the next call overwrites: a captured call would replay another
        // call's tasks, so capture is refused
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &cs) != cudaSuccess)
            return noalloc_fail(IAAT_ERR_CUDA, "cudaStreamIsCapturing failed");
        if (cs != cudaStreamCaptureStatusNone)
            return noalloc_fail(IAAT_ERR_UNSUPPORTED,
                                "the allocation-free entry point cannot be captured in a CUDA graph "
                                "(it copies each call's plan from reused host arrays)");
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mutex);
    if (!g_noalloc_dev[dev]) {
        // set-up, once per device, with that device current
        char *ptr = nullptr;
        if (cudaGetSymbolAddress((void **)&ptr, g_noalloc_scratch) != cudaSuccess || !ptr)
            return noalloc_fail(IAAT_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
        if (noalloc_prepare(dev) != IAAT_OK)
            return noalloc_fail(IAAT_ERR_CUDA, "kernel attribute set-up failed");
        g_noalloc_dev[dev] = ptr;
    }
    char *scratch = g_noalloc_dev[dev];
    int64_t nt = 0, ng = 0;
    iaat_status_t st = noalloc_plan(descs, count, esz, kNoAllocMaxTasks, g_na_tasks, g_na_bytes, g_na_cost,
                                    g_na_order, g_na_sorted, g_na_gbeg, &nt, &ng);
    if (st != IAAT_OK)
        return st;
    if (ng == 0)
        return IAAT_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // The host arrays are pageable, so each copy has taken its data when it
    // returns; the arrays can be reused by the next call at once.
    if (cudaMemsetAsync(scratch, 0, sizeof(int32_t), s) != cudaSuccess ||
        cudaMemcpyAsync(scratch + kNoAllocGbegOff, g_na_gbeg, (size_t)(ng + 1) * sizeof(int32_t),
                        cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(scratch + kNoAllocTasksOff, g_na_sorted, (size_t)nt * sizeof(TaskDesc),
                        cudaMemcpyHostToDevice, s) != cudaSuccess)
        return noalloc_fail(IAAT_ERR_CUDA, "copy into the scratch array failed");
    KParams kp;
    memset(&kp, 0, sizeof kp);
    kp.p.tasks = reinterpret_cast<const TaskDesc *>(scratch + kNoAllocTasksOff);
    kp.p.gbeg = reinterpret_cast<const int32_t *>(scratch + kNoAllocGbegOff);
    kp.p.ngroups = (int32_t)ng;
    kp.p.err = reinterpret_cast<int32_t *>(scratch);
    const int grid = (int)(ng < noalloc_sm_count(dev) ? ng : noalloc_sm_count(dev));
    if (launch_fma(esz == 4 ? 0 : 1, kp, grid, s) != cudaSuccess)
        return noalloc_fail(IAAT_ERR_CUDA, "kernel launch failed");
    return IAAT_OK;
}

// Error word of the allocation-free entry point (for iaat_plan_check(NULL)).
cudaError_t iaat::noalloc_err_ptr(int32_t **p)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev >= 0 && dev < 64 && g_noalloc_dev[dev]) {
        *p = reinterpret_cast<int32_t *>(g_noalloc_dev[dev]);
        return cudaSuccess;
    }
    *p = nullptr;
    return cudaSuccess;
}
