// Host-side declarations of the kernel launchers (defined in the .cu files).
#pragma once
#include <cuda_runtime.h>
#include "common.cuh"
#include "tw_types.cuh"
#include "wd_types.cuh"
#include "../../include/iaat.h"

namespace iaat {
cudaError_t prepare_fma(int dtype);
// warp-stream FP32 kernel (ws.cuh)
cudaError_t prepare_ws();
cudaError_t launch_ws(const WsParams &p, int grid, cudaStream_t stream);
cudaError_t launch_fma(int dtype, const KParams &kp, int grid, cudaStream_t stream);
cudaError_t single_call_err_ptr(int32_t **p);
cudaError_t measure_fma_peak(int dtype, double *gflops);   // 0 FP32 FFMA, 1 FP64 DFMA
// tcgen05 kernel, precision 1 = 3xBF16, 2 = TF32, 3 = FP16 (iaat_precision_t)
cudaError_t prepare_tc(int precision);
cudaError_t launch_tc(int precision, const KParams &kp, int grid, cudaStream_t stream);
int tc_group_cap(int precision);        // largest stage footprint (bytes)
// pack-stream tensor-core kernel (tc2.cuh)
cudaError_t prepare_tc2(int precision);
cudaError_t launch_tc2(int precision, const Tc2Params &p, int grid, cudaStream_t stream);
int tc2_ring_bytes(int precision);      // staging ring of one warp group (bytes)
// warp-tile tensor-core kernel (tw.cuh)
cudaError_t prepare_tw(int precision);
cudaError_t launch_tw(int precision, const TwParams &p, int grid, cudaStream_t stream);
int tw_ring_bytes(int precision);       // staging ring of one warp (bytes)
// warp-direct CUDA-core kernel (wd.cuh), esz 4 = FP32, 8 = FP64
cudaError_t prepare_wd(int esz);
cudaError_t launch_wd(int esz, const WdParams &p, int grid, cudaStream_t stream);
// complex kernel (CGEMM / ZGEMM), dtype IAAT_C32 or IAAT_C64
cudaError_t prepare_cplx(int dtype);
cudaError_t launch_cplx(int dtype, const KParams &kp, int grid, cudaStream_t stream);
// The staging ring of each kernel: byte offset from the shared-memory base and size.
void fma_ring(int esz, uint32_t *off, uint32_t *bytes);
void tc_ring(int precision, uint32_t *off, uint32_t *bytes);
void cplx_ring(uint32_t *off, uint32_t *bytes);
cudaError_t cplx_single_scratch(char **p, size_t *bytes);   // device scratch of iaat_cgemm / iaat_zgemm
constexpr int kTcPackRows = 128;        // rows of one MMA tile
constexpr int kTcPackCols = 128;        // columns of one MMA tile
// Allocation-free planning into caller-supplied arrays (host.cpp); used by
// iaat_gemm_grouped_noalloc (kernels_fma.cu).
iaat_status_t noalloc_plan(const iaat_gemm_desc_t *descs, int64_t count, int esz, int max_tasks, TaskDesc *tasks,
                           uint32_t *bytes, double *cost, int32_t *order, TaskDesc *out, int32_t *gbeg,
                           int64_t *ntasks_out, int64_t *ngroups_out);
iaat_status_t noalloc_fail(iaat_status_t st, const char *msg);
iaat_status_t noalloc_prepare(int dev);
int noalloc_sm_count(int dev);
cudaError_t noalloc_err_ptr(int32_t **p);   // NULL until the entry point's first call on the device
// host.cpp: set the calling thread's error message and return st; the
// argument checks of one instance (index idx in messages)
iaat_status_t host_fail(iaat_status_t st, const char *msg);
iaat_status_t validate_instance(int64_t idx, const iaat_gemm_desc_t &g, int esz);
}  // namespace iaat
