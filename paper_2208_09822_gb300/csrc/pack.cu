// The pack step of a conventional GEMM as a GPU kernel -- kept only for the
// ablation that measures its share of the time (the GPU analogue of the
// paper's Fig. 3).
//
// Sec. I: a traditional GEMM blocks, packs and computes; the pack step copies
// operand blocks into the contiguous layout its single kernel expects, and for
// small matrices that extra pass over memory is a large share of the run time,
// which is why the paper's kernels read the matrices where they are.  Here the
// pack step copies op(A) and op(B) of every instance into a workspace as tight
// column-major M x K and K x N matrices (every case becomes NN) and rewrites the
// descriptors to point there; the library's grouped plan can then run on the
// packed copies.  The library's own path never packs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/iaat.h"
#include "launch.h"

namespace iaat {

// One matrix to pack: packed element (i, j), i < rows, j < cols, at
// dst[i + j*rows] is  trans ? src[j + i*ld] : src[i + j*ld].
struct PackJob {
    const char *src;
    char *dst;
    int32_t rows, cols, ld, trans;
};
static_assert(sizeof(PackJob) == 32, "PackJob layout");

// 256 threads (32 x 8) per CTA walk the jobs; each job in 32 x 32 tiles.  A
// transposed source goes through a shared tile so both the reads (along the
// stored columns) and the writes (along the packed columns) are coalesced.
// Every thread of a CTA works on the same job and tile, so the barriers are
// reached uniformly.
template <typename T>
__global__ void __launch_bounds__(256) pack_kernel(const PackJob *jobs, int njobs)
{
    __shared__ T tile[32][33];
    const int tx = (int)(threadIdx.x & 31u), ty = (int)(threadIdx.x >> 5);
    for (int jb = blockIdx.x; jb < njobs; jb += gridDim.x) {
        const PackJob J = jobs[jb];
        const T *src = reinterpret_cast<const T *>(J.src);
        T *dst = reinterpret_cast<T *>(J.dst);
        const int64_t ld = J.ld, rows = J.rows;
        for (int i0 = 0; i0 < J.rows; i0 += 32)
            for (int j0 = 0; j0 < J.cols; j0 += 32) {
                if (!J.trans) {
                    for (int r = ty; r < 32; r += 8) {
                        const int i = i0 + tx, j = j0 + r;
                        if (i < J.rows && j < J.cols)
                            dst[i + j * rows] = src[i + j * ld];
                    }
                } else {
                    for (int r = ty; r < 32; r += 8) {
                        const int i = i0 + r, j = j0 + tx;
                        if (i < J.rows && j < J.cols)
                            tile[r][tx] = src[j + i * ld];
                    }
                    __syncthreads();
                    for (int r = ty; r < 32; r += 8) {
                        const int i = i0 + tx, j = j0 + r;
                        if (i < J.rows && j < J.cols)
                            dst[i + j * rows] = tile[tx][r];
                    }
                    __syncthreads();
                }
            }
    }
}

}  // namespace iaat

struct iaat_pack_s {
    int device = 0;
    int esz = 4;
    char *d_ws = nullptr;
    iaat::PackJob *d_jobs = nullptr;
    int64_t njobs = 0;
    int grid = 0;
};

// See include/iaat.h.
extern "C" iaat_status_t iaat_pack_create(const iaat_gemm_desc_t *descs, int64_t count, iaat_dtype_t dtype,
                                          iaat_gemm_desc_t *packed, int64_t *bytes_moved, iaat_pack_t *out)
{
    using namespace iaat;
    if (!out)
        return host_fail(IAAT_ERR_INVALID_VALUE, "out is NULL");
    *out = nullptr;
    if (count < 0 || (count > 0 && (!descs || !packed)))
        return host_fail(IAAT_ERR_INVALID_VALUE, "bad descriptor arrays");
    if (dtype != IAAT_F32 && dtype != IAAT_F64)
        return host_fail(IAAT_ERR_INVALID_VALUE, "the pack step takes IAAT_F32 or IAAT_F64");
    const int esz = dtype == IAAT_F32 ? 4 : 8;
    std::vector<PackJob> jobs;
    std::vector<size_t> offs;   // workspace offset of each job's destination
    size_t ws = 0;
    int64_t moved = 0;
    auto round16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
    for (int64_t i = 0; i < count; ++i) {
        const iaat_gemm_desc_t &g = descs[i];
        const iaat_status_t st = validate_instance(i, g, esz);
        if (st != IAAT_OK)
            return st;
        iaat_gemm_desc_t &p = packed[i];
        p = g;
        p.transA = 0;
        p.transB = 0;
        p.lda = std::max(1, g.M);
        p.ldb = std::max(1, g.K);
        p.A = nullptr;
        p.B = nullptr;
        if (g.M == 0 || g.N == 0 || g.K == 0 || g.alpha == 0.0)
            continue;   // A and B are never read
        const size_t a_bytes = (size_t)g.M * g.K * esz, b_bytes = (size_t)g.K * g.N * esz;
        jobs.push_back(PackJob{static_cast<const char *>(g.A), nullptr, g.M, g.K, g.lda, g.transA});
        offs.push_back(ws);
        ws += round16(a_bytes);
        jobs.push_back(PackJob{static_cast<const char *>(g.B), nullptr, g.K, g.N, g.ldb, g.transB});
        offs.push_back(ws);
        ws += round16(b_bytes);
        moved += 2 * (int64_t)(a_bytes + b_bytes);
    }
    if (jobs.size() > (size_t)0x7fffffff)
        return host_fail(IAAT_ERR_UNSUPPORTED, "too many matrices to pack");
    iaat_pack_s *pk = new (std::nothrow) iaat_pack_s;
    if (!pk)
        return host_fail(IAAT_ERR_OOM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&pk->device);
    if (e == cudaSuccess)
        e = cudaMalloc(&pk->d_ws, std::max<size_t>(16, ws));
    if (e == cudaSuccess)
        e = cudaMalloc(reinterpret_cast<void **>(&pk->d_jobs), std::max<size_t>(1, jobs.size()) * sizeof(PackJob));
    if (e != cudaSuccess) {
        iaat_pack_destroy(pk);
        return host_fail(IAAT_ERR_OOM, (std::string("pack workspace: ") + cudaGetErrorString(e)).c_str());
    }
    // destinations, and the packed descriptors that point at them
    size_t k = 0;
    for (int64_t i = 0; i < count; ++i) {
        const iaat_gemm_desc_t &g = descs[i];
        if (g.M == 0 || g.N == 0 || g.K == 0 || g.alpha == 0.0)
            continue;
        jobs[k].dst = pk->d_ws + offs[k];
        packed[i].A = jobs[k].dst;
        jobs[k + 1].dst = pk->d_ws + offs[k + 1];
        packed[i].B = jobs[k + 1].dst;
        k += 2;
    }
    if (!jobs.empty() &&
        (e = cudaMemcpy(pk->d_jobs, jobs.data(), jobs.size() * sizeof(PackJob), cudaMemcpyHostToDevice)) !=
            cudaSuccess) {
        iaat_pack_destroy(pk);
        return host_fail(IAAT_ERR_CUDA, (std::string("upload the pack jobs: ") + cudaGetErrorString(e)).c_str());
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, pk->device) != cudaSuccess || sms <= 0)
        sms = 1;
    pk->esz = esz;
    pk->njobs = (int64_t)jobs.size();
    pk->grid = (int)std::min<int64_t>(pk->njobs, (int64_t)sms * 8);
    if (bytes_moved)
        *bytes_moved = moved;
    *out = pk;
    return IAAT_OK;
}

extern "C" iaat_status_t iaat_pack_run(iaat_pack_t pack, void *stream)
{
    using namespace iaat;
    if (!pack)
        return host_fail(IAAT_ERR_INVALID_VALUE, "pack is NULL");
    if (pack->njobs == 0)
        return IAAT_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (pack->esz == 4)
        pack_kernel<float><<<pack->grid, 256, 0, s>>>(pack->d_jobs, (int)pack->njobs);
    else
        pack_kernel<double><<<pack->grid, 256, 0, s>>>(pack->d_jobs, (int)pack->njobs);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return host_fail(IAAT_ERR_CUDA, (std::string("pack kernel launch: ") + cudaGetErrorString(e)).c_str());
    return IAAT_OK;
}

extern "C" iaat_status_t iaat_pack_destroy(iaat_pack_t pack)
{
    if (!pack)
        return IAAT_OK;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != pack->device)
        cudaSetDevice(pack->device);
    cudaDeviceSynchronize();
    if (pack->d_ws)
        cudaFree(pack->d_ws);
    if (pack->d_jobs)
        cudaFree(pack->d_jobs);
    if (cur >= 0 && cur != pack->device)
        cudaSetDevice(cur);
    delete pack;
    return IAAT_OK;
}
