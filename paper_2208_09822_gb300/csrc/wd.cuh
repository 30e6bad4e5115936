// Warp-direct grouped small-GEMM kernel on the CUDA cores (FFMA / DFMA): the
// "kernel executing plan" of Sec. V-B cut down to one warp per block with no
// staging pipeline, for batches of many tiny instances, where the per-task
// control work of a staged pipeline costs more than the data movement.
//
// The planner cuts every instance into warp blocks -- at most 32 rows and
// wd_max_cols columns of C with the instance's whole K -- and deals them to
// the warps of the grid ahead of time, largest first, each to the least
// loaded warp (no atomics; the launch replays from a CUDA graph unchanged).
// Within a block the warp's lanes form g column groups of m rows (m*g <= 32,
// so a 6-row block keeps 30 lanes busy instead of 6):
//
//  * each lane loads its row of op(A) straight into registers;
//  * the warp copies the op(B) block element by element into its own slice
//    of shared memory (consecutive lanes on consecutive addresses of the
//    stored B, whatever the transpose), and each lane copies the C0 values of
//    its own columns there too, so every load of the block is in flight at
//    once and the warp waits for memory once per block;
//  * each lane then runs Algorithm 1's k-loop for one column at a time -- the
//    op(B) column read as 16-byte vectors, which the lanes of one column group
//    share -- and stores alpha*acc + beta*C0 (the same operation order as the
//    stage-program kernel, so both give identical results).
//
// K runs in one pass of KR values held in registers, KR the smallest of
// 4, 8, 16, 32 (FP64: 4, 8, 16) that holds K; larger K runs in chunks of the
// largest, with the accumulators of at most kWdChunkIters columns per lane in
// registers.  There are no waits on other warps; a malformed task record sets
// the plan's error word and is skipped.
#pragma once
#include "wd_types.cuh"

namespace iaat {

__device__ __forceinline__ void wd_cp16(void *dst, const void *src)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
// one element, global to shared, without passing through registers
template <typename T>
__device__ __forceinline__ void wd_cp_elem(T *dst, const T *src)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void wd_cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void wd_cp_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void wd_cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// e / d for 0 <= e < 1024 and 1 <= d <= 32: the exact (e + 0.5) / d lies at
// least 0.5 / d >= 2^-6 from an integer, and the reciprocal and the product,
// each rounded to float, move it by under 512 * 2^-23 < 2^-13.
__device__ __forceinline__ int wd_div(int e, float rcp) { return __float2int_rz(((float)e + 0.5f) * rcp); }

template <typename T>
__device__ __forceinline__ T wd_alpha(const WdTask &r)
{
    if constexpr (sizeof(T) == 4)
        return r.ab.f[0];
    else
        return r.ab.d[0];
}
template <typename T>
__device__ __forceinline__ T wd_beta(const WdTask &r)
{
    if constexpr (sizeof(T) == 4)
        return r.ab.f[1];
    else
        return r.ab.d[1];
}

// What one block needs to find its operands.
template <typename T>
struct WdGeom {
    const T *B;          // op(B)(0, 0) of the block
    int64_t ldb;
    bool tb;
    int n, g, q, iters, lane;
    bool act;
    const T *C0;         // the lane's first C element (row i, column q)
    int64_t cstep;       // g columns of C
};

// The block's staging copies, all issued before anything waits for them:
// op(B)(k0 + k, j) for the kc x n elements e = 32*u + lane of the copy (in
// the stored order, so that consecutive lanes read consecutive addresses)
// into sB at j*pitch + k; and with readc the lane's C0 values of its column
// steps into sC at step*32 + lane.
template <typename T>
__device__ __forceinline__ void wd_stage(const WdGeom<T> &G, T *sB, T *sC, int k0, int kc, int pitch, bool stage_b,
                                         bool readc)
{
    if (stage_b) {
        const int ne = kc * G.n;
        const int dv = G.tb ? G.n : kc;   // the fastest index of the stored order
        const float rcp = __frcp_rn((float)dv);
#pragma unroll 4
        for (int e = G.lane; e < ne; e += 32) {
            const int s = wd_div(e, rcp), f = e - s * dv;   // slow, fast index
            const int k = G.tb ? s : f, j = G.tb ? f : s;
            wd_cp_elem(sB + j * pitch + k,
                       G.B + (G.tb ? (int64_t)(k0 + k) * G.ldb + j : (int64_t)j * G.ldb + (k0 + k)));
        }
    }
    if (readc && G.act) {
        const T *c = G.C0;
#pragma unroll 4
        for (int t = 0; t < G.iters; ++t, c += G.cstep)
            if (G.q + G.g * t < G.n)
                wd_cp_elem(sC + t * 32 + G.lane, c);
    }
}

// acc += sum over kk < kc of a[kk] * b[kk], in k order, b read as 16-byte vectors.
template <typename T, int KR>
__device__ __forceinline__ T wd_dot(const T (&a)[KR], const T *b, int kc, T acc)
{
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int k4 = 0; k4 < KR; k4 += 4) {
            const float4 w = *reinterpret_cast<const float4 *>(b + k4);
            if (k4 + 0 < kc) acc = fmaf(a[k4 + 0], w.x, acc);
            if (k4 + 1 < kc) acc = fmaf(a[k4 + 1], w.y, acc);
            if (k4 + 2 < kc) acc = fmaf(a[k4 + 2], w.z, acc);
            if (k4 + 3 < kc) acc = fmaf(a[k4 + 3], w.w, acc);
        }
    } else {
#pragma unroll
        for (int k2 = 0; k2 < KR; k2 += 2) {
            const double2 w = *reinterpret_cast<const double2 *>(b + k2);
            if (k2 + 0 < kc) acc = fma(a[k2 + 0], w.x, acc);
            if (k2 + 1 < kc) acc = fma(a[k2 + 1], w.y, acc);
        }
    }
    return acc;
}

template <typename T, int KR>
__device__ __forceinline__ void wd_load_a(T (&a)[KR], const T *Ai, int64_t astep, int kc, bool act)
{
#pragma unroll
    for (int kk = 0; kk < KR; ++kk)
        a[kk] = (act && kk < kc) ? __ldg(Ai + kk * astep) : T(0);
}

// One block whose K fits one pass of KR values.  The kernel loop has issued
// the staging copies (wd_stage) and waited for them.
template <typename T, int KR>
__device__ __forceinline__ void wd_block(const WdTask &r, const WdGeom<T> &G, const T (&a)[KR], const T *sB,
                                         const T *sC)
{
    constexpr int P = wd_pitch((int)sizeof(T), KR);
    const int K = r.K;
    const bool readc = (r.flags & kWdReadC) != 0;
    const T alpha = wd_alpha<T>(r), beta = wd_beta<T>(r);
    T *Cl = const_cast<T *>(G.C0);
#pragma unroll 1
    for (int t = 0; t < G.iters; ++t) {
        const int j = G.q + G.g * t;
        T acc = T(0);
        if (K > 0)
            acc = wd_dot<T, KR>(a, sB + min(j, G.n - 1) * P, K, acc);
        T v = alpha * acc;
        if (readc)
            v = fma(beta, sC[t * 32 + G.lane], v);
        if (G.act && j < G.n)
            Cl[t * G.cstep] = v;
    }
}

// Issue the staging copies and the loads of op(A) for a block of one pass,
// then (after the record prefetch) wait for the copies and run it.
template <typename T, int KR>
__device__ __forceinline__ void wd_run(const WdTask &r, const WdGeom<T> &G, T *sB, T *sC, int i, const void *next_rec,
                                       void *next_slot)
{
    constexpr int P = wd_pitch((int)sizeof(T), KR);
    const int K = r.K;
    T a[KR];
    if (K > 0) {
        const bool ta = (r.flags & kWdTransA) != 0;
        const int64_t lda = r.lda;
        wd_load_a<T, KR>(a, reinterpret_cast<const T *>(r.A) + (ta ? (int64_t)i * lda : (int64_t)i), ta ? 1 : lda, K,
                         G.act);
    }
    wd_stage<T>(G, sB, sC, 0, K, P, K > 0, (r.flags & kWdReadC) != 0);
    wd_cp_commit();
    if (next_rec && G.lane < 4)
        wd_cp16(static_cast<char *>(next_slot) + 16 * G.lane, static_cast<const char *>(next_rec) + 16 * G.lane);
    wd_cp_commit();
    wd_cp_wait1();   // the staging copies (the record may still be in flight)
    __syncwarp();
    wd_block<T, KR>(r, G, a, sB, sC);
}

// One block whose K runs in chunks of KR = wd_max_k values (iters <=
// kWdChunkIters): the lane's partial sums wait between chunks in the C0 area
// past its C0 values, at sC[(kWdChunkIters + t)*32 + lane].
template <typename T>
__device__ __forceinline__ void wd_run_chunked(const WdTask &r, const WdGeom<T> &G, T *sB, T *sC, int i,
                                               const void *next_rec, void *next_slot)
{
    constexpr int KR = wd_max_k((int)sizeof(T));
    constexpr int P = wd_pitch((int)sizeof(T), KR);
    static_assert(2 * kWdChunkIters <= wd_max_cols((int)sizeof(T)), "partial sums fit the C0 area");
    const int K = r.K;
    const bool readc = (r.flags & kWdReadC) != 0;
    const bool ta = (r.flags & kWdTransA) != 0;
    const int64_t lda = r.lda;
    const T *Ai = reinterpret_cast<const T *>(r.A) + (ta ? (int64_t)i * lda : (int64_t)i);
    const int64_t astep = ta ? 1 : lda;
    T *sAcc = sC + kWdChunkIters * 32 + G.lane;
    if (next_rec && G.lane < 4)
        wd_cp16(static_cast<char *>(next_slot) + 16 * G.lane, static_cast<const char *>(next_rec) + 16 * G.lane);
    wd_cp_commit();
    for (int k0 = 0; k0 < K; k0 += KR) {
        const int kc = min(KR, K - k0);
        __syncwarp();   // the previous chunk's reads of sB are done
        T a[KR];
        wd_load_a<T, KR>(a, Ai + k0 * astep, astep, kc, G.act);
        wd_stage<T>(G, sB, sC, k0, kc, P, true, readc && k0 == 0);   // C0 with the first chunk
        wd_cp_commit();
        wd_cp_wait0();
        __syncwarp();
#pragma unroll 1
        for (int t = 0; t < G.iters; ++t)
            sAcc[t * 32] = wd_dot<T, KR>(a, sB + min(G.q + G.g * t, G.n - 1) * P, kc, k0 == 0 ? T(0) : sAcc[t * 32]);
    }
    const T alpha = wd_alpha<T>(r), beta = wd_beta<T>(r);
    T *Cl = const_cast<T *>(G.C0);
#pragma unroll 1
    for (int t = 0; t < G.iters; ++t) {
        T v = alpha * sAcc[t * 32];
        if (readc)
            v = fma(beta, sC[t * 32 + G.lane], v);
        if (G.act && G.q + G.g * t < G.n)
            Cl[t * G.cstep] = v;
    }
}

template <typename T>
__global__ void __launch_bounds__(kWdThreads, kWdCtasPerSm) wd_kernel(const WdParams p)
{
    extern __shared__ __align__(16) unsigned char smem_wd[];
    constexpr int ESZ = (int)sizeof(T);
    const int lane = (int)(threadIdx.x & 31);
    const int wl = (int)(threadIdx.x >> 5);
    const int w = (int)blockIdx.x * kWdWarps + wl;
    if (w >= p.nwarps)
        return;
    unsigned char *base = smem_wd + wl * wd_warp_bytes(ESZ);
    WdTask *sR = reinterpret_cast<WdTask *>(base);   // two record slots
    T *sB = reinterpret_cast<T *>(base + kWdRecBytes);
    T *sC = sB + wd_b_elems(ESZ);
    const int t0 = p.wbeg[w], t1 = p.wbeg[w + 1];
    // records arrive by cp.async one block ahead: lanes 0..3 copy 16 bytes each
    if (t0 < t1 && lane < 4)
        wd_cp16(reinterpret_cast<char *>(sR) + 16 * lane, reinterpret_cast<const char *>(p.tasks + t0) + 16 * lane);
    wd_cp_commit();
    for (int t = t0; t < t1; ++t) {
        wd_cp_wait0();   // this block's record has landed
        __syncwarp();    // (and the previous block's reads of the staging area are done)
        const WdTask &r = sR[(t - t0) & 1];   // fields read where used
        const void *next_rec = t + 1 < t1 ? static_cast<const void *>(p.tasks + t + 1) : nullptr;
        void *next_slot = sR + ((t + 1 - t0) & 1);
        const int m = r.m, g = r.g, n = r.n, K = r.K, iters = r.iters;
        const bool chunked = K > wd_max_k(ESZ);
        const int q = (lane * (int)r.magic) >> 15;   // lane / m
        const int i = lane - q * m;
        // the checks that keep every access inside the block and the staging
        // area: a lane's row within the block, iters = ceil(n / g)
        const bool bad = m < 1 || m > kWdMaxRows || g < 1 || m * g > 32 || n < 1 || n > wd_max_cols(ESZ) || K < 0 ||
                         iters * g < n || (iters - 1) * g >= n || (chunked && iters > kWdChunkIters) || i < 0 ||
                         i >= m;
        if (__any_sync(0xffffffffu, bad)) {
            if (lane == 0 && p.err)
                atomicOr(p.err, kErrBadGroup);
            __syncwarp();
            if (next_rec && lane < 4)
                wd_cp16(static_cast<char *>(next_slot) + 16 * lane, static_cast<const char *>(next_rec) + 16 * lane);
            wd_cp_commit();
            continue;
        }
        WdGeom<T> G;
        G.B = reinterpret_cast<const T *>(r.B);
        G.ldb = r.ldb;
        G.tb = (r.flags & kWdTransB) != 0;
        G.n = n;
        G.g = g;
        G.q = q;
        G.iters = iters;
        G.lane = lane;
        G.act = q < g;
        G.C0 = reinterpret_cast<const T *>(r.C) + i + (int64_t)q * r.ldc;
        G.cstep = (int64_t)g * r.ldc;
        if (chunked)
            wd_run_chunked<T>(r, G, sB, sC, i, next_rec, next_slot);
        else if (K <= 4)
            wd_run<T, 4>(r, G, sB, sC, i, next_rec, next_slot);
        else if (K <= 8)
            wd_run<T, 8>(r, G, sB, sC, i, next_rec, next_slot);
        else if (ESZ == 8 || K <= 16)
            wd_run<T, 16>(r, G, sB, sC, i, next_rec, next_slot);
        else
            wd_run<T, wd_max_k(ESZ)>(r, G, sB, sC, i, next_rec, next_slot);
    }
    wd_cp_wait0();   // no copy outlives the kernel
}

}  // namespace iaat
