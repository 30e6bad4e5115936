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
//  * the warp copies the op(A) and op(B) blocks element by element into its
//    own slice of shared memory with cp.async (consecutive lanes on
//    consecutive addresses of the stored matrices, whatever the transpose),
//    and each lane copies the C0 values of its own columns there too; the
//    next block's record is fetched meanwhile, and the warp waits for memory
//    once per block;
//  * each lane takes its row of op(A) into registers and runs Algorithm 1's
//    k-loop for one column at a time -- compiled for the block's exact K up
//    to wd_k1, so there are no bounds checks in it, and for K rounded up to a
//    multiple of 4 (the last four checked) up to wd_k2; the op(B) column read
//    as 16-byte vectors, which the lanes of one column group share -- and
//    stores alpha*acc + beta*C0 (the same operation order as the
//    stage-program kernel, so both give identical results).
//
// Blocks with K above wd_k1 are at most 16 rows by half the columns, so their
// longer op(A) rows and op(B) columns fit the same staging area; K above
// wd_k2 runs in chunks of wd_k2 values, the partial sums of the lane's at most
// kWdChunkIters column steps kept in the C0 area between chunks.  There are
// no waits on other warps; a malformed task record sets the plan's error
// word and is skipped.
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
__device__ __forceinline__ void wd_cp_elem(uint32_t dst, const T *src)
{
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void wd_cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void wd_cp_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void wd_cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// 1/d rounded to float, d = 1..32 (entry 0 unused): folded by the compiler.
__constant__ float c_wd_rcp[33] = {
    0.0f,        1.0f / 1,  1.0f / 2,  1.0f / 3,  1.0f / 4,  1.0f / 5,  1.0f / 6,  1.0f / 7,  1.0f / 8,
    1.0f / 9,    1.0f / 10, 1.0f / 11, 1.0f / 12, 1.0f / 13, 1.0f / 14, 1.0f / 15, 1.0f / 16, 1.0f / 17,
    1.0f / 18,   1.0f / 19, 1.0f / 20, 1.0f / 21, 1.0f / 22, 1.0f / 23, 1.0f / 24, 1.0f / 25, 1.0f / 26,
    1.0f / 27,   1.0f / 28, 1.0f / 29, 1.0f / 30, 1.0f / 31, 1.0f / 32};

// e / d for 0 <= e < 1024 and 1 <= d <= 32, rcp = c_wd_rcp[d]: the exact
// (e + 0.5) / d lies at least 0.5 / d >= 2^-6 from an integer, and the
// rounded reciprocal and product move it by under 512 * 2^-23 < 2^-13.
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

// What one block needs to find its operands and results.
template <typename T>
struct WdGeom {
    const T *A;          // op(A)(0, 0) of the block
    const T *B;          // op(B)(0, 0) of the block
    int64_t lda, ldb;
    bool ta, tb, readc;
    int m, n, g, q, i, iters, lane;
    int nt;              // the lane's column steps: those with q + g*t < n (0 unless q < g)
    int sa, pitch;       // staged op(A) row stride and op(B) column pitch of the block's shape
    T *C0;               // the lane's first C element (row i, column q)
    int64_t cstep;       // g columns of C
};

// Copy the kr x cnt block of a stored matrix X whose element (k, c) -- k the
// K index, c the row (op(A)) or column (op(B)) -- sits at X[c + k*ld]
// (kfast = false) or X[k + c*ld] (kfast = true), into shared memory at
// dst + k*sk + c*sc (elements).  The lanes split into gs = 32 / dv groups of
// dv = the fastest index's range: lane f + dv*s0 copies the elements (f, s)
// for s = s0, s0 + gs, ... of the slow index, so consecutive lanes read
// consecutive addresses and each step is a copy and two pointer increments.
template <typename T>
__device__ __forceinline__ void wd_stage_block(uint32_t dst, const T *X, int64_t ld, bool kfast, int k0, int kr,
                                               int cnt, int sk, int sc, int lane)
{
    const int dv = kfast ? kr : cnt, sv = kfast ? cnt : kr;   // fast, slow range
    const float rcp = c_wd_rcp[dv];
    const int gs = wd_div(32, rcp), s0 = wd_div(lane, rcp), f = lane - s0 * dv;
    if (s0 >= gs)
        return;   // lanes past the last whole group
    const int k = kfast ? f : s0, c = kfast ? s0 : f;
    const T *src = X + (kfast ? (int64_t)c * ld + (k0 + k) : (int64_t)(k0 + k) * ld + c);
    uint32_t d = dst + (uint32_t)((k * sk + c * sc) * (int)sizeof(T));
    const int64_t src_step = (int64_t)gs * ld;                                   // the slow index moves by gs
    const uint32_t d_step = (uint32_t)(gs * (kfast ? sc : sk) * (int)sizeof(T));
#pragma unroll 1
    for (int s = s0; s < sv; s += gs, src += src_step, d += d_step)
        wd_cp_elem<T>(d, src);
}

// Issue the copies of one K range [k0, k0 + kc) of the block: op(A) into sA,
// op(B) into sB and, with c0, the lane's C0 values into sC (its nt column
// steps).
template <typename T>
__device__ __forceinline__ void wd_stage(const WdGeom<T> &G, uint32_t sA, uint32_t sB, uint32_t sC, int k0, int kc,
                                         bool c0)
{
    if (kc > 0) {
        // op(A)(i, k): A[i + k*lda] (not transposed) or A[k + i*lda], to sA[k*sa + i]
        wd_stage_block<T>(sA, G.A, G.lda, G.ta, k0, kc, G.m, G.sa, 1, G.lane);
        // op(B)(k, j): B[k + j*ldb] (not transposed) or B[j + k*ldb], to sB[j*pitch + k]
        wd_stage_block<T>(sB, G.B, G.ldb, !G.tb, k0, kc, G.n, 1, G.pitch, G.lane);
    }
    if (c0) {
        const T *c = G.C0;
        uint32_t d = sC + (uint32_t)(G.lane * (int)sizeof(T));
#pragma unroll 2
        for (int t = 0; t < G.nt; ++t, c += G.cstep, d += 32 * (int)sizeof(T))
            wd_cp_elem<T>(d, c);
    }
}

// The column steps of a block, or of one K chunk of it, with kc values of
// k: acc = sum_k op(A)(i, k) * op(B)(k, j) in k order, then alpha*acc +
// beta*C0 stored (last), or the partial sum kept at sP[t*32 + lane] for the
// next chunk (first: no partial sum to add to).  The code is compiled for
// KR values of k, the last TAIL of them checked against kc (TAIL = 0: kc is
// KR).  CHUNK: first and last come at run time (else both hold).
template <typename T, int KR, int SA, int P, int TAIL, bool CHUNK>
__device__ __forceinline__ void wd_cols(int kc, bool first, bool last, const WdGeom<T> &G, const T *sA, const T *sB,
                                        const T *sC, T *sP, T alpha, T beta)
{
    if constexpr (!CHUNK)
        first = last = true;
    T a[KR];
#pragma unroll
    for (int k = 0; k < KR; ++k)
        a[k] = (k < KR - TAIL || k < kc) ? sA[k * SA + G.i] : T(0);
    T *Cl = G.C0;
    const T *b = sB + G.q * P;
#pragma unroll 1
    for (int t = 0; t < G.nt; ++t, b += G.g * P) {
        T acc = first ? T(0) : sP[t * 32 + G.lane];
        if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int k4 = 0; k4 < KR; k4 += 4) {
                const float4 w = *reinterpret_cast<const float4 *>(b + k4);
                const float wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (k4 + u < KR && (k4 + u < KR - TAIL || k4 + u < kc))
                        acc = fmaf(a[k4 + u], wv[u], acc);
            }
        } else {
#pragma unroll
            for (int k2 = 0; k2 < KR; k2 += 2) {
                const double2 w = *reinterpret_cast<const double2 *>(b + k2);
                if (k2 < KR - TAIL || k2 < kc)
                    acc = fma(a[k2], w.x, acc);
                if (k2 + 1 < KR && (k2 + 1 < KR - TAIL || k2 + 1 < kc))
                    acc = fma(a[k2 + 1], w.y, acc);
            }
        }
        if (last) {
            T v = alpha * acc;
            if (G.readc)
                v = fma(beta, sC[t * 32 + G.lane], v);
            Cl[t * G.cstep] = v;
        } else {
            sP[t * 32 + G.lane] = acc;
        }
    }
}

// K = 0 (alpha = 0): C = beta*C0 (alpha*0 first, as everywhere else).
template <typename T>
__device__ __forceinline__ void wd_cols0(const WdGeom<T> &G, const T *sC, T alpha, T beta)
{
#pragma unroll 1
    for (int t = 0; t < G.nt; ++t) {
        T v = alpha * T(0);
        if (G.readc)
            v = fma(beta, sC[t * 32 + G.lane], v);
        G.C0[t * G.cstep] = v;
    }
}

// One pass of the whole K of a block, 1 <= K <= wd_k2: exact code for
// K <= wd_k1 (32-row blocks), code for K rounded up to a multiple of 4
// beyond (16-row blocks).
template <typename T>
__device__ __forceinline__ void wd_cols_pass(int K, const WdGeom<T> &G, const T *sA, const T *sB, const T *sC, T *sP,
                                             T alpha, T beta)
{
    constexpr int E = (int)sizeof(T), P1 = wd_pitch1(E), P2 = wd_pitch2(E);
#define IAAT_WD_EXACT(k)                                                                       \
    case k:                                                                                    \
        wd_cols<T, k, 32, P1, 0, false>(k, true, true, G, sA, sB, sC, sP, alpha, beta);        \
        break;
#define IAAT_WD_WIDE(k)                                                                        \
    case (k) / 4:                                                                              \
        wd_cols<T, k, 16, P2, 4, false>(K, true, true, G, sA, sB, sC, sP, alpha, beta);        \
        break;
    if (K <= wd_k1(E)) {
        switch (K) {
            IAAT_WD_EXACT(1) IAAT_WD_EXACT(2) IAAT_WD_EXACT(3) IAAT_WD_EXACT(4)
            IAAT_WD_EXACT(5) IAAT_WD_EXACT(6) IAAT_WD_EXACT(7) IAAT_WD_EXACT(8)
        default:
            if constexpr (E == 4) {
                switch (K) {
                    IAAT_WD_EXACT(9) IAAT_WD_EXACT(10) IAAT_WD_EXACT(11) IAAT_WD_EXACT(12)
                    IAAT_WD_EXACT(13) IAAT_WD_EXACT(14) IAAT_WD_EXACT(15) IAAT_WD_EXACT(16)
                default:
                    break;
                }
            }
            break;
        }
    } else if constexpr (E == 4) {
        switch ((K + 3) / 4) {
            IAAT_WD_WIDE(20) IAAT_WD_WIDE(24) IAAT_WD_WIDE(28) IAAT_WD_WIDE(32)
        default:
            break;
        }
    } else {
        switch ((K + 3) / 4) {
            IAAT_WD_WIDE(12) IAAT_WD_WIDE(16)
        default:
            break;
        }
    }
#undef IAAT_WD_EXACT
#undef IAAT_WD_WIDE
}

// One K chunk of a 16-row block: kc values (1..wd_k2), code for kc rounded
// up to a multiple of 8 (the last 8 checked).
template <typename T>
__device__ __forceinline__ void wd_cols_chunk(int kc, bool first, bool last, const WdGeom<T> &G, const T *sA,
                                              const T *sB, const T *sC, T *sP, T alpha, T beta)
{
    constexpr int E = (int)sizeof(T), P2 = wd_pitch2(E);
#define IAAT_WD_CHUNK(k)                                                                       \
    case (k) / 8:                                                                              \
        wd_cols<T, k, 16, P2, 8, true>(kc, first, last, G, sA, sB, sC, sP, alpha, beta);       \
        break;
    switch ((kc + 7) / 8) {
        IAAT_WD_CHUNK(8) IAAT_WD_CHUNK(16)
    default:
        if constexpr (E == 4) {
            switch ((kc + 7) / 8) {
                IAAT_WD_CHUNK(24) IAAT_WD_CHUNK(32)
            default:
                break;
            }
        }
        break;
    }
#undef IAAT_WD_CHUNK
}

template <typename T>
__global__ void __launch_bounds__(kWdThreads, kWdCtasPerSm) wd_kernel(const WdParams p)
{
    extern __shared__ __align__(16) unsigned char smem_wd[];
    constexpr int ESZ = (int)sizeof(T);
    constexpr int K1 = wd_k1(ESZ), K2 = wd_k2(ESZ);
    const int lane = (int)(threadIdx.x & 31);
    const int wl = (int)(threadIdx.x >> 5);
    const int w = (int)blockIdx.x * kWdWarps + wl;
    if (w >= p.nwarps)
        return;
    unsigned char *base = smem_wd + wl * wd_warp_bytes(ESZ);
    WdTask *sR = reinterpret_cast<WdTask *>(base);   // two record slots
    T *sA = reinterpret_cast<T *>(base + kWdRecBytes);
    T *sB = sA + wd_a_elems(ESZ);
    T *sC = sB + wd_b_elems(ESZ);
    const uint32_t uA = (uint32_t)__cvta_generic_to_shared(sA), uB = (uint32_t)__cvta_generic_to_shared(sB),
                   uC = (uint32_t)__cvta_generic_to_shared(sC);
    T *sP = sC + kWdChunkIters * 32;   // partial sums between K chunks (16-row blocks: steps < 8)
    // records arrive by cp.async one block ahead, lanes 0..3 copying 16 bytes
    // each; the first from the warp's own copy, in flight with the loads of
    // its task range
    if (lane < 4)
        wd_cp16(reinterpret_cast<char *>(sR) + 16 * lane, reinterpret_cast<const char *>(p.first + w) + 16 * lane);
    wd_cp_commit();
    const int t0 = p.wbeg[w], t1 = p.wbeg[w + 1];
    for (int t = t0; t < t1; ++t) {
        wd_cp_wait0();   // this block's record has landed
        __syncwarp();    // (and the previous block's reads of the staging area are done)
        const WdTask &r = sR[(t - t0) & 1];   // fields read where used
        const int m = r.m, g = r.g, n = r.n, K = r.K, iters = r.iters;
        const bool wide = K > K1;   // the 16-row shape
        const int q = (lane * (int)r.magic) >> 15;   // lane / m
        const int i = lane - q * m;
        // the checks that keep every access inside the block and the staging
        // area: the shape's limits, a lane's row within the block, iters =
        // ceil(n / g)
        const bool bad = m < 1 || m > (wide ? kWdRows2 : kWdMaxRows) || g < 1 || m * g > 32 || n < 1 ||
                         n > (wide ? wd_max_cols(ESZ) / 2 : wd_max_cols(ESZ)) || K < 0 || iters * g < n ||
                         (iters - 1) * g >= n || i < 0 || i >= m;
        const bool skip = __any_sync(0xffffffffu, bad);
        WdGeom<T> G;
        G.A = reinterpret_cast<const T *>(r.A);
        G.B = reinterpret_cast<const T *>(r.B);
        G.lda = r.lda;
        G.ldb = r.ldb;
        G.ta = (r.flags & kWdTransA) != 0;
        G.tb = (r.flags & kWdTransB) != 0;
        G.readc = (r.flags & kWdReadC) != 0;
        G.m = m;
        G.n = n;
        G.g = g;
        G.q = q;
        G.i = i;
        G.iters = iters;
        G.lane = lane;
        // steps t with q + g*t < n: ceil((n - q) / g) = floor((n - q - 1 + 0.5) / g) + 1
        G.nt = q < g ? wd_div(n - q - 1, c_wd_rcp[g]) + 1 : 0;
        G.C0 = reinterpret_cast<T *>(r.C) + i + (int64_t)q * r.ldc;
        G.cstep = (int64_t)g * r.ldc;
        G.sa = wide ? kWdRows2 : kWdMaxRows;
        G.pitch = wide ? wd_pitch2(ESZ) : wd_pitch1(ESZ);
        const T alpha = wd_alpha<T>(r), beta = wd_beta<T>(r);
        if (!skip)
            wd_stage<T>(G, uA, uB, uC, 0, min(K, K2), G.readc);
        wd_cp_commit();
        if (t + 1 < t1 && lane < 4)   // the next record, into the other slot
            wd_cp16(reinterpret_cast<char *>(sR + ((t + 1 - t0) & 1)) + 16 * lane,
                    reinterpret_cast<const char *>(p.tasks + t + 1) + 16 * lane);
        wd_cp_commit();
        wd_cp_wait1();   // the staging copies (the record may still be in flight)
        __syncwarp();
        if (skip) {
            if (lane == 0 && p.err)
                atomicOr(p.err, kErrBadGroup);
            continue;
        }
        if (K == 0) {
            wd_cols0<T>(G, sC, alpha, beta);
        } else if (K <= K2) {
            wd_cols_pass<T>(K, G, sA, sB, sC, sP, alpha, beta);
        } else {
            // K in chunks of K2 (16-row blocks: at most 8 column steps per lane)
            wd_cols_chunk<T>(K2, true, false, G, sA, sB, sC, sP, alpha, beta);
            for (int k0 = K2; k0 < K; k0 += K2) {
                const int kc = min(K2, K - k0);
                __syncwarp();   // the previous chunk's reads of sA and sB are done
                wd_stage<T>(G, uA, uB, uC, k0, kc, false);
                wd_cp_commit();
                wd_cp_wait0();   // this chunk (and the next record)
                __syncwarp();
                wd_cols_chunk<T>(kc, false, k0 + kc >= K, G, sA, sB, sC, sP, alpha, beta);
            }
        }
    }
    wd_cp_wait0();   // no copy outlives the kernel
}

}  // namespace iaat
