// Persistent grouped small-GEMM kernel on the tcgen05 tensor cores, FP32 in
// and out: 3xBF16 split products, TF32, or FP16 inputs, FP32 accumulation in
// tensor memory.
//
// The producer warp and the staging ring are those of the CUDA-core kernel.
// The eight consumer warps take a stage's tasks pack by pack: a pack is a set
// of tasks stacked into one 128-row MMA tile (task t owns rows R_t.., and the
// columns C_t.. of the concatenated B), so several small instances share one
// tensor-core pass and only the diagonal blocks of the product are kept.
// Per pack:
//   1. convert op(A) rows and op(B) columns of every task from the staged
//      FP32 data into the canonical K-major (no swizzle) operand layout,
//      splitting X = Xh + Xl for 3xBF16 (zero past each task's K);
//   2. one thread issues the MMAs (K/16 or K/8 steps; three products per
//      step for 3xBF16) into one of two TMEM accumulators and commits them to
//      an mbarrier;
//   3. while those run, the warps write the previous pack's results:
//      tcgen05.ld of the accumulator rows, alpha*acc + beta*C0, stores of
//      exactly the task's elements.
// Every wait is bounded; a time-out sets the error word and the kernel frees
// its tensor memory and returns.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "grouped.cuh"

namespace iaat {

constexpr int kTc3xBF16 = 1, kTcTF32 = 2, kTcFP16 = 3;
constexpr int kTcRows = 128;          // MMA M (TMEM lanes)
constexpr int kTcMaxCols = 128;       // columns of one pack (MMA N <= 128)
constexpr int kTcMaxK = 80;           // largest K of a task
constexpr int kTcConsumerWarps = 8;
constexpr int kTcThreads = 32 * (kTcConsumerWarps + 1);
constexpr int kTcTmemCols = 256;      // two accumulators of 128 columns

template <int P> struct TcTraits;
template <> struct TcTraits<kTc3xBF16> {
    static constexpr int kOpBytes = 2, kTerms = 2, kKStep = 16;
};
template <> struct TcTraits<kTcTF32> {
    static constexpr int kOpBytes = 4, kTerms = 1, kKStep = 8;
};
template <> struct TcTraits<kTcFP16> {
    static constexpr int kOpBytes = 2, kTerms = 1, kKStep = 16;
};

// Canonical K-major layout, no swizzle: core matrices of 8 rows x 16 bytes,
// stored as 128 contiguous bytes; core matrices adjacent along K are 128 B
// apart (leading byte offset), 8-row groups are kTcSBO<P> apart (stride byte
// offset).  One operand buffer holds 128 rows x kTcMaxK.
template <int P> IAAT_CE int tc_sbo() { return (kTcMaxK * TcTraits<P>::kOpBytes / 16) * 128; }
template <int P> IAAT_CE int tc_operand_bytes() { return (kTcRows / 8) * tc_sbo<P>(); }
template <int P> IAAT_CE int tc_operands_total() { return 2 * TcTraits<P>::kTerms * tc_operand_bytes<P>(); }

// shared-memory map (bytes)
constexpr int kTcMmaBar = 192;        // two mbarriers
constexpr int kTcTmemSlot = 208;      // tcgen05.alloc result
constexpr int kTcFlag = 212;          // consumer-wide status word
constexpr int kTcOperands = (kSmemCanon + 1023) & ~1023;
template <int P> IAAT_CE int tc_ring_offset() { return kTcOperands + tc_operands_total<P>(); }
template <int P> IAAT_CE int tc_ring_bytes() { return (kSmemTotal - tc_ring_offset<P>()) & ~127; }
template <int P> IAAT_CE int tc_max_group_bytes() { return tc_ring_bytes<P>() / 2; }

// ------------------------------------------------------------ tcgen05 PTX

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void consumer_bar() { asm volatile("bar.sync 1, %0;" ::"n"(kTcConsumerWarps * 32) : "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t slot_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot_smem), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version for tcgen05
    return d;                  // base offset 0, swizzle none
}

template <int P>
__device__ __forceinline__ uint32_t tc_idesc(int n)
{
    // D = F32; A/B = BF16 (1), F16 (0) or TF32 (2); both K-major; N>>3, M>>4
    constexpr uint32_t fmt = (P == kTc3xBF16) ? 1u : (P == kTcTF32 ? 2u : 0u);
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
}

template <int P>
__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    if constexpr (P == kTcTF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
            : "memory");
    }
}

__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i)
        v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------- conversions
// Round an FP32 value to TF32 (10 explicit mantissa bits), nearest-even;
// the tensor core then reads the top 19 bits unchanged.
__device__ __forceinline__ uint32_t tf32_rn(float x)
{
    uint32_t u = __float_as_uint(x);
    if ((u & 0x7f800000u) == 0x7f800000u)
        return u;   // Inf / NaN unchanged
    u += 0x0fffu + ((u >> 13) & 1u);
    return u & 0xffffe000u;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);   // .x = lo (low half), .y = hi
    return *reinterpret_cast<uint32_t *>(&h);
}

__device__ __forceinline__ uint32_t pack_f16(float lo, float hi)
{
    __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}

// Convert the 16-byte core-matrix row of VPR FP32 values x[] and store it
// (hi, and lo for 3xBF16) at byte offset `off` of the term buffers.
template <int P>
__device__ __forceinline__ void store_row(char *t0, char *t1, uint32_t off, const float *x)
{
    if constexpr (P == kTc3xBF16) {
        uint32_t h[4], l[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            h[q] = pack_bf16(x[2 * q], x[2 * q + 1]);
            const float r0 = x[2 * q] - __uint_as_float(h[q] << 16);
            const float r1 = x[2 * q + 1] - __uint_as_float(h[q] & 0xffff0000u);
            l[q] = pack_bf16(r0, r1);
        }
        *reinterpret_cast<uint4 *>(t0 + off) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4 *>(t1 + off) = make_uint4(l[0], l[1], l[2], l[3]);
    } else if constexpr (P == kTcFP16) {
        uint32_t h[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            h[q] = pack_f16(x[2 * q], x[2 * q + 1]);
        *reinterpret_cast<uint4 *>(t0 + off) = make_uint4(h[0], h[1], h[2], h[3]);
    } else {
        *reinterpret_cast<uint4 *>(t0 + off) = make_uint4(tf32_rn(x[0]), tf32_rn(x[1]), tf32_rn(x[2]), tf32_rn(x[3]));
    }
}

// Convert rows [0, rows) of one operand of a task into canonical rows
// [row0, row0 + rows) of the term buffers, K-groups [0, ngroups).
// raw(i, k) = src + i*si + k*sk (bytes); values with k >= K are zero.
// kfast: lanes run along the K-groups (raw contiguous in k), else along rows.
template <int P>
__device__ __forceinline__ void convert_operand(char *t0, char *t1, const char *src, int si, int sk, int rows,
                                                int K, int row0, int ngroups, bool kfast)
{
    constexpr int VPR = 16 / TcTraits<P>::kOpBytes;   // values per core-matrix row
    constexpr int SBO = tc_sbo<P>();
    const int lane = (int)lane_id();
    if (rows <= 0 || ngroups <= 0)
        return;
    int lg_fast;   // log2 of lanes along the fast dimension
    const int fast_len = kfast ? ngroups : rows;
    lg_fast = fast_len >= 32 ? 5 : (32 - __clz(fast_len - 1));   // ceil(log2)
    if (fast_len <= 1)
        lg_fast = 0;
    const int nfast = 1 << lg_fast;
    const int lf = lane & (nfast - 1);
    const int ls = lane >> lg_fast;
    const int sstep = 32 >> lg_fast;
    const int slow_len = kfast ? rows : ngroups;
#pragma unroll 1
    for (int s0 = 0; s0 < slow_len; s0 += sstep) {
        const int s = s0 + ls;
#pragma unroll 1
        for (int f = lf; f < fast_len && s < slow_len; f += nfast) {
            const int i = kfast ? s : f;
            const int g = kfast ? f : s;
            const int k0 = g * VPR;
            float x[8];
            const char *p = src + i * si + k0 * sk;
#pragma unroll
            for (int e = 0; e < VPR; ++e)
                x[e] = (k0 + e < K) ? *reinterpret_cast<const float *>(p + e * sk) : 0.0f;
            const int r = row0 + i;
            const uint32_t off = (uint32_t)((r >> 3) * SBO + g * 128 + (r & 7) * 16);
            store_row<P>(t0, t1, off, x);
        }
    }
}

template <int P>
__device__ void tc_epilogue(const SmemMap &S, const TaskRec *recs, unsigned mask, bool zero_acc, int NT, int cw,
                            uint32_t dtmem);

struct PackTask {   // fields of one task as the consumer warps need them
    int M, N, K, R, Cc, ta, tb, offA, offB, csA, csB;
};

template <int P>
__device__ void tc_consumer(const KParams &KP, const SmemMap &S, int cw, uint32_t tmem)
{
    const Params &P_ = KP.p;
    const int lane = (int)lane_id();
    constexpr int KS = TcTraits<P>::kKStep;
    constexpr int VPR = 16 / TcTraits<P>::kOpBytes;
    constexpr int OPB = tc_operand_bytes<P>();
    char *const opbase = S.base + kTcOperands;
    char *const A0 = opbase;
    char *const A1 = opbase + OPB;                                   // 3xBF16: lo
    char *const B0 = opbase + TcTraits<P>::kTerms * OPB;
    char *const B1 = B0 + OPB;
    volatile int32_t *flag = reinterpret_cast<volatile int32_t *>(S.base + kTcFlag);
    const uint32_t mbar0 = S.sbase + kTcMmaBar;
    uint32_t mma_phase[2] = {0u, 0u};
    int buf = 0;
    bool alive = true;

    for (int i = 0; alive; ++i) {
        const int g = sched_group(i, blockIdx.x, gridDim.x);
        if (g >= P_.ngroups)
            break;
        const int slot = i % kNumSlots;
        if (cw == 0) {
            int ok = 1;
            if (lane == 0)
                ok = mbar_wait(S.full(slot), (uint32_t)((i / kNumSlots) & 1), kWaitLimitNs) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (lane == 0) {
                *flag = ok;
                if (!ok)
                    set_error(P_.err, kErrTimeoutFull);
            }
        }
        consumer_bar();
        if (!*flag) {
            alive = false;
            break;
        }
        const SlotHeader *hd = S.header(slot);
        const TaskRec *recs = S.recs(slot);
        const int nt = hd->ntasks;
        // lane t keeps task t's fields
        PackTask me{0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        int pack = 1 << 20;
        if (lane < nt) {
            const TaskRec &r = recs[lane];
            me = PackTask{r.M, r.N, r.K, r.nbm, r.nbn, r.ta, r.tb, r.offA, r.offB, r.csA, r.csB};
            pack = r.variant;
        }
        int npacks = lane < nt ? pack + 1 : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            npacks = max(npacks, __shfl_xor_sync(0xffffffffu, npacks, o));

        unsigned prev_mask = 0;
        int prev_nt = 0;
        bool prev_zero = false;
        for (int p = 0; p < npacks && alive; ++p) {
            const unsigned mask = __ballot_sync(0xffffffffu, lane < nt && pack == p);
            int kmax = (mask >> lane) & 1 ? me.K : 0;
            int cmax = (mask >> lane) & 1 ? me.Cc + me.N : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
                cmax = max(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
            }
            const int KT = (kmax + KS - 1) / KS * KS;
            const int NT = max(16, (cmax + 15) & ~15);
            const int ngroups = KT / VPR;
            // 1. conversion: the pack's tasks dealt round-robin to the warps
            if (KT > 0) {
                int q = 0;
                for (unsigned m = mask; m; m &= m - 1, ++q) {
                    const int t = __ffs(m) - 1;
                    if ((q % kTcConsumerWarps) != cw)
                        continue;
                    PackTask tk;
                    tk.M = __shfl_sync(0xffffffffu, me.M, t);
                    tk.N = __shfl_sync(0xffffffffu, me.N, t);
                    tk.K = __shfl_sync(0xffffffffu, me.K, t);
                    tk.R = __shfl_sync(0xffffffffu, me.R, t);
                    tk.Cc = __shfl_sync(0xffffffffu, me.Cc, t);
                    tk.ta = __shfl_sync(0xffffffffu, me.ta, t);
                    tk.tb = __shfl_sync(0xffffffffu, me.tb, t);
                    tk.offA = __shfl_sync(0xffffffffu, me.offA, t);
                    tk.offB = __shfl_sync(0xffffffffu, me.offB, t);
                    tk.csA = __shfl_sync(0xffffffffu, me.csA, t);
                    tk.csB = __shfl_sync(0xffffffffu, me.csB, t);
                    // op(A)(i, k): stored A[i + k*lda] (N) or A[k + i*lda] (T)
                    const int ai = tk.ta ? tk.csA : 4, ak = tk.ta ? 4 : tk.csA;
                    convert_operand<P>(A0, A1, S.base + tk.offA, ai, ak, tk.M, tk.K, tk.R, ngroups, tk.ta != 0);
                    // op(B)(k, n) as an N x K operand: stored B[k + n*ldb] (N) or B[n + k*ldb] (T)
                    const int bi = tk.tb ? 4 : tk.csB, bk = tk.tb ? tk.csB : 4;
                    convert_operand<P>(B0, B1, S.base + tk.offB, bi, bk, tk.N, tk.K, tk.Cc, ngroups, tk.tb == 0);
                }
            }
            fence_proxy_async();
            tc_fence_before();
            consumer_bar();
            // 2. MMAs of this pack into accumulator `buf`
            if (cw == 0 && lane == 0 && KT > 0) {
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(buf * kTcMaxCols);
                const uint32_t idesc = tc_idesc<P>(NT);
                const uint32_t a0 = smem_addr(A0), a1 = smem_addr(A1), b0 = smem_addr(B0), b1 = smem_addr(B1);
                constexpr uint32_t SBO = (uint32_t)tc_sbo<P>();
                for (int ks = 0; ks < KT / KS; ++ks) {
                    const uint32_t o = (uint32_t)ks * 256u;   // two core matrices along K
                    if constexpr (P == kTc3xBF16) {
                        tc_mma<P>(d, smem_desc(a1 + o, 128, SBO), smem_desc(b0 + o, 128, SBO), idesc, ks > 0);
                        tc_mma<P>(d, smem_desc(a0 + o, 128, SBO), smem_desc(b1 + o, 128, SBO), idesc, 1);
                        tc_mma<P>(d, smem_desc(a0 + o, 128, SBO), smem_desc(b0 + o, 128, SBO), idesc, 1);
                    } else {
                        tc_mma<P>(d, smem_desc(a0 + o, 128, SBO), smem_desc(b0 + o, 128, SBO), idesc, ks > 0);
                    }
                }
                tc_commit(mbar0 + 8u * (uint32_t)buf);
            }
            // 3. results of the previous pack while these MMAs run
            if (p > 0)
                tc_epilogue<P>(S, recs, prev_mask, prev_zero, prev_nt, cw, tmem + (uint32_t)((buf ^ 1) * kTcMaxCols));
            // wait for this pack's MMAs: the operand buffers are free again
            if (cw == 0) {
                int ok = 1;
                if (lane == 0 && KT > 0) {
                    ok = mbar_wait(mbar0 + 8u * (uint32_t)buf, mma_phase[buf], kWaitLimitNs) ? 1 : 0;
                    if (!ok)
                        set_error(P_.err, kErrTimeoutFull);
                }
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (lane == 0)
                    *flag = ok;
            }
            if (KT > 0)
                mma_phase[buf] ^= 1u;
            tc_fence_before();
            consumer_bar();
            tc_fence_after();
            if (!*flag) {
                alive = false;
                break;
            }
            prev_mask = mask;
            prev_zero = KT == 0;   // no product: the accumulator is not read
            prev_nt = NT;
            buf ^= 1;
        }
        if (!alive)
            break;
        if (npacks > 0)
            tc_epilogue<P>(S, recs, prev_mask, prev_zero, prev_nt, cw, tmem + (uint32_t)((buf ^ 1) * kTcMaxCols));
        tc_fence_before();
        consumer_bar();
        if (cw == 0 && lane == 0)
            mbar_arrive(S.empty(slot));
    }
    // leave: every consumer warp reaches this barrier on both paths
    tc_fence_before();
    consumer_bar();
    tc_fence_after();
    if (cw == 0)
        tmem_dealloc(tmem, kTcTmemCols);
}

// Results of one pack: thread (warp cw, lane) owns accumulator row
// 32*(cw%4) + lane; warps cw < 4 take the even 16-column chunks, the others
// the odd ones.  `mask` bit t: task t is in the pack; zero_acc: the pack
// had no product (K = 0 or alpha = 0 everywhere), acc = 0.
template <int P>
__device__ void tc_epilogue(const SmemMap &S, const TaskRec *recs, unsigned mask, bool zero_acc, int NT, int cw,
                            uint32_t dtmem)
{
    const int lane = (int)lane_id();
    const int row = 32 * (cw & 3) + lane;
    // find this row's task
    int t = -1;
    for (unsigned m = mask; m; m &= m - 1) {
        const int c = __ffs(m) - 1;
        const int R = recs[c].nbm, M = recs[c].M;
        if (row >= R && row < R + M)
            t = c;
    }
    int Cc = 0, N = 0, i = 0, ldc = 0, csC = 0, offC = 0;
    float alpha = 0.f, beta = 0.f;
    bool readc = false;
    float *C = nullptr;
    if (t >= 0) {
        const TaskRec &r = recs[t];
        Cc = r.nbn; N = r.N; i = row - r.nbm; ldc = r.ldc; csC = r.csC; offC = r.offC;
        alpha = (float)r.alpha; beta = (float)r.beta;
        readc = (r.flags & kFlagReadC) != 0;
        C = reinterpret_cast<float *>(r.C);
    }
    const uint32_t taddr = dtmem + ((uint32_t)(32 * (cw & 3)) << 16);
    for (int ch = (cw >> 2); ch * 16 < NT; ch += 2) {
        const int j0 = ch * 16;
        const bool need = t >= 0 && Cc < j0 + 16 && j0 < Cc + N;
        if (!__any_sync(0xffffffffu, need))
            continue;
        float v[16];
        if (zero_acc) {
#pragma unroll
            for (int u = 0; u < 16; ++u)
                v[u] = 0.f;
        } else {
            tmem_ld16(taddr + (uint32_t)j0, v);
        }
        if (need) {
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int j = j0 + u - Cc;
                if (j >= 0 && j < N) {
                    float c = alpha * v[u];
                    if (readc)
                        c = fmaf(beta, *reinterpret_cast<const float *>(S.base + offC + j * csC + i * 4), c);
                    C[i + (int64_t)j * ldc] = c;
                }
            }
        }
    }
}

template <int P>
__global__ void __launch_bounds__(kTcThreads, 1) grouped_tc_kernel(const __grid_constant__ KParams KP)
{
    extern __shared__ __align__(1024) char smem_tc[];
    char *smem = smem_tc;
    SmemMap S;
    S.base = smem;
    S.sbase = smem_addr(smem);
    S.ring_off = (uint32_t)tc_ring_offset<P>();
    S.ring_bytes = (uint32_t)tc_ring_bytes<P>();
    const int warp = threadIdx.x / 32;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kNumSlots; ++s) {
            mbar_init(S.full(s), 1);
            mbar_init(S.empty(s), 1);
        }
        mbar_init(S.sbase + kTcMmaBar, 1);
        mbar_init(S.sbase + kTcMmaBar + 8, 1);
        fence_barrier_init();
    }
    if (warp == 0)
        tmem_alloc(S.sbase + kTcTmemSlot, kTcTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t *>(smem + kTcTmemSlot);
    if (warp == kTcConsumerWarps)
        producer_loop<4>(KP, S);
    else
        tc_consumer<P>(KP, S, warp, tmem);
}

}  // namespace iaat
