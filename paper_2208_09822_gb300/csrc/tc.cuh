// Persistent grouped small-GEMM kernel on the tcgen05 tensor cores, FP32 in
// and out: 3xBF16 split products, TF32, or FP16 inputs, FP32 accumulation in
// tensor memory.
//
// Packs: the planner stacks the tasks of a stage into packs of at most 128
// rows and 128 columns; task t owns rows R_t.. of the MMA tile and columns
// C_t.. of the concatenated B, so several small instances share one
// tensor-core pass and only the diagonal blocks of the product are kept
// (the pack index, R_t and C_t travel in the task's variant/nbm/nbn fields).
//
// Warp roles (18 warps):
//   0-7  converters: per 32-wide K-chunk of a pack, every thread converts one
//        row of the 128-row tile -- warps 0-3 the rows of op(A), warps 4-7
//        the rows of op(B)^T -- from the staged FP32 data into the canonical
//        K-major (no swizzle) operand layout of one of two operand stages:
//        X = Xh + Xl (BF16) for 3xBF16, RN-rounded TF32, or FP16, with zeros
//        past the row's K;
//   8-15 epilogue: when a pack's accumulator is complete, read each row of
//        it from tensor memory (warps 8+q and 12+q own lanes 32q..32q+31 and
//        take alternate 16-column chunks) and write alpha*acc + beta*C0 to
//        exactly the task's elements;
//   16   producer: streams stages into the shared-memory ring (shared with
//        the CUDA-core kernel);
//   17   MMA: one lane issues the chunk's MMAs into one of two accumulators
//        and commits them to mbarriers that free the operand stage and, after
//        a pack's last chunk, hand the accumulator to the epilogue.
// Conversion of chunk c+1, the MMAs of chunk c and the epilogue of the
// previous pack run at the same time.  Every wait is bounded; a time-out sets
// the error word, every role leaves its loop, and the CTA frees its tensor
// memory before returning.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "grouped.cuh"

namespace iaat {

constexpr int kTc3xBF16 = 1, kTcTF32 = 2, kTcFP16 = 3;
constexpr int kTcRows = 128;           // MMA M (TMEM lanes)
constexpr int kTcMaxCols = 128;        // columns of one pack (MMA N <= 128)
constexpr int kTcKC = 32;              // K per operand stage
constexpr int kTcStages = 2;           // operand stages
constexpr int kTcConvWarps = 8, kTcEpiWarps = 8;
constexpr int kTcWarpProducer = 16, kTcWarpMma = 17;
constexpr int kTcThreads = 576;
constexpr int kTcTmemCols = 256;       // two accumulators of 128 columns

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
// apart (leading byte offset), 8-row groups are tc_sbo() apart (stride byte
// offset).  One operand buffer holds 128 rows x kTcKC.
template <int P> IAAT_CE int tc_vpr() { return 16 / TcTraits<P>::kOpBytes; }          // values per core row
template <int P> IAAT_CE int tc_kgroups() { return kTcKC / tc_vpr<P>(); }             // core matrices along K
template <int P> IAAT_CE int tc_sbo() { return tc_kgroups<P>() * 128; }
template <int P> IAAT_CE int tc_operand_bytes() { return (kTcRows / 8) * tc_sbo<P>(); }
template <int P> IAAT_CE int tc_stage_bytes() { return 2 * TcTraits<P>::kTerms * tc_operand_bytes<P>(); }

// shared-memory map (bytes): the ring's barriers and stage records as in the
// CUDA-core kernel, then this kernel's own barriers, then the operand stages
constexpr int kTcExtra = kSmemSlots + kNumSlots * kSlotBytes;
constexpr int kTcBarOpFull = kTcExtra;          // [2], 4 converter-warp arrivals
constexpr int kTcBarOpEmpty = kTcExtra + 16;    // [2], tcgen05.commit
constexpr int kTcBarAccFull = kTcExtra + 32;    // [2], tcgen05.commit
constexpr int kTcBarAccEmpty = kTcExtra + 48;   // [2], 4 epilogue-warp arrivals
constexpr int kTcTmemSlot = kTcExtra + 64;      // tcgen05.alloc result
constexpr int kTcChunkInfo = kTcExtra + 80;     // [2] x 16 B
constexpr int kTcOperands = (kTcExtra + 128 + 1023) & ~1023;
static_assert(kTcExtra % 16 == 0, "barrier alignment");
template <int P> IAAT_CE int tc_ring_offset() { return kTcOperands + kTcStages * tc_stage_bytes<P>(); }
template <int P> IAAT_CE int tc_ring_bytes() { return (kSmemTotal - tc_ring_offset<P>()) & ~127; }
template <int P> IAAT_CE int tc_max_group_bytes() { return tc_ring_bytes<P>() / 2; }

struct ChunkInfo {      // converters -> MMA warp, one per operand stage
    int32_t nt;         // MMA N of the pack
    int32_t kc;         // K of this chunk (multiple of the MMA K step; 0: no product)
    int32_t flags;      // bit 0 first chunk of the pack, bit 1 last, bit 2 end of work
    int32_t pad;
};
constexpr int kChunkFirst = 1, kChunkLast = 2, kChunkEnd = 4;

// ------------------------------------------------------------ tcgen05 PTX

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

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

// Convert one 16-byte core-matrix row (tc_vpr<P>() FP32 values) and store it
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

// Convert one task operand's K-chunk [k0, k0 + kc) into canonical rows
// [row0, row0 + rows) of an operand stage.  raw(i, k) = src + i*si + k*sk.
// Values with k >= K are zero.  kcontig: the staged data is contiguous along
// k, so a lane takes one core-matrix row (lanes: rows x K-groups); otherwise
// it is contiguous along the rows and lanes run along the rows.
template <int P>
__device__ __forceinline__ void convert_chunk(char *t0, char *t1, const char *src, int si, int sk, int rows, int K,
                                              int row0, int k0, int kc, bool kcontig)
{
    constexpr int VPR = tc_vpr<P>();
    constexpr int KGM = tc_kgroups<P>();
    constexpr int SBO = tc_sbo<P>();
    const int lane = (int)lane_id();
    const int ng = kc / VPR;
    if (kcontig) {
        constexpr int RPS = 32 / KGM;            // rows per warp step
        const int g = lane % KGM, rr = lane / KGM;
        if (g < ng) {
            const int kb = k0 + g * VPR;
#pragma unroll 1
            for (int r = rr; r < rows; r += RPS) {
                const char *p = src + r * si + kb * sk;
                float x[8];
#pragma unroll
                for (int e = 0; e < VPR; ++e)
                    x[e] = (kb + e < K) ? *reinterpret_cast<const float *>(p + e * sk) : 0.0f;
                const int row = row0 + r;
                store_row<P>(t0, t1, (uint32_t)((row >> 3) * SBO + g * 128 + (row & 7) * 16), x);
            }
        }
    } else {
#pragma unroll 1
        for (int r = lane; r < rows; r += 32) {
            const int row = row0 + r;
            const char *p = src + r * si;
#pragma unroll 1
            for (int g = 0; g < ng; ++g) {
                const int kb = k0 + g * VPR;
                float x[8];
#pragma unroll
                for (int e = 0; e < VPR; ++e)
                    x[e] = (kb + e < K) ? *reinterpret_cast<const float *>(p + (kb + e) * sk) : 0.0f;
                store_row<P>(t0, t1, (uint32_t)((row >> 3) * SBO + g * 128 + (row & 7) * 16), x);
            }
        }
    }
}

struct TcSmem {
    SmemMap S;
    __device__ uint32_t op_full(int b) const { return S.sbase + kTcBarOpFull + 8 * b; }
    __device__ uint32_t op_empty(int b) const { return S.sbase + kTcBarOpEmpty + 8 * b; }
    __device__ uint32_t acc_full(int a) const { return S.sbase + kTcBarAccFull + 8 * a; }
    __device__ uint32_t acc_empty(int a) const { return S.sbase + kTcBarAccEmpty + 8 * a; }
    __device__ ChunkInfo *info(int b) const { return reinterpret_cast<ChunkInfo *>(S.base + kTcChunkInfo) + b; }
};

// Per-warp view of a stage's tasks: lane t holds task t's fields.
struct LaneTask {
    int M, N, K, R, Cc, pack, ta, tb, offA, offB, csA, csB;
};

__device__ __forceinline__ LaneTask load_lane_task(const TaskRec *recs, int nt)
{
    const int lane = (int)lane_id();
    LaneTask me{0, 0, 0, 0, 0, 1 << 20, 0, 0, 0, 0, 0, 0};
    if (lane < nt) {
        const TaskRec &r = recs[lane];
        me = LaneTask{r.M, r.N, r.K, r.nbm, r.nbn, r.variant, r.ta, r.tb, r.offA, r.offB, r.csA, r.csB};
    }
    return me;
}

__device__ __forceinline__ int warp_max(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Pack p's task mask, K (rounded to the MMA K step) and MMA N.
template <int P>
__device__ __forceinline__ void pack_shape(const LaneTask &me, int nt, int p, unsigned &mask, int &KT, int &NT)
{
    constexpr int KS = TcTraits<P>::kKStep;
    const int lane = (int)lane_id();
    const bool in = lane < nt && me.pack == p;
    mask = __ballot_sync(0xffffffffu, in);
    const int kmax = warp_max(in ? me.K : 0);
    const int cmax = warp_max(in ? me.Cc + me.N : 0);
    KT = (kmax + KS - 1) / KS * KS;
    NT = max(16, (cmax + 15) & ~15);
}

// Bounded wait on an mbarrier phase by every lane of a warp.  Each lane
// performs the acquire itself, so each lane's later reads of what was
// published with the barrier (stage records, chunk records, operand data)
// see the new values; lanes that only learned of the phase from another lane
// could read stale records, take different branches and deadlock the warp at
// its next collective.  The outcome is made warp-uniform.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity)
{
    // lane 0 does the (suspending) wait; then every lane confirms the
    // completed phase with its own try_wait, which is its acquire
    int ok = 1;
    if (lane_id() == 0)
        ok = mbar_wait(bar, parity, kWaitLimitNs) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    const bool mine = ok && mbar_wait(bar, parity, kWaitLimitNs);
    return __all_sync(0xffffffffu, mine);
}

template <int P>
__device__ void tc_converters(const KParams &KP, const TcSmem &T, int cw)
{
    const Params &Pm = KP.p;
    const int lane = (int)lane_id();
    constexpr int OPB = tc_operand_bytes<P>();
    constexpr int VPR = tc_vpr<P>();
    const int side = cw >> 2;                 // 0: A rows, 1: B rows
    const int row = 32 * (cw & 3) + lane;     // this thread's pack row
    int b = 0;
    uint32_t bpar = 0;     // parity of the operand stages' current round
    int uses = 0;          // chunks handed to the MMA warp so far
    bool alive = true;
    for (int i = 0; alive; ++i) {
        const int g = sched_group(i, blockIdx.x, gridDim.x);
        if (g >= Pm.ngroups)
            break;
        const int slot = i % kNumSlots;
        if (!warp_wait(T.S.full(slot), (uint32_t)((i / kNumSlots) & 1))) {
            if (lane == 0)
                set_error(Pm.err, kErrTimeoutFull);
            alive = false;
            break;
        }
        const TaskRec *recs = T.S.recs(slot);
        const int nt = T.S.header(slot)->ntasks;
        const LaneTask me = load_lane_task(recs, nt);
        const int npacks = warp_max(lane < nt ? me.pack + 1 : 0);
        for (int p = 0; p < npacks && alive; ++p) {
            unsigned mask;
            int KT, NT;
            pack_shape<P>(me, nt, p, mask, KT, NT);
            const int nch = KT > 0 ? (KT + kTcKC - 1) / kTcKC : 1;
            // the task owning this thread's row of the pack (A rows for warps
            // 0-3, B rows for warps 4-7), and where that row's data sits
            int my_task = -1;
            for (unsigned m = mask; m; m &= m - 1) {
                const int c = __ffs(m) - 1;
                const int lo = __shfl_sync(0xffffffffu, side == 0 ? me.R : me.Cc, c);
                const int len = __shfl_sync(0xffffffffu, side == 0 ? me.M : me.N, c);
                if (row >= lo && row < lo + len)
                    my_task = c;
            }
            const int src_lane = my_task >= 0 ? my_task : 0;
            const int t_lo = __shfl_sync(0xffffffffu, side == 0 ? me.R : me.Cc, src_lane);
            const int my_K = __shfl_sync(0xffffffffu, me.K, src_lane);
            const int t_tr = __shfl_sync(0xffffffffu, side == 0 ? me.ta : me.tb, src_lane);
            const int t_off = __shfl_sync(0xffffffffu, side == 0 ? me.offA : me.offB, src_lane);
            const int t_cs = __shfl_sync(0xffffffffu, side == 0 ? me.csA : me.csB, src_lane);
            // A row i: stored A[i + k*lda] (N) or A[k + i*lda] (T);
            // B row n (column n of op(B)): stored B[k + n*ldb] (N) or B[n + k*ldb] (T)
            const bool kcontig = side == 0 ? t_tr != 0 : t_tr == 0;
            const int my_si = kcontig ? t_cs : 4;
            const int my_sk = kcontig ? 4 : t_cs;
            const char *my_src = T.S.base + t_off + (row - t_lo) * my_si;
            const uint32_t row_off = (uint32_t)((row >> 3) * tc_sbo<P>() + (row & 7) * 16);
            // this row's operand bytes must have landed (each thread acquires
            // the barrier of its own task)
            {
                const bool ok = my_task < 0 || mbar_wait(T.S.task(slot, my_task),
                                                         (uint32_t)((i / kNumSlots) & 1), kWaitLimitNs);
                if (!__all_sync(0xffffffffu, ok)) {
                    if (lane == 0)
                        set_error(Pm.err, kErrTimeoutFull);
                    alive = false;
                    break;
                }
            }
            for (int c = 0; c < nch; ++c) {
                // the MMAs that read this stage one round ago must be done
                if (uses >= kTcStages && !warp_wait(T.op_empty(b), bpar ^ 1u)) {
                    if (lane == 0)
                        set_error(Pm.err, kErrTimeoutEmpty);
                    alive = false;
                    break;
                }
                const int k0 = c * kTcKC;
                const int kc = KT > 0 ? min(kTcKC, KT - k0) : 0;
                char *base = T.S.base + kTcOperands + b * tc_stage_bytes<P>();
                char *A0 = base, *A1 = base + OPB;
                char *B0 = base + TcTraits<P>::kTerms * OPB, *B1 = B0 + OPB;
                if (kc > 0 && my_task >= 0) {
                    // this thread's pack row: its K-groups of the chunk
                    char *t0 = side == 0 ? A0 : B0;
                    char *t1 = side == 0 ? A1 : B1;
                    const int ng = kc / VPR;
#pragma unroll 1
                    for (int gi = 0; gi < ng; ++gi) {
                        const int kb = k0 + gi * VPR;
                        const char *p = my_src + kb * my_sk;
                        float x[8];
                        if (kb + VPR <= my_K) {
#pragma unroll
                            for (int e = 0; e < VPR; ++e)
                                x[e] = *reinterpret_cast<const float *>(p + e * my_sk);
                        } else {
#pragma unroll
                            for (int e = 0; e < VPR; ++e)
                                x[e] = (kb + e < my_K) ? *reinterpret_cast<const float *>(p + e * my_sk) : 0.0f;
                        }
                        store_row<P>(t0, t1, row_off + (uint32_t)(gi * 128), x);
                    }
                }
                if (cw == 0 && lane == 0) {
                    ChunkInfo *ci = T.info(b);
                    ci->nt = NT;
                    ci->kc = kc;
                    ci->flags = (c == 0 ? kChunkFirst : 0) | (c == nch - 1 ? kChunkLast : 0);
                }
                fence_proxy_async();
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(T.op_full(b));
                ++uses;
                if (++b == kTcStages) {
                    b = 0;
                    bpar ^= 1u;
                }
            }
        }
        __syncwarp();
        if (lane == 0)
            mbar_arrive(T.S.empty(slot));
    }
    // end-of-work marker for the MMA warp
    if (alive && (uses < kTcStages || warp_wait(T.op_empty(b), bpar ^ 1u))) {
        if (cw == 0 && lane == 0) {
            ChunkInfo *ci = T.info(b);
            ci->nt = 16;
            ci->kc = 0;
            ci->flags = kChunkEnd;
        }
        __syncwarp();
        if (lane == 0)
            mbar_arrive(T.op_full(b));
    }
}

template <int P>
__device__ void tc_mma_warp(const KParams &KP, const TcSmem &T, uint32_t tmem)
{
    const Params &Pm = KP.p;
    const int lane = (int)lane_id();
    constexpr int KS = TcTraits<P>::kKStep;
    constexpr int OPB = tc_operand_bytes<P>();
    constexpr uint32_t SBO = (uint32_t)tc_sbo<P>();
    int b = 0, a = 0;
    uint32_t bpar = 0;
    uint32_t apar[2] = {0u, 0u};
    int acc_uses[2] = {0, 0};
    int commits[kTcStages] = {0, 0};   // tcgen05.commit arrivals sent to op_empty[b]
    for (;;) {
        if (!warp_wait(T.op_full(b), bpar)) {
            if (lane == 0)
                set_error(Pm.err, kErrTimeoutFull);
            break;
        }
        const ChunkInfo ci = *T.info(b);
        if (ci.flags & kChunkEnd)
            break;
        if ((ci.flags & kChunkFirst) && acc_uses[a] > 0) {
            // the epilogue must have drained this accumulator
            if (!warp_wait(T.acc_empty(a), apar[a] ^ 1u)) {
                if (lane == 0)
                    set_error(Pm.err, kErrTimeoutEmpty);
                break;
            }
        }
        if (lane == 0) {
            tc_fence_after();
            if (ci.kc > 0) {
                const uint32_t d = tmem + (uint32_t)(a * kTcMaxCols);
                const uint32_t idesc = tc_idesc<P>(ci.nt);
                const uint32_t base = smem_addr(T.S.base + kTcOperands + b * tc_stage_bytes<P>());
                const uint32_t a0 = base, a1 = base + OPB;
                const uint32_t b0 = base + TcTraits<P>::kTerms * OPB, b1 = b0 + OPB;
                const bool first = (ci.flags & kChunkFirst) != 0;
                for (int ks = 0; ks < ci.kc / KS; ++ks) {
                    const uint32_t o = (uint32_t)ks * 256u;   // two core matrices along K
                    const uint32_t accum = (first && ks == 0) ? 0u : 1u;
                    if constexpr (P == kTc3xBF16) {
                        tc_mma<P>(d, smem_desc(a1 + o, 128, SBO), smem_desc(b0 + o, 128, SBO), idesc, accum);
                        tc_mma<P>(d, smem_desc(a0 + o, 128, SBO), smem_desc(b1 + o, 128, SBO), idesc, 1);
                        tc_mma<P>(d, smem_desc(a0 + o, 128, SBO), smem_desc(b0 + o, 128, SBO), idesc, 1);
                    } else {
                        tc_mma<P>(d, smem_desc(a0 + o, 128, SBO), smem_desc(b0 + o, 128, SBO), idesc, accum);
                    }
                }
            }
            tc_commit(T.op_empty(b));
            if (ci.flags & kChunkLast)
                tc_commit(T.acc_full(a));
        }
        __syncwarp();
        ++commits[b];
        if (ci.flags & kChunkLast) {
            ++acc_uses[a];
            apar[a] ^= 1u;
            a ^= 1;
        }
        if (++b == kTcStages) {
            b = 0;
            bpar ^= 1u;
        }
    }
    // No asynchronous arrival may reach this CTA's shared memory after it
    // exits: wait (bounded) for the last commit to each operand-stage barrier,
    // which no other role waits for.  (The accumulator commits are all
    // waited for by the epilogue.)
    if (lane == 0) {
        for (int bb = 0; bb < kTcStages; ++bb)
            if (commits[bb] > 0 &&
                !mbar_wait(T.op_empty(bb), (uint32_t)((commits[bb] - 1) & 1), kWaitLimitNs))
                set_error(Pm.err, kErrTimeoutFull);
    }
    __syncwarp();
}

template <int P>
__device__ void tc_epilogue_warps(const KParams &KP, const TcSmem &T, int ew, uint32_t tmem)
{
    const Params &Pm = KP.p;
    const int lane = (int)lane_id();
    const int q = ew & 3;                           // TMEM lane quarter (warp index mod 4)
    const int half = ew >> 2;                       // which alternate 16-column chunks
    const int row = 32 * q + lane;                  // accumulator row (TMEM lane) of this thread
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    int a = 0;
    uint32_t apar[2] = {0u, 0u};
    for (int i = 0;; ++i) {
        const int g = sched_group(i, blockIdx.x, gridDim.x);
        if (g >= Pm.ngroups)
            break;
        const int slot = i % kNumSlots;
        if (!warp_wait(T.S.full(slot), (uint32_t)((i / kNumSlots) & 1))) {
            if (lane == 0)
                set_error(Pm.err, kErrTimeoutFull);
            return;
        }
        const TaskRec *recs = T.S.recs(slot);
        const int nt = T.S.header(slot)->ntasks;
        const LaneTask me = load_lane_task(recs, nt);
        const int npacks = warp_max(lane < nt ? me.pack + 1 : 0);
        for (int p = 0; p < npacks; ++p) {
            unsigned mask;
            int KT, NT;
            pack_shape<P>(me, nt, p, mask, KT, NT);
            if (!warp_wait(T.acc_full(a), apar[a])) {
                if (lane == 0)
                    set_error(Pm.err, kErrTimeoutFull);
                return;
            }
            apar[a] ^= 1u;
            tc_fence_after();
            const uint32_t dt = tmem + (uint32_t)(a * kTcMaxCols) + lane_base;
            // tasks whose rows meet this warp's 32 rows
            const unsigned rows_mask = __ballot_sync(
                0xffffffffu, ((mask >> lane) & 1) && me.R < 32 * q + 32 && me.R + me.M > 32 * q);
            for (unsigned m = rows_mask; m; m &= m - 1) {
                const int t = __ffs(m) - 1;
                const TaskRec &r = recs[t];
                const int R = r.nbm, M = r.M, Cc = r.nbn, N = r.N;
                const bool mine = row >= R && row < R + M;
                if (mine && (r.flags & kFlagReadC) &&
                    !mbar_wait(T.S.task(slot, t), (uint32_t)((i / kNumSlots) & 1), kWaitLimitNs))
                    set_error(Pm.err, kErrTimeoutFull);
                const int i_ = mine ? row - R : 0;
                const float alpha = (float)r.alpha, beta = (float)r.beta;
                const bool readc = (r.flags & kFlagReadC) != 0;
                float *C = reinterpret_cast<float *>(r.C) + i_;
                const int64_t ldc = r.ldc;
                const char *c0 = T.S.base + r.offC + i_ * 4;
                const int csC = r.csC;
                for (int j0 = (Cc & ~15) + 16 * half; j0 < Cc + N; j0 += 32) {
                    float v[16];
                    if (KT > 0) {
                        tmem_ld16(dt + (uint32_t)j0, v);
                    } else {
#pragma unroll
                        for (int u = 0; u < 16; ++u)
                            v[u] = 0.f;
                    }
                    if (mine) {
                        // columns j0.. of the tile are columns j0-Cc.. of C
                        const int jlo = max(j0, Cc) - Cc, jhi = min(j0 + 16, Cc + N) - Cc;
                        float *cp = C + jlo * ldc;
                        const char *c0p = c0 + jlo * csC;
#pragma unroll
                        for (int u = 0; u < 16; ++u) {
                            const int j = j0 + u - Cc;
                            if (j >= jlo && j < jhi) {
                                float c = alpha * v[u];
                                if (readc)
                                    c = fmaf(beta, *reinterpret_cast<const float *>(c0p), c);
                                *cp = c;
                                cp += ldc;
                                c0p += csC;
                            }
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0)
                mbar_arrive(T.acc_empty(a));
            a ^= 1;
        }
        __syncwarp();
        if (lane == 0)
            mbar_arrive(T.S.empty(slot));
    }
}

template <int P>
__global__ void __launch_bounds__(kTcThreads, 1) grouped_tc_kernel(const __grid_constant__ KParams KP)
{
    extern __shared__ __align__(1024) char smem_tc[];
    TcSmem T;
    T.S.base = smem_tc;
    T.S.sbase = smem_addr(smem_tc);
    T.S.ring_off = (uint32_t)tc_ring_offset<P>();
    T.S.ring_bytes = (uint32_t)tc_ring_bytes<P>();
    const int warp = threadIdx.x / 32;
    if (threadIdx.x < kNumSlots * kMaxGroupTasks)
        mbar_init(T.S.task(threadIdx.x / kMaxGroupTasks, threadIdx.x % kMaxGroupTasks), 1);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kNumSlots; ++s) {
            mbar_init(T.S.full(s), 1);
            mbar_init(T.S.empty(s), kTcConvWarps + kTcEpiWarps);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(T.op_full(b), kTcConvWarps);
            mbar_init(T.op_empty(b), 1);
            mbar_init(T.acc_full(b), 1);
            mbar_init(T.acc_empty(b), kTcEpiWarps);
        }
        fence_barrier_init();
    }
    if (warp == 0)
        tmem_alloc(T.S.sbase + kTcTmemSlot, kTcTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t *>(smem_tc + kTcTmemSlot);
    if (warp < kTcConvWarps)
        tc_converters<P>(KP, T, warp);
    else if (warp < kTcConvWarps + kTcEpiWarps)
        tc_epilogue_warps<P>(KP, T, warp - kTcConvWarps, tmem);
    else if (warp == kTcWarpProducer)
        producer_loop<4>(KP, T.S);
    else
        tc_mma_warp<P>(KP, T, tmem);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        tmem_dealloc(tmem, kTcTmemCols);
}

}  // namespace iaat
