// Persistent grouped small-GEMM kernel on the tcgen05 tensor cores, FP32 in
// and out: 3xBF16 split products, TF32, or FP16 inputs, FP32 accumulation in
// tensor memory.
//
// Packs: the planner places the tasks of a stage into packs, one 128-row MMA
// tile each.  A task owns whole 32-row quarters of the tile (its rows start
// at R_t, a multiple of 32) and a run of 16-column blocks (its columns start
// at C_t, a multiple of 16), so several small instances share one
// tensor-core pass and only the diagonal blocks of the product are kept.
// The quarters matter because tensor-memory lanes 32q..32q+31 can only be
// read by the warps of SM sub-partition q: one task per quarter spreads each
// pack's epilogue over all four sub-partitions.
//
// Warp roles (20 warps; 16 and 17 only pad, see kTcWarpProducer):
//   0-7  converters: per 32-wide K-chunk of a pack, every thread converts one
//        row of a 128-row operand tile -- warps 0-3 the rows of op(A) (one
//        quarter each), warps 4-7 those of op(B)^T (in reverse order of
//        quarters) -- from the staged FP32
//        data into the canonical K-major (no swizzle) layout of one of
//        kTcStages operand stages: X = Xh + Xl (BF16) for 3xBF16,
//        X = Xh + Xm + Xl for 6xBF16, RN-rounded TF32, or FP16, with zeros
//        past the row's K;
//   8-15 epilogue: warp 8+e reads quarter e&3 of the accumulator of every
//        pack whose sequence number is e>>2 modulo kTcEpiPhases, batching two
//        16-column tensor-memory loads per wait, and writes alpha*acc +
//        beta*C0 to exactly the task's elements;
//   18   producer: streams stages into the shared-memory ring (shared with
//        the CUDA-core kernel) and copies each pack's summary (PackInfo);
//   19   MMA: one lane issues each chunk's MMAs into one of kTcAccs
//        accumulators and commits them to mbarriers that free the operand
//        stage and, after a pack's last chunk, hand the accumulator over.
// Conversion of the next chunks, the MMAs of this one and the epilogue of up
// to kTcAccs - 1 earlier packs run at the same time.  Every wait is bounded;
// a time-out sets the error word, every role leaves its loop, and the CTA
// frees its tensor memory before returning.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "grouped.cuh"

namespace iaat {

constexpr int kTc3xBF16 = 1, kTcTF32 = 2, kTcFP16 = 3, kTc6xBF16 = 4;
constexpr int kTcRows = 128;           // MMA M (tensor-memory lanes)
constexpr int kTcMaxCols = 128;        // columns of one pack (MMA N <= 128)
constexpr int kTcKC = 32;              // K per operand stage
constexpr int kTcStages = 2;           // operand stages
constexpr int kTcAccs = 4;             // accumulators of kTcMaxCols columns
constexpr int kTcConvWarps = 8;       // 4 for the rows of op(A), 4 for op(B)^T (16: two per row)
constexpr int kTcEpiWarps = 8;        // a multiple of 4: one per lane quarter and pack phase
constexpr int kTcEpiPhases = kTcEpiWarps / 4;   // packs in flight in the epilogue per quarter
// The producer and the MMA thread run on SM sub-partitions 2 and 3 (warp
// index mod 4), whose converter and epilogue warps -- lane quarters 2 and 3
// of a pack, the ones a pack fills last -- have the least work; the two warps
// before them only pad the block to get there.
constexpr int kTcWarpProducer = kTcConvWarps + kTcEpiWarps + 2, kTcWarpMma = kTcWarpProducer + 1;
static_assert(kTcWarpProducer % 4 == 2 && kTcWarpMma % 4 == 3, "role placement");
constexpr int kTcThreads = 32 * (kTcWarpMma + 1);
constexpr int kTcTmemCols = kTcAccs * kTcMaxCols;

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
template <> struct TcTraits<kTc6xBF16> {
    static constexpr int kOpBytes = 2, kTerms = 3, kKStep = 16;
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
// CUDA-core kernel, then this kernel's own barriers and pack summaries, then
// the operand stages
constexpr int kTcExtra = kSmemSlots + kNumSlots * kSlotBytes;
constexpr int kTcBarOpFull = kTcExtra;          // [kTcStages], kTcConvWarps arrivals
constexpr int kTcBarOpEmpty = kTcExtra + 32;    // [kTcStages], tcgen05.commit
constexpr int kTcBarAccFull = kTcExtra + 64;    // [kTcAccs], tcgen05.commit
constexpr int kTcBarAccEmpty = kTcExtra + 96;   // [kTcAccs], 4 epilogue-warp arrivals (one per quarter)
constexpr int kTcBarCFull = kTcExtra + 128;     // [kNumSlots], the stage's C copies
constexpr int kTcTmemSlot = kTcExtra + 192;     // tcgen05.alloc result
constexpr int kTcChunkInfo = kTcExtra + 256;    // [kTcStages] x 16 B
constexpr int kTcPackInfo = kTcExtra + 320;     // PackInfo[kNumSlots][kMaxGroupTasks]
constexpr int kTcOperands = (kTcPackInfo + kNumSlots * kMaxGroupTasks * (int)sizeof(PackInfo) + 1023) & ~1023;
static_assert(kTcExtra % 16 == 0, "barrier alignment");
static_assert(kTcStages <= 4 && kTcAccs <= 4 && kNumSlots <= 8, "barrier space");
static_assert((kTcAccs & (kTcAccs - 1)) == 0 && kTcEpiWarps % 4 == 0 && (kTcConvWarps == 8 || kTcConvWarps == 16),
              "accumulator rotation, lane quarters, converter split");
template <int P> IAAT_CE int tc_ring_offset() { return kTcOperands + kTcStages * tc_stage_bytes<P>(); }
template <int P> IAAT_CE int tc_ring_bytes() { return (kSmemTotal - tc_ring_offset<P>()) & ~127; }
// A stage may take at most a third of the ring, so three are in flight.
template <int P> IAAT_CE int tc_max_group_bytes() { return tc_ring_bytes<P>() / 3; }

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
    constexpr uint32_t fmt = (P == kTc3xBF16 || P == kTc6xBF16) ? 1u : (P == kTcTF32 ? 2u : 0u);
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

// 16 consecutive accumulator columns of this warp's 32 tensor-memory lanes
// into r[OFF..OFF+15] (thread t gets lane 32q + t); completes at tmem_wait_ld.
template <int OFF>
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[OFF + 0]), "=r"(r[OFF + 1]), "=r"(r[OFF + 2]), "=r"(r[OFF + 3]), "=r"(r[OFF + 4]),
          "=r"(r[OFF + 5]), "=r"(r[OFF + 6]), "=r"(r[OFF + 7]), "=r"(r[OFF + 8]), "=r"(r[OFF + 9]),
          "=r"(r[OFF + 10]), "=r"(r[OFF + 11]), "=r"(r[OFF + 12]), "=r"(r[OFF + 13]), "=r"(r[OFF + 14]),
          "=r"(r[OFF + 15])
        : "r"(taddr));
}

// Wait for this thread's outstanding tensor-memory loads.  The destination
// registers pass through the statement so that no use of them can be
// scheduled ahead of the wait.
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&r)[32])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                   "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]),
                   "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]),
                   "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]),
                   "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

// ------------------------------------------------------- conversions
// Round an FP32 value to TF32 (10 explicit mantissa bits), nearest-even, with
// the conversion instruction (one per value; it gave the same bits as adding
// 0xfff plus the kept LSB and clearing the low 13 bits on 2^30 finite values,
// ties included, and took TF32 from 0.84 to 0.75 ms on the uneven batch);
// the tensor core then reads the top 19 bits unchanged.
__device__ __forceinline__ uint32_t tf32_rn(float x)
{
    uint32_t r;
    asm("cvt.rn.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
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
// (hi; lo for 3xBF16; hi, mid, lo for 6xBF16) at byte offset `off` of the
// term buffers.
template <int P>
__device__ __forceinline__ void store_row(char *t0, char *t1, char *t2, uint32_t off, const float *x)
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
    } else if constexpr (P == kTc6xBF16) {
        // each term is the BF16 rounding of what the terms before it leave;
        // the differences are exact in FP32
        uint32_t h[4], m[4], l[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            h[q] = pack_bf16(x[2 * q], x[2 * q + 1]);
            const float r0 = x[2 * q] - __uint_as_float(h[q] << 16);
            const float r1 = x[2 * q + 1] - __uint_as_float(h[q] & 0xffff0000u);
            m[q] = pack_bf16(r0, r1);
            const float s0 = r0 - __uint_as_float(m[q] << 16);
            const float s1 = r1 - __uint_as_float(m[q] & 0xffff0000u);
            l[q] = pack_bf16(s0, s1);
        }
        *reinterpret_cast<uint4 *>(t0 + off) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4 *>(t1 + off) = make_uint4(m[0], m[1], m[2], m[3]);
        *reinterpret_cast<uint4 *>(t2 + off) = make_uint4(l[0], l[1], l[2], l[3]);
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

struct TcSmem {
    SmemMap S;
    __device__ uint32_t op_full(int b) const { return S.sbase + kTcBarOpFull + 8 * b; }
    __device__ uint32_t op_empty(int b) const { return S.sbase + kTcBarOpEmpty + 8 * b; }
    __device__ uint32_t acc_full(int a) const { return S.sbase + kTcBarAccFull + 8 * a; }
    __device__ uint32_t acc_empty(int a) const { return S.sbase + kTcBarAccEmpty + 8 * a; }
    __device__ ChunkInfo *info(int b) const { return reinterpret_cast<ChunkInfo *>(S.base + kTcChunkInfo) + b; }
};

// Bounded wait on an mbarrier phase by every lane of a warp.  Each lane
// performs the acquire itself, so each lane's later reads of what was
// published with the barrier (stage records, pack summaries, staged data)
// see the new values.  The outcome is made warp-uniform.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity)
{
    const bool ok = mbar_wait(bar, parity, kWaitLimitNs);
    return __all_sync(0xffffffffu, ok);
}

template <int P>
__device__ void tc_converters(const KParams &KP, const TcSmem &T, int cw)
{
    const Params &Pm = KP.p;
    const int lane = (int)lane_id();
    constexpr int OPB = tc_operand_bytes<P>();
    constexpr int VPR = tc_vpr<P>();
    constexpr int KS = TcTraits<P>::kKStep;
    const int side = (cw >> 2) & 1;           // 0: rows of op(A), 1: rows of op(B)^T
    const int gfirst = cw >> 3;               // with 16 converter warps, two share each row:
    constexpr int GSTEP = kTcConvWarps / 8;   // this warp takes K-groups gfirst, gfirst + GSTEP, ...
    // this thread's row of the operand tile: op(A) rows 32q.. run on sub-
    // partition q, op(B)^T rows 32(3-q).. too, so the busy low rows of both
    // operands (packs fill from row 0) share the sub-partitions evenly
    const int row = 32 * (side == 0 ? (cw & 3) : 3 - (cw & 3)) + lane;
    const uint32_t row_off = (uint32_t)((row >> 3) * tc_sbo<P>() + (row & 7) * 16);
    int b = 0;
    uint32_t bpar = 0;     // parity of the operand stages' current round
    int uses = 0;          // chunks handed to the MMA warp so far
    bool alive = true;
    for (int i = 0; alive; ++i) {
        const int g = sched_group(i, blockIdx.x, gridDim.x);
        if (g >= Pm.ngroups)
            break;
        const int slot = i % kNumSlots;
        const uint32_t par = (uint32_t)((i / kNumSlots) & 1);
        if (!warp_wait(T.S.full(slot), par)) {
            if (lane == 0)
                set_error(Pm.err, kErrTimeoutFull);
            alive = false;
            break;
        }
        const TaskRec *recs = T.S.recs(slot);
        const PackInfo *pis = T.S.pinfo(slot);
        const int npk = T.S.header(slot)->npacks;
        for (int p = 0; p < npk && alive; ++p) {
            const PackInfo &pi = pis[p];
            const int t = side == 0 ? pi.qtask[cw & 3] : pi.btask[row >> 4];
            const int KT = ((int)pi.kmax + KS - 1) / KS * KS;
            const int NT = pi.nt;
            const int nch = KT > 0 ? (KT + kTcKC - 1) / kTcKC : 1;
            // this thread's row: row r of task t's op(A), or column r of its op(B)
            bool valid = false;
            int myK = 0, sk = 4;
            const char *src = T.S.base;
            if (t >= 0) {
                const TaskRec &rc = recs[t];
                const int r = row - (side == 0 ? (int)rc.nbm : (int)rc.nbn);
                valid = r < (side == 0 ? (int)rc.M : (int)rc.N);
                // A row i: stored A[i + k*lda] (N) or A[k + i*lda] (T);
                // B row n (column n of op(B)): stored B[k + n*ldb] (N) or B[n + k*ldb] (T)
                const int tr = side == 0 ? rc.ta : rc.tb;
                const bool kcontig = side == 0 ? tr != 0 : tr == 0;
                const int cs = side == 0 ? rc.csA : rc.csB;
                sk = kcontig ? 4 : cs;
                src += (side == 0 ? rc.offA : rc.offB) + r * (kcontig ? cs : 4);
                myK = rc.K;
            }
            // the operand bytes of this thread's task must have landed
            {
                const bool ok = !valid || mbar_wait(T.S.task(slot, t), par, kWaitLimitNs);
                if (!__all_sync(0xffffffffu, ok)) {
                    if (lane == 0)
                        set_error(Pm.err, kErrTimeoutFull);
                    alive = false;
                    break;
                }
            }
            for (int c = 0; c < nch; ++c) {
                if (uses >= kTcStages) {
                    // the MMAs that read this stage one round ago are complete
                    int ok = 1;
                    if (lane == 0)
                        ok = mbar_wait(T.op_empty(b), bpar ^ 1u, kWaitLimitNs) ? 1 : 0;
                    ok = __shfl_sync(0xffffffffu, ok, 0);
                    __syncwarp();
                    if (!ok) {
                        if (lane == 0)
                            set_error(Pm.err, kErrTimeoutEmpty);
                        alive = false;
                        break;
                    }
                }
                const int k0 = c * kTcKC;
                const int kc = KT > 0 ? min(kTcKC, KT - k0) : 0;
                char *t0 = T.S.base + kTcOperands + b * tc_stage_bytes<P>() + side * TcTraits<P>::kTerms * OPB;
                char *t1 = t0 + OPB;
                char *t2 = t1 + OPB;   // 6xBF16 only
                if (valid && kc > 0) {
                    const int ng = kc / VPR;
#pragma unroll 1
                    for (int gi = gfirst; gi < ng; gi += GSTEP) {
                        const int kb = k0 + gi * VPR;
                        const char *q = src + kb * sk;
                        float x[8];
                        if (kb + VPR <= myK) {
#pragma unroll
                            for (int e = 0; e < VPR; ++e)
                                x[e] = *reinterpret_cast<const float *>(q + e * sk);
                        } else {
#pragma unroll
                            for (int e = 0; e < VPR; ++e)
                                x[e] = (kb + e < myK) ? *reinterpret_cast<const float *>(q + e * sk) : 0.0f;
                        }
                        store_row<P>(t0, t1, t2, row_off + (uint32_t)(gi * 128), x);
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
    if (alive) {
        int ok = 1;
        if (uses >= kTcStages && lane == 0)
            ok = mbar_wait(T.op_empty(b), bpar ^ 1u, kWaitLimitNs) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        __syncwarp();
        if (ok) {
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
}

// The MMA role: run by one thread.
template <int P>
__device__ void tc_mma_thread(const KParams &KP, const TcSmem &T, uint32_t tmem)
{
    const Params &Pm = KP.p;
    constexpr int KS = TcTraits<P>::kKStep;
    constexpr int OPB = tc_operand_bytes<P>();
    constexpr uint32_t SBO = (uint32_t)tc_sbo<P>();
    int b = 0;
    uint32_t bpar = 0;
    uint32_t pk = 0;     // packs completed
    int total = 0;       // chunks consumed (each sends one commit to its stage's op_empty)
    const uint32_t ops = smem_addr(T.S.base + kTcOperands);
    for (;;) {
        if (!mbar_wait(T.op_full(b), bpar, kWaitLimitNs)) {
            set_error(Pm.err, kErrTimeoutFull);
            break;
        }
        const ChunkInfo ci = *T.info(b);
        if (ci.flags & kChunkEnd)
            break;
        const int a = (int)(pk & (kTcAccs - 1));
        // before a pack's first chunk: the epilogue has drained this accumulator's previous use
        if ((ci.flags & kChunkFirst) && pk >= (uint32_t)kTcAccs &&
            !mbar_wait(T.acc_empty(a), ((pk / kTcAccs) - 1u) & 1u, kWaitLimitNs)) {
            set_error(Pm.err, kErrTimeoutEmpty);
            break;
        }
        tc_fence_after();
        if (ci.kc > 0) {
            const uint32_t d = tmem + (uint32_t)(a * kTcMaxCols);
            const uint32_t idesc = tc_idesc<P>(ci.nt);
            const uint32_t base = ops + (uint32_t)(b * tc_stage_bytes<P>());
            // descriptors of the chunk's first K step; each step moves 256
            // bytes (two core matrices) along K, 16 in the address field
            uint64_t da0 = smem_desc(base, 128, SBO), db0 = smem_desc(base + TcTraits<P>::kTerms * OPB, 128, SBO);
            uint64_t da1 = da0 + (OPB >> 4), db1 = db0 + (OPB >> 4);
            uint64_t da2 = da1 + (OPB >> 4), db2 = db1 + (OPB >> 4);
            uint32_t accum = (ci.flags & kChunkFirst) ? 0u : 1u;
            for (int ks = 0; ks < ci.kc / KS; ++ks) {
                if constexpr (P == kTc6xBF16) {
                    // smallest products first: mm, lh, hl, mh, hm, hh
                    tc_mma<P>(d, da1, db1, idesc, accum);
                    tc_mma<P>(d, da2, db0, idesc, 1u);
                    tc_mma<P>(d, da0, db2, idesc, 1u);
                    tc_mma<P>(d, da1, db0, idesc, 1u);
                    tc_mma<P>(d, da0, db1, idesc, 1u);
                    tc_mma<P>(d, da0, db0, idesc, 1u);
                    da1 += 16;
                    db1 += 16;
                    da2 += 16;
                    db2 += 16;
                } else if constexpr (P == kTc3xBF16) {
                    tc_mma<P>(d, da1, db0, idesc, accum);
                    tc_mma<P>(d, da0, db1, idesc, 1u);
                    tc_mma<P>(d, da0, db0, idesc, 1u);
                    da1 += 16;
                    db1 += 16;
                } else {
                    tc_mma<P>(d, da0, db0, idesc, accum);
                }
                da0 += 16;
                db0 += 16;
                accum = 1u;
            }
        }
        tc_commit(T.op_empty(b));
        if (ci.flags & kChunkLast) {
            tc_commit(T.acc_full(a));
            ++pk;
        }
        ++total;
        if (++b == kTcStages) {
            b = 0;
            bpar ^= 1u;
        }
    }
    // No asynchronous arrival may reach this CTA's shared memory after it
    // exits: wait (bounded) for the last commit to each operand stage, which
    // no other role is left to wait for.  (The epilogue waits for every
    // accumulator commit.)
    for (int bb = 0; bb < kTcStages; ++bb) {
        const int n = total / kTcStages + (bb < total % kTcStages ? 1 : 0);
        if (n > 0 && !mbar_wait(T.op_empty(bb), (uint32_t)((n - 1) & 1), kWaitLimitNs))
            set_error(Pm.err, kErrTimeoutFull);
    }
}

template <int P>
__device__ void tc_epilogue_warps(const KParams &KP, const TcSmem &T, int ew, uint32_t tmem)
{
    const Params &Pm = KP.p;
    const int lane = (int)lane_id();
    const int q = ew & 3;                           // tensor-memory lane quarter (= warp index mod 4)
    const int phase = ew >> 2;                      // packs pk with pk % kTcEpiPhases == phase
    const int row = 32 * q + lane;                  // accumulator row (tensor-memory lane) of this thread
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    uint32_t pk = 0;                                // pack sequence number
    for (int i = 0;; ++i) {
        const int g = sched_group(i, blockIdx.x, gridDim.x);
        if (g >= Pm.ngroups)
            break;
        const int slot = i % kNumSlots;
        const uint32_t par = (uint32_t)((i / kNumSlots) & 1);
        if (!warp_wait(T.S.full(slot), par) || !warp_wait(T.S.cfull(slot), par)) {
            if (lane == 0)
                set_error(Pm.err, kErrTimeoutFull);
            return;
        }
        const TaskRec *recs = T.S.recs(slot);
        const PackInfo *pis = T.S.pinfo(slot);
        const int npk = T.S.header(slot)->npacks;
        for (int p = 0; p < npk; ++p, ++pk) {
            if ((int)(pk % kTcEpiPhases) != phase)
                continue;
            const int a = (int)(pk & (kTcAccs - 1));
            if (!warp_wait(T.acc_full(a), (pk / kTcAccs) & 1u)) {
                if (lane == 0)
                    set_error(Pm.err, kErrTimeoutFull);
                return;
            }
            tc_fence_after();
            const PackInfo &pi = pis[p];
            const int t = pi.qtask[q];
            const bool product = pi.kmax > 0;
            if (t >= 0) {
                const TaskRec &rc = recs[t];
                const int r = row - (int)rc.nbm;           // this thread's row of C
                const bool valid = r < (int)rc.M;
                const int N = rc.N;
                const float alpha = rc.alpha.f, beta = rc.beta.f;
                const bool readc = (rc.flags & kFlagReadC) != 0;
                float *Cp = reinterpret_cast<float *>(rc.C) + r;
                const int64_t ldc = rc.ldc;
                const char *c0p = T.S.base + rc.offC + r * 4;
                const int csC = rc.csC;
                const uint32_t dt = tmem + (uint32_t)(a * kTcMaxCols + (int)rc.nbn) + lane_base;
                const int nchunk = (N + 15) >> 4;
                for (int cb = 0; cb < nchunk; cb += 2) {
                    uint32_t v[32];
                    if (product) {
                        tmem_ld16<0>(dt + (uint32_t)(16 * cb), v);
                        if (cb + 1 < nchunk)
                            tmem_ld16<16>(dt + (uint32_t)(16 * cb + 16), v);
                        tmem_wait_ld(v);
                    } else {
#pragma unroll
                        for (int e = 0; e < 32; ++e)
                            v[e] = 0u;
                    }
                    // all of a chunk's C0 loads first, then its stores:
                    // predicated, so nothing waits on a branch
#pragma unroll
                    for (int cc = 0; cc < 2; ++cc) {
                        const int j0 = 16 * (cb + cc);
                        if (j0 < N) {
                            const int jn = min(16, N - j0);
                            const char *c0c = c0p + j0 * csC;
                            float c0v[16];
#pragma unroll
                            for (int u = 0; u < 16; ++u)
                                c0v[u] = (readc && valid && u < jn) ? *reinterpret_cast<const float *>(c0c + u * csC)
                                                                      : 0.0f;
                            float *cpc = Cp + j0 * ldc;
#pragma unroll
                            for (int u = 0; u < 16; ++u)
                                if (valid && u < jn)
                                    cpc[u * ldc] = fmaf(beta, c0v[u], alpha * __uint_as_float(v[16 * cc + u]));
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0)
                mbar_arrive(T.acc_empty(a));
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
    T.S.pinfo_off = (uint32_t)kTcPackInfo;
    T.S.cbar_off = (uint32_t)kTcBarCFull;
    const int warp = threadIdx.x / 32;
    if (threadIdx.x < kNumSlots * kMaxGroupTasks)
        mbar_init(T.S.task(threadIdx.x / kMaxGroupTasks, threadIdx.x % kMaxGroupTasks), 1);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kNumSlots; ++s) {
            mbar_init(T.S.full(s), 1);
            mbar_init(T.S.empty(s), kTcConvWarps + kTcEpiWarps);
            mbar_init(T.S.cfull(s), 1);
        }
        for (int b = 0; b < kTcStages; ++b) {
            mbar_init(T.op_full(b), kTcConvWarps);
            mbar_init(T.op_empty(b), 1);
        }
        for (int a = 0; a < kTcAccs; ++a) {
            mbar_init(T.acc_full(a), 1);
            mbar_init(T.acc_empty(a), 4);
        }
        fence_barrier_init();
    }
    if (warp == 0)
        tmem_alloc(T.S.sbase + kTcTmemSlot, kTcTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t *>(smem_tc + kTcTmemSlot);
    if (warp < kTcConvWarps) {
        tc_converters<P>(KP, T, warp);
    } else if (warp < kTcConvWarps + kTcEpiWarps) {
        tc_epilogue_warps<P>(KP, T, warp - kTcConvWarps, tmem);
    } else if (warp < kTcWarpProducer) {
        // padding warps: nothing to do until the final barrier
    } else if (warp == kTcWarpProducer) {
        producer_loop<4, true>(KP, T.S);
    } else {
        if (lane_id() == 0)
            tc_mma_thread<P>(KP, T, tmem);
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        tmem_dealloc(tmem, kTcTmemCols);
}

}  // namespace iaat
