// Shared host / device definitions of the warp-tile tensor-core kernel
// (tw.cuh): its task record, launch parameters and ring-item sizes.
#pragma once
#include "common.cuh"

namespace iaat {

// ----------------------------------------- warp-tile tensor-core kernel
// (tw.cuh) Every warp runs its own list of warp tasks -- blocks of at most
// 32 x 32 of C with a K range -- through a private shared-memory ring and its
// own 32 accumulator columns of tensor memory.  One warp task, 64 bytes; the
// first ring item of a task starts with a copy of it.
struct alignas(16) TwTask {
    const char *A;        // op(A) element (r0, 0) of the block in the stored A
    const char *B;        // op(B) element (0, c0) of the block in the stored B
    char *C;              // C element (r0, c0)
    int32_t lda, ldb, ldc;
    int32_t K;            // K (0: no product)
    int16_t M, N;         // block rows, block columns (1..32)
    uint8_t ta, tb, flags;
    uint8_t kseg16;       // K values per ring item / 16 (the last item takes the rest)
    float alpha, beta;
    int32_t pad[2];
};
static_assert(sizeof(TwTask) == 64, "TwTask layout");

struct TwParams {
    const TwTask *tasks;   // warp w's tasks: tasks[wbeg[w] .. wbeg[w+1])
    const int32_t *wbeg;
    int32_t *err;
    int32_t nwarps;        // gridDim.x * kTwWarps
    int32_t pad;
};

constexpr int kTwWarps = 12;      // warps per CTA (one CTA per SM)
constexpr int kTwKC = 16;         // K values per converted operand chunk (one MMA K step of BF16 / FP16)
constexpr int kTwMaxOut = 8;      // ring items in flight per warp
constexpr int kTwBlockM = 32;     // largest block height: one lane quarter of tensor memory
constexpr int kTwBlockN = 32;     // largest block width: the warp's accumulator columns (16 or 32)
constexpr int kTwThreads = 32 * kTwWarps;

// Ring items.  An operand block is R runs of len elements each (the
// contiguous stretches of its stored columns, ld elements apart).  It is
// staged either run by run -- each run as the 16-byte granules that cover it,
// in a slot of tw_run_slot(4*len) bytes, its first element at the slot start
// plus the address's offset within its granule (0, 4, 8 or 12) -- or, when
// the ld padding between runs is small, as one span from its first element
// to its last (the padding included): one run of 4*((R-1)*ld + len) bytes.
IAAT_HD uint32_t tw_run_slot(int64_t xbytes) { return (uint32_t)((xbytes + 27) >> 4) << 4; }
IAAT_HD uint32_t tw_op_bytes(int runs, int len, int64_t ld, bool span)
{
    if (runs <= 0 || len <= 0)
        return 0u;
    return span ? tw_run_slot(4 * ((int64_t)(runs - 1) * ld + len)) : (uint32_t)runs * tw_run_slot(4 * (int64_t)len);
}
// The block of op(A) (mh rows x a K range of kl values): runs along k when A
// is not transposed (one per k, mh long), along the rows when it is; of
// op(B) (kl x nw): one per column (kl long) when B is not transposed, one per
// k (nw long) when it is; of C: one per column (mh long).
IAAT_HD uint32_t tw_a_bytes(int ta, int mh, int kl, int64_t lda, bool span)
{
    return ta ? tw_op_bytes(mh, kl, lda, span) : tw_op_bytes(kl, mh, lda, span);
}
IAAT_HD uint32_t tw_b_bytes(int tb, int nw, int kl, int64_t ldb, bool span)
{
    return tb ? tw_op_bytes(kl, nw, ldb, span) : tw_op_bytes(nw, kl, ldb, span);
}
IAAT_HD uint32_t tw_c_bytes(int mh, int nw, int64_t ldc, bool span) { return tw_op_bytes(nw, mh, ldc, span); }
// Record flags beside kFlagReadC: which operands are staged as one span.
constexpr uint8_t kTwSpanA = 2, kTwSpanB = 4, kTwSpanC = 8;
// A task's items: its K range cut into kseg-value pieces (one empty item for
// K = 0); then, when C is read, one C item.
IAAT_HD uint32_t tw_ab_item_bytes(const TwTask &t, int kl)
{
    return tw_a_bytes(t.ta, t.M, kl, t.lda, (t.flags & kTwSpanA) != 0) +
           tw_b_bytes(t.tb, t.N, kl, t.ldb, (t.flags & kTwSpanB) != 0);
}
IAAT_HD uint32_t tw_c_item_bytes(const TwTask &t) { return tw_c_bytes(t.M, t.N, t.ldc, (t.flags & kTwSpanC) != 0); }

}  // namespace iaat
