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

constexpr int kTwWarps = 12;      // warps per CTA (one CTA per SM), 32 accumulator columns of tensor memory each
constexpr int kTwKC = 16;         // K values per converted operand chunk (one MMA K step of BF16 / FP16)
constexpr int kTwMaxOut = 8;      // ring items in flight per warp
constexpr int kTwBlock = 32;      // largest block side
constexpr int kTwThreads = 32 * kTwWarps;

// Ring items.  A run is a contiguous stretch of one stored column (X bytes);
// it is copied as the 16-byte granules that cover it into a slot of
// tw_run_slot(X) bytes, its first element at the slot start plus the
// address's offset within its granule (0, 4, 8 or 12).
IAAT_HD uint32_t tw_run_slot(int xbytes) { return (uint32_t)((xbytes + 27) >> 4) << 4; }
// op(A) rows r0.. (mh of them) x K range of kl values: runs along k (not
// transposed: one per k) or along the rows (transposed: one per row)
IAAT_HD uint32_t tw_a_bytes(int ta, int mh, int kl)
{
    return kl <= 0 ? 0u : (ta ? (uint32_t)mh * tw_run_slot(4 * kl) : (uint32_t)kl * tw_run_slot(4 * mh));
}
IAAT_HD uint32_t tw_b_bytes(int tb, int nw, int kl)
{
    return kl <= 0 ? 0u : (tb ? (uint32_t)kl * tw_run_slot(4 * nw) : (uint32_t)nw * tw_run_slot(4 * kl));
}
// A task's items: its K range cut into kseg-value pieces (one item for K = 0),
// the first one led by the task record; then, when C is read, one C item.
IAAT_HD uint32_t tw_ab_item_bytes(int ta, int tb, int mh, int nw, int kl, bool first)
{
    return (first ? 64u : 0u) + tw_a_bytes(ta, mh, kl) + tw_b_bytes(tb, nw, kl);
}
IAAT_HD uint32_t tw_c_item_bytes(int mh, int nw) { return (uint32_t)nw * tw_run_slot(4 * mh); }

}  // namespace iaat
