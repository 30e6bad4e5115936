// Shared host / device definitions of the warp-direct CUDA-core kernel
// (wd.cuh): its task record, launch parameters and block limits.
#pragma once
#include "common.cuh"

namespace iaat {

// One warp task, 64 bytes: a block of at most 32 rows and wd_max_cols(esz)
// columns of one instance's C with the instance's whole K.  The warp's lanes
// are laid out as g column groups of m rows: lane q*m + i computes row i of
// the columns q, q+g, q+2g, ... of the block (iters of them at most).
struct alignas(16) WdTask {
    const char *A;        // op(A) element (r0, 0) of the block in the stored A
    const char *B;        // op(B) element (0, c0) of the block in the stored B
    char *C;              // C element (r0, c0)
    int32_t lda, ldb, ldc;
    int32_t K;            // K (0: C = beta*C0)
    uint8_t m, g;         // block rows (1..32), column groups (m*g <= 32)
    uint8_t flags;        // kWdTransA | kWdTransB | kWdReadC
    uint8_t iters;        // ceil(n / g): column steps of a lane
    uint16_t n;           // block columns (1..wd_max_cols)
    uint16_t magic;       // ceil(32768 / m): lane / m == (lane * magic) >> 15
    union {
        double d[2];      // FP64 plans: alpha, beta
        float f[2];       // FP32 plans: alpha, beta rounded to float
    } ab;
};
static_assert(sizeof(WdTask) == 64, "WdTask layout");

constexpr uint8_t kWdTransA = 1;
constexpr uint8_t kWdTransB = 2;
constexpr uint8_t kWdReadC = 4;

struct WdParams {
    const WdTask *tasks;   // warp w's tasks: tasks[wbeg[w] .. wbeg[w+1])
    const int32_t *wbeg;
    const WdTask *first;   // first[w]: a copy of warp w's first task (zeros if none), fetched
                           // without waiting for wbeg
    int32_t *err;
    int32_t nwarps;        // warps of the grid that own tasks
    int32_t pad;
};

constexpr int kWdWarps = 4;          // warps per CTA
constexpr int kWdThreads = 32 * kWdWarps;
constexpr int kWdCtasPerSm = 6;      // 24 warps per SM (80 registers a thread)
constexpr int kWdMaxRows = 32;       // block height: one row per lane
// Two block shapes.  Up to wd_k1 values of K: at most 32 rows and
// wd_max_cols columns, row i of op(A) at sA[k*32 + i], op(B) column j at
// sB[j*wd_pitch1].  Beyond: at most 16 rows and wd_max_cols / 2 columns,
// K in passes of up to wd_k2 values (one pass, or chunks of wd_k2 with the
// partial sums of the lane's at most 8 column steps kept between chunks),
// row i at sA[k*16 + i], column j at sB[j*wd_pitch2].  Both fit the same
// staging area.
IAAT_HD constexpr int wd_k1(int esz) { return esz == 4 ? 16 : 8; }
IAAT_HD constexpr int wd_k2(int esz) { return esz == 4 ? 32 : 16; }
IAAT_HD constexpr int wd_max_cols(int esz) { return esz == 4 ? 32 : 16; }
constexpr int kWdRows2 = 16;         // block height beyond wd_k1
constexpr int kWdChunkIters = 8;     // column steps per lane of a 16-row block (g >= 2)
// Staged op(B) column pitches (elements): whole, odd numbers of 16-byte
// groups, so that consecutive columns start in different 16-byte bank groups.
IAAT_HD constexpr int wd_pitch1(int esz) { return esz == 4 ? 20 : 10; }
IAAT_HD constexpr int wd_pitch2(int esz) { return esz == 4 ? 36 : 18; }
// A warp's slice of shared memory: two task records (the next one lands
// while the current block runs), the op(A) block, the op(B) block, then 32
// lanes' C0 values per column step (rows 8..15 hold partial sums between K
// chunks).
constexpr int kWdRecBytes = 2 * (int)sizeof(WdTask);
IAAT_HD constexpr int wd_a_elems(int esz) { return wd_k1(esz) * kWdMaxRows; }   // == wd_k2 * kWdRows2
IAAT_HD constexpr int wd_b_elems(int esz) { return wd_max_cols(esz) * wd_pitch1(esz); }
IAAT_HD constexpr int wd_stage_elems(int esz) { return wd_a_elems(esz) + wd_b_elems(esz) + wd_max_cols(esz) * 32; }
IAAT_HD constexpr int wd_warp_bytes(int esz) { return kWdRecBytes + wd_stage_elems(esz) * esz; }
static_assert(wd_k2(4) * kWdRows2 <= wd_a_elems(4) && wd_k2(8) * kWdRows2 <= wd_a_elems(8), "op(A) fits");
static_assert(wd_max_cols(4) / 2 * wd_pitch2(4) <= wd_b_elems(4) && wd_max_cols(8) / 2 * wd_pitch2(8) <= wd_b_elems(8),
              "op(B) fits");

}  // namespace iaat
