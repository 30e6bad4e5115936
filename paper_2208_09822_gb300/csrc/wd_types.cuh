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
    int32_t *err;
    int32_t nwarps;        // warps of the grid that own tasks
    int32_t pad;
};

constexpr int kWdWarps = 4;          // warps per CTA
constexpr int kWdThreads = 32 * kWdWarps;
constexpr int kWdCtasPerSm = 5;      // 20 warps per SM (96 registers a thread)
constexpr int kWdMaxRows = 32;       // block height: one row per lane
constexpr int kWdChunkIters = 8;     // column steps per lane when K runs in chunks
// The largest K one pass holds in registers (larger K runs in chunks of it,
// with at most kWdChunkIters column steps per lane) and the block width.
IAAT_HD constexpr int wd_max_k(int esz) { return esz == 4 ? 32 : 16; }
IAAT_HD constexpr int wd_max_cols(int esz) { return esz == 4 ? 32 : 16; }
// Staged op(B) column pitch (elements) for a pass of kr values of K: at least
// kr, a whole number of 16-byte groups, and an odd number of them (or one),
// so that consecutive columns start in different 16-byte bank groups.
IAAT_HD constexpr int wd_pitch(int esz, int kr) { return esz == 4 ? (kr == 4 ? 4 : kr + 4) : kr + 2; }
// A warp's slice of shared memory: two task records (the next one lands
// while the current block runs), the op(B) block, then 32 lanes' C0 values
// per column step.
constexpr int kWdRecBytes = 2 * (int)sizeof(WdTask);
IAAT_HD constexpr int wd_b_elems(int esz) { return wd_max_cols(esz) * wd_pitch(esz, wd_max_k(esz)); }
IAAT_HD constexpr int wd_stage_elems(int esz) { return wd_b_elems(esz) + wd_max_cols(esz) * 32; }
IAAT_HD constexpr int wd_warp_bytes(int esz) { return kWdRecBytes + wd_stage_elems(esz) * esz; }

}  // namespace iaat
