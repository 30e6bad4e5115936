// Definitions shared by the host planner and the device kernels.
//
// Work model (the GPU form of the paper's two stages):
//  * install time (Sec. IV): a fixed family of warp-level register-tile
//    kernels, one per (MR x NR register tile, LM x LN lane grid), compiled
//    ahead of time for sm_103a -- the "kernel array" of Table I;
//  * run time (Sec. V): the host tiler splits each instance's C into warp
//    blocks of one variant (the input-aware choice), the planner packs the
//    pieces into pipeline stages, and one persistent kernel executes the
//    whole plan (the "kernel executing plan", Sec. V-B).
#pragma once
#include <cstdint>
#include <cstddef>

#if defined(__CUDACC__)
#define IAAT_HD __host__ __device__ __forceinline__
#define IAAT_CE __host__ __device__ constexpr
#else
#define IAAT_HD inline
#define IAAT_CE constexpr
#endif

namespace iaat {

// ---------------------------------------------------------------- limits
constexpr int kMaxDim = 80;          // cbrt(MNK) <= 80 bounds every size used here
constexpr int kMaxGroupTasks = 32;   // tasks per pipeline stage (one per producer lane)
constexpr int kNumSlots = 8;         // pipeline stages in flight per CTA
constexpr int kConsumerWarps = 8;    // compute warps per CTA (FP64; FP32 uses Traits<4>::kWarps)

// One piece of work: a whole instance, or a column range of it.  Pointers
// address element (0,0) of the piece's stored A, B, C.  64 bytes.
struct alignas(16) TaskDesc {
    const char *A;
    const char *B;
    char *C;
    int32_t lda, ldb, ldc;
    int16_t M, N, K;      // C rows, C columns of this piece; K = 0: no product
    uint8_t ta, tb;
    uint8_t variant;      // register-tile variant of every block of the piece
    uint8_t flags;        // bit 0: beta != 0 (C is read)
    uint8_t nbm, nbn;     // warp blocks along M and along N
    double alpha, beta;
};
static_assert(sizeof(TaskDesc) == 64, "TaskDesc layout");
constexpr uint8_t kFlagReadC = 1;

// alpha or beta of a task record, in the plan's precision: FP64 plans read
// the double, FP32 plans the float (no FP64 conversion on the device).
// Complex plans keep alpha and beta in a table of the plan; the record's
// alpha then holds the address of the instance's entry (re(alpha),
// im(alpha), re(beta), im(beta) in the component type).
union RecScalar {
    double d;
    float f;
    const void *p;
};

// What the consumer warps see of a task once its operands sit in shared
// memory: element (i, j) of the stored X is at byte off + j*cs + i*esz.
struct alignas(16) TaskRec {
    char *C;
    int32_t ldc;
    int32_t offA, offB, offC;
    int32_t csA, csB, csC;
    int16_t M, N, K;
    uint8_t ta, tb, variant, flags, nbm, nbn;
    RecScalar alpha, beta;
};
static_assert(sizeof(TaskRec) == 64, "TaskRec layout");

IAAT_HD void set_scalars(TaskRec &r, double alpha, double beta, int esz)
{
    r.alpha.d = 0.0;
    r.beta.d = 0.0;
    if (esz == 4) {
        r.alpha.f = (float)alpha;
        r.beta.f = (float)beta;
    } else {
        r.alpha.d = alpha;
        r.beta.d = beta;
    }
}

// Tensor-core kernel: one pack (one 128-row MMA tile) of a stage, as the
// producer summarises it for the converter, MMA and epilogue roles.
struct alignas(16) PackInfo {
    int8_t qtask[4];   // task owning each 32-row quarter of the tile (-1: none)
    int8_t btask[8];   // task owning each 16-column block (-1: none)
    int16_t kmax;      // largest K of the pack's tasks
    uint8_t nt;        // MMA N: end of the last task's 16-column blocks (>= 16)
    uint8_t pad;
};
static_assert(sizeof(PackInfo) == 16, "PackInfo layout");

struct alignas(16) SlotHeader {
    int32_t ntasks;
    int32_t nblocks;
    int32_t npacks;   // tensor-core kernel: packs of the stage
    int32_t pad;
    int32_t prefix[kMaxGroupTasks];  // inclusive prefix of blocks per task
};
constexpr int kSlotBytes = sizeof(SlotHeader) + kMaxGroupTasks * sizeof(TaskRec);

// ----------------------------------------------- raw staging of a matrix
// A stored sub-matrix (h rows, w columns, leading dimension ld elements)
// starting at address p is copied into shared memory as whole aligned
// 16-byte granules: either as one span from the granule of its first element
// to the granule of its last (span mode), or column by column (column mode,
// when the ld padding would make the span much larger than the data).  In
// both modes element (i, j) lands at  base + (p & 15) + j*cs + i*esz,  so
// global and shared addresses agree modulo 16 and every copy is a legal
// 16-byte-aligned bulk copy.
struct Stage {
    uint32_t bytes;      // shared bytes reserved (multiple of 16)
    uint32_t cs;         // column stride in shared memory (bytes)
    uint32_t copies;     // bulk copies issued
    uint32_t tx;         // bytes the copies deliver
    uint8_t span;        // 1: one span copy
};

IAAT_HD uint32_t round16(uint64_t x) { return (uint32_t)((x + 15) & ~(uint64_t)15); }

IAAT_HD Stage plan_stage(uint64_t p, int h, int w, int ld, int esz)
{
    Stage s{0, 0, 0, 0, 1};
    if (h <= 0 || w <= 0)
        return s;
    uint64_t beg = p & ~(uint64_t)15;
    uint64_t last = p + ((uint64_t)(w - 1) * (uint64_t)ld + (uint64_t)h) * (uint64_t)esz;
    uint32_t span = (uint32_t)(((last + 15) & ~(uint64_t)15) - beg);
    uint32_t ldb = (uint32_t)ld * (uint32_t)esz;
    uint32_t cs = round16((uint64_t)h * esz + 32) + (ldb & 15u);
    uint32_t head = (uint32_t)(p & 15);
    uint32_t colbytes = round16((uint64_t)head + (uint64_t)(w - 1) * cs + (uint64_t)h * esz);
    if (w == 1 || (uint64_t)span <= (uint64_t)colbytes + (colbytes >> 3) + 256) {
        s.bytes = span; s.cs = ldb; s.copies = 1; s.tx = span; s.span = 1;
    } else {
        s.bytes = colbytes; s.cs = cs; s.copies = (uint32_t)w; s.span = 0;
        // each column delivers the granules covering its own elements
        uint32_t tx = 0;
        for (int j = 0; j < w; ++j) {
            uint64_t c0 = p + (uint64_t)j * ldb;
            uint64_t c1 = c0 + (uint64_t)h * esz;
            tx += (uint32_t)(((c1 + 15) & ~(uint64_t)15) - (c0 & ~(uint64_t)15));
        }
        s.tx = tx;
    }
    return s;
}

// Stored shapes of a task's operands.
IAAT_HD void stored_dims(const TaskDesc &t, int &ha, int &wa, int &hb, int &wb)
{
    ha = t.ta ? t.K : t.M; wa = t.ta ? t.M : t.K;
    hb = t.tb ? t.N : t.K; wb = t.tb ? t.K : t.N;
}

struct TaskStages {
    Stage a, b, c;
    IAAT_HD uint32_t total() const { return a.bytes + b.bytes + c.bytes; }
};

IAAT_HD TaskStages plan_task(const TaskDesc &t, int esz)
{
    TaskStages s;
    int ha, wa, hb, wb;
    stored_dims(t, ha, wa, hb, wb);
    bool prod = t.K > 0;
    s.a = plan_stage((uint64_t)(uintptr_t)t.A, prod ? ha : 0, prod ? wa : 0, t.lda, esz);
    s.b = plan_stage((uint64_t)(uintptr_t)t.B, prod ? hb : 0, prod ? wb : 0, t.ldb, esz);
    bool readc = (t.flags & kFlagReadC) != 0;
    s.c = plan_stage((uint64_t)(uintptr_t)t.C, readc ? t.M : 0, readc ? t.N : 0, t.ldc, esz);
    return s;
}

// ------------------------------------------- register-tile kernel family
// Variant v: every lane holds an MR x NR tile of C; the 32 lanes form an
// LM x LN grid, so one warp block covers (LM*MR) x (LN*NR) of C.  This is the
// GPU counterpart of Table I's m_c x n_c kernels: each is fully unrolled for
// its tile, and the tiler picks one per instance.
struct Variant {
    int8_t mr, nr, lm, ln;
};

// FP32 family.
constexpr int kNumVariantsF32 = 5;
constexpr Variant kVariantsF32[kNumVariantsF32] = {
    {4, 8, 8, 4},   // 0: 32 x 32
    {4, 4, 8, 4},   // 1: 32 x 16
    {4, 4, 4, 8},   // 2: 16 x 32
    {2, 4, 8, 4},   // 3: 16 x 16
    {1, 2, 8, 4},   // 4: 8 x 8
};

// FP64 family (DFMA; each accumulator takes two registers).  DFMA-bound
// work pays a DFMA slot for every idle lane of a partly filled tile, so the
// family adds narrow tiles (32 x 8 down to 32 x 1, and 8 x 4) for
// instances whose width is not a multiple of 16.
constexpr int kNumVariantsF64 = 10;
constexpr Variant kVariantsF64[kNumVariantsF64] = {
    {4, 8, 8, 4},    // 0: 32 x 32
    {4, 4, 8, 4},    // 1: 32 x 16
    {4, 4, 4, 8},    // 2: 16 x 32
    {2, 4, 8, 4},    // 3: 16 x 16
    {1, 2, 8, 4},    // 4: 8 x 8
    {4, 2, 8, 4},    // 5: 32 x 8
    {4, 1, 8, 4},    // 6: 32 x 4
    {2, 1, 16, 2},   // 7: 32 x 2
    {1, 1, 32, 1},   // 8: 32 x 1
    {1, 1, 8, 4},    // 9: 8 x 4
};

// Complex families (CGEMM / ZGEMM, Table I rows 3-4): an accumulator is a
// (re, im) pair, so a complex-float tile takes the registers of an FP64 tile
// of the same shape and a complex-double tile twice that; the complex-double
// tiles are at most 32 x 16.  Complex double runs at the DFMA rate, where
// every lane of a partly filled block costs a DFMA slot, so its family adds
// one-element-per-lane tiles in every lane-grid shape: with them the tiler
// fills about 80% of the DFMA slots on log-uniform sizes in [1, 80],
// against about 61% with the five larger tiles alone (flop-weighted model).
constexpr int kNumVariantsC32 = 5;
constexpr Variant kVariantsC32[kNumVariantsC32] = {
    {4, 8, 8, 4},   // 0: 32 x 32
    {4, 4, 8, 4},   // 1: 32 x 16
    {4, 4, 4, 8},   // 2: 16 x 32
    {2, 4, 8, 4},   // 3: 16 x 16
    {1, 2, 8, 4},   // 4: 8 x 8
};
constexpr int kNumVariantsC64 = 11;
constexpr Variant kVariantsC64[kNumVariantsC64] = {
    {4, 4, 8, 4},    // 0: 32 x 16
    {4, 4, 4, 8},    // 1: 16 x 32
    {2, 4, 8, 4},    // 2: 16 x 16
    {2, 2, 8, 4},    // 3: 16 x 8
    {1, 2, 8, 4},    // 4: 8 x 8
    {1, 1, 8, 4},    // 5: 8 x 4
    {1, 1, 4, 8},    // 6: 4 x 8
    {1, 1, 16, 2},   // 7: 16 x 2
    {1, 1, 2, 16},   // 8: 2 x 16
    {1, 1, 32, 1},   // 9: 32 x 1
    {1, 1, 1, 32},   // 10: 1 x 32
};

// K is consumed in chunks of kKC (FP32) / kKC64 (FP64) staged per warp.
constexpr int kKC = 16;
constexpr int kKC64 = 8;
constexpr int kMaxBM = 32, kMaxBN = 32;  // largest warp block over both families

// Per-warp canonical operand buffers: As[KC][BM], Bs[KC][BN].
template <int ESZ> struct Traits;
// kWarps: consumer warps per CTA (one more warp is the producer).  FP32 runs
// 16 so each scheduler has four warps to hide shared-memory latency with;
// FP64 keeps 8 because its register tiles need twice the registers.
template <> struct Traits<4> {
    static constexpr int KC = kKC;
    static constexpr int kCanonBytes = KC * (kMaxBM + kMaxBN) * 4;   // 4 KB
    static constexpr int kWarps = 16;
};
template <> struct Traits<8> {
    static constexpr int KC = kKC64;
    static constexpr int kCanonBytes = KC * (kMaxBM + kMaxBN) * 8;   // 4 KB
    static constexpr int kWarps = kConsumerWarps;
};
template <int ESZ> IAAT_CE int kernel_threads() { return 32 * (Traits<ESZ>::kWarps + 1); }

// Shared-memory map of the persistent kernel (byte offsets).
constexpr int kSmemBarriers = 0;                          // full[], empty[], ring ranges
constexpr int kSmemTaskBars = 256;                        // per-task readiness [slot][task]
constexpr int kSmemSlots = kSmemTaskBars + kNumSlots * kMaxGroupTasks * 8;
constexpr int kSmemCanon = kSmemSlots + kNumSlots * kSlotBytes;
template <int ESZ> IAAT_CE int smem_ring_offset()
{
    return ((kSmemCanon + Traits<ESZ>::kWarps * Traits<ESZ>::kCanonBytes) + 127) & ~127;
}
constexpr int kSmemTotal = 227 * 1024;
template <int ESZ> IAAT_CE int ring_bytes() { return (kSmemTotal - smem_ring_offset<ESZ>()) & ~127; }
// A stage may take at most half the ring, so two always fit.
template <int ESZ> IAAT_CE int max_group_bytes() { return ring_bytes<ESZ>() / 2; }

// Complex kernel: kCplxWarps consumer warps that read the staged operands in
// place (no per-warp buffers), so its ring starts right after the slots.
constexpr int kCplxWarps = 8;
IAAT_CE int cplx_ring_offset() { return (kSmemCanon + 127) & ~127; }
IAAT_CE int cplx_ring_bytes() { return (kSmemTotal - cplx_ring_offset()) & ~127; }
IAAT_CE int cplx_max_group_bytes() { return cplx_ring_bytes() / 2; }

// Order in which the CTAs take the cost-sorted stages: stage i of CTA `cta`
// is group sched_group(i, cta, ncta), a snake over the groups that balances
// like LPT without atomics.
IAAT_HD int sched_group(int i, int cta, int ncta)
{
    return i * ncta + ((i & 1) ? (ncta - 1 - cta) : cta);
}

// ------------------------------------------------------- stage programs
// iaat_plan_create turns the plan into one program per stage, executed by the
// producer warp of the CTA that runs the stage: everything about the stage
// that does not change between launches -- where its operands go in the
// staging ring, which earlier stage must release the space first, the task
// records and pack summaries the consumers read, the bytes each readiness
// barrier expects, and the list of bulk copies -- is computed once on the
// host.  Program layout (16-byte aligned, at poff[g] for group g):
//   StageProg | uint32 tx[32] | CopyCmd[ncmd] | SlotHeader + TaskRec[nt] | PackInfo[npk]
struct alignas(16) StageProg {
    int32_t wait;        // stage of this CTA's sequence that must be released first (-1: none)
    uint32_t rec_bytes;  // SlotHeader + TaskRec[nt]: copied to the stage's slot
    uint16_t ncmd;       // copy commands
    uint8_t nt, npk;     // tasks, packs (tensor-core kernel: PackInfo[npk] follows the records)
    uint32_t ctx;        // tensor-core kernel: bytes of the stage's C copies (one barrier)
};
static_assert(sizeof(StageProg) == 16, "StageProg layout");
struct alignas(16) CopyCmd {
    const char *src;     // 16-byte aligned global address
    uint32_t dst;        // byte offset from the shared-memory base, 16-byte aligned
    uint32_t meta;       // bytes (bits 0-23, a multiple of 16) | barrier << 24 (task t, or 32: C barrier)
};
static_assert(sizeof(CopyCmd) == 16, "CopyCmd layout");
constexpr int kProgTx = 16;
constexpr int kProgCmds = kProgTx + 4 * kMaxGroupTasks;
constexpr uint32_t kCmdBarC = 32;

// Kernel parameters.
struct Params {
    const TaskDesc *tasks;
    const int32_t *gbeg;      // group g = tasks [gbeg[g], gbeg[g+1])
    const char *prog;         // stage programs (plans); NULL: plan on the device
    const int64_t *poff;      // program of group g at prog + poff[g]
    int32_t ngroups;
    int32_t pad;
    int32_t *err;             // device error word (0 = fine)
};

// Kernel parameters: either plan arrays in global memory, or (single call)
// up to kInline tasks carried inline in the parameter block.
constexpr int kInline = 32;
struct KParams {
    Params p;
    TaskDesc inline_tasks[kInline];
    int32_t inline_gbeg[kInline + 1];
};
static_assert(sizeof(KParams) <= 4096, "kernel parameter block");

// ------------------------------------------------ warp-stream kernel
// (ws.cuh) The FP32 CUDA-core plans run a kernel in which every warp streams
// its own list of warp tasks through a private shared-memory ring.
// One warp task.  64 bytes; the first 64 bytes of every ring item are a copy.
struct alignas(16) WsTask {
    const char *A;        // op(A) element (r0, 0) of the block in the stored A
    const char *B;        // op(B) element (0, c0) of the block in the stored B
    char *C;              // C element (r0, c0)
    int32_t lda, ldb, ldc;
    int32_t K;            // K (0: no product); streamed in chunks, so any K of the domain
    int16_t M, N;         // block rows, block columns
    uint8_t ta, tb, variant, flags;
    float alpha, beta;
    int32_t pad[2];
};
static_assert(sizeof(WsTask) == 64, "WsTask layout");

struct WsParams {
    const WsTask *tasks;   // warp w's tasks: tasks[wbeg[w] .. wbeg[w+1])
    const int32_t *wbeg;
    int32_t *err;
    int32_t nwarps;        // gridDim.x * kWsWarps
    int32_t pad;
};

constexpr int kWsWarps = 16;                 // warps per CTA, one CTA per SM
constexpr int kWsKC = 16;                    // K values per item
constexpr int kWsMaxOut = 8;                 // items in flight per warp
constexpr int kWsHdr = 80;                   // item header: task record + 16 bytes of chunk info
constexpr int kWsCStride = 32;               // column stride (floats) of the staged C block
constexpr int kWsRingBytes = (kSmemTotal / kWsWarps) & ~127;   // 14464 bytes per warp
constexpr int kWsMaxItem = kWsHdr + 2 * kWsKC * 32 * 4 + kWsCStride * 32 * 4;
static_assert(kWsMaxItem <= kWsRingBytes, "one item of the largest tile must fit the ring");
constexpr int kWsThreads = 32 * kWsWarps;

// ------------------------------------------- pack-stream tensor-core kernel
// (tc2.cuh) Tensor-core plans run a kernel with four independent groups of
// four warps per SM; each group streams its own list of packs (one 128-row
// MMA tile of up to kT2MaxTasks tasks).  A pack's program in global memory is
//   Tc2Hdr | Tc2Rec[ntasks] | (unused record slots) | CopyCmd[ncmd]
// (16-byte aligned), the commands always kT2CmdOff bytes after the header so
// that one fixed window holds the header, the records and the first
// commands; the header and records are copied to the start of the pack's
// staging item, the commands bring the raw operands after them.
struct alignas(16) Tc2Hdr {
    int32_t ntasks;       // tasks of the pack (1..kT2MaxTasks)
    int32_t ncmd;         // copy commands
    int32_t kpack;        // MMA K: the largest K of the pack, rounded up to the MMA K step (0: no product)
    int32_t nt;           // MMA N: the end of the last task's columns, a multiple of 16 (16..kT2Cols)
    uint32_t item_bytes;  // staging bytes of the pack (multiple of 16)
    uint32_t rec_bytes;   // header + records (copied first)
    uint32_t tx_bytes;    // bytes all copies of the pack deliver, records included
    int32_t pad0;
    int64_t next[2];      // programs of the next two packs of the same warp group (-1: none)
    int32_t pad1[4];
};
static_assert(sizeof(Tc2Hdr) == 64, "Tc2Hdr layout");

// One task of a pack: element (r, c) of its stored X sits at item + offX +
// c*csX + r*4 in the staging item.  Its rows are rows row0.. of the MMA tile
// (tensor-memory lanes) and its columns columns col0.. of the accumulator.
struct alignas(16) Tc2Rec {
    char *C;
    int32_t ldc;
    int32_t offA, offB, offC;
    int32_t csA, csB, csC;
    int32_t K;
    int16_t M, N;
    uint8_t ta, tb, row0, col0;
    uint8_t flags, pad0;
    int16_t pad1;
    float alpha, beta;
};
static_assert(sizeof(Tc2Rec) == 64, "Tc2Rec layout");

struct Tc2Params {
    const char *prog;        // pack programs
    const int64_t *poff;     // program of pack p at prog + poff[p]
    const int32_t *gbeg;     // group gg runs packs [gbeg[gg], gbeg[gg+1])
    int32_t *err;
    int32_t ngroups;         // gridDim.x * kT2Groups
    int32_t pad;
};

constexpr int kT2Groups = 4;              // warp groups per CTA (one CTA per SM)
constexpr int kT2Threads = 32 * 5 * kT2Groups;   // per group four warps and a producer warp
constexpr int kT2KC = 16;                 // K values per converted operand chunk
constexpr int kT2Inflight = 4;            // packs in flight per group
constexpr int kT2Cols = 128;              // accumulator columns of a group
constexpr int kT2MaxTasks = 8;            // tasks per pack
constexpr int kT2CmdOff = 64 + kT2MaxTasks * 64;           // byte offset of the commands in a program
constexpr int kT2WinCmds = 64;                             // commands in the prefetched window
constexpr int kT2Window = kT2CmdOff + kT2WinCmds * 16;     // bytes of a program the issuing warp prefetches

constexpr int32_t kErrTimeoutFull = 1;
constexpr int32_t kErrTimeoutEmpty = 2;
constexpr int32_t kErrBadGroup = 4;

}  // namespace iaat
