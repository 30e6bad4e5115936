// Persistent grouped small-GEMM kernel on the CUDA cores (FP32 FFMA, FP64
// DFMA): the "kernel executing plan" of Sec. V-B run by one launch.
//
// Each CTA walks its share of the plan's stages (groups of <= 32 tasks):
//  * the producer warp (one lane per task) sizes each task's A, B, C, claims
//    a contiguous piece of the shared-memory ring, publishes the task records
//    and issues 1-D bulk copies that complete on the stage's mbarrier;
//  * the consumer warps take the stage's warp blocks round-robin.  A block is
//    computed K-chunk by K-chunk: the warp re-packs op(A) rows and op(B)
//    columns of the chunk into its own canonical buffers (zero-padded, so the
//    inner loop has no bounds checks -- the paper's "no boundary processing"),
//    then every lane runs its MR x NR register tile as rank-1 updates
//    (Algorithm 1's k-loop), and finally writes alpha*acc + beta*C0.
// Every wait is bounded; on time-out the kernel records an error code in
// *err and stops instead of hanging.
#pragma once
#include "common.cuh"
#include "ptx.cuh"

namespace iaat {

constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s per wait

__device__ __forceinline__ void set_error(int32_t *err, int32_t code)
{
    if (err)
        atomicOr(err, code);
}

struct SmemMap {
    char *base;
    uint32_t sbase;
    uint32_t ring_off;     // byte offset of the staging ring from base
    uint32_t ring_bytes;   // its size
    uint32_t pinfo_off;    // tensor-core kernel: PackInfo[kNumSlots][kMaxGroupTasks]
    uint32_t cbar_off;     // tensor-core kernel: per-slot barrier of the C copies
    // full(s): the stage's records are published; task(s, t): the operands
    // of task t of the stage have landed (one barrier per task, so consumers
    // start on the first tasks of a stage while later ones are in flight).
    __device__ uint32_t full(int s) const { return sbase + kSmemBarriers + 8 * s; }
    __device__ uint32_t task(int s, int t) const { return sbase + kSmemTaskBars + 8 * (s * kMaxGroupTasks + t); }
    __device__ uint32_t empty(int s) const { return sbase + kSmemBarriers + 64 + 8 * s; }
    __device__ uint32_t *range_beg() const { return reinterpret_cast<uint32_t *>(base + 128); }
    __device__ uint32_t *range_end() const { return reinterpret_cast<uint32_t *>(base + 160); }
    __device__ PackInfo *pinfo(int s) const
    {
        return reinterpret_cast<PackInfo *>(base + pinfo_off) + s * kMaxGroupTasks;
    }
    __device__ uint32_t cfull(int s) const { return sbase + cbar_off + 8 * s; }
    __device__ SlotHeader *header(int s) const
    {
        return reinterpret_cast<SlotHeader *>(base + kSmemSlots + s * kSlotBytes);
    }
    __device__ TaskRec *recs(int s) const
    {
        return reinterpret_cast<TaskRec *>(base + kSmemSlots + s * kSlotBytes + sizeof(SlotHeader));
    }
};

__device__ __forceinline__ void issue_stage(const Stage &st, const char *p, int h, int w, int ld, int esz,
                                            uint32_t dst, uint32_t bar)
{
    if (st.bytes == 0)
        return;
    uint64_t pa = reinterpret_cast<uint64_t>(p);
    if (st.span) {
        bulk_g2s(dst, reinterpret_cast<const void *>(pa & ~15ull), st.bytes, bar);
        return;
    }
    uint32_t head = (uint32_t)(pa & 15);
    uint64_t ldb = (uint64_t)ld * esz;
    for (int j = 0; j < w; ++j) {
        uint64_t c0 = pa + (uint64_t)j * ldb;
        uint64_t g0 = c0 & ~15ull;
        uint64_t g1 = (c0 + (uint64_t)h * esz + 15) & ~15ull;
        uint32_t d = dst + ((head + (uint32_t)j * st.cs) & ~15u);
        bulk_g2s(d, reinterpret_cast<const void *>(g0), (uint32_t)(g1 - g0), bar);
    }
}

// Producer of a plan launched without stage programs (the single-call and
// allocation-free entry points, CUDA-core kernel): sizes each stage's tasks,
// claims ring space and writes the records itself.  Lane t handles task t.
template <int ESZ>
__device__ void producer_dyn(const KParams &KP, const SmemMap &S)
{
    const Params &P = KP.p;
    const TaskDesc *tasks = P.tasks ? P.tasks : KP.inline_tasks;
    const int32_t *gbeg = P.gbeg ? P.gbeg : KP.inline_gbeg;
    const uint32_t lane = lane_id();
    const uint32_t ring_off = S.ring_off;
    const uint32_t RING = S.ring_bytes;
    uint32_t *rbeg = S.range_beg(), *rend = S.range_end();
    uint32_t head = 0;
    int oldest = 0;
    int i = 0;
    // Descriptor loads run ahead of the stage being issued: the stage index
    // of stage i+2 and the task descriptors of stage i+1 are in flight while
    // stage i is sized and its copies issued.
    auto load_bounds = [&](int ii, int &b0, int &b1) {
        const int gg = sched_group(ii, blockIdx.x, gridDim.x);
        b0 = b1 = 0;
        if (gg < P.ngroups) {
            b0 = gbeg[gg];
            b1 = gbeg[gg + 1];
        }
    };
    auto load_desc = [&](int b0, int b1, TaskDesc &d) {
        const int nt = b1 - b0;
        if ((int)lane < nt && nt <= kMaxGroupTasks) {
            d = tasks[b0 + lane];
        } else {
            d.A = d.B = nullptr; d.C = nullptr;
            d.lda = d.ldb = d.ldc = 1; d.M = d.N = d.K = 0; d.ta = d.tb = 0;
            d.variant = 0; d.flags = 0; d.nbm = d.nbn = 1; d.alpha = d.beta = 0.0;
        }
    };
    int cb0, cb1, nb0, nb1;
    load_bounds(0, cb0, cb1);
    load_bounds(1, nb0, nb1);
    TaskDesc d_cur;
    load_desc(cb0, cb1, d_cur);
    for (;; ++i) {
        const int g = sched_group(i, blockIdx.x, gridDim.x);
        if (g >= P.ngroups)
            break;
        const int slot = i % kNumSlots;
        const int nt = cb1 - cb0;
        if (nt < 0 || nt > kMaxGroupTasks) {
            if (lane == 0)
                set_error(P.err, kErrBadGroup);
            break;
        }
        const bool has = (int)lane < nt;
        const TaskDesc d = d_cur;
        load_desc(nb0, nb1, d_cur);
        cb0 = nb0;
        cb1 = nb1;
        load_bounds(i + 2, nb0, nb1);
        TaskStages st = plan_task(d, ESZ);
        const uint32_t f = has ? st.total() : 0u;
        const uint32_t tx = has ? (st.a.tx + st.b.tx + st.c.tx) : 0u;
        const int nb = has ? (int)d.nbm * (int)d.nbn : 0;
        uint32_t incl = f;
        int nbi = nb;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            int w = __shfl_up_sync(0xffffffffu, nbi, o);
            if ((int)lane >= o) {
                incl += v;
                nbi += w;
            }
        }
        const uint32_t F = __shfl_sync(0xffffffffu, incl, 31);
        const int NB = __shfl_sync(0xffffffffu, nbi, 31);
        const uint32_t excl = incl - f;

        // claim ring space [a, a+F); wait until no live stage overlaps it
        uint32_t a = 0;
        int ok = 1;
        if (lane == 0) {
            a = (head + F <= RING) ? head : 0u;
            int need = i - kNumSlots;   // the slot's previous user
            for (int s = i - 1; s >= oldest && s > need; --s) {
                const int ss = s % kNumSlots;
                if (F > 0 && rbeg[ss] < a + F && a < rend[ss]) {
                    need = s;
                    break;
                }
            }
            if (need >= oldest) {
                ok = mbar_wait(S.empty(need % kNumSlots), (uint32_t)((need / kNumSlots) & 1), kWaitLimitNs);
                oldest = need + 1;
            }
            rbeg[slot] = a;
            rend[slot] = a + F;
            head = a + F;
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
            if (lane == 0)
                set_error(P.err, kErrTimeoutEmpty);
            break;
        }
        a = __shfl_sync(0xffffffffu, a, 0);

        const uint32_t base = ring_off + a + excl;   // offset from the smem base
        SlotHeader *hd = S.header(slot);
        if (has) {
            TaskRec r;
            r.C = d.C;
            r.ldc = d.ldc;
            r.offA = (int32_t)(base + ((uint32_t)reinterpret_cast<uintptr_t>(d.A) & 15u));
            r.offB = (int32_t)(base + st.a.bytes + ((uint32_t)reinterpret_cast<uintptr_t>(d.B) & 15u));
            r.offC = (int32_t)(base + st.a.bytes + st.b.bytes + ((uint32_t)reinterpret_cast<uintptr_t>(d.C) & 15u));
            r.csA = (int32_t)st.a.cs;
            r.csB = (int32_t)st.b.cs;
            r.csC = (int32_t)st.c.cs;
            r.M = d.M; r.N = d.N; r.K = d.K;
            r.ta = d.ta; r.tb = d.tb; r.variant = d.variant; r.flags = d.flags;
            r.nbm = d.nbm; r.nbn = d.nbn;
            set_scalars(r, d.alpha, d.beta, ESZ);
            S.recs(slot)[lane] = r;
        }
        hd->prefix[lane] = has ? nbi : 0x7fffffff;
        if (lane == 0) {
            hd->ntasks = nt;
            hd->nblocks = NB;
            hd->npacks = 0;
        }
        __syncwarp();
        if (lane == 0)
            mbar_arrive(S.full(slot));
        // every lane arms its task's barrier (no bytes for lanes without a
        // task, so all 32 complete once per use of the slot), then issues
        // that task's copies
        mbar_arrive_expect_tx(S.task(slot, (int)lane), tx);
        if (has) {
            int ha, wa, hb, wb;
            stored_dims(d, ha, wa, hb, wb);
            const uint32_t bar = S.task(slot, (int)lane);
            const uint32_t dst = S.sbase + base;
            const bool prod = d.K > 0;
            issue_stage(st.a, d.A, prod ? ha : 0, prod ? wa : 0, d.lda, ESZ, dst, bar);
            issue_stage(st.b, d.B, prod ? hb : 0, prod ? wb : 0, d.ldb, ESZ, dst + st.a.bytes, bar);
            issue_stage(st.c, d.C, d.M, d.N, d.ldc, ESZ, dst + st.a.bytes + st.b.bytes, bar);
        }
    }
    // Copies still in flight target this CTA's shared memory: before leaving,
    // wait (bounded) until every issued stage has landed.
    const int first = i - kNumSlots > 0 ? i - kNumSlots : 0;
    for (int s = first; s < i; ++s)
        if (!mbar_wait(S.task(s % kNumSlots, (int)lane), (uint32_t)((s / kNumSlots) & 1), kWaitLimitNs))
            set_error(P.err, kErrTimeoutFull);
}

// Producer of a plan with stage programs: per stage it waits for the release
// the program names, copies the precomputed records (and, TC, the pack
// summaries) into the slot on its full barrier, arms the readiness barriers
// and issues the program's bulk copies.  TC: the stage feeds the tensor-core
// kernel, whose C copies complete on the slot's cfull barrier (the epilogue
// reads C long after the operands, so one wait per stage serves it).
// The programs of the next stages are loaded ahead: the offset of stage
// i+3, the header of stage i+2, and the barrier bytes and first 64 copy
// commands of stage i+1 are in flight while stage i is issued.
template <int ESZ, bool TC>
__device__ void producer_prog(const KParams &KP, const SmemMap &S)
{
    const Params &P = KP.p;
    const int lane = (int)lane_id();
    const uint32_t lo = S.ring_off, hi = S.ring_off + S.ring_bytes;
    auto prog_off = [&](int ii) -> int64_t {
        const int gg = sched_group(ii, blockIdx.x, gridDim.x);
        return gg < P.ngroups ? P.poff[gg] : (int64_t)-1;
    };
    auto load_hdr = [&](int64_t off) -> uint4 {
        return off >= 0 ? *reinterpret_cast<const uint4 *>(P.prog + off) : make_uint4(0u, 0u, 0u, 0u);
    };
    struct Body {
        uint32_t tx;
        uint4 c0, c1;
    };
    auto load_body = [&](int64_t off, const uint4 &h, Body &b) {
        b.tx = 0u;
        b.c0 = b.c1 = make_uint4(0u, 0u, 0u, 0u);
        if (off < 0)
            return;
        const int ncmd = (int)(h.z & 0xffffu);
        b.tx = reinterpret_cast<const uint32_t *>(P.prog + off + kProgTx)[lane];
        const uint4 *cm = reinterpret_cast<const uint4 *>(P.prog + off + kProgCmds);
        if (lane < ncmd)
            b.c0 = cm[lane];
        if (lane + 32 < ncmd)
            b.c1 = cm[lane + 32];
    };
    int64_t off_c = prog_off(0), off_n = prog_off(1), off_nn = prog_off(2);
    uint4 h_c = load_hdr(off_c), h_n = load_hdr(off_n);
    Body b_c;
    load_body(off_c, h_c, b_c);
    int oldest = 0;
    int i = 0;
    bool bad = false;
    for (;; ++i) {
        if (off_c < 0)
            break;
        const int slot = i % kNumSlots;
        const int wait = (int)h_c.x;
        const uint32_t rec_bytes = h_c.y;
        const int ncmd = (int)(h_c.z & 0xffffu);
        const int nt = (int)((h_c.z >> 16) & 0xffu), npk = (int)(h_c.z >> 24);
        const uint32_t ctx = h_c.w;
        const char *pg = P.prog + off_c;
        const Body b = b_c;
        // loads for the next stages
        load_body(off_n, h_n, b_c);
        const uint4 h_nn = load_hdr(off_nn);
        const int64_t off_nnn = prog_off(i + 3);
        if (nt > kMaxGroupTasks || npk > kMaxGroupTasks || wait >= i ||
            rec_bytes != (uint32_t)(sizeof(SlotHeader) + nt * sizeof(TaskRec)) || (!TC && npk != 0)) {
            if (lane == 0)
                set_error(P.err, kErrBadGroup);
            bad = true;
            break;
        }
        // the release that frees this stage's slot and ring space
        int ok = 1;
        if (lane == 0 && wait >= oldest) {
            ok = mbar_wait(S.empty(wait % kNumSlots), (uint32_t)((wait / kNumSlots) & 1), kWaitLimitNs) ? 1 : 0;
            oldest = wait + 1;
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
            if (lane == 0)
                set_error(P.err, kErrTimeoutEmpty);
            bad = true;
            break;
        }
        if (lane == 0) {
            const uint32_t pkb = (uint32_t)npk * (uint32_t)sizeof(PackInfo);
            mbar_arrive_expect_tx(S.full(slot), rec_bytes + pkb);
            const char *img = pg + kProgCmds + ncmd * (int)sizeof(CopyCmd);
            bulk_g2s(smem_addr(S.header(slot)), img, rec_bytes, S.full(slot));
            if (TC && npk > 0)
                bulk_g2s(smem_addr(S.pinfo(slot)), img + rec_bytes, pkb, S.full(slot));
            if (TC)
                mbar_arrive_expect_tx(S.cfull(slot), ctx);
        }
        __syncwarp();
        // every lane arms its task's barrier (0 bytes without a task, so all
        // 32 complete once per use of the slot)
        mbar_arrive_expect_tx(S.task(slot, lane), b.tx);
        __syncwarp();
        auto issue = [&](const uint4 &c) {
            const uint32_t bytes = c.w & 0xffffffu, bar = c.w >> 24;
            if (c.z < lo || c.z + bytes > hi || ((c.z | bytes | c.x) & 15u) != 0u || bar > (TC ? kCmdBarC : 31u)) {
                set_error(P.err, kErrBadGroup);
                return;
            }
            const char *src = reinterpret_cast<const char *>(((uint64_t)c.y << 32) | c.x);
            bulk_g2s(S.sbase + c.z, src, bytes, bar == kCmdBarC ? S.cfull(slot) : S.task(slot, (int)bar));
        };
        if (lane < ncmd)
            issue(b.c0);
        if (lane + 32 < ncmd)
            issue(b.c1);
        const uint4 *cm = reinterpret_cast<const uint4 *>(pg + kProgCmds);
        for (int k = lane + 64; k < ncmd; k += 32)
            issue(cm[k]);
        off_c = off_n;
        h_c = h_n;
        off_n = off_nn;
        h_n = h_nn;
        off_nn = off_nnn;
    }
    (void)bad;
    // Copies still in flight target this CTA's shared memory: before leaving,
    // wait (bounded) until every issued stage has landed.
    const int first = i - kNumSlots > 0 ? i - kNumSlots : 0;
    for (int s = first; s < i; ++s) {
        const uint32_t par = (uint32_t)((s / kNumSlots) & 1);
        if (!mbar_wait(S.task(s % kNumSlots, lane), par, kWaitLimitNs) ||
            !mbar_wait(S.full(s % kNumSlots), par, kWaitLimitNs) ||
            (TC && !mbar_wait(S.cfull(s % kNumSlots), par, kWaitLimitNs)))
            set_error(P.err, kErrTimeoutFull);
    }
}

template <int ESZ, bool TC = false>
__device__ void producer_loop(const KParams &KP, const SmemMap &S)
{
    if (KP.p.prog)
        producer_prog<ESZ, TC>(KP, S);
    else if constexpr (!TC)
        producer_dyn<ESZ>(KP, S);
    else if (lane_id() == 0)
        set_error(KP.p.err, kErrBadGroup);   // tensor-core launches always carry programs
}

// Position of element m of canonical row kk: 16-byte groups XOR-swizzled by
// the row so both re-pack directions and the tile loads avoid bank conflicts.
template <int BM, int VE>
__device__ __forceinline__ int swz(int m, int kk)
{
    constexpr int G0 = BM / VE;
    constexpr int G = G0 >= 8 ? 8 : (G0 >= 1 ? G0 : 1);
    return m ^ ((kk & (G - 1)) * VE);
}

// Re-pack one chunk of an operand into canonical rows X[kk][m], kk < kcp.
// raw(m, kk) = src + m*sm + kk*sk.  Elements with m >= mh or kk >= kc are 0.
// MFAST: lanes run along m (raw contiguous in m), else along kk.
template <typename T, int BM, int KC, bool MFAST>
__device__ __forceinline__ void repack(T *X, const char *src, int sm, int sk, int mh, int kc, int kcp)
{
    constexpr int VE = 16 / (int)sizeof(T);
    const int lane = (int)lane_id();
    if (MFAST) {
        constexpr int STEP_ROWS = BM >= 32 ? 1 : 32 / BM;
        constexpr int PER_ROW = BM >= 32 ? BM / 32 : 1;
        const int m_l = BM >= 32 ? lane : (lane % BM);
        const int kk_l = BM >= 32 ? 0 : (lane / BM);
#pragma unroll 1
        for (int kk0 = 0; kk0 < kcp; kk0 += STEP_ROWS) {
            const int kk = kk0 + kk_l;
#pragma unroll
            for (int q = 0; q < PER_ROW; ++q) {
                const int m = m_l + 32 * q;
                T v = T(0);
                if (m < mh && kk < kc)
                    v = *reinterpret_cast<const T *>(src + m * sm + kk * sk);
                if (kk < kcp)
                    X[kk * BM + swz<BM, VE>(m, kk)] = v;
            }
        }
    } else {
        constexpr int KL = KC;               // lanes along kk
        constexpr int MSTEP = 32 / KL;       // m values per sweep
        const int kk = lane % KL;
        const int mo = lane / KL;
        if (kk < kcp) {
            const bool kin = kk < kc;
            const char *s = src + kk * sk;
#pragma unroll 4
            for (int m = mo; m < BM; m += MSTEP) {
                T v = T(0);
                if (kin && m < mh)
                    v = *reinterpret_cast<const T *>(s + m * sm);
                X[kk * BM + swz<BM, VE>(m, kk)] = v;
            }
        }
    }
}

// One k step of the register tile: the lane's MR values of op(A) and NR of
// op(B) at k, then MR x NR FMAs.  ADIR / BDIR: the operand is read where it
// was staged (aoff / boff: byte offsets of the lane's rows / columns);
// otherwise from the warp's canonical chunk buffer, row kk.
template <typename T, int MR, int NR, int LM, int LN, bool ADIR, bool BDIR>
__device__ __forceinline__ void k_step(T (&acc)[MR][NR], const char *ak_, const char *bk_, const int (&aoff)[MR],
                                       const int (&boff)[NR], const T *As, const T *Bs, int kk, int li, int lj)
{
    constexpr int ESZ = (int)sizeof(T);
    constexpr int BM = LM * MR, BN = LN * NR;
    constexpr int VE = 16 / ESZ;
    T av[MR], bv[NR];
    if constexpr (ADIR) {
#pragma unroll
        for (int a = 0; a < MR; ++a)
            av[a] = *reinterpret_cast<const T *>(ak_ + aoff[a]);
    } else {
        const T *arow = As + kk * BM;
        if constexpr (MR >= VE) {
#pragma unroll
            for (int q = 0; q < MR / VE; ++q) {
                const int pos = swz<BM, VE>(li * MR + q * VE, kk);
                if constexpr (ESZ == 4) {
                    float4 t4 = *reinterpret_cast<const float4 *>(arow + pos);
                    av[q * 4 + 0] = t4.x; av[q * 4 + 1] = t4.y;
                    av[q * 4 + 2] = t4.z; av[q * 4 + 3] = t4.w;
                } else {
                    double2 t2 = *reinterpret_cast<const double2 *>(arow + pos);
                    av[q * 2 + 0] = t2.x; av[q * 2 + 1] = t2.y;
                }
            }
        } else {
            const int pos = swz<BM, VE>(li * MR, kk);
#pragma unroll
            for (int q = 0; q < MR; ++q)
                av[q] = arow[pos + q];
        }
    }
    if constexpr (BDIR) {
#pragma unroll
        for (int b = 0; b < NR; ++b)
            bv[b] = *reinterpret_cast<const T *>(bk_ + boff[b]);
    } else {
        const T *brow = Bs + kk * BN;
        if constexpr (NR >= VE) {
#pragma unroll
            for (int q = 0; q < NR / VE; ++q) {
                const int pos = swz<BN, VE>(lj * NR + q * VE, kk);
                if constexpr (ESZ == 4) {
                    float4 t4 = *reinterpret_cast<const float4 *>(brow + pos);
                    bv[q * 4 + 0] = t4.x; bv[q * 4 + 1] = t4.y;
                    bv[q * 4 + 2] = t4.z; bv[q * 4 + 3] = t4.w;
                } else {
                    double2 t2 = *reinterpret_cast<const double2 *>(brow + pos);
                    bv[q * 2 + 0] = t2.x; bv[q * 2 + 1] = t2.y;
                }
            }
        } else {
            const int pos = swz<BN, VE>(lj * NR, kk);
#pragma unroll
            for (int q = 0; q < NR; ++q)
                bv[q] = brow[pos + q];
        }
    }
#pragma unroll
    for (int a = 0; a < MR; ++a)
#pragma unroll
        for (int b = 0; b < NR; ++b)
            acc[a][b] = fma(av[a], bv[b], acc[a][b]);
}

// The block's k-loop, K-chunk by K-chunk: operands not read in place are
// re-packed into the canonical buffers first, then the k steps run.
template <typename T, int MR, int NR, int LM, int LN, bool ADIR, bool BDIR>
__device__ __forceinline__ void k_loop(T (&acc)[MR][NR], const char *Ab, const char *Bb, int am, int ak, int bk,
                                       int bn, int mh, int nw, int K, const int (&aoff)[MR], const int (&boff)[NR],
                                       T *As, T *Bs, int li, int lj)
{
    constexpr int BM = LM * MR, BN = LN * NR;
    constexpr int KC = Traits<(int)sizeof(T)>::KC;
#pragma unroll 1
    for (int k0 = 0; k0 < K; k0 += KC) {
        const int kc = min(KC, K - k0);
        const int kcp = (kc + 3) & ~3;
        if constexpr (!ADIR) {
            if (am != (int)sizeof(T))
                repack<T, BM, KC, false>(As, Ab + k0 * ak, am, ak, mh, kc, kcp);
            else
                repack<T, BM, KC, true>(As, Ab + k0 * ak, am, ak, mh, kc, kcp);
        }
        if constexpr (!BDIR) {
            if (bn == (int)sizeof(T))
                repack<T, BN, KC, true>(Bs, Bb + k0 * bk, bn, bk, nw, kc, kcp);
            else
                repack<T, BN, KC, false>(Bs, Bb + k0 * bk, bn, bk, nw, kc, kcp);
        }
        if constexpr (!ADIR || !BDIR)
            __syncwarp();
        const char *ak_ = Ab + k0 * ak;
        const char *bk_ = Bb + k0 * bk;
        // both operands re-packed: their zero padding lets the steps run to
        // the chunk's K rounded up to 4, four at a time; an operand read in
        // place has no padding, so then the steps stop at K exactly
        const int kend = (!ADIR && !BDIR) ? kcp : kc;
        int kk = 0;
#pragma unroll 1
        for (; kk + 4 <= kend; kk += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
                k_step<T, MR, NR, LM, LN, ADIR, BDIR>(acc, ak_ + (kk + u) * ak, bk_ + (kk + u) * bk, aoff, boff,
                                                      As, Bs, kk + u, li, lj);
        }
        if constexpr (ADIR || BDIR) {
#pragma unroll 1
            for (; kk < kc; ++kk)
                k_step<T, MR, NR, LM, LN, ADIR, BDIR>(acc, ak_ + kk * ak, bk_ + kk * bk, aoff, boff, As, Bs, kk, li,
                                                      lj);
        }
        if constexpr (!ADIR || !BDIR)
            __syncwarp();
    }
}

template <typename T, int MR, int NR, int LM, int LN>
__device__ __forceinline__ void run_block(const char *smem, const TaskRec &r, int bi, int bj, T *As, T *Bs)
{
    constexpr int ESZ = (int)sizeof(T);
    const int lane = (int)lane_id();
    const int M = r.M, N = r.N, K = r.K;
    const int bh = (M + r.nbm - 1) / r.nbm;
    const int bw = (N + r.nbn - 1) / r.nbn;
    const int r0 = bi * bh, c0 = bj * bw;
    const int mh = min(bh, M - r0), nw = min(bw, N - c0);
    const int li = lane % LM, lj = lane / LM;

    T acc[MR][NR];
#pragma unroll
    for (int a = 0; a < MR; ++a)
#pragma unroll
        for (int b = 0; b < NR; ++b)
            acc[a][b] = T(0);

    if (K > 0) {
        const int am = r.ta ? r.csA : ESZ, ak = r.ta ? ESZ : r.csA;
        const int bk = r.tb ? r.csB : ESZ, bn = r.tb ? ESZ : r.csB;
        const char *Ab = smem + r.offA + r0 * am;
        const char *Bb = smem + r.offB + c0 * bn;
        // FP64: A not transposed has a lane's MR rows of one column
        // consecutive in the staged data, B transposed its NR columns of one
        // row; those operands are read in place (rows / columns past the block
        // clamped to its last one, their results never stored) instead of
        // being re-packed (fc64: 9.8 -> 9.1 ms).  FP32 re-packs every operand:
        // its 16-warp kernel ran slower with the four k-loop versions (the
        // instruction footprint and register pressure grow).
        int aoff[MR], boff[NR];
#pragma unroll
        for (int a = 0; a < MR; ++a)
            aoff[a] = min(li * MR + a, mh - 1) * ESZ;
#pragma unroll
        for (int b = 0; b < NR; ++b)
            boff[b] = min(lj * NR + b, nw - 1) * ESZ;
        if constexpr (ESZ == 4) {
            constexpr int BM = LM * MR, BN = LN * NR;
            constexpr int KC = Traits<ESZ>::KC;
            constexpr int VE = 16 / ESZ;
#pragma unroll 1
            for (int k0 = 0; k0 < K; k0 += KC) {
                const int kc = min(KC, K - k0);
                const int kcp = (kc + 3) & ~3;
                if (r.ta)
                    repack<T, BM, KC, false>(As, Ab + k0 * ak, am, ak, mh, kc, kcp);
                else
                    repack<T, BM, KC, true>(As, Ab + k0 * ak, am, ak, mh, kc, kcp);
                if (r.tb)
                    repack<T, BN, KC, true>(Bs, Bb + k0 * bk, bn, bk, nw, kc, kcp);
                else
                    repack<T, BN, KC, false>(Bs, Bb + k0 * bk, bn, bk, nw, kc, kcp);
                __syncwarp();
#pragma unroll 1
                for (int kk0 = 0; kk0 < kcp; kk0 += 4) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int kk = kk0 + u;
                        const T *arow = As + kk * BM;
                        const T *brow = Bs + kk * BN;
                        T av[MR], bv[NR];
                        if constexpr (MR >= VE) {
#pragma unroll
                            for (int q = 0; q < MR / VE; ++q) {
                                const int pos = swz<BM, VE>(li * MR + q * VE, kk);
                                if constexpr (ESZ == 4) {
                                    float4 t4 = *reinterpret_cast<const float4 *>(arow + pos);
                                    av[q * 4 + 0] = t4.x; av[q * 4 + 1] = t4.y;
                                    av[q * 4 + 2] = t4.z; av[q * 4 + 3] = t4.w;
                                } else {
                                    double2 t2 = *reinterpret_cast<const double2 *>(arow + pos);
                                    av[q * 2 + 0] = t2.x; av[q * 2 + 1] = t2.y;
                                }
                            }
                        } else {
                            const int pos = swz<BM, VE>(li * MR, kk);
#pragma unroll
                            for (int q = 0; q < MR; ++q)
                                av[q] = arow[pos + q];
                        }
                        if constexpr (NR >= VE) {
#pragma unroll
                            for (int q = 0; q < NR / VE; ++q) {
                                const int pos = swz<BN, VE>(lj * NR + q * VE, kk);
                                if constexpr (ESZ == 4) {
                                    float4 t4 = *reinterpret_cast<const float4 *>(brow + pos);
                                    bv[q * 4 + 0] = t4.x; bv[q * 4 + 1] = t4.y;
                                    bv[q * 4 + 2] = t4.z; bv[q * 4 + 3] = t4.w;
                                } else {
                                    double2 t2 = *reinterpret_cast<const double2 *>(brow + pos);
                                    bv[q * 2 + 0] = t2.x; bv[q * 2 + 1] = t2.y;
                                }
                            }
                        } else {
                            const int pos = swz<BN, VE>(lj * NR, kk);
#pragma unroll
                            for (int q = 0; q < NR; ++q)
                                bv[q] = brow[pos + q];
                        }
#pragma unroll
                        for (int a = 0; a < MR; ++a)
#pragma unroll
                            for (int b = 0; b < NR; ++b)
                                acc[a][b] = fma(av[a], bv[b], acc[a][b]);
                    }
                }
                __syncwarp();
            }
        } else if (r.ta == 0) {
            if (r.tb)
                k_loop<T, MR, NR, LM, LN, true, true>(acc, Ab, Bb, am, ak, bk, bn, mh, nw, K, aoff, boff, As, Bs, li, lj);
            else
                k_loop<T, MR, NR, LM, LN, true, false>(acc, Ab, Bb, am, ak, bk, bn, mh, nw, K, aoff, boff, As, Bs, li, lj);
        } else {
            if (r.tb)
                k_loop<T, MR, NR, LM, LN, false, true>(acc, Ab, Bb, am, ak, bk, bn, mh, nw, K, aoff, boff, As, Bs, li, lj);
            else
                k_loop<T, MR, NR, LM, LN, false, false>(acc, Ab, Bb, am, ak, bk, bn, mh, nw, K, aoff, boff, As, Bs, li, lj);
        }
    }

    // epilogue: C = alpha*acc + beta*C0, exact elements only
    T alpha, beta;
    if constexpr (ESZ == 4) {
        alpha = r.alpha.f;
        beta = r.beta.f;
    } else {
        alpha = r.alpha.d;
        beta = r.beta.d;
    }
    const bool readc = (r.flags & kFlagReadC) != 0;
    const char *Craw = smem + r.offC;
    T *Cg = reinterpret_cast<T *>(r.C);
    const int64_t ldc = r.ldc;
#pragma unroll
    for (int b = 0; b < NR; ++b) {
        const int j = lj * NR + b;
        if (j < nw) {
            const int gj = c0 + j;
#pragma unroll
            for (int a = 0; a < MR; ++a) {
                const int i = li * MR + a;
                if (i < mh) {
                    const int gi = r0 + i;
                    T v = alpha * acc[a][b];
                    if (readc)
                        v = fma(beta, *reinterpret_cast<const T *>(Craw + gj * r.csC + gi * ESZ), v);
                    Cg[gi + gj * ldc] = v;
                }
            }
        }
    }
}

template <typename T>
__device__ __forceinline__ void dispatch_block(const char *smem, const TaskRec &r, int bi, int bj, T *As, T *Bs);

template <>
__device__ __forceinline__ void dispatch_block<float>(const char *smem, const TaskRec &r, int bi, int bj, float *As,
                                                      float *Bs)
{
#define IAAT_V(id)                                                                                    \
    case id:                                                                                          \
        run_block<float, kVariantsF32[id].mr, kVariantsF32[id].nr, kVariantsF32[id].lm, kVariantsF32[id].ln>( \
            smem, r, bi, bj, As, Bs);                                                                 \
        break;
    switch (r.variant) {
        IAAT_V(0) IAAT_V(1) IAAT_V(2) IAAT_V(3) IAAT_V(4)
    default:
        break;
    }
#undef IAAT_V
}

template <>
__device__ __forceinline__ void dispatch_block<double>(const char *smem, const TaskRec &r, int bi, int bj,
                                                       double *As, double *Bs)
{
#define IAAT_V(id)                                                                                    \
    case id:                                                                                          \
        run_block<double, kVariantsF64[id].mr, kVariantsF64[id].nr, kVariantsF64[id].lm, kVariantsF64[id].ln>( \
            smem, r, bi, bj, As, Bs);                                                                 \
        break;
    switch (r.variant) {
        IAAT_V(0) IAAT_V(1) IAAT_V(2) IAAT_V(3) IAAT_V(4) IAAT_V(5) IAAT_V(6) IAAT_V(7) IAAT_V(8) IAAT_V(9)
    default:
        break;
    }
#undef IAAT_V
}

template <typename T>
__device__ void consumer_loop(const KParams &KP, const SmemMap &S, int warp)
{
    constexpr int ESZ = (int)sizeof(T);
    const Params &P = KP.p;
    const int lane = (int)lane_id();
    T *As = reinterpret_cast<T *>(S.base + kSmemCanon + warp * Traits<ESZ>::kCanonBytes);
    T *Bs = As + Traits<ESZ>::KC * kMaxBM;
    int rot = 0;   // blocks taken so far over the CTA's stages, modulo the warps
    for (int i = 0;; ++i) {
        const int g = sched_group(i, blockIdx.x, gridDim.x);
        if (g >= P.ngroups)
            break;
        const int slot = i % kNumSlots;
        if (!mbar_wait(S.full(slot), (uint32_t)((i / kNumSlots) & 1), kWaitLimitNs)) {
            if (lane == 0)
                set_error(P.err, kErrTimeoutFull);
            return;
        }
        const SlotHeader *hd = S.header(slot);
        const TaskRec *recs = S.recs(slot);
        const int nb = hd->nblocks;
        const int pre = hd->prefix[lane];
        // the rotation continues across stages, so the warp that takes a
        // stage's extra block is a different one each time
        for (int b = (warp - rot + Traits<ESZ>::kWarps) % Traits<ESZ>::kWarps; b < nb; b += Traits<ESZ>::kWarps) {
            const int t = __popc(__ballot_sync(0xffffffffu, pre <= b));
            const int before = __shfl_sync(0xffffffffu, pre, t > 0 ? t - 1 : 0);
            const int lb = b - (t > 0 ? before : 0);
            if (!mbar_wait(S.task(slot, t), (uint32_t)((i / kNumSlots) & 1), kWaitLimitNs)) {
                if (lane == 0)
                    set_error(P.err, kErrTimeoutFull);
                return;
            }
            const TaskRec r = recs[t];
            const int bi = lb % r.nbm, bj = lb / r.nbm;
            dispatch_block<T>(S.base, r, bi, bj, As, Bs);
        }
        __syncwarp();
        if (lane == 0)
            mbar_arrive(S.empty(slot));
        rot = (rot + nb) % Traits<ESZ>::kWarps;
    }
}

template <typename T>
__global__ void __launch_bounds__(kernel_threads<(int)sizeof(T)>(), 1) grouped_kernel(const __grid_constant__ KParams KP)
{
    constexpr int kWarps = Traits<(int)sizeof(T)>::kWarps;
    extern __shared__ __align__(128) char smem[];
    SmemMap S;
    S.base = smem;
    S.sbase = smem_addr(smem);
    S.ring_off = (uint32_t)smem_ring_offset<(int)sizeof(T)>();
    S.ring_bytes = (uint32_t)ring_bytes<(int)sizeof(T)>();
    S.pinfo_off = 0;
    S.cbar_off = 0;
    const int warp = threadIdx.x / 32;
    if (threadIdx.x < kNumSlots * kMaxGroupTasks)
        mbar_init(S.task(threadIdx.x / kMaxGroupTasks, threadIdx.x % kMaxGroupTasks), 1);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kNumSlots; ++s) {
            mbar_init(S.full(s), 1);
            mbar_init(S.empty(s), kWarps);
        }
    }
    fence_barrier_init();
    __syncthreads();
    if (warp == kWarps)
        producer_loop<(int)sizeof(T)>(KP, S);
    else
        consumer_loop<T>(KP, S, warp);
}

}  // namespace iaat
