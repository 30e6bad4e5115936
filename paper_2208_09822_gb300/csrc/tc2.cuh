// Pack-stream grouped small-GEMM kernel on the tcgen05 tensor cores, FP32 in
// and out (3xBF16 split products, TF32, FP16 or 6xBF16 inputs; FP32
// accumulation in tensor memory).
//
// A CTA (one per SM) runs four independent groups of four warps, each fed
// by a producer warp of its own.  Warp q of a group sits on SM sub-partition q and owns
// tensor-memory lanes 32q..32q+31; the group owns 128 accumulator columns,
// one operand buffer (one K-chunk of the 128-row A tile and of the B tile,
// every split term) and one staging ring.  The planner puts up to
// kT2MaxTasks tasks (instances, or pieces of large ones) into a pack -- one
// 128-row MMA tile; a task owns a run of rows of the tile (tasks of up to 32
// rows inside one 32-row quarter) and a run of 16-column blocks -- and deals
// the packs to the groups ahead of time (largest first, least loaded group).
//
//  * producer warp: up to kT2Inflight packs ahead of its group, it reads
//    the pack's host-built program (prefetched into shared memory by a bulk
//    copy) and issues the pack's 1-D bulk copies (records and raw operand
//    spans) into the group's ring, completing on the pack's mbarrier; the
//    group gives ring space back through per-pack "empty" mbarriers.  Copy
//    issue costs a warp about 230 cycles per bulk copy (the tensor memory
//    accelerator overlaps the copies of several issuing warps), so it never
//    runs on a group's warps, and the four producers issue in parallel;
//  * convert: per K-chunk, the group's 128 threads turn the staged FP32 rows
//    of every task's op(A) and op(B)^T into the canonical K-major operand
//    layout (Xh, Xl BF16 terms for 3xBF16), only the tasks' real rows, zeros
//    past each task's K;
//  * MMA: after a named barrier of the group, one thread issues the chunk's
//    tcgen05.mma (three products for 3xBF16) and commits them to the group's
//    MMA barrier;
//  * epilogue: each warp reads the accumulator rows of its quarter
//    (tcgen05.ld, lane = row) and writes alpha*acc + beta*C0 for the task of
//    each row -- C0 read from the staged C, consecutive lanes on consecutive
//    rows of a column, so the stores are coalesced -- then the group's
//    barrier frees the pack's accumulator and its staging.
//
// Every wait is bounded; a time-out or a malformed program sets the error
// word and the group's abort flag, the group stops at the next pack boundary,
// the producer stops issuing for it and waits for its copies in flight, and
// the CTA frees its tensor memory.
#pragma once
#include <cstddef>

#include "tc.cuh"

namespace iaat {

template <int P> IAAT_CE int t2_vpr() { return 16 / TcTraits<P>::kOpBytes; }   // values per 16-byte core row
template <int P> IAAT_CE int t2_kgroups() { return kT2KC / t2_vpr<P>(); }     // core matrices along K per chunk
template <int P> IAAT_CE int t2_sbo() { return t2_kgroups<P>() * 128; }        // 8-row group stride
template <int P> IAAT_CE int t2_opb() { return (kTcRows / 8) * t2_sbo<P>(); }  // one term of one operand
template <int P> IAAT_CE int t2_buf_bytes() { return 2 * TcTraits<P>::kTerms * t2_opb<P>(); }

// shared-memory map: per group 256 bytes of barriers and state, the tensor
// memory slot, the operand buffers, two program windows per group, then the
// staging rings.  Group state (byte offsets):
constexpr int kT2GsFull = 0;        // [kT2Inflight] mbarriers: a pack's staging has landed
constexpr int kT2GsEmpty = 32;      // [kT2Inflight] mbarriers: the group is done with a pack
constexpr int kT2GsWin = 64;        // [2] mbarriers: a program window has landed
constexpr int kT2GsMma = 80;        // mbarrier: the group's MMAs have completed
constexpr int kT2GsAbort = 88;      // int32 abort flag
constexpr int kT2GsOff = 96;        // [kT2Inflight] uint32 ring offsets of the packs in flight
constexpr int kT2GroupState = 128;
constexpr int kT2TmemSlot = kT2Groups * kT2GroupState;
constexpr int kT2Ops = 2048;




template <int P> IAAT_CE int t2_win_off() { return kT2Ops + kT2Groups * t2_buf_bytes<P>(); }
template <int P> IAAT_CE int t2_ring_off() { return t2_win_off<P>() + kT2Groups * 2 * kT2Window; }
template <int P> IAAT_CE int t2_ring_bytes() { return ((kSmemTotal - t2_ring_off<P>()) / kT2Groups) & ~127; }
static_assert(kT2TmemSlot + 16 <= kT2Ops && kT2Window % 16 == 0, "group state, program windows");

__device__ __forceinline__ void group_sync(int g)
{
    asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(128) : "memory");
}

__device__ __forceinline__ void cpa16(uint32_t dst, const void *src) { cp_async16(dst, src); }

// arrive on `bar` once every cp.async this thread issued so far has landed
__device__ __forceinline__ void cpa_arrive(uint32_t bar)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

// Convert K-chunk c of every task of the pack into the operand buffer.  The
// group's 128 threads share a flattened list of work items: per task its
// op(A) rows, then the rows of op(B)^T (its columns), each row cut into
// 16-byte core rows of t2_vpr values of k.
template <int P>
__device__ __forceinline__ void t2_convert(const char *item, int ntasks, char *ops, int c, int tid)
{
    constexpr int VPR = t2_vpr<P>();
    constexpr int G = t2_kgroups<P>();
    constexpr int LG = G == 2 ? 1 : (G == 4 ? 2 : 0);
    static_assert((1 << LG) == G, "core rows per chunk");
    constexpr int OPB = t2_opb<P>();
    constexpr int SBO = t2_sbo<P>();
    constexpr int TERMS = TcTraits<P>::kTerms;
    const Tc2Rec *recs = reinterpret_cast<const Tc2Rec *>(item + sizeof(Tc2Hdr));
    int pre[kT2MaxTasks];   // inclusive prefix of work items per task
#pragma unroll
    for (int t = 0; t < kT2MaxTasks; ++t) {
        const int rows = t < ntasks ? (int)recs[t].M + (int)recs[t].N : 0;
        pre[t] = (t ? pre[t - 1] : 0) + rows * G;
    }
    const int total = pre[kT2MaxTasks - 1];
    const int k0 = c * kT2KC;
#pragma unroll 2
    for (int e = tid; e < total; e += 128) {
        int t = 0, base = 0;
#pragma unroll
        for (int u = 0; u < kT2MaxTasks - 1; ++u) {
            if (e >= pre[u]) {
                t = u + 1;
                base = pre[u];
            }
        }
        const Tc2Rec &tr = recs[t];
        const int l = e - base;
        const int rr = l >> LG, gi = l & (G - 1);
        const int M = tr.M;
        const int side = rr >= M ? 1 : 0;
        const int r = rr - side * M;
        const int kb = k0 + gi * VPR;
        // op(A)(r, k): stored A(r, k) (N) or A(k, r) (T); op(B)^T row r = op(B)(k, r):
        // stored B(k, r) (N) or B(r, k) (T)
        const bool kcontig = side == 0 ? tr.ta != 0 : tr.tb == 0;
        const int cs = side == 0 ? tr.csA : tr.csB;
        const int sk = kcontig ? 4 : cs;
        const char *src = item + (side == 0 ? tr.offA : tr.offB) + (kcontig ? r * cs : r * 4) + kb * sk;
        const int kleft = tr.K - kb;
        float x[8];
#pragma unroll
        for (int v = 0; v < VPR; ++v)
            x[v] = v < kleft ? *reinterpret_cast<const float *>(src + v * sk) : 0.0f;
        const int row = (side == 0 ? (int)tr.row0 : (int)tr.col0) + r;
        char *t0 = ops + side * TERMS * OPB;
        store_row<P>(t0, t0 + OPB, t0 + 2 * OPB, (uint32_t)((row >> 3) * SBO + (row & 7) * 16 + gi * 128), x);
    }
}

// The MMAs of one K-chunk (kc values, a multiple of the MMA K step).
template <int P>
__device__ __forceinline__ void t2_mma(uint32_t ops, uint32_t dtmem, int nt, int kc, uint32_t accum)
{
    constexpr int KS = TcTraits<P>::kKStep;
    constexpr int OPB = t2_opb<P>();
    constexpr uint32_t SBO = (uint32_t)t2_sbo<P>();
    const uint32_t idesc = tc_idesc<P>(nt);
    uint64_t da0 = smem_desc(ops, 128, SBO), db0 = smem_desc(ops + TcTraits<P>::kTerms * OPB, 128, SBO);
    uint64_t da1 = da0 + (OPB >> 4), db1 = db0 + (OPB >> 4);
    uint64_t da2 = da1 + (OPB >> 4), db2 = db1 + (OPB >> 4);
    for (int ks = 0; ks < kc / KS; ++ks) {
        if constexpr (P == kTc6xBF16) {
            tc_mma<P>(dtmem, da1, db1, idesc, accum);
            tc_mma<P>(dtmem, da2, db0, idesc, 1u);
            tc_mma<P>(dtmem, da0, db2, idesc, 1u);
            tc_mma<P>(dtmem, da1, db0, idesc, 1u);
            tc_mma<P>(dtmem, da0, db1, idesc, 1u);
            tc_mma<P>(dtmem, da0, db0, idesc, 1u);
            da1 += 16; db1 += 16; da2 += 16; db2 += 16;
        } else if constexpr (P == kTc3xBF16) {
            tc_mma<P>(dtmem, da1, db0, idesc, accum);
            tc_mma<P>(dtmem, da0, db1, idesc, 1u);
            tc_mma<P>(dtmem, da0, db0, idesc, 1u);
            da1 += 16; db1 += 16;
        } else {
            tc_mma<P>(dtmem, da0, db0, idesc, accum);
        }
        da0 += 16;   // one K step: two core matrices along K, 256 bytes
        db0 += 16;
        accum = 1u;
    }
}

// Epilogue of the warp on lane quarter q: lane l holds row 32q + l of the
// tile, which belongs to at most one task; the warp reads the accumulator
// columns its lanes' tasks span, 32 at a time, and each lane stores the
// columns of its own task (alpha*acc + beta*C0, C0 from the staging).
__device__ __forceinline__ void t2_epilogue(const char *item, int ntasks, uint32_t tmem, int q, int lane, bool product)
{
    const Tc2Rec *recs = reinterpret_cast<const Tc2Rec *>(item + sizeof(Tc2Hdr));
    const int row = 32 * q + lane;
    int mt = -1;
#pragma unroll
    for (int t = 0; t < kT2MaxTasks; ++t)
        if (t < ntasks && row >= (int)recs[t].row0 && row < (int)recs[t].row0 + (int)recs[t].M)
            mt = t;
    if (__ballot_sync(0xffffffffu, mt >= 0) == 0u)
        return;
    const Tc2Rec &r = recs[mt >= 0 ? mt : 0];
    const int c0 = r.col0, N = mt >= 0 ? (int)r.N : 0;
    const int lo = __reduce_min_sync(0xffffffffu, mt >= 0 ? c0 : 4096);
    const int hi = __reduce_max_sync(0xffffffffu, mt >= 0 ? c0 + N : 0);
    const int cbeg = lo & ~15;
    const int tr = row - (int)r.row0;   // this lane's row of its task's C
    const float alpha = r.alpha, beta = r.beta;
    const bool readc = (r.flags & kFlagReadC) != 0;
    const int64_t ldc = r.ldc;
    const int csC = r.csC;
    const uint32_t dt = tmem + ((uint32_t)(32 * q) << 16);
    for (int cb = cbeg; cb < hi; cb += 32) {
        uint32_t v[32];
        if (product) {
            // 16 columns at a time, never past the pack's last 16-column block
            tmem_ld16<0>(dt + (uint32_t)cb, v);
            if (cb + 16 < hi)
                tmem_ld16<16>(dt + (uint32_t)(cb + 16), v);
            tmem_wait_ld(v);
        } else {
#pragma unroll
            for (int e = 0; e < 32; ++e)
                v[e] = 0u;
        }
        const int j0 = cb - c0;   // task column of v[0]
        float *cp = reinterpret_cast<float *>(r.C) + tr + (int64_t)j0 * ldc;
        const char *sp = item + r.offC + tr * 4 + j0 * csC;
#pragma unroll
        for (int u = 0; u < 32; ++u) {
            if ((unsigned)(j0 + u) < (unsigned)N) {
                float x = alpha * __uint_as_float(v[u]);
                if (readc)
                    x = fmaf(beta, *reinterpret_cast<const float *>(sp), x);
                __stcs(cp, x);
            }
            cp += ldc;
            sp += csC;
        }
    }
}

__device__ __forceinline__ bool t2_wait(uint32_t bar, uint32_t parity)
{
    return mbar_wait(bar, parity, kWaitLimitNs);
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// The producer warp of group g: issues the bulk copies of the group's packs.
template <int P>
__device__ void t2_producer(const Tc2Params &Pm, char *sm2, uint32_t sb, int g, int lane)
{
    constexpr uint32_t RING = (uint32_t)t2_ring_bytes<P>();
    char *gs = sm2 + g * kT2GroupState;
    const uint32_t gbar = sb + (uint32_t)(g * kT2GroupState);
    volatile int32_t *abort_flag = reinterpret_cast<volatile int32_t *>(gs + kT2GsAbort);
    volatile uint32_t *item_off = reinterpret_cast<volatile uint32_t *>(gs + kT2GsOff);
    const uint32_t ring = sb + (uint32_t)(t2_ring_off<P>() + g * (int)RING);
    auto fetch_window = [&](int s, int64_t o) {
        if (o >= 0 && lane == 0) {
            const uint32_t bar = gbar + kT2GsWin + 8 * s;
            mbar_arrive_expect_tx(bar, (uint32_t)kT2Window);
            bulk_g2s(sb + (uint32_t)(t2_win_off<P>() + (g * 2 + s) * kT2Window), Pm.prog + o, (uint32_t)kT2Window, bar);
        }
    };
    const int gg = (int)blockIdx.x * kT2Groups + g;
    int pi = gg < Pm.ngroups ? Pm.gbeg[gg] : 0;
    const int pe = gg < Pm.ngroups ? Pm.gbeg[gg + 1] : 0;
    int64_t o0 = pi < pe ? Pm.poff[pi] : -1, o1 = pi + 1 < pe ? Pm.poff[pi + 1] : -1;   // packs pi, pi + 1
    fetch_window(0, o0);
    fetch_window(1, o1);
    int issued = 0, rel = 0;
    uint32_t head = 0;
    uint64_t idle_since = global_ns();
    while (pi < pe && !*abort_flag) {
        // packs the group has given back
        while (rel < issued &&
               mbar_test(gbar + kT2GsEmpty + 8 * (rel % kT2Inflight), (uint32_t)((rel / kT2Inflight) & 1)))
            ++rel;
        bool progress = false;
        while (issued - rel < kT2Inflight && pi < pe) {
            const int ws = issued & 1;
            if (!t2_wait(gbar + kT2GsWin + 8 * ws, (uint32_t)((issued >> 1) & 1))) {
                if (lane == 0) {
                    set_error(Pm.err, kErrTimeoutFull);
                    *abort_flag = 1;
                }
                break;
            }
            const char *w = sm2 + t2_win_off<P>() + (g * 2 + ws) * kT2Window;
            const uint4 h0 = *reinterpret_cast<const uint4 *>(w);
            const uint4 h1 = *reinterpret_cast<const uint4 *>(w + 16);
            const int ntasks = (int)h0.x, ncmd = (int)h0.y;
            const uint32_t size = h1.x, recb = h1.y, tx = h1.z;
            const int slot = issued % kT2Inflight;
            const char *prog = Pm.prog + o0;
            auto cmd_at = [&](int k) -> uint4 {
                return k < kT2WinCmds ? *reinterpret_cast<const uint4 *>(w + kT2CmdOff + 16 * k)
                                      : *reinterpret_cast<const uint4 *>(prog + kT2CmdOff + 16 * k);
            };
            bool ok = ntasks >= 1 && ntasks <= kT2MaxTasks && ncmd >= 0 && ncmd <= 4096 && size <= RING &&
                      (size & 15u) == 0u && recb == (uint32_t)(sizeof(Tc2Hdr) + ntasks * sizeof(Tc2Rec)) &&
                      recb <= size && (int)h0.w >= 16 && (int)h0.w <= kT2Cols && (h0.w & 15u) == 0u;
            uint32_t off = 0;
            if (ok) {
                off = head + size <= RING ? head : 0u;
                if (issued > rel) {
                    const uint32_t tail = item_off[rel % kT2Inflight];
                    const bool fits = head > tail ? (off == head || size <= tail) : (off == head && head + size <= tail);
                    if (!fits)
                        break;
                } else {
                    off = 0;
                }
                for (int k = lane; ok && k < ncmd; k += 32) {
                    const uint4 cmd = cmd_at(k);
                    const uint32_t bytes = cmd.w & 0xffffffu;
                    ok = cmd.z + bytes <= size && cmd.z >= recb && ((cmd.x | cmd.z | bytes) & 15u) == 0u;
                }
            }
            ok = __all_sync(0xffffffffu, ok);
            const uint32_t full = gbar + kT2GsFull + 8 * slot;
            if (!ok) {
                if (lane == 0) {
                    set_error(Pm.err, kErrBadGroup);
                    *abort_flag = 1;
                    item_off[slot] = 0u;
                    mbar_arrive(full);   // wake the group; it sees the abort flag
                }
                ++issued;
                break;
            }
            if (lane == 0) {
                item_off[slot] = off;
                mbar_arrive_expect_tx(full, tx);
                bulk_g2s(ring + off, prog, recb, full);
            }
            __syncwarp();
            for (int k = lane; k < ncmd; k += 32) {
                const uint4 cmd = cmd_at(k);
                const char *src = reinterpret_cast<const char *>(((uint64_t)cmd.y << 32) | cmd.x);
                bulk_g2s(ring + off + cmd.z, src, cmd.w & 0xffffffu, full);
            }
            // the window has been read: refill it with the program two packs ahead
            const int64_t o2 = *reinterpret_cast<const int64_t *>(w + offsetof(Tc2Hdr, next) + 8);
            __syncwarp();
            fetch_window(ws, pi + 2 < pe ? o2 : (int64_t)-1);
            head = off + size;
            ++issued;
            ++pi;
            o0 = o1;
            o1 = pi + 1 < pe ? o2 : (int64_t)-1;
            progress = true;
        }
        if (progress) {
            idle_since = global_ns();
        } else if (global_ns() - idle_since > kWaitLimitNs) {
            if (lane == 0) {
                set_error(Pm.err, kErrTimeoutEmpty);
                *abort_flag = 1;
            }
        } else {
            __nanosleep(32);
        }
    }
    // copies still in flight target this CTA's shared memory: wait for the
    // group's last packs (it has consumed the others)
    const int first = issued > kT2Inflight ? issued - kT2Inflight : 0;
    for (int k = first; k < issued; ++k)
        if (!t2_wait(gbar + kT2GsFull + 8 * (k % kT2Inflight), (uint32_t)((k / kT2Inflight) & 1)) && lane == 0)
            set_error(Pm.err, kErrTimeoutFull);
}

template <int P>
__global__ void __launch_bounds__(kT2Threads, 1) tc2_kernel(const __grid_constant__ Tc2Params Pm)
{
    extern __shared__ __align__(1024) char sm2[];
    const uint32_t sb = smem_addr(sm2);
    const int warp = (int)(threadIdx.x >> 5), lane = (int)lane_id();
    const int g = warp >> 2, q = warp & 3;
    const int tid = (int)threadIdx.x & 127;
    const bool producer = warp >= 4 * kT2Groups;   // warp 16 + g feeds group g
    if (threadIdx.x < kT2Groups * 16) {
        // group threadIdx.x / 16: barriers 0-3 full, 4-7 empty, 8-9 window, 10 MMA
        const int gq = (int)threadIdx.x >> 4, b = (int)threadIdx.x & 15;
        const uint32_t base = sb + (uint32_t)(gq * kT2GroupState);
        if (b < 4)
            mbar_init(base + kT2GsFull + 8 * b, 1);
        else if (b < 8)
            mbar_init(base + kT2GsEmpty + 8 * (b - 4), 1);
        else if (b < 10)
            mbar_init(base + kT2GsWin + 8 * (b - 8), 1);
        else if (b == 10)
            mbar_init(base + kT2GsMma, 1);
        else if (b == 11)
            *reinterpret_cast<volatile int32_t *>(sm2 + gq * kT2GroupState + kT2GsAbort) = 0;
    }
    fence_barrier_init();
    if (warp == 0)
        tmem_alloc(sb + kT2TmemSlot, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (producer) {
        t2_producer<P>(Pm, sm2, sb, warp - 4 * kT2Groups, lane);
    } else {
        const int gg = (int)blockIdx.x * kT2Groups + g;
        char *gstate = sm2 + g * kT2GroupState;
        const uint32_t gbar = sb + (uint32_t)(g * kT2GroupState);
        const uint32_t bar_mma = gbar + kT2GsMma;
        volatile int32_t *abort_flag = reinterpret_cast<volatile int32_t *>(gstate + kT2GsAbort);
        volatile uint32_t *item_off = reinterpret_cast<volatile uint32_t *>(gstate + kT2GsOff);
        const uint32_t tmem = *reinterpret_cast<volatile uint32_t *>(sm2 + kT2TmemSlot) + (uint32_t)(g * kT2Cols);
        char *ops = sm2 + kT2Ops + g * t2_buf_bytes<P>();
        const uint32_t ops_addr = smem_addr(ops);
        constexpr uint32_t RING = (uint32_t)t2_ring_bytes<P>();
        char *ring = sm2 + t2_ring_off<P>() + g * (int)RING;
        const int npk = gg < Pm.ngroups ? Pm.gbeg[gg + 1] - Pm.gbeg[gg] : 0;
        uint32_t mma_n = 0;   // MMA commits so far
        for (int done = 0; done < npk; ++done) {
            // the pack's staging has landed (every lane acquires it itself)
            const int slot = done % kT2Inflight;
            if (!t2_wait(gbar + kT2GsFull + 8 * slot, (uint32_t)((done / kT2Inflight) & 1))) {
                if (lane == 0)
                    set_error(Pm.err, kErrTimeoutFull);
                *abort_flag = 1;
            }
            group_sync(g);
            if (*abort_flag)
                break;
            const char *item = ring + item_off[slot];
            const Tc2Hdr &h = *reinterpret_cast<const Tc2Hdr *>(item);
            const int ntasks = h.ntasks, kpack = h.kpack, nt = h.nt;
            const int nch = kpack > 0 ? (kpack + kT2KC - 1) / kT2KC : 0;
            bool ok = true;
            for (int c = 0; c < nch; ++c) {
                if (c > 0 && !t2_wait(bar_mma, (mma_n - 1) & 1u)) {   // chunk c - 1 has read the operands
                    ok = false;
                    if (lane == 0)
                        set_error(Pm.err, kErrTimeoutFull);
                }
                t2_convert<P>(item, ntasks, ops, c, tid);
                fence_proxy_async();
                tc_fence_before();
                group_sync(g);
                if (tid == 0) {
                    tc_fence_after();
                    t2_mma<P>(ops_addr, tmem, nt, min(kT2KC, kpack - c * kT2KC), c == 0 ? 0u : 1u);
                    tc_commit(bar_mma);
                }
                ++mma_n;
            }
            if (nch > 0) {
                if (!t2_wait(bar_mma, (mma_n - 1) & 1u)) {
                    ok = false;
                    if (lane == 0)
                        set_error(Pm.err, kErrTimeoutFull);
                }
                tc_fence_after();
            }
            if (__all_sync(0xffffffffu, ok))
                t2_epilogue(item, ntasks, tmem, q, lane, nch > 0);
            else
                *abort_flag = 1;
            tc_fence_before();
            group_sync(g);   // the pack's accumulator and staging are free
            if (tid == 0)
                mbar_arrive(gbar + kT2GsEmpty + 8 * slot);
            if (*abort_flag)
                break;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        tmem_dealloc(*reinterpret_cast<volatile uint32_t *>(sm2 + kT2TmemSlot), 512);
}

}  // namespace iaat
