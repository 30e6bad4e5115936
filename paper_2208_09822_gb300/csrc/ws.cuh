// Warp-stream grouped small-GEMM kernel on the CUDA cores (FP32 FFMA): the
// "kernel executing plan" of Sec. V-B with every warp its own pipeline.
//
// The planner cuts every instance into warp tasks -- one warp block of C
// (at most 32 x 32, one register-tile variant of the kernel family, the
// input-aware choice of Sec. V-A) with the instance's whole K -- and deals
// them to the warps of the grid ahead of time, largest first, each to the
// least loaded warp (so the persistent launch needs no atomics and replays
// from a CUDA graph unchanged).  Each warp then streams its own task list
// through a private ring of shared memory:
//
//  * an item is one K-chunk (16 values of k) of one task: the task record,
//    op(A) rows x 16 and 16 x op(B) columns, and with the task's last chunk
//    its C block.  The warp's lanes copy the elements one by one with 4-byte
//    cp.async straight into the layout the register tile reads (K-chunk
//    rows, XOR-swizzled 16-byte groups), so the copy is also the re-pack and
//    the paper's "no packing" holds: nothing is written twice.  Rows and
//    columns past the block are never written (their results are never
//    stored); only the K padding of the last chunk is zeroed.
//  * up to kWsMaxOut items are in flight per warp (cp.async groups), so about
//    sixteen warps x a few KB per SM keep HBM busy; items are released in
//    order, and the ring space of an item is reused as soon as it is
//    computed -- there is no hand-off between warps and no barrier.
//  * the k-loop is Algorithm 1's rank-1 update on an MR x NR register tile
//    per lane (16-byte shared loads, FMAs, no bounds checks), and the
//    epilogue writes alpha*acc + beta*C0 back into the staged C block, then
//    stores the block column by column with consecutive lanes on consecutive
//    rows (coalesced).
//
// There are no spin waits: cp.async.wait_group only waits for the warp's own
// copies.  A malformed task record sets the plan's error word and is skipped.
#pragma once
#include "grouped.cuh"

namespace iaat {

// Run-time description of a variant for the copy side (the compute side
// has it as template arguments): block height and width; the A / B swizzle
// masks (16-byte group g of K-chunk row kk holds group g ^ (kk & mask));
// and the C-block swizzle, element (i, j) at j*32 + (i ^ s(j)) with
// s(j) = ((l & m0) << p0) | ((l >> q1) << p1), l = j >> nrs (the lane column
// that owns column j), chosen so that the 32 lanes of one epilogue access
// hit 32 different banks.
struct WsVarRt {
    uint8_t bm, bn, ga, gb, nrs, m0, p0, q1, p1, pad[3];
};

// per variant of kVariantsF32: 32x32, 32x16, 16x32, 16x16, 8x8
__constant__ WsVarRt c_ws_var[kNumVariantsF32] = {
    {32, 32, 7, 7, 3, 3, 0, 2, 0, {0, 0, 0}},
    {32, 16, 7, 3, 2, 3, 0, 2, 0, {0, 0, 0}},
    {16, 32, 3, 7, 2, 3, 0, 2, 4, {0, 0, 0}},
    {16, 16, 3, 3, 2, 1, 4, 1, 0, {0, 0, 0}},
    {8, 8, 1, 1, 1, 3, 3, 2, 0, {0, 0, 0}},
};

// ceil(65536 / L), L = 1..32: floor(x / L) = (x * magic) >> 16 for x < 2048.
__constant__ uint32_t c_ws_magic[33] = {
    0,     65536, 32768, 21846, 16384, 13108, 10923, 9363, 8192, 7282, 6554,
    5958,  5462,  5042,  4682,  4370,  4096,  3856,  3641, 3450, 3277, 3121,
    2979,  2850,  2731,  2622,  2521,  2428,  2341,  2260, 2185, 2115, 2048};

__device__ __forceinline__ uint32_t ws_sC(const WsVarRt &v, int j)
{
    const uint32_t l = (uint32_t)j >> v.nrs;
    return ((l & v.m0) << v.p0) | ((l >> v.q1) << v.p1);
}

// Compile-time twin of ws_sC for the variant <MR, NR, LM, LN>.
template <int MR, int NR, int LM, int LN>
__device__ __forceinline__ int ws_sC_ct(int lj)
{
    if constexpr (LM * MR == 32)
        return lj & 3;                                   // 32 x 32, 32 x 16
    else if constexpr (LM * MR == 16 && LN == 8)
        return (lj & 3) | ((lj >> 2) << 4);              // 16 x 32
    else if constexpr (LM * MR == 16)
        return ((lj & 1) << 4) | (lj >> 1);              // 16 x 16
    else
        return lj << 3;                                  // 8 x 8
}

// Copy a region of 4-byte elements into shared memory.  x runs along the
// region's contiguous direction in global memory (L <= 32 elements, 4 bytes
// apart), y along the other (Y lines, sy bytes apart); the warp covers
// floor(32 / L) lines per instruction, consecutive lanes on consecutive x.
template <class F>
__device__ __forceinline__ void ws_copy(const char *src, int L, int Y, int64_t sy, int lane, F dst)
{
    if (L <= 0 || Y <= 0)
        return;
    const uint32_t mg = c_ws_magic[L];
    const int yl = (int)(((uint32_t)lane * mg) >> 16);
    const int step = (int)((32u * mg) >> 16);
    if (yl >= step)
        return;
    const int xl = lane - yl * L;
    const char *s = src + (int64_t)xl * 4 + (int64_t)yl * sy;
    const int64_t ds = (int64_t)step * sy;
#pragma unroll 2
    for (int y = yl; y < Y; y += step, s += ds)
        cp_async4(dst(xl, y), s);
}

// Bytes of the ring item holding chunk c (of nch) of a task of variant vr.
__device__ __forceinline__ uint32_t ws_item_bytes(const WsVarRt &vr, int K, int c, int nch)
{
    uint32_t b = kWsHdr;
    if (K > 0) {
        const int kc = min(kWsKC, K - c * kWsKC);
        b += (uint32_t)((kc + 3) & ~3) * (vr.bm + vr.bn) * 4u;
    }
    if (c == nch - 1)
        b += (uint32_t)kWsCStride * vr.bn * 4u;
    return b;
}

// Issue the copies of chunk c (of nch) of task t into the item at shared
// address `item`; `g` is the task's record in global memory.
__device__ __forceinline__ void ws_issue(const WsTask &t, const WsTask *g, int c, int nch, uint32_t item, int lane)
{
    if (lane < 4)
        cp_async16(item + 16u * lane, reinterpret_cast<const char *>(g) + 16 * lane);
    const WsVarRt vr = c_ws_var[t.variant];
    const int K = t.K, mh = t.M, nw = t.N;
    const bool last = c == nch - 1;
    int kc = 0, kcp = 0;
    if (K > 0) {
        kc = min(kWsKC, K - c * kWsKC);
        kcp = (kc + 3) & ~3;
    }
    if (lane == 0)
        st_shared_v4(item + 64, c, kcp, last ? 1 : 0, 0);
    const uint32_t aS = item + kWsHdr;
    const uint32_t bS = aS + (uint32_t)kcp * vr.bm * 4u;
    const uint32_t cS = bS + (uint32_t)kcp * vr.bn * 4u;
    const int bm = vr.bm, bn = vr.bn, ga = vr.ga, gb = vr.gb;
    auto dA = [&](int m, int kk) { return aS + 4u * (uint32_t)(kk * bm + (m ^ ((kk & ga) << 2))); };
    auto dB = [&](int n, int kk) { return bS + 4u * (uint32_t)(kk * bn + (n ^ ((kk & gb) << 2))); };
    if (K > 0) {
        const int k0 = c * kWsKC;
        const int64_t la = (int64_t)t.lda * 4, lb = (int64_t)t.ldb * 4;
        // op(A)(i, k): A[i + k*lda] (N) or A[k + i*lda] (T)
        if (!t.ta)
            ws_copy(t.A + k0 * la, mh, kc, la, lane, [&](int x, int y) { return dA(x, y); });
        else
            ws_copy(t.A + (int64_t)k0 * 4, kc, mh, la, lane, [&](int x, int y) { return dA(y, x); });
        // op(B)(k, j): B[k + j*ldb] (N) or B[j + k*ldb] (T)
        if (!t.tb)
            ws_copy(t.B + (int64_t)k0 * 4, kc, nw, lb, lane, [&](int x, int y) { return dB(y, x); });
        else
            ws_copy(t.B + k0 * lb, nw, kc, lb, lane, [&](int x, int y) { return dB(x, y); });
        // the K padding of the last chunk: zeros in the real rows / columns
        const int pk = kcp - kc;
        if (pk > 0) {
            const uint32_t ma = c_ws_magic[mh], mb = c_ws_magic[nw];
            for (int e = lane; e < pk * mh; e += 32) {
                const int q = (int)(((uint32_t)e * ma) >> 16);
                st_shared_u32(dA(e - q * mh, kc + q), 0u);
            }
            for (int e = lane; e < pk * nw; e += 32) {
                const int q = (int)(((uint32_t)e * mb) >> 16);
                st_shared_u32(dB(e - q * nw, kc + q), 0u);
            }
        }
    }
    if (last && (t.flags & kFlagReadC))
        ws_copy(t.C, mh, nw, (int64_t)t.ldc * 4, lane,
                [&](int i, int j) { return cS + 4u * (uint32_t)(j * kWsCStride + (i ^ (int)ws_sC(vr, j))); });
}

// One K-chunk of a warp block: kcp (a multiple of 4) rank-1 updates of the
// lane's MR x NR tile from the staged, swizzled chunk rows.
template <int MR, int NR, int LM, int LN>
__device__ __forceinline__ void ws_chunk(float (&acc)[32], const float *As, const float *Bs, int kcp, int li, int lj)
{
    constexpr int BM = LM * MR, BN = LN * NR;
    constexpr int VE = 4;
#pragma unroll 1
    for (int kk0 = 0; kk0 < kcp; kk0 += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int kk = kk0 + u;
            const float *arow = As + kk * BM;
            const float *brow = Bs + kk * BN;
            float av[MR], bv[NR];
            if constexpr (MR >= VE) {
#pragma unroll
                for (int q = 0; q < MR / VE; ++q) {
                    const float4 t4 = *reinterpret_cast<const float4 *>(arow + swz<BM, VE>(li * MR + q * VE, kk));
                    av[q * 4 + 0] = t4.x; av[q * 4 + 1] = t4.y; av[q * 4 + 2] = t4.z; av[q * 4 + 3] = t4.w;
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
                    const float4 t4 = *reinterpret_cast<const float4 *>(brow + swz<BN, VE>(lj * NR + q * VE, kk));
                    bv[q * 4 + 0] = t4.x; bv[q * 4 + 1] = t4.y; bv[q * 4 + 2] = t4.z; bv[q * 4 + 3] = t4.w;
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
                    acc[a * NR + b] = fmaf(av[a], bv[b], acc[a * NR + b]);
        }
    }
}

// Epilogue of a warp block: alpha*acc + beta*C0 into the staged C block
// (C0 read there when beta != 0), then the block stored column by column.
template <int MR, int NR, int LM, int LN>
__device__ __forceinline__ void ws_epilogue(const float (&acc)[32], float *Cs, const WsTask &r, const WsVarRt &vr,
                                            int li, int lj, int lane)
{
    const int mh = r.M, nw = r.N;
    const float alpha = r.alpha, beta = r.beta;
    const bool readc = (r.flags & kFlagReadC) != 0;
    const int s = ws_sC_ct<MR, NR, LM, LN>(lj);
#pragma unroll
    for (int b = 0; b < NR; ++b) {
        const int j = lj * NR + b;
#pragma unroll
        for (int a = 0; a < MR; ++a) {
            const int i = li * MR + a;
            if (i < mh && j < nw) {
                float *p = Cs + j * kWsCStride + (i ^ s);
                float v = alpha * acc[a * NR + b];
                if (readc)
                    v = fmaf(beta, *p, v);
                *p = v;
            }
        }
    }
    __syncwarp();
    float *Cg = reinterpret_cast<float *>(r.C);
    const int64_t ldc = r.ldc;
    const uint32_t mg = c_ws_magic[mh];
    const int n = mh * nw;
    for (int e = lane; e < n; e += 32) {
        const int j = (int)(((uint32_t)e * mg) >> 16);
        const int i = e - j * mh;
        __stcs(Cg + i + j * ldc, Cs[j * kWsCStride + (i ^ (int)ws_sC(vr, j))]);
    }
}

template <int MR, int NR, int LM, int LN>
__device__ __forceinline__ void ws_item(float (&acc)[32], char *item, const WsTask &r, const WsVarRt &vr, int kcp,
                                        bool first, bool last, int lane)
{
    constexpr int BM = LM * MR, BN = LN * NR;
    const int li = lane % LM, lj = lane / LM;
    if (first) {
#pragma unroll
        for (int e = 0; e < 32; ++e)
            acc[e] = 0.0f;
    }
    const float *As = reinterpret_cast<const float *>(item + kWsHdr);
    const float *Bs = As + kcp * BM;
    if (kcp > 0)
        ws_chunk<MR, NR, LM, LN>(acc, As, Bs, kcp, li, lj);
    if (last)
        ws_epilogue<MR, NR, LM, LN>(acc, const_cast<float *>(Bs + kcp * BN), r, vr, li, lj, lane);
}

__device__ __forceinline__ bool ws_task_ok(const WsTask &t)
{
    if (t.variant >= kNumVariantsF32)
        return false;
    const WsVarRt vr = c_ws_var[t.variant];
    return t.M >= 1 && t.M <= vr.bm && t.N >= 1 && t.N <= vr.bn && t.K >= 0;
}

__global__ void __launch_bounds__(kWsThreads, 1) ws_kernel(const __grid_constant__ WsParams P)
{
    extern __shared__ __align__(128) char smem_ws[];
    const int wic = (int)(threadIdx.x >> 5);
    const int lane = (int)lane_id();
    const int w = blockIdx.x * kWsWarps + wic;
    if (w >= P.nwarps)
        return;
    int ti = P.wbeg[w];
    const int te = P.wbeg[w + 1];
    char *ring = smem_ws + wic * kWsRingBytes;
    const uint32_t rs = smem_addr(ring);

    // issue side: the record of task ti (pt) and of ti + 1 (pn, loaded ahead)
    WsTask pt{}, pn{};
    if (ti < te)
        pt = P.tasks[ti];
    if (ti + 1 < te)
        pn = P.tasks[ti + 1];
    int pc = 0;                      // next chunk of task ti to issue
    uint32_t head = 0;               // ring offset after the newest item
    int issued = 0, consumed = 0;
    uint32_t qoff = 0;               // lane q: ring offset of item q (mod 32)
    float acc[32];
#pragma unroll
    for (int e = 0; e < 32; ++e)
        acc[e] = 0.0f;

    for (;;) {
        // issue items while fewer than kWsMaxOut are in flight and the ring has room
        while (issued - consumed < kWsMaxOut && ti < te) {
            if (!ws_task_ok(pt)) {
                if (lane == 0)
                    atomicOr(P.err, kErrBadGroup);
                pc = 0;
                ++ti;
                pt = pn;
                if (ti + 1 < te)
                    pn = P.tasks[ti + 1];
                continue;
            }
            const WsVarRt vr = c_ws_var[pt.variant];
            const int nch = pt.K > 0 ? (pt.K + kWsKC - 1) / kWsKC : 1;
            const uint32_t size = ws_item_bytes(vr, pt.K, pc, nch);
            uint32_t off = head + size <= (uint32_t)kWsRingBytes ? head : 0u;
            if (issued > consumed) {
                const uint32_t tail = __shfl_sync(0xffffffffu, qoff, consumed & 31);
                const bool ok = head > tail ? (off == head || size <= tail) : (off == head && head + size <= tail);
                if (!ok)
                    break;
            } else {
                off = 0;
            }
            ws_issue(pt, P.tasks + ti, pc, nch, rs + off, lane);
            cp_async_commit();
            if (lane == (issued & 31))
                qoff = off;
            head = off + size;
            ++issued;
            if (++pc == nch) {
                pc = 0;
                ++ti;
                pt = pn;
                if (ti + 1 < te)
                    pn = P.tasks[ti + 1];
            }
        }
        if (consumed == issued)
            break;
        // consume the oldest item
        const uint32_t off = __shfl_sync(0xffffffffu, qoff, consumed & 31);
        cp_async_wait_upto(issued - consumed - 1);
        __syncwarp();
        char *item = ring + off;
        const WsTask &r = *reinterpret_cast<const WsTask *>(item);
        const int4 meta = *reinterpret_cast<const int4 *>(item + 64);
        const int v = r.variant;
        const WsVarRt vr = c_ws_var[v];
        const bool first = meta.x == 0, last = meta.z != 0;
        const int kcp = meta.y;
        switch (v) {
#define IAAT_WS_V(id)                                                                                          \
    case id:                                                                                                   \
        ws_item<kVariantsF32[id].mr, kVariantsF32[id].nr, kVariantsF32[id].lm, kVariantsF32[id].ln>(          \
            acc, item, r, vr, kcp, first, last, lane);                                                         \
        break;
            IAAT_WS_V(0) IAAT_WS_V(1) IAAT_WS_V(2) IAAT_WS_V(3) IAAT_WS_V(4)
#undef IAAT_WS_V
        default:
            break;
        }
        __syncwarp();
        ++consumed;
    }
}

}  // namespace iaat
