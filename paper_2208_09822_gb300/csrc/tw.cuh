// Warp-tile grouped small-GEMM kernel on the tcgen05 tensor cores, FP32 in
// and out (3xBF16 split products, TF32, FP16 or 6xBF16 inputs; FP32
// accumulation in tensor memory): the kernel executing plan of Sec. V-B with
// every warp its own pipeline.
//
// The planner cuts every instance into warp tasks -- blocks of at most
// kTwBlockM x kTwBlockN (32 x 32) of C, each with the instance's whole K --
// and deals them to the warps of the grid ahead of time, largest first, each
// to the least loaded warp.  A warp then runs its list alone; no other warp
// waits for it:
//
//  * staging: the warp's lanes copy each task's raw operands into the warp's
//    private ring with 16-byte cp.async (L2 to shared memory), as runs --
//    the contiguous stretches of the stored columns, each as the 16-byte
//    granules that cover it -- or, where the ld padding is small, as one span
//    over all of them, cut by K into items that fit half the ring,
//    up to kTwMaxOut items ahead of the one being computed, each item one
//    cp.async group;
//  * convert, per K-chunk of 16: lane i turns row i of the block's op(A)
//    into its split terms (Xh, Xl BF16 for 3xBF16) and stores them into
//    tensor memory (tcgen05.st, lane i of the warp's lane quarter); the lanes
//    together turn the rows of op(B)^T into the canonical K-major layout
//    (core matrices of 8 rows x 16 bytes) of the warp's shared-memory tile,
//    only the block's real rows, zeros past K;
//  * MMA: lane 0 issues the chunk's tcgen05.mma (M = 128, A from tensor
//    memory, B from shared memory) into the warp's 32 accumulator columns
//    and commits them to the warp's mbarrier.  Warp w runs on SM
//    sub-partition w mod 4 and reaches only tensor-memory lanes 32(w mod 4)
//    .. +31, so its rows of op(A) are lane quarter w mod 4 of A columns that
//    the four warps of its quad share; the other quarters' products land in
//    accumulator lanes the warp never reads.  A in tensor memory keeps the
//    MMA's shared-memory reads to the B tile (a 128-row A tile read from
//    shared memory would take four times the bandwidth the staging needs);
//  * epilogue: lane i holds row i of the block (tcgen05.ld 32x32b) and writes
//    alpha*acc + beta*C0 column by column, consecutive lanes on consecutive
//    rows (coalesced), C0 from the staged C item.
//
// Every wait on the tensor core is bounded; a time-out or a malformed task
// record sets the plan's error word (the warp stops, or skips the task).
#pragma once
#include "tc.cuh"
#include "tw_types.cuh"

namespace iaat {

template <int P> IAAT_CE int tw_vpr() { return 16 / TcTraits<P>::kOpBytes; }       // values per core row
template <int P> IAAT_CE int tw_groups() { return kTwKC / tw_vpr<P>(); }          // core rows per tile row
template <int P> IAAT_CE int tw_sbo() { return tw_groups<P>() * 128; }            // 8-row group stride
template <int P> IAAT_CE int tw_tile() { return (kTwBlockN / 8) * tw_sbo<P>(); }  // the rows of op(B)^T, one term
template <int P> IAAT_CE int tw_region() { return kTwWarps * tw_tile<P>(); }      // one term of every warp
// tensor-memory columns of one chunk of op(A), one term (32-bit columns)
template <int P> IAAT_CE int tw_acols() { return kTwKC * TcTraits<P>::kOpBytes / 4; }
// tensor memory: the warps' accumulators (kTwBlockN columns each), then per
// quad of warps the A columns of every term
constexpr int kTwAccCols = kTwBlockN * kTwWarps;
template <int P> IAAT_CE int tw_tmem_cols() { return kTwAccCols + (kTwWarps / 4) * TcTraits<P>::kTerms * tw_acols<P>(); }
constexpr uint32_t kTwTmemAlloc = 512;
// shared memory: the warps' mbarriers and the tensor-memory slot, then the
// B tiles (one region per term), the warps' task-record rings, the warps'
// staging rings
constexpr int kTwCtl = 2048;
constexpr int kTwItemBars = 1024;   // per warp kTwMaxOut mbarriers: staging item i landed (slot i mod kTwMaxOut)
constexpr int kTwRecSlots = 32;   // task records a warp holds (a power of two)
constexpr int kTwRecAhead = 9;    // records are copied this many tasks ahead of their staging
template <int P> IAAT_CE int tw_opB() { return kTwCtl; }
template <int P> IAAT_CE int tw_rec_off() { return kTwCtl + TcTraits<P>::kTerms * tw_region<P>(); }
template <int P> IAAT_CE int tw_ring_off() { return tw_rec_off<P>() + kTwWarps * kTwRecSlots * 64; }
template <int P> IAAT_CE int tw_ring() { return ((kSmemTotal - tw_ring_off<P>()) / kTwWarps) & ~127; }
static_assert(kTwWarps % 4 == 0 && kTwBlockM == 32 && (kTwBlockN == 16 || kTwBlockN == 32),
              "quads of warps, one lane quarter per block, MMA N of 16 or 32");
static_assert(tw_tmem_cols<kTc6xBF16>() <= (int)kTwTmemAlloc && tw_tmem_cols<kTcTF32>() <= (int)kTwTmemAlloc,
              "tensor-memory columns");
static_assert(kTwMaxOut == 8, "queue slots in lanes 0..7");
static_assert(kTwItemBars + kTwWarps * kTwMaxOut * 8 <= kTwCtl, "control area");
// The record of task t is copied in the cp.async group of task t - 9's first
// item.  When task t is begun, at most kTwMaxOut items are in flight and the
// first items of tasks t-8 .. t-1 came after that one, so the consumer has
// already waited for its group; the slot is reused for task t + 32, copied
// with task t + 23's first item, once the consumer is at least 16 items past
// task t's first one.
static_assert(kTwRecAhead > kTwMaxOut && kTwRecSlots >= kTwRecAhead + 2 * kTwMaxOut + 1 &&
                  (kTwRecSlots & (kTwRecSlots - 1)) == 0,
              "record ring");

constexpr uint32_t kTwFirst = 1;   // the task's first item
constexpr uint32_t kTwCItem = 2;   // the item holds the staged C block
constexpr uint32_t kTwEpi = 4;     // the block's epilogue follows this item

// Copy R runs of X bytes, run r starting at global address src + r*S, as the
// 16-byte granules covering each: run r's granules go to dst + r*D
// (D = tw_run_slot(X)), so its first element lands at dst + r*D +
// ((src + r*S) & 15).  Lane e of every 32 takes granule slot e: run
// floor(e / L), granule e mod L (L = D / 16), the quotient taken in FP32 --
// exact: (e + 1/2) / L is at least 1/(2L) from an integer, and with a
// reciprocal good to 2 ulp the product's relative error stays below 2^-21,
// so for e < 2^20 the floor is right.
__device__ __forceinline__ void tw_copy_runs(uint32_t dst, const char *src, int64_t S, int R, int X, int lane)
{
    const int L = (X + 27) >> 4;
    const int n = R * L;
    const float inv = __fdividef(1.0f, (float)L);
    for (int e = lane; e < n; e += 32) {
        const int r = (int)(((float)e + 0.5f) * inv);
        const int g = e - r * L;
        const uintptr_t s = reinterpret_cast<uintptr_t>(src) + (uintptr_t)((int64_t)r * S);
        if (g < (int)(((s & 15u) + (uintptr_t)X + 15u) >> 4))
            cp_async16(dst + 16u * (uint32_t)e,
                       reinterpret_cast<const void *>((s & ~(uintptr_t)15) + 16u * (uint32_t)g));
    }
}

// The 16-byte granules that cover `bytes` bytes from global address src:
// their aligned start, and their count times 16.
__device__ __forceinline__ void tw_span_granules(const char *src, int64_t bytes, const char **a, uint32_t *n)
{
    const uintptr_t s = reinterpret_cast<uintptr_t>(src);
    *a = reinterpret_cast<const char *>(s & ~(uintptr_t)15);
    *n = (uint32_t)((((int64_t)(s & 15u) + bytes + 15) >> 4) << 4);
}

// The task the warp is computing, from the record at the start of its first item.
struct TwCur {
    const char *A, *B;
    float *C;
    int lda, ldb, ldc, K, M, N, ta, tb, readc, flags;
    float alpha, beta;
};

__device__ __forceinline__ TwCur tw_read_record(const char *rec)
{
    const TwTask &t = *reinterpret_cast<const TwTask *>(rec);
    TwCur c;
    c.A = t.A;
    c.B = t.B;
    c.C = reinterpret_cast<float *>(t.C);
    c.lda = t.lda;
    c.ldb = t.ldb;
    c.ldc = t.ldc;
    c.K = t.K;
    c.M = t.M;
    c.N = t.N;
    c.ta = t.ta;
    c.tb = t.tb;
    c.readc = (t.flags & kFlagReadC) != 0;
    c.flags = t.flags;
    c.alpha = t.alpha;
    c.beta = t.beta;
    return c;
}

// Staged operand geometry of one item.  krun: the stored runs go along k (one
// per k), element (row, k) at sec + k*D + mis(k) + 4*row; otherwise one run
// per row, element (row, k) at sec + row*D + mis(row) + 4*k; mis(r) =
// (b0 + r*s16) & 15, k relative to the item's K range.  Staged run by run:
// D = tw_run_slot(4 len), s16 = 4 ld mod 16; as one span: D = 4 ld, s16 = 0.
// Chunks and core rows start at multiples of 4 runs, and 4*s16 is a multiple
// of 16, so the offsets of the values of a core row repeat from one to the
// next.
struct TwSide {
    const char *sec;
    int D, b0, s16;
    bool krun;
};

// 16 tensor-memory columns of this warp's lane quarter from r[0..N-1]
template <int N>
__device__ __forceinline__ void tmem_st(uint32_t taddr, const uint32_t *r)
{
    if constexpr (N == 8) {
        asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
                     "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                     : "memory");
    } else {
        static_assert(N == 16, "tcgen05.st width");
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::
                "r"(taddr),
            "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
            "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
            : "memory");
    }
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Row `lane` of op(A), K-chunk [kc, kc + 16) of the item's kl values, split
// into its terms and stored into the quad's A columns at `ta_addr` (lane
// quarter of this warp; term h tw_acols() columns further on).  Two values
// per column for 16-bit terms (the lower k in the low half), one for TF32.
// Every lane stores (the instruction is warp-wide); rows past M store
// whatever they computed, into accumulator rows nobody reads.
template <int P>
__device__ __forceinline__ void tw_convert_a(const TwSide &s, int M, int kc, int kl, uint32_t ta_addr, int lane)
{
    constexpr int AC = tw_acols<P>();
    float x[kTwKC];
    const int row = lane < M ? lane : 0;
    const char *p = s.krun ? s.sec + kc * s.D + 4 * row : s.sec + row * s.D + ((s.b0 + row * s.s16) & 15) + 4 * kc;
#pragma unroll
    for (int v = 0; v < kTwKC; ++v)
        x[v] = kc + v < kl ? *reinterpret_cast<const float *>(p + (s.krun ? v * s.D + ((s.b0 + v * s.s16) & 15) : 4 * v))
                           : 0.0f;
    if constexpr (P == kTcTF32) {
        uint32_t w[16];
#pragma unroll
        for (int v = 0; v < 16; ++v)
            w[v] = tf32_rn(x[v]);
        tmem_st<16>(ta_addr, w);
    } else if constexpr (P == kTcFP16) {
        uint32_t w[8];
#pragma unroll
        for (int c = 0; c < 8; ++c)
            w[c] = pack_f16(x[2 * c], x[2 * c + 1]);
        tmem_st<8>(ta_addr, w);
    } else {
        uint32_t h[8], m[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            h[c] = pack_bf16(x[2 * c], x[2 * c + 1]);
            x[2 * c] -= __uint_as_float(h[c] << 16);
            x[2 * c + 1] -= __uint_as_float(h[c] & 0xffff0000u);
            m[c] = pack_bf16(x[2 * c], x[2 * c + 1]);
        }
        tmem_st<8>(ta_addr, h);
        tmem_st<8>(ta_addr + AC, m);
        if constexpr (P == kTc6xBF16) {
            uint32_t l[8];
#pragma unroll
            for (int c = 0; c < 8; ++c)
                l[c] = pack_bf16(x[2 * c] - __uint_as_float(m[c] << 16),
                                 x[2 * c + 1] - __uint_as_float(m[c] & 0xffff0000u));
            tmem_st<8>(ta_addr + 2 * AC, l);
        }
    }
}

// K-chunk [kc, kc + 16) of the rows of op(B)^T (rows = N of them) into the
// warp's canonical tiles t0.. (one per term); the lanes share the (row, core
// row) work items.
template <int P>
__device__ __forceinline__ void tw_convert_b(const TwSide &s, int rows, int kc, int kl, char *t0, char *t1, char *t2,
                                             int lane)
{
    constexpr int V = tw_vpr<P>();
    constexpr int G = tw_groups<P>();
    constexpr int LG = G == 2 ? 1 : (G == 4 ? 2 : 0);
    static_assert((1 << LG) == G, "core rows per tile row");
    constexpr int SBO = tw_sbo<P>();
    int o[V];
#pragma unroll
    for (int v = 0; v < V; ++v)
        o[v] = s.krun ? v * s.D + ((s.b0 + v * s.s16) & 15) : 4 * v;
    const int n = rows * G;
    for (int e = lane; e < n; e += 32) {
        const int row = e >> LG, g = e & (G - 1);
        const int k = kc + g * V;   // first k of this core row
        const char *p = s.krun ? s.sec + k * s.D + 4 * row : s.sec + row * s.D + ((s.b0 + row * s.s16) & 15) + 4 * k;
        float x[8];
#pragma unroll
        for (int v = 0; v < V; ++v)
            x[v] = k + v < kl ? *reinterpret_cast<const float *>(p + o[v]) : 0.0f;
        store_row<P>(t0, t1, t2, (uint32_t)((row >> 3) * SBO + (row & 7) * 16 + g * 128), x);
    }
}

template <int P>
__device__ __forceinline__ void tw_mma1(uint32_t dtmem, uint32_t atmem, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    if constexpr (P == kTcTF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(dtmem),
            "r"(atmem), "l"(bdesc), "r"(idesc), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(dtmem),
            "r"(atmem), "l"(bdesc), "r"(idesc), "r"(acc)
            : "memory");
    }
}

// The MMAs of one K-chunk: A from the quad's tensor-memory columns `at`
// (term h tw_acols() columns further on), B from the warp's tile at `bw`
// (term h tw_region() bytes further on).
template <int P>
__device__ __forceinline__ void tw_mma(uint32_t at, uint32_t bw, uint32_t dtmem, int nt, uint32_t accum)
{
    constexpr int KS = TcTraits<P>::kKStep;
    constexpr uint32_t SBO = (uint32_t)tw_sbo<P>();
    constexpr uint64_t TS = (uint64_t)tw_region<P>() >> 4;   // term stride in descriptor units
    constexpr uint32_t AC = (uint32_t)tw_acols<P>();
    constexpr uint32_t ASTEP = (uint32_t)(KS * TcTraits<P>::kOpBytes / 4);   // A columns per K step
    const uint32_t idesc = tc_idesc<P>(nt);
    uint64_t db0 = smem_desc(bw, 128, SBO);
    uint64_t db1 = db0 + TS, db2 = db1 + TS;
    uint32_t a0 = at, a1 = at + AC, a2 = at + 2 * AC;
#pragma unroll
    for (int ks = 0; ks < kTwKC / KS; ++ks) {
        if constexpr (P == kTc6xBF16) {
            tw_mma1<P>(dtmem, a1, db1, idesc, accum);
            tw_mma1<P>(dtmem, a2, db0, idesc, 1u);
            tw_mma1<P>(dtmem, a0, db2, idesc, 1u);
            tw_mma1<P>(dtmem, a1, db0, idesc, 1u);
            tw_mma1<P>(dtmem, a0, db1, idesc, 1u);
            tw_mma1<P>(dtmem, a0, db0, idesc, 1u);
        } else if constexpr (P == kTc3xBF16) {
            tw_mma1<P>(dtmem, a1, db0, idesc, accum);
            tw_mma1<P>(dtmem, a0, db1, idesc, 1u);
            tw_mma1<P>(dtmem, a0, db0, idesc, 1u);
        } else {
            tw_mma1<P>(dtmem, a0, db0, idesc, accum);
        }
        // one K step: two core matrices of B along K (256 bytes); ASTEP columns of A
        db0 += 16; db1 += 16; db2 += 16;
        a0 += ASTEP; a1 += ASTEP; a2 += ASTEP;
        accum = 1u;
    }
}

// Lane i (< M) writes row i of the block: alpha*acc + beta*C0, C0 from the
// staged C item (one run per column, or one span).
__device__ __forceinline__ void tw_epilogue(const TwCur &t, const char *citem, uint32_t taddr, bool product, int nt,
                                            int lane)
{
    uint32_t acc[32];
    if (product) {
        tmem_ld16<0>(taddr, acc);
        if (nt > 16)
            tmem_ld16<16>(taddr + 16u, acc);
        tmem_wait_ld(acc);
    } else {
#pragma unroll
        for (int j = 0; j < 32; ++j)
            acc[j] = 0u;
    }
    if (lane >= t.M)
        return;
    float *cp = t.C + lane;
    const int64_t ldc = t.ldc;
    // C0 is read only when beta != 0 (it may hold anything otherwise)
    const bool span = (t.flags & kTwSpanC) != 0;
    const int DC = span ? (int)(4 * ldc) : (int)tw_run_slot(4 * t.M);
    const int c0 = (int)(reinterpret_cast<uintptr_t>(t.C) & 15u), s16 = span ? 0 : (int)((4 * ldc) & 15);
    int mis[4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
        mis[u] = (c0 + u * s16) & 15;
    const char *sp = citem + 4 * lane;
    const float beta = t.readc ? t.beta : 0.0f;
    // eight columns at a time: their C0 loads issue together
#pragma unroll
    for (int j0 = 0; j0 < 32; j0 += 8) {
        if (j0 >= t.N)
            break;
        float c[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            c[u] = t.readc && j0 + u < t.N ? *reinterpret_cast<const float *>(sp + u * DC + mis[u & 3]) : 0.0f;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (j0 + u < t.N)
                __stcs(cp, fmaf(beta, c[u], t.alpha * __uint_as_float(acc[j0 + u])));
            cp += ldc;
        }
        sp += 8 * DC;
    }
}

template <int P>
__global__ void __launch_bounds__(kTwThreads, 1) tw_kernel(const TwParams p)
{
    extern __shared__ __align__(1024) char smem_tw[];
    char *const smem = smem_tw;
    constexpr uint32_t RING = (uint32_t)tw_ring<P>();
    constexpr int T = TcTraits<P>::kTerms;
    const int warp = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31u), q = warp & 3;
    const uint32_t sb = smem_addr(smem);
    const uint32_t bar = sb + 8u * (uint32_t)warp;
    if (threadIdx.x == 0) {
        for (int w = 0; w < kTwWarps; ++w)
            mbar_init(sb + 8u * (uint32_t)w, 1);
        // one arrival by lane 0 (with the bulk copies' byte count); the
        // lanes' cp.async copies are tracked by arrivals that add their own
        for (int i = 0; i < kTwWarps * kTwMaxOut; ++i)
            mbar_init(sb + (uint32_t)(kTwItemBars + 8 * i), 1);
        fence_barrier_init();
    }
    if (warp == 0)
        tmem_alloc(sb + 512u, kTwTmemAlloc);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t *>(smem + 512);
    const uint32_t lq = (uint32_t)(32 * q) << 16;                              // the warp's lane quarter
    const uint32_t dcol = tmem + (uint32_t)(kTwBlockN * warp);                 // its accumulator (MMA D)
    const uint32_t acol = tmem + (uint32_t)(kTwAccCols + (warp >> 2) * T * tw_acols<P>());   // its quad's A
    char *tB0 = smem + tw_opB<P>() + warp * tw_tile<P>();
    char *tB1 = tB0 + tw_region<P>(), *tB2 = tB1 + tw_region<P>();
    const uint32_t bw = sb + (uint32_t)(tw_opB<P>() + warp * tw_tile<P>());
    const char *ring = smem + tw_ring_off<P>() + warp * (int)RING;
    const uint32_t ring_s = sb + (uint32_t)tw_ring_off<P>() + (uint32_t)warp * RING;
    const uint32_t ibar = sb + (uint32_t)(kTwItemBars + 8 * kTwMaxOut * warp);   // + 8 * slot

    const int gw = (int)blockIdx.x * kTwWarps + warp;
    int it = 0, te = 0;
    if (gw < p.nwarps) {
        it = p.wbeg[gw];
        te = p.wbeg[gw + 1];
    }
    // the warp's record ring: task t's record in slot t mod kTwRecSlots
    const char *recs = smem + tw_rec_off<P>() + warp * kTwRecSlots * 64;
    const uint32_t recs_s = sb + (uint32_t)(tw_rec_off<P>() + warp * kTwRecSlots * 64);
    auto fetch_rec = [&](int t) {
        if (lane < 4 && t < te)
            cp_async16(recs_s + (uint32_t)((t & (kTwRecSlots - 1)) * 64 + 16 * lane),
                       reinterpret_cast<const char *>(p.tasks + t) + 16 * lane);
    };
    for (int r = 0; r < kTwRecAhead; ++r)
        fetch_rec(it + r);
    cp_async_commit();
    cp_async_wait<0>();
    __syncwarp();
    TwTask ir{};   // the task being staged
    int ireadc = 0, ikseg = 16, inseg = 1, iseg = 0;
    // take task it's record; false (and the error word set) for a record the kernel must refuse
    auto begin = [&]() -> bool {
        ir = *reinterpret_cast<const TwTask *>(recs + (it & (kTwRecSlots - 1)) * 64);
        ireadc = ir.flags & kFlagReadC;
        ikseg = 16 * (int)ir.kseg16;
        iseg = 0;
        inseg = ir.K > 0 && ikseg > 0 ? (ir.K + ikseg - 1) / ikseg : 1;
        const bool ok = ir.M >= 1 && ir.M <= kTwBlockM && ir.N >= 1 && ir.N <= kTwBlockN && ir.K >= 0 &&
                        ir.ta <= 1 && ir.tb <= 1 && (ir.K == 0 || ikseg > 0) && ir.lda > 0 && ir.ldb > 0 &&
                        ir.ldc > 0 && tw_ab_item_bytes(ir, ir.K < ikseg ? ir.K : ikseg) <= RING / 2 &&
                        tw_c_item_bytes(ir) <= RING / 2;
        if (!ok && lane == 0)
            set_error(p.err, kErrBadGroup);
        return ok;
    };
    // move past refused records: their later records' copies are in no
    // group the consumer waits for, so wait for every copy here (error path)
    auto skip_refused = [&]() {
        bool skipped = false;
        while (it < te && !begin()) {
            fetch_rec(it + kTwRecAhead);
            ++it;
            cp_async_commit();
            cp_async_wait<0>();
            __syncwarp();
            skipped = true;
        }
        return skipped;
    };
    skip_refused();

    uint32_t head = 0, hoff = 0, tail = 0;   // ring: bytes allocated and freed (monotonic), offset of head
    int issued = 0, consumed = 0;
    // in-flight items: slot s (= item number mod kTwMaxOut) in lane s
    uint32_t q_off = 0, q_end = 0, q_fl = 0;
    int q_k0 = 0, q_k1 = 0, q_t = 0;
    // Stage the next item of the current task if the ring has room for it.
    auto issue_one = [&]() -> bool {
        if (it >= te)
            return false;
        const bool citem = iseg == inseg;
        int k0 = 0, k1 = 0;
        uint32_t bytes;
        if (citem) {
            bytes = tw_c_item_bytes(ir);
        } else {
            k0 = iseg * ikseg;
            k1 = min(ir.K, k0 + ikseg);
            bytes = tw_ab_item_bytes(ir, k1 - k0);
        }
        uint32_t off = hoff, pad = 0;
        if (off + bytes > RING) {
            pad = RING - off;
            off = 0;
        }
        if (head + pad + bytes - tail > RING)
            return false;
        head += pad + bytes;
        hoff = off + bytes;
        uint32_t fl = 0;
        // the item's operand blocks (C; or op(A) then op(B)), one copy call site
        const int kl = k1 - k0;
        if (citem) {
            fl = kTwCItem | kTwEpi;
        } else {
            if (iseg == 0) {
                fl |= kTwFirst;
                fetch_rec(it + kTwRecAhead);
            }
            if (iseg == inseg - 1 && !ireadc)
                fl |= kTwEpi;
        }
        uint32_t d = ring_s + off;
        const int nops = citem ? 1 : (kl > 0 ? 2 : 0);
        // spans go as bulk copies issued by lane 0 below, runs as the lanes'
        // cp.async; item completion: the slot's mbarrier
        const char *bsrc[2] = {nullptr, nullptr};
        uint32_t bdst[2] = {0u, 0u}, bn[2] = {0u, 0u};
        for (int o = 0; o < nops; ++o) {
            const bool isb = o == 1;
            const int tr = citem ? 0 : (isb ? ir.tb : ir.ta);
            const int64_t ld = citem ? ir.ldc : (isb ? ir.ldb : ir.lda);
            const int rows = citem || !isb ? ir.M : ir.N;   // block rows of C / op(A), columns of op(B)
            const bool span = (ir.flags & (citem ? kTwSpanC : (isb ? kTwSpanB : kTwSpanA))) != 0;
            // runs along k: op(A) not transposed, op(B) transposed; else one run per row / column
            const bool krun = !citem && (isb ? tr != 0 : tr == 0);
            const char *base = citem ? ir.C : (isb ? ir.B : ir.A);
            const char *src = citem ? base : base + 4 * (krun ? (int64_t)k0 * ld : (int64_t)k0);
            const int R = citem ? ir.N : (krun ? kl : rows);
            const int len = citem ? ir.M : (krun ? rows : kl);
            if (R > 0 && len > 0) {
                if (span) {
                    tw_span_granules(src, 4 * ((int64_t)(R - 1) * ld + len), &bsrc[o], &bn[o]);
                    bdst[o] = d;
                } else {
                    tw_copy_runs(d, src, 4 * ld, R, 4 * len, lane);
                }
            }
            d += tw_op_bytes(R, len, ld, span);
        }
        const uint32_t bar_i = ibar + 8u * (uint32_t)(issued & (kTwMaxOut - 1));
        asm volatile("cp.async.mbarrier.arrive.shared::cta.b64 [%0];" ::"r"(bar_i) : "memory");
        __syncwarp();
        if (lane == 0) {
            mbar_arrive_expect_tx(bar_i, bn[0] + bn[1]);
            for (int o = 0; o < 2; ++o)
                if (bn[o])
                    bulk_g2s(bdst[o], bsrc[o], bn[o], bar_i);
        }
        if (lane == (issued & (kTwMaxOut - 1))) {
            q_off = off;
            q_end = head;
            q_k0 = k0;
            q_k1 = k1;
            q_fl = fl;
            q_t = it;
        }
        ++issued;
        if (++iseg == inseg + ireadc) {
            ++it;
            skip_refused();
        }
        return true;
    };

    TwCur cur{};
    uint32_t ph = 0;
    bool pending = false, abort = false;
    // wait for the warp's MMAs in flight (all lanes acquire; warp-uniform outcome)
    auto wait_mma = [&]() {
        if (pending) {
            if (!warp_wait(bar, ph)) {
                if (lane == 0)
                    set_error(p.err, kErrTimeoutFull);
                abort = true;
            }
            ph ^= 1u;
            pending = false;
        }
    };
    for (;;) {
        while (issued - consumed < kTwMaxOut && issue_one()) {
        }
        if (issued == consumed)
            break;
        const int s = consumed & (kTwMaxOut - 1);
        const uint32_t off = __shfl_sync(0xffffffffu, q_off, s), end = __shfl_sync(0xffffffffu, q_end, s);
        const uint32_t fl = __shfl_sync(0xffffffffu, q_fl, s);
        const int k0 = __shfl_sync(0xffffffffu, q_k0, s), k1 = __shfl_sync(0xffffffffu, q_k1, s);
        const int ct = __shfl_sync(0xffffffffu, q_t, s);
        if (!warp_wait(ibar + 8u * (uint32_t)s, (uint32_t)((consumed / kTwMaxOut) & 1))) {
            if (lane == 0)
                set_error(p.err, kErrTimeoutFull);
            abort = true;
            break;
        }
        const char *item = ring + off;
        if (!(fl & kTwCItem)) {
            const char *sec = item;
            if (fl & kTwFirst)
                cur = tw_read_record(recs + (ct & (kTwRecSlots - 1)) * 64);
            const int kl = k1 - k0;
            if (kl > 0) {
                TwSide a, b;
                a.krun = cur.ta == 0;
                b.krun = cur.tb != 0;
                a.sec = sec;
                const bool sa = (cur.flags & kTwSpanA) != 0, sbb = (cur.flags & kTwSpanB) != 0;
                b.sec = sec + tw_a_bytes(cur.ta, cur.M, kl, cur.lda, sa);
                a.D = sa ? 4 * cur.lda : (int)tw_run_slot(a.krun ? 4 * cur.M : 4 * kl);
                b.D = sbb ? 4 * cur.ldb : (int)tw_run_slot(b.krun ? 4 * cur.N : 4 * kl);
                a.b0 = (int)((reinterpret_cast<uintptr_t>(cur.A) +
                              (uintptr_t)(a.krun ? 4 * (int64_t)k0 * cur.lda : 4 * (int64_t)k0)) & 15u);
                b.b0 = (int)((reinterpret_cast<uintptr_t>(cur.B) +
                              (uintptr_t)(b.krun ? 4 * (int64_t)k0 * cur.ldb : 4 * (int64_t)k0)) & 15u);
                a.s16 = sa ? 0 : (4 * cur.lda) & 15;
                b.s16 = sbb ? 0 : (4 * cur.ldb) & 15;
                const int nt = cur.N > 16 ? 32 : 16;
                for (int kc = 0; kc < kl; kc += kTwKC) {
                    wait_mma();   // the A columns and the B tile are free once the last chunk's MMAs are done
                    if (abort)
                        break;
                    tc_fence_after();
                    tw_convert_a<P>(a, cur.M, kc, kl, acol + lq, lane);
                    tw_convert_b<P>(b, cur.N, kc, kl, tB0, tB1, tB2, lane);
                    tmem_wait_st();
                    fence_proxy_async();
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) {
                        tc_fence_after();
                        tw_mma<P>(acol, bw, dcol, nt, (k0 + kc) > 0 ? 1u : 0u);
                        tc_commit(bar);
                    }
                    __syncwarp();
                    pending = true;
                }
                if (abort)
                    break;
            }
        }
        // the block's epilogue: after its C item, or after its last item when C is not read
        if (fl & kTwEpi) {
            wait_mma();
            if (abort)
                break;
            tc_fence_after();
            tw_epilogue(cur, item, dcol + lq, cur.K > 0, cur.N > 16 ? 32 : 16, lane);
            tc_fence_before();
        }
        __syncwarp();
        tail = end;
        ++consumed;
    }
    // after a time-out, wait (bounded) for the copies still in flight into
    // this warp's ring before the CTA's shared memory is given up
    for (int i = consumed; abort && i < issued; ++i)
        mbar_wait(ibar + 8u * (uint32_t)(i & (kTwMaxOut - 1)), (uint32_t)((i / kTwMaxOut) & 1), kWaitLimitNs);
    cp_async_wait<0>();
    wait_mma();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, kTwTmemAlloc);
    }
}

}  // namespace iaat
