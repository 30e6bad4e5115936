// Persistent grouped complex small-GEMM kernel on the CUDA cores: CGEMM
// (complex float, FFMA) and ZGEMM (complex double, DFMA), the complex types of
// Table I, with the paper's four cases NN, NT, TN, TT (no conjugation).
//
// The plan, the stage programs and the producer warp are those of the real
// kernel (grouped.cuh): only the element size differs (8 or 16 bytes, a
// (re, im) pair).  The consumer warps differ in two ways:
//  * a complex multiply-add is four real FMAs (re += ar*br - ai*bi,
//    im += ar*bi + ai*br), the 8 flops per term that Eq. 2 counts, so a
//    warp block does four times the arithmetic per staged byte of the real
//    kernel and the operands are read where they were staged, with no
//    re-pack into per-warp buffers (the shared-memory loads stay well below
//    the FMA issue rate; the ring takes the space instead);
//  * alpha and beta are complex and come from the plan's scalar table
//    (TaskRec::alpha.p), read once per warp block.
// Every wait is bounded, as in the real kernel.
#pragma once
#include "grouped.cuh"

namespace iaat {

template <typename T> struct Cplx;
template <> struct Cplx<float> {
    using V = float2;
};
template <> struct Cplx<double> {
    using V = double2;
};

// One k term of the register tile: the lane's MR elements of op(A) and NR of
// op(B) (byte offsets aoff / boff from the term's row of the staged data),
// then MR x NR complex multiply-adds.
template <typename T, int MR, int NR>
__device__ __forceinline__ void cmac(T (&re)[MR][NR], T (&im)[MR][NR], const char *ak, const char *bk,
                                     const int (&aoff)[MR], const int (&boff)[NR])
{
    using V = typename Cplx<T>::V;
    V av[MR], bv[NR];
#pragma unroll
    for (int a = 0; a < MR; ++a)
        av[a] = *reinterpret_cast<const V *>(ak + aoff[a]);
#pragma unroll
    for (int b = 0; b < NR; ++b)
        bv[b] = *reinterpret_cast<const V *>(bk + boff[b]);
#pragma unroll
    for (int a = 0; a < MR; ++a)
#pragma unroll
        for (int b = 0; b < NR; ++b) {
            re[a][b] = fma(av[a].x, bv[b].x, re[a][b]);
            re[a][b] = fma(-av[a].y, bv[b].y, re[a][b]);
            im[a][b] = fma(av[a].x, bv[b].y, im[a][b]);
            im[a][b] = fma(av[a].y, bv[b].x, im[a][b]);
        }
}

// Warp block (bi, bj) of task r: lane (li, lj) of the LM x LN lane grid owns
// rows li*MR.. and columns lj*NR.. of the block.  Rows and columns past the
// block are clamped to its last one (their results are never stored), so the
// k-loop has no bounds checks.
template <typename T, int MR, int NR, int LM, int LN>
__device__ __forceinline__ void run_block_c(const char *smem, const TaskRec &r, int bi, int bj)
{
    using V = typename Cplx<T>::V;
    constexpr int E = (int)sizeof(V);
    const int lane = (int)lane_id();
    const int M = r.M, N = r.N, K = r.K;
    const int bh = (M + r.nbm - 1) / r.nbm;
    const int bw = (N + r.nbn - 1) / r.nbn;
    const int r0 = bi * bh, c0 = bj * bw;
    const int mh = min(bh, M - r0), nw = min(bw, N - c0);
    const int li = lane % LM, lj = lane / LM;
    const V *sc = reinterpret_cast<const V *>(r.alpha.p);
    const V alpha = __ldg(sc), beta = __ldg(sc + 1);

    T re[MR][NR], im[MR][NR];
#pragma unroll
    for (int a = 0; a < MR; ++a)
#pragma unroll
        for (int b = 0; b < NR; ++b)
            re[a][b] = im[a][b] = T(0);

    if (K > 0) {
        // element (i, k) of op(A) at Ab + i*am + k*ak; (k, j) of op(B) at Bb + k*bk + j*bn
        const int am = r.ta ? r.csA : E, ak = r.ta ? E : r.csA;
        const int bk = r.tb ? r.csB : E, bn = r.tb ? E : r.csB;
        const char *Ab = smem + r.offA + r0 * am;
        const char *Bb = smem + r.offB + c0 * bn;
        int aoff[MR], boff[NR];
#pragma unroll
        for (int a = 0; a < MR; ++a)
            aoff[a] = min(li * MR + a, mh - 1) * am;
#pragma unroll
        for (int b = 0; b < NR; ++b)
            boff[b] = min(lj * NR + b, nw - 1) * bn;
        // complex float: two k terms per trip, so the loads of one overlap
        // the FMAs of the other; complex double needs the registers for its
        // larger accumulators and runs one term per trip
        int k = 0;
        if constexpr (sizeof(T) == 4) {
#pragma unroll 1
            for (; k + 2 <= K; k += 2) {
                cmac<T, MR, NR>(re, im, Ab + k * ak, Bb + k * bk, aoff, boff);
                cmac<T, MR, NR>(re, im, Ab + (k + 1) * ak, Bb + (k + 1) * bk, aoff, boff);
            }
        }
#pragma unroll 1
        for (; k < K; ++k)
            cmac<T, MR, NR>(re, im, Ab + k * ak, Bb + k * bk, aoff, boff);
    }

    // epilogue: C = alpha*acc + beta*C0 (complex), exact elements only
    const bool readc = (r.flags & kFlagReadC) != 0;
    const char *Craw = smem + r.offC;
    V *Cg = reinterpret_cast<V *>(r.C);
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
                    T vr = fma(alpha.x, re[a][b], -alpha.y * im[a][b]);
                    T vi = fma(alpha.x, im[a][b], alpha.y * re[a][b]);
                    if (readc) {
                        const V c = *reinterpret_cast<const V *>(Craw + gj * r.csC + gi * E);
                        vr = fma(beta.x, c.x, fma(-beta.y, c.y, vr));
                        vi = fma(beta.x, c.y, fma(beta.y, c.x, vi));
                    }
                    V out;
                    out.x = vr;
                    out.y = vi;
                    Cg[gi + gj * ldc] = out;
                }
            }
        }
    }
}

template <typename T>
__device__ __forceinline__ void dispatch_block_c(const char *smem, const TaskRec &r, int bi, int bj);

template <>
__device__ __forceinline__ void dispatch_block_c<float>(const char *smem, const TaskRec &r, int bi, int bj)
{
#define IAAT_V(id)                                                                                             \
    case id:                                                                                                   \
        run_block_c<float, kVariantsC32[id].mr, kVariantsC32[id].nr, kVariantsC32[id].lm, kVariantsC32[id].ln>( \
            smem, r, bi, bj);                                                                                  \
        break;
    switch (r.variant) {
        IAAT_V(0) IAAT_V(1) IAAT_V(2) IAAT_V(3) IAAT_V(4)
    default:
        break;
    }
#undef IAAT_V
}

template <>
__device__ __forceinline__ void dispatch_block_c<double>(const char *smem, const TaskRec &r, int bi, int bj)
{
#define IAAT_V(id)                                                                                              \
    case id:                                                                                                    \
        run_block_c<double, kVariantsC64[id].mr, kVariantsC64[id].nr, kVariantsC64[id].lm, kVariantsC64[id].ln>( \
            smem, r, bi, bj);                                                                                   \
        break;
    switch (r.variant) {
        IAAT_V(0) IAAT_V(1) IAAT_V(2) IAAT_V(3) IAAT_V(4) IAAT_V(5) IAAT_V(6) IAAT_V(7) IAAT_V(8) IAAT_V(9)
        IAAT_V(10)
    default:
        break;
    }
#undef IAAT_V
}

// The consumer warps' walk over the CTA's stages (same schedule, barriers
// and block assignment as the real kernel's consumer_loop).
template <typename T>
__device__ void consumer_loop_c(const KParams &KP, const SmemMap &S, int warp)
{
    const Params &P = KP.p;
    const int lane = (int)lane_id();
    int rot = 0;   // blocks taken so far over the CTA's stages, modulo the warps
    for (int i = 0;; ++i) {
        const int g = sched_group(i, blockIdx.x, gridDim.x);
        if (g >= P.ngroups)
            break;
        const int slot = i % kNumSlots;
        const uint32_t par = (uint32_t)((i / kNumSlots) & 1);
        if (!mbar_wait(S.full(slot), par, kWaitLimitNs)) {
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
        for (int b = (warp - rot + kCplxWarps) % kCplxWarps; b < nb; b += kCplxWarps) {
            const int t = __popc(__ballot_sync(0xffffffffu, pre <= b));
            const int before = __shfl_sync(0xffffffffu, pre, t > 0 ? t - 1 : 0);
            const int lb = b - (t > 0 ? before : 0);
            if (!mbar_wait(S.task(slot, t), par, kWaitLimitNs)) {
                if (lane == 0)
                    set_error(P.err, kErrTimeoutFull);
                return;
            }
            const TaskRec r = recs[t];
            dispatch_block_c<T>(S.base, r, lb % r.nbm, lb / r.nbm);
        }
        __syncwarp();
        if (lane == 0)
            mbar_arrive(S.empty(slot));
        rot = (rot + nb) % kCplxWarps;
    }
}

template <typename T>
__global__ void __launch_bounds__(32 * (kCplxWarps + 1), 1) grouped_cplx_kernel(const __grid_constant__ KParams KP)
{
    extern __shared__ __align__(128) char smem[];
    SmemMap S;
    S.base = smem;
    S.sbase = smem_addr(smem);
    S.ring_off = (uint32_t)cplx_ring_offset();
    S.ring_bytes = (uint32_t)cplx_ring_bytes();
    S.pinfo_off = 0;
    S.cbar_off = 0;
    const int warp = threadIdx.x / 32;
    if (threadIdx.x < kNumSlots * kMaxGroupTasks)
        mbar_init(S.task(threadIdx.x / kMaxGroupTasks, threadIdx.x % kMaxGroupTasks), 1);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kNumSlots; ++s) {
            mbar_init(S.full(s), 1);
            mbar_init(S.empty(s), kCplxWarps);
        }
    }
    fence_barrier_init();
    __syncthreads();
    if (warp == kCplxWarps) {
        // complex launches always carry stage programs
        if (KP.p.prog)
            producer_prog<2 * (int)sizeof(T), false>(KP, S);
        else if (lane_id() == 0)
            set_error(KP.p.err, kErrBadGroup);
    } else {
        consumer_loop_c<T>(KP, S, warp);
    }
}

}  // namespace iaat
