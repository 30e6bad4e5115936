// Host side of the C ABI: argument checks, the run-time tiler (Sec. V-A),
// the planner that turns a batch into pipeline stages, and the launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <queue>
#include <vector>

#include "../../include/iaat.h"
#include "common.cuh"
#include "launch.h"
#include "tuning.h"

using namespace iaat;

// ------------------------------------------------------------- errors

static thread_local char g_last_error[512];

static iaat_status_t fail(iaat_status_t st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof g_last_error, fmt, ap);
    va_end(ap);
    return st;
}

static iaat_status_t cuda_fail(cudaError_t e, const char *what)
{
    return fail(IAAT_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

extern "C" const char *iaat_last_error(void) { return g_last_error; }

extern "C" const char *iaat_version(void) { return "iaat-gb300 0.1 (sm_103a)"; }

// ------------------------------------------------------- validation

static iaat_status_t check_instance(int64_t idx, int M, int N, int K, int lda, int ldb, int ldc, int ta, int tb,
                                    const void *A, const void *B, const void *C, double alpha, int esz)
{
    if (M < 0 || N < 0 || K < 0)
        return fail(IAAT_ERR_INVALID_VALUE, "instance %lld: negative size (M=%d N=%d K=%d)", (long long)idx, M, N, K);
    if ((ta != 0 && ta != 1) || (tb != 0 && tb != 1))
        return fail(IAAT_ERR_INVALID_VALUE, "instance %lld: trans flags must be 0 or 1", (long long)idx);
    const int ra = ta ? K : M, rb = tb ? N : K;
    if (lda < std::max(1, ra) || ldb < std::max(1, rb) || ldc < std::max(1, M))
        return fail(IAAT_ERR_INVALID_VALUE, "instance %lld: leading dimension too small (lda=%d ldb=%d ldc=%d)",
                    (long long)idx, lda, ldb, ldc);
    const int64_t mnk = (int64_t)M * N * K;
    const int64_t lim = (ta == 1 && tb == 0) ? 32768 : 512000;
    if (mnk > lim)
        return fail(IAAT_ERR_NOT_SMALL, "instance %lld: M*N*K = %lld is outside the small-GEMM domain (<= %lld)",
                    (long long)idx, (long long)mnk, (long long)lim);
    if (M > 0 && N > 0) {
        if (!C)
            return fail(IAAT_ERR_INVALID_VALUE, "instance %lld: C is NULL", (long long)idx);
        if (K > 0 && alpha != 0.0 && (!A || !B))
            return fail(IAAT_ERR_INVALID_VALUE, "instance %lld: A or B is NULL", (long long)idx);
        const uintptr_t mask = (uintptr_t)esz - 1;
        if (((uintptr_t)C & mask) || (K > 0 && alpha != 0.0 && (((uintptr_t)A & mask) || ((uintptr_t)B & mask))))
            return fail(IAAT_ERR_MISALIGNED, "instance %lld: pointer not aligned to %d bytes", (long long)idx, esz);
    }
    return IAAT_OK;
}

// ------------------------------------------------------------ tiler
// Cost, in warp issue slots, of one warp block of variant v with K terms:
// the FMAs and tile loads of the k-loop, the re-pack of each K-chunk (the
// memops term of Sec. V-A: m_i + n_i values per k), and a fixed epilogue.

static bool is_complex(int dt) { return dt == IAAT_C32 || dt == IAAT_C64; }
static int dtype_esz(int dt) { return dt == IAAT_F32 ? 4 : (dt == IAAT_C64 ? 16 : 8); }

static const Variant *variants(int dt, int *n)
{
    switch (dt) {
    case IAAT_F32:
        *n = kNumVariantsF32;
        return kVariantsF32;
    case IAAT_C32:
        *n = kNumVariantsC32;
        return kVariantsC32;
    case IAAT_C64:
        *n = kNumVariantsC64;
        return kVariantsC64;
    default:
        *n = kNumVariantsF64;
        return kVariantsF64;
    }
}

namespace iaat {
// The tiler's cost model without the tuned per-variant scale (the
// autotuner calibrates against it).
double model_block_cost(const Variant &v, int esz, int K);
}

// Complex tiles read the staged operands in place: per k term MR + NR
// element loads and 4*MR*NR FMAs (Eq. 2's four real products per complex
// one), then a complex epilogue.  Complex double is bound by the DFMA pipe,
// which takes a warp's DFMA in 64 clocks while other instructions issue in
// one and overlap it, so there a block costs almost only its DFMA slots --
// idle lanes of a partly filled tile included.
constexpr double kComplexDfmaWeight = 32.0;

static double block_cost(const Variant &v, int dt, int K)
{
    if (!is_complex(dt))
        return iaat::model_block_cost(v, dtype_esz(dt), K);
    const double fma = 4.0 * v.mr * v.nr * (dt == IAAT_C64 ? kComplexDfmaWeight : 1.0);
    return (double)K * (fma + v.mr + v.nr) + 2.0 * tuning().epilogue_weight * v.mr * v.nr + tuning().block_overhead;
}

double iaat::model_block_cost(const Variant &v, int esz, int K)
{
    const int ve = 16 / esz;
    const int kc = esz == 4 ? kKC : kKC64;
    const int bm = v.lm * v.mr, bn = v.ln * v.nr;
    const double fma = (double)v.mr * v.nr * (esz == 8 ? tuning().dfma_weight : 1.0);
    const double lds = (v.mr >= ve ? v.mr / ve : v.mr) + (v.nr >= ve ? v.nr / ve : v.nr);
    const int kp = (K + 3) & ~3;
    const int chunks = (K + kc - 1) / kc;
    const double repack = chunks * ((double)kc * (bm + bn) / 32.0) * tuning().repack_weight;
    return kp * (fma + lds) + repack + tuning().epilogue_weight * v.mr * v.nr + tuning().block_overhead;
}

struct TileChoice {
    int variant, nbm, nbn;
    double cost;
};

// scaled: weigh the variants by the autotuner's measured scales (the
// CUDA-core kernel); the tensor-core planner only uses the cost as an
// ordering key and takes the plain model, so that tuning the CUDA-core
// kernel does not reorder tensor-core stages.  min_blocks: the cheapest
// tiling with at least that many warp blocks (else the one with the most).
static TileChoice choose_tiling(int dt, int M, int N, int K, int force_variant, bool scaled = true,
                                int min_blocks = 1)
{
    int nv;
    const Variant *vs = variants(dt, &nv);
    scaled = scaled && !is_complex(dt);   // the autotuner calibrates the real families
    TileChoice best{0, 1, 1, 1e300};
    bool best_ok = false;
    int best_blocks = 0;
    for (int v = 0; v < nv; ++v) {
        if (force_variant >= 0 && v != force_variant)
            continue;
        const int bm = vs[v].lm * vs[v].mr, bn = vs[v].ln * vs[v].nr;
        const int nbm = std::max(1, (M + bm - 1) / bm), nbn = std::max(1, (N + bn - 1) / bn);
        if (nbm > 255 || nbn > 255)
            continue;
        const double c =
            (double)nbm * nbn * block_cost(vs[v], dt, K) * (scaled ? tuning().variant_scale(dtype_esz(dt), v) : 1.0);
        const bool ok = nbm * nbn >= min_blocks;
        const bool better = ok ? (!best_ok || c < best.cost)
                               : (!best_ok && (nbm * nbn > best_blocks || (nbm * nbn == best_blocks && c < best.cost)));
        if (better) {
            best = TileChoice{v, nbm, nbn, c};
            best_ok = ok;
            best_blocks = nbm * nbn;
        }
    }
    return best;
}

// Consumer warps of the CUDA-core kernels (real FP32, real FP64, complex).
static int fma_warps(int dt) { return dt == IAAT_F32 ? Traits<4>::kWarps : (is_complex(dt) ? kCplxWarps : kConsumerWarps); }

extern "C" int64_t iaat_tile(iaat_dtype_t dtype, int transA, int transB, int M, int N, int K, int32_t *blocks,
                             int64_t cap)
{
    (void)transA;
    (void)transB;
    if (dtype < IAAT_F32 || dtype > IAAT_C64 || M < 0 || N < 0 || K < 0 || cap < 0 || (cap > 0 && !blocks))
        return -1;
    if (M == 0 || N == 0)
        return 0;
    const TileChoice t = choose_tiling(dtype, M, N, K, -1);
    const int bh = (M + t.nbm - 1) / t.nbm, bw = (N + t.nbn - 1) / t.nbn;
    int64_t n = 0;
    for (int bj = 0; bj < t.nbn; ++bj)
        for (int bi = 0; bi < t.nbm; ++bi) {
            const int r0 = bi * bh, c0 = bj * bw;
            if (r0 >= M || c0 >= N)
                continue;
            if (n < cap) {
                blocks[4 * n + 0] = r0;
                blocks[4 * n + 1] = c0;
                blocks[4 * n + 2] = std::min(bh, M - r0);
                blocks[4 * n + 3] = std::min(bw, N - c0);
            }
            ++n;
        }
    return n;
}

// Exact-cover tiler under the paper's memops objective (Sec. V-A): row strips
// of kernel heights, each strip cut into the fewest blocks its widths allow
// (equal widths), minimising sum(m_i + n_i).  Dynamic programming over the
// rows; ties keep the taller strip first.
extern "C" int64_t iaat_tile_exact(int M, int N, const int32_t *heights, const int32_t *max_width, int nheights,
                                   int32_t *blocks, int64_t cap, int64_t *sum_out)
{
    if (M < 0 || N < 0 || nheights <= 0 || !heights || !max_width || cap < 0 || (cap > 0 && !blocks))
        return -1;
    if (M == 0 || N == 0) {
        if (sum_out)
            *sum_out = 0;
        return 0;
    }
    const int64_t INF = INT64_MAX / 4;
    std::vector<int64_t> f(M + 1, INF);
    std::vector<int> pick(M + 1, -1);
    f[0] = 0;
    for (int m = 1; m <= M; ++m) {
        for (int h = 0; h < nheights; ++h) {
            const int hh = heights[h], w = max_width[h];
            if (hh <= 0 || w <= 0 || hh > m || f[m - hh] >= INF)
                continue;
            const int64_t nblk = (N + w - 1) / w;
            const int64_t c = f[m - hh] + nblk * hh + N;
            if (c < f[m] || (c == f[m] && pick[m] >= 0 && hh > heights[pick[m]])) {
                f[m] = c;
                pick[m] = h;
            }
        }
    }
    if (f[M] >= INF)
        return -1;
    if (sum_out)
        *sum_out = f[M];
    std::vector<int> strips;
    for (int m = M; m > 0; m -= heights[pick[m]])
        strips.push_back(pick[m]);
    int64_t n = 0;
    int row = 0;
    for (int s : strips) {
        const int hh = heights[s], w = max_width[s];
        const int nblk = (N + w - 1) / w;
        int col = 0;
        for (int b = 0; b < nblk; ++b) {
            const int width = N / nblk + (b < N % nblk ? 1 : 0);
            if (n < cap) {
                blocks[4 * n + 0] = row;
                blocks[4 * n + 1] = col;
                blocks[4 * n + 2] = hh;
                blocks[4 * n + 3] = width;
            }
            ++n;
            col += width;
        }
        row += hh;
    }
    return n;
}

// ---------------------------------------------------------- planner

struct iaat_plan_s {
    int device = 0;
    int esz = 4;
    iaat_dtype_t dtype = IAAT_F32;
    iaat_precision_t precision = IAAT_PREC_DEFAULT;
    char *d_prog = nullptr;        // stage programs
    int64_t *d_poff = nullptr;     // program offset per group
    int32_t *d_err = nullptr;
    char *d_scal = nullptr;        // complex plans: alpha, beta of every instance
    iaat_plan_s *sub = nullptr;    // routed plans: the FP32 CUDA-core plan of the small-K instances
    bool tc2 = false;              // pack-stream tensor-core kernel
    int32_t *d_gbeg = nullptr;     // its packs per warp group
    Tc2Params t2p{};
    bool ws = false;               // warp-stream kernel (FP32 CUDA-core plans)
    char *d_ws = nullptr;          // its warp tasks, per-warp ranges and error word
    WsParams wsp{};
    bool tw = false;               // warp-tile tensor-core kernel
    char *d_tw = nullptr;          // its warp tasks, per-warp ranges and error word
    TwParams twp{};
    bool wd = false;               // warp-direct CUDA-core kernel
    char *d_wd = nullptr;          // its warp tasks, per-warp ranges and error word
    WdParams wdp{};
    int64_t ntasks = 0, ngroups = 0;
    int grid = 0;
    iaat_plan_info_t info{};
};

namespace {

struct HostTask {
    TaskDesc d;
    uint32_t bytes;   // shared-memory footprint
    double cost;      // ordering key
};

std::mutex g_prep_mutex;
bool g_prepared[64][19];

// kind: 0 = FP32 FFMA (stage programs), 1 = FP64 DFMA, 2..5 = tcgen05
// precision (kind - 1), 6 = complex float, 7 = complex double, 8 = FP32 FFMA
// warp-stream kernel, 9..12 = pack-stream tensor-core kernel, precision kind - 8,
// 13..16 = warp-tile tensor-core kernel, precision kind - 12, 17 / 18 =
// warp-direct kernel FP32 / FP64
iaat_status_t prepare_device(int dev, int kind)
{
    std::lock_guard<std::mutex> lk(g_prep_mutex);
    if (dev < 0 || dev >= 64)
        return fail(IAAT_ERR_CUDA, "device index %d out of range", dev);
    if (!g_prepared[dev][kind]) {
        cudaError_t e = kind > 16   ? prepare_wd(kind == 17 ? 4 : 8)
                        : kind < 2  ? prepare_fma(kind)
                        : kind < 6  ? prepare_tc(kind - 1)
                        : kind == 8 ? prepare_ws()
                        : kind > 12 ? prepare_tw(kind - 12)
                        : kind > 8  ? prepare_tc2(kind - 8)
                                    : prepare_cplx(kind == 6 ? IAAT_C32 : IAAT_C64);
        if (e != cudaSuccess)
            return cuda_fail(e, "cudaFuncSetAttribute");
        g_prepared[dev][kind] = true;
    }
    return IAAT_OK;
}

int kernel_kind(int dt, iaat_precision_t prec)
{
    if (is_complex(dt))
        return dt == IAAT_C32 ? 6 : 7;
    return prec != IAAT_PREC_DEFAULT ? 1 + (int)prec : (dt == IAAT_F32 ? 0 : 1);
}

int g_sm_count[64];

int sm_count(int dev)
{
    if (dev >= 0 && dev < 64 && g_sm_count[dev] > 0)
        return g_sm_count[dev];
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
        n = 1;
    if (dev >= 0 && dev < 64)
        g_sm_count[dev] = n;
    return n;
}

// ------------------------------------------------------ instance pieces
// An instance whose operands do not fit one pipeline stage, or that exceeds
// a kernel's tile limits (at most kPieceRows x kPieceCols for the CUDA-core
// kernel, one 128 x 128 MMA tile for the tensor-core kernel), is cut into
// pm x pn pieces: its rows into pm near-equal ranges and its columns into pn.
// Every piece computes its own block of C with the whole K, so the pieces are
// independent.  K itself is never cut (its pieces would have to accumulate
// into the same C); an instance whose A and B columns for one output element
// do not fit a stage is rejected.
constexpr int kPieceRows = 256, kPieceCols = 256;

void piece_range(int n, int parts, int idx, int &start, int &len)
{
    const int base = n / parts, extra = n % parts;
    start = idx * base + std::min(idx, extra);
    len = base + (idx < extra ? 1 : 0);
}

TaskDesc make_piece(const iaat_gemm_desc_t &g, int esz, int Keff, int r0, int h, int c0, int w)
{
    TaskDesc d{};
    d.A = g.A ? static_cast<const char *>(g.A) + (size_t)(g.transA ? (int64_t)r0 * g.lda : (int64_t)r0) * esz
              : nullptr;
    d.B = g.B ? static_cast<const char *>(g.B) + (size_t)(g.transB ? (int64_t)c0 : (int64_t)c0 * g.ldb) * esz
              : nullptr;
    d.C = static_cast<char *>(g.C) + (size_t)((int64_t)r0 + (int64_t)c0 * g.ldc) * esz;
    d.lda = g.lda;
    d.ldb = g.ldb;
    d.ldc = g.ldc;
    d.M = (int16_t)h;
    d.N = (int16_t)w;
    d.K = (int16_t)Keff;
    d.ta = (uint8_t)g.transA;
    d.tb = (uint8_t)g.transB;
    d.flags = (g.beta != 0.0) ? kFlagReadC : 0;
    d.alpha = esz == 4 ? (double)(float)g.alpha : g.alpha;
    d.beta = esz == 4 ? (double)(float)g.beta : g.beta;
    return d;
}

bool split_fits(const iaat_gemm_desc_t &g, int esz, int Keff, int pm, int pn, uint32_t cap)
{
    for (int i = 0; i < pm; ++i) {
        int r0, h;
        piece_range(g.M, pm, i, r0, h);
        for (int j = 0; j < pn; ++j) {
            int c0, w;
            piece_range(g.N, pn, j, c0, w);
            if (plan_task(make_piece(g, esz, Keff, r0, h, c0, w), esz).total() > cap)
                return false;
        }
    }
    return true;
}

// Smallest split (growing the longer side of the pieces first) whose every
// piece fits `cap` bytes of staging and mcap x ncap elements of C.
bool choose_split(const iaat_gemm_desc_t &g, int esz, int Keff, uint32_t cap, int mcap, int ncap, int &pm, int &pn)
{
    if (Keff > 32767)
        return false;
    pm = (g.M + mcap - 1) / mcap;
    pn = (g.N + ncap - 1) / ncap;
    for (;;) {
        if (split_fits(g, esz, Keff, pm, pn, cap))
            return true;
        const int h = (g.M + pm - 1) / pm, w = (g.N + pn - 1) / pn;
        if (h >= w && pm < g.M)
            ++pm;
        else if (pn < g.N)
            ++pn;
        else if (pm < g.M)
            ++pm;
        else
            return false;
    }
}

// Parallelism of the consumer warps of a CUDA-core kernel: its staging ring
// (two stage caps) holds about ring / bytes tasks of a task's size at a time,
// and only their blocks can be computed, so a task too large for the ring to
// hold one per warp is tiled into at least warps / that many blocks.
static int stage_min_blocks(const TaskDesc &d, int dt, uint32_t cap)
{
    const uint32_t bytes = std::max<uint32_t>(1, plan_task(d, dtype_esz(dt)).total());
    const int resident = (int)std::max<uint32_t>(1, 2 * cap / bytes);
    return resident < fma_warps(dt) ? (fma_warps(dt) + resident - 1) / resident : 1;
}

// Build the tasks of one instance: one, or its pieces.  piece > 0: cut C into
// pieces of at most piece x piece as well (the single-call path spreads one
// instance over several SMs that way).
// Complex plans (dt IAAT_C32 / IAAT_C64): g carries alpha and beta only as
// markers (alpha 0 or 1; beta 0, 1 or 2 for "other"), and each task's alpha
// field holds the instance index, which build_programs turns into the address
// of the instance's entry in the plan's scalar table.
static void push_task(int64_t idx, const iaat_gemm_desc_t &g, int dt, int Keff, int r0, int h, int c0, int w,
                      const TileChoice &t, std::vector<HostTask> &out, int64_t *blocks_out)
{
    const int esz = dtype_esz(dt);
    TaskDesc d = make_piece(g, esz, Keff, r0, h, c0, w);
    if (is_complex(dt)) {
        d.alpha = (double)idx;
        d.beta = 0.0;
    }
    d.variant = (uint8_t)t.variant;
    d.nbm = (uint8_t)t.nbm;
    d.nbn = (uint8_t)t.nbn;
    const TaskStages st = plan_task(d, esz);
    *blocks_out += (int64_t)d.nbm * d.nbn;
    out.push_back(HostTask{d, st.total(), (double)(st.a.tx + st.b.tx + st.c.tx) + tuning().cost_per_slot * t.cost});
}

// Mixed-shape tiling of one instance (Sec. V-A: one C tiled with several
// block shapes, the cheapest under the cost model), for the DFMA-bound types,
// where the idle lanes of a partly filled register tile still cost DFMA
// slots: besides the uniform grid of one variant, C may be cut into a part
// that is an exact multiple of a variant's block width (or height) and a
// remainder, each tiled with its own variant, when the model says that is at
// least 3 % cheaper, counting the operand the remainder stages a second
// time (op(A) for a column cut, op(B) for a row cut) at one cost unit per 16
// bytes (without that term 60 % of the fc64 batch was cut and it ran 4 %
// slower; ZGEMM gained 1.4 %).
static iaat_status_t make_mixed_tasks(int64_t idx, const iaat_gemm_desc_t &g, int dt, int Keff, uint32_t cap,
                                      std::vector<HostTask> &out, int64_t *blocks_out)
{
    const int M = g.M, N = g.N, esz = dtype_esz(dt);
    auto choose = [&](int r0, int h, int c0, int w) {
        const TaskDesc d = make_piece(g, esz, Keff, r0, h, c0, w);
        return choose_tiling(dt, h, w, Keff, -1, true, stage_min_blocks(d, dt, cap));
    };
    const TileChoice whole = choose(0, M, 0, N);
    double best = 0.97 * whole.cost;
    int split = 0;   // > 0: columns [0, split) and [split, N); < 0: rows [0, -split) and [-split, M)
    TileChoice ta{}, tb{};
    int nv;
    const Variant *vs = variants(dt, &nv);
    for (int v = 0; v < nv; ++v) {
        const int bn = vs[v].ln * vs[v].nr, bm = vs[v].lm * vs[v].mr;
        const int w1 = (N / bn) * bn, h1 = (M / bm) * bm;
        const double restage_a = (double)M * Keff * esz / 16.0, restage_b = (double)Keff * N * esz / 16.0;
        if (w1 > 0 && w1 < N) {
            const TileChoice a = choose(0, M, 0, w1), b = choose(0, M, w1, N - w1);
            if (a.cost + b.cost + restage_a < best) {
                best = a.cost + b.cost + restage_a;
                split = w1;
                ta = a;
                tb = b;
            }
        }
        if (h1 > 0 && h1 < M) {
            const TileChoice a = choose(0, h1, 0, N), b = choose(h1, M - h1, 0, N);
            if (a.cost + b.cost + restage_b < best) {
                best = a.cost + b.cost + restage_b;
                split = -h1;
                ta = a;
                tb = b;
            }
        }
    }
    if (split > 0) {
        push_task(idx, g, dt, Keff, 0, M, 0, split, ta, out, blocks_out);
        push_task(idx, g, dt, Keff, 0, M, split, N - split, tb, out, blocks_out);
    } else if (split < 0) {
        push_task(idx, g, dt, Keff, 0, -split, 0, N, ta, out, blocks_out);
        push_task(idx, g, dt, Keff, -split, M + split, 0, N, tb, out, blocks_out);
    } else {
        push_task(idx, g, dt, Keff, 0, M, 0, N, whole, out, blocks_out);
    }
    return IAAT_OK;
}

iaat_status_t make_tasks(int64_t idx, const iaat_gemm_desc_t &g, int dt, bool tc, int force_variant, uint32_t cap,
                         std::vector<HostTask> &out, int64_t *blocks_out, int piece = 0)
{
    const int esz = dtype_esz(dt);
    const int M = g.M, N = g.N;
    if (M == 0 || N == 0)
        return IAAT_OK;
    const int Keff = (g.alpha == 0.0) ? 0 : g.K;
    if (Keff == 0 && g.beta == 1.0)
        return IAAT_OK;   // C = 1*C: nothing to do
    int pm = 1, pn = 1;
    const int mcap = piece > 0 ? piece : (tc ? kTcPackRows : kPieceRows);
    const int ncap = piece > 0 ? piece : (tc ? kTcPackCols : kPieceCols);
    if (!choose_split(g, esz, Keff, cap, mcap, ncap, pm, pn))
        return fail(IAAT_ERR_UNSUPPORTED, "instance %lld: operands do not fit a pipeline stage (M=%d N=%d K=%d)",
                    (long long)idx, M, N, g.K);
    if (pm * pn == 1 && !tc && piece == 0 && force_variant < 0 && (dt == IAAT_F64 || dt == IAAT_C64))
        return make_mixed_tasks(idx, g, dt, Keff, cap, out, blocks_out);
    for (int i = 0; i < pm; ++i) {
        int r0, h;
        piece_range(M, pm, i, r0, h);
        for (int j = 0; j < pn; ++j) {
            int c0, w;
            piece_range(N, pn, j, c0, w);
            TaskDesc d = make_piece(g, esz, Keff, r0, h, c0, w);
            if (is_complex(dt)) {
                d.alpha = (double)idx;
                d.beta = 0.0;
            }
            // a single call's pieces run one per CTA: give each enough warp
            // blocks for the consumer warps (DFMA-bound pieces use every
            // sub-partition's pipe that way)
            const int min_blocks = (tc || force_variant >= 0) ? 1
                                   : piece > 0                 ? fma_warps(dt)
                                                               : stage_min_blocks(d, dt, cap);
            const TileChoice t = choose_tiling(dt, h, w, Keff, force_variant, !tc, min_blocks);
            d.variant = (uint8_t)t.variant;
            d.nbm = (uint8_t)t.nbm;
            d.nbn = (uint8_t)t.nbn;
            const TaskStages st = plan_task(d, esz);
            *blocks_out += (int64_t)d.nbm * d.nbn;
            out.push_back(HostTask{d, st.total(),
                                   (double)(st.a.tx + st.b.tx + st.c.tx) + tuning().cost_per_slot * t.cost});
        }
    }
    return IAAT_OK;
}

// Order tasks by cost (largest first) and cut them into stages of at most
// max_tasks tasks and `cap` bytes of shared memory (half the staging ring, so
// two stages always fit).  Each task of a stage has its own readiness
// barrier, so a large stage still lets the consumers start early.
void make_groups(std::vector<HostTask> &tasks, uint32_t cap, int max_tasks, std::vector<TaskDesc> &flat,
                 std::vector<int32_t> &gbeg)
{
    std::stable_sort(tasks.begin(), tasks.end(),
                     [](const HostTask &a, const HostTask &b) { return a.cost > b.cost; });
    flat.clear();
    gbeg.clear();
    uint32_t used = 0;
    int count = 0;
    for (const auto &t : tasks) {
        if (count == 0 || count >= max_tasks || used + t.bytes > cap) {
            gbeg.push_back((int32_t)flat.size());
            used = 0;
            count = 0;
        }
        flat.push_back(t.d);
        used += t.bytes;
        ++count;
    }
    gbeg.push_back((int32_t)flat.size());
}

// tcgen05 plans: inside each stage, order the tasks by K (largest first) and
// place them into packs, one 128-row MMA tile each.  A task takes whole
// 32-row quarters of the tile (the four tensor-memory lane quarters, each
// read back by the warps of one SM sub-partition), so its rows start at a
// multiple of 32 and the epilogue of a pack is spread over all four
// sub-partitions; its columns start at a multiple of 16 (one tensor-memory
// load), and a pack holds at most 128 columns.  A task's pack index, first
// row and first column travel in its variant/nbm/nbn fields.
// It also writes each pack's summary (PackInfo: the task, by its index in the
// stage, owning every quarter and every 16-column block, the largest K and
// the MMA N) and, per stage, the index of its first pack.
void make_packs(std::vector<TaskDesc> &flat, const std::vector<int32_t> &gbeg, std::vector<PackInfo> &packs,
                std::vector<int32_t> &pbeg)
{
    packs.clear();
    pbeg.clear();
    for (size_t g = 0; g + 1 < gbeg.size(); ++g) {
        pbeg.push_back((int32_t)packs.size());
        auto b = flat.begin() + gbeg[g], e = flat.begin() + gbeg[g + 1];
        std::stable_sort(b, e, [](const TaskDesc &x, const TaskDesc &y) { return x.K > y.K; });
        int quarters = 4, cols = 0;
        for (auto it = b; it != e; ++it) {
            const int q = (it->M + 31) / 32, w = (it->N + 15) & ~15;
            if (quarters + q > kTcPackRows / 32 || cols + w > kTcPackCols) {
                PackInfo pi{};
                for (int k = 0; k < 4; ++k)
                    pi.qtask[k] = -1;
                for (int k = 0; k < 8; ++k)
                    pi.btask[k] = -1;
                packs.push_back(pi);
                quarters = 0;
                cols = 0;
            }
            PackInfo &pi = packs.back();
            const int t = (int)(it - b);
            it->variant = (uint8_t)(packs.size() - 1 - pbeg.back());
            it->nbm = (uint8_t)(32 * quarters);
            it->nbn = (uint8_t)cols;
            for (int k = 0; k < q; ++k)
                pi.qtask[quarters + k] = (int8_t)t;
            for (int k = 0; k < w / 16; ++k)
                pi.btask[cols / 16 + k] = (int8_t)t;
            pi.kmax = (int16_t)std::max<int>(pi.kmax, it->K);
            quarters += q;
            cols += w;
            pi.nt = (uint8_t)std::max(16, cols);
        }
    }
    pbeg.push_back((int32_t)packs.size());
}

// Stage programs (see common.cuh): the producer's whole per-stage work,
// computed once per plan.  The ring placement follows each CTA's sequence of
// stages: a stage takes the F bytes after the previous one (wrapping to the
// ring's start when they do not fit), and before writing it must see the
// release of the latest earlier stage whose bytes it overlaps, or of the
// previous user of its slot -- releases happen in stage order, so that one
// wait covers every earlier stage.
void emit_copies(const Stage &st, const char *p, int h, int w, int ld, int esz, uint32_t dst, uint32_t bar,
                 std::vector<CopyCmd> &cmds)
{
    if (st.bytes == 0)
        return;
    const uint64_t pa = (uint64_t)(uintptr_t)p;
    if (st.span) {
        cmds.push_back(CopyCmd{reinterpret_cast<const char *>(pa & ~15ull), dst, st.bytes | (bar << 24)});
        return;
    }
    const uint32_t head = (uint32_t)(pa & 15);
    const uint64_t ldb = (uint64_t)ld * esz;
    for (int j = 0; j < w; ++j) {
        const uint64_t c0 = pa + (uint64_t)j * ldb;
        const uint64_t g0 = c0 & ~15ull, g1 = (c0 + (uint64_t)h * esz + 15) & ~15ull;
        cmds.push_back(CopyCmd{reinterpret_cast<const char *>(g0), dst + ((head + (uint32_t)j * st.cs) & ~15u),
                               (uint32_t)(g1 - g0) | (bar << 24)});
    }
}

iaat_status_t build_programs(const std::vector<TaskDesc> &flat, const std::vector<int32_t> &gbeg,
                             const std::vector<PackInfo> &packs, const std::vector<int32_t> &pbeg, int esz, bool tc,
                             int grid, uint32_t ring_off, uint32_t ring_bytes, const char *scal, uint32_t scal_stride,
                             std::vector<char> &prog, std::vector<int64_t> &poff)
{
    const int ng = (int)gbeg.size() - 1;
    poff.assign((size_t)std::max(ng, 1), 0);
    prog.clear();
    std::vector<CopyCmd> cmds;
    std::vector<TaskRec> recs;
    for (int c = 0; c < grid; ++c) {
        uint32_t head = 0, rbeg[kNumSlots] = {}, rend[kNumSlots] = {};
        int oldest = 0;
        for (int i = 0;; ++i) {
            const int g = sched_group(i, c, grid);
            if (g >= ng)
                break;
            const int t0 = gbeg[g], nt = gbeg[g + 1] - t0;
            const int npk = tc ? pbeg[g + 1] - pbeg[g] : 0;
            if (nt < 0 || nt > kMaxGroupTasks || npk < 0 || npk > kMaxGroupTasks)
                return fail(IAAT_ERR_INVALID_VALUE, "stage %d has %d tasks", g, nt);
            TaskStages st[kMaxGroupTasks];
            uint32_t F = 0;
            for (int t = 0; t < nt; ++t) {
                st[t] = plan_task(flat[t0 + t], esz);
                F += st[t].total();
            }
            if (F > ring_bytes)
                return fail(IAAT_ERR_UNSUPPORTED, "stage %d needs %u bytes of staging", g, F);
            const uint32_t a = (head + F <= ring_bytes) ? head : 0u;
            int need = i - kNumSlots;   // the slot's previous user
            for (int s = i - 1; s >= oldest && s > need; --s) {
                const int ss = s % kNumSlots;
                if (F > 0 && rbeg[ss] < a + F && a < rend[ss]) {
                    need = s;
                    break;
                }
            }
            int wait = -1;
            if (need >= oldest) {
                wait = need;
                oldest = need + 1;
            }
            rbeg[i % kNumSlots] = a;
            rend[i % kNumSlots] = a + F;
            head = a + F;

            SlotHeader hd{};
            hd.ntasks = nt;
            hd.npacks = npk;
            uint32_t tx[kMaxGroupTasks] = {};
            uint32_t ctx = 0, excl = 0;
            int nbi = 0;
            cmds.clear();
            recs.assign((size_t)nt, TaskRec{});
            for (int t = 0; t < nt; ++t) {
                const TaskDesc &d = flat[t0 + t];
                const TaskStages &s = st[t];
                const uint32_t base = ring_off + a + excl;
                TaskRec &r = recs[t];
                r.C = d.C;
                r.ldc = d.ldc;
                r.offA = (int32_t)(base + ((uint32_t)(uintptr_t)d.A & 15u));
                r.offB = (int32_t)(base + s.a.bytes + ((uint32_t)(uintptr_t)d.B & 15u));
                r.offC = (int32_t)(base + s.a.bytes + s.b.bytes + ((uint32_t)(uintptr_t)d.C & 15u));
                r.csA = (int32_t)s.a.cs;
                r.csB = (int32_t)s.b.cs;
                r.csC = (int32_t)s.c.cs;
                r.M = d.M; r.N = d.N; r.K = d.K;
                r.ta = d.ta; r.tb = d.tb; r.variant = d.variant; r.flags = d.flags;
                r.nbm = d.nbm; r.nbn = d.nbn;
                if (scal)   // complex plan: the instance's scalar-table entry
                    r.alpha.p = scal + (int64_t)d.alpha * scal_stride;
                else
                    set_scalars(r, d.alpha, d.beta, esz);
                nbi += (int)d.nbm * (int)d.nbn;
                hd.prefix[t] = nbi;
                tx[t] = s.a.tx + s.b.tx + (tc ? 0u : s.c.tx);
                if (tc)
                    ctx += s.c.tx;
                int ha, wa, hb, wb;
                stored_dims(d, ha, wa, hb, wb);
                const bool prod = d.K > 0;
                emit_copies(s.a, d.A, prod ? ha : 0, prod ? wa : 0, d.lda, esz, base, (uint32_t)t, cmds);
                emit_copies(s.b, d.B, prod ? hb : 0, prod ? wb : 0, d.ldb, esz, base + s.a.bytes, (uint32_t)t, cmds);
                emit_copies(s.c, d.C, d.M, d.N, d.ldc, esz, base + s.a.bytes + s.b.bytes, tc ? kCmdBarC : (uint32_t)t,
                            cmds);
                excl += s.total();
            }
            for (int t = nt; t < kMaxGroupTasks; ++t)
                hd.prefix[t] = 0x7fffffff;
            hd.nblocks = nbi;
            if (cmds.size() > 0xffff)
                return fail(IAAT_ERR_UNSUPPORTED, "stage %d needs %zu copies", g, cmds.size());

            StageProg h{};
            h.wait = wait;
            h.rec_bytes = (uint32_t)(sizeof(SlotHeader) + nt * sizeof(TaskRec));
            h.ncmd = (uint16_t)cmds.size();
            h.nt = (uint8_t)nt;
            h.npk = (uint8_t)npk;
            h.ctx = ctx;
            poff[g] = (int64_t)prog.size();
            auto put = [&prog](const void *p, size_t n) {
                const char *c = static_cast<const char *>(p);
                prog.insert(prog.end(), c, c + n);
            };
            put(&h, sizeof h);
            put(tx, sizeof tx);
            put(cmds.data(), cmds.size() * sizeof(CopyCmd));
            put(&hd, sizeof hd);
            put(recs.data(), recs.size() * sizeof(TaskRec));
            if (npk > 0)
                put(&packs[pbeg[g]], (size_t)npk * sizeof(PackInfo));
        }
    }
    return IAAT_OK;
}

}  // namespace

// ------------------------------------------------ warp-stream planner
// FP32 CUDA-core plans run the warp-stream kernel (ws.cuh): every instance
// is cut into warp tasks (one warp block of C each, the whole K), and the
// tasks are dealt to the warps of the grid ahead of time.

// Warp instructions that copy a region of Y lines of L elements each (one
// 4-byte cp.async per element, floor(32 / L) lines per instruction).
static double ws_copy_instr(int L, int Y)
{
    if (L <= 0 || Y <= 0)
        return 0.0;
    const int step = 32 / std::min(L, 32);
    return (double)((Y + step - 1) / step);
}

// Issue slots of one warp task: per K-chunk the rank-1 updates (FMAs and
// 16-byte shared loads), the copies of op(A) and op(B) (about six issue
// slots per copy instruction with its address arithmetic) and a fixed cost;
// then the copy of C0, the epilogue and a fixed cost per task.
constexpr double kWsCopySlots = 6.0, kWsChunkSlots = 60.0, kWsTaskSlots = 80.0;

static double ws_task_cost(const Variant &v, int mh, int nw, int K, int ta, int tb, bool readc)
{
    double c = kWsTaskSlots;
    const double lds = (v.mr >= 4 ? v.mr / 4 : v.mr) + (v.nr >= 4 ? v.nr / 4 : v.nr);
    for (int k0 = 0; k0 < K; k0 += kWsKC) {
        const int kc = std::min(kWsKC, K - k0), kcp = (kc + 3) & ~3;
        c += kcp * (v.mr * v.nr + lds) + kWsChunkSlots;
        c += kWsCopySlots * ((ta ? ws_copy_instr(kc, mh) : ws_copy_instr(mh, kc)) +
                             (tb ? ws_copy_instr(nw, kc) : ws_copy_instr(kc, nw)));
    }
    if (K == 0)
        c += kWsChunkSlots;
    if (readc)
        c += kWsCopySlots * ws_copy_instr(mh, nw);
    return c + 3.0 * v.mr * v.nr + 6.0 * ((mh * nw + 31) / 32);
}

// Cost of tiling an M x N (x K) instance with variant v: its rows cut into
// ceil(M / bm) near-equal block heights and its columns likewise.
static double ws_tiling_cost(const Variant &v, int M, int N, int K, int ta, int tb, bool readc, int64_t *nblocks)
{
    const int bm = v.lm * v.mr, bn = v.ln * v.nr;
    const int nbm = (M + bm - 1) / bm, nbn = (N + bn - 1) / bn;
    *nblocks = (int64_t)nbm * nbn;
    // near-equal split: M % nbm blocks of ceil(M / nbm) rows, the rest floor
    const int hr = M / nbm, wr = N / nbn;
    const int64_t nh1 = M % nbm, nh0 = nbm - nh1, nw1 = N % nbn, nw0 = nbn - nw1;
    double c = 0.0;
    if (nh0 && nw0) c += (double)(nh0 * nw0) * ws_task_cost(v, hr, wr, K, ta, tb, readc);
    if (nh0 && nw1) c += (double)(nh0 * nw1) * ws_task_cost(v, hr, wr + 1, K, ta, tb, readc);
    if (nh1 && nw0) c += (double)(nh1 * nw0) * ws_task_cost(v, hr + 1, wr, K, ta, tb, readc);
    if (nh1 && nw1) c += (double)(nh1 * nw1) * ws_task_cost(v, hr + 1, wr + 1, K, ta, tb, readc);
    return c;
}

// Weight of one byte of HBM traffic in the assignment cost, in issue slots:
// at the HBM roof an SM moves about 45 GB/s while it issues about 8,300
// warp instructions per microsecond, so one byte is worth about 0.19 slots.
constexpr double kWsByteSlots = 0.19;

static iaat_status_t plan_create_ws(const iaat_gemm_desc_t *descs, int64_t count, const iaat_plan_options_t *opts,
                                    int force_variant, iaat_plan_t *out, const int64_t *index_map)
{
    std::vector<WsTask> tasks;
    std::vector<double> cost;
    tasks.reserve((size_t)count * 2);
    cost.reserve((size_t)count * 2);
    iaat_plan_info_t info{};
    info.instances = count;
    info.dtype = IAAT_F32;
    info.precision = IAAT_PREC_DEFAULT;
    for (int64_t i = 0; i < count; ++i) {
        const iaat_gemm_desc_t &g = descs[i];
        const int64_t gi = index_map ? index_map[i] : i;
        iaat_status_t st = check_instance(gi, g.M, g.N, g.K, g.lda, g.ldb, g.ldc, g.transA, g.transB, g.A, g.B, g.C,
                                          g.alpha, 4);
        if (st != IAAT_OK)
            return st;
        const int M = g.M, N = g.N;
        if (M == 0 || N == 0)
            continue;
        const int K = (g.alpha == 0.0) ? 0 : g.K;
        if (K == 0 && g.beta == 1.0)
            continue;   // C = 1*C: nothing to do
        const bool readc = g.beta != 0.0;
        info.active += 1;
        info.flops += 2 * (int64_t)M * N * K;
        info.algorithmic_bytes += ((int64_t)M * K + (int64_t)K * N + (int64_t)M * N + (readc ? (int64_t)M * N : 0)) * 4;
        int best = 0;
        double best_cost = 1e300;
        for (int v = 0; v < kNumVariantsF32; ++v) {
            if (force_variant >= 0 && v != force_variant)
                continue;
            int64_t nb = 0;
            const double c = ws_tiling_cost(kVariantsF32[v], M, N, K, g.transA, g.transB, readc, &nb);
            if (c < best_cost) {
                best_cost = c;
                best = v;
            }
        }
        const Variant &vv = kVariantsF32[best];
        const int bm = vv.lm * vv.mr, bn = vv.ln * vv.nr;
        const int nbm = (M + bm - 1) / bm, nbn = (N + bn - 1) / bn;
        for (int bj = 0; bj < nbn; ++bj) {
            int c0, nw;
            piece_range(N, nbn, bj, c0, nw);
            for (int bi = 0; bi < nbm; ++bi) {
                int r0, mh;
                piece_range(M, nbm, bi, r0, mh);
                WsTask t{};
                if (K > 0) {
                    t.A = static_cast<const char *>(g.A) + (size_t)(g.transA ? (int64_t)r0 * g.lda : (int64_t)r0) * 4;
                    t.B = static_cast<const char *>(g.B) + (size_t)(g.transB ? (int64_t)c0 : (int64_t)c0 * g.ldb) * 4;
                }
                t.C = static_cast<char *>(g.C) + (size_t)((int64_t)r0 + (int64_t)c0 * g.ldc) * 4;
                t.lda = g.lda;
                t.ldb = g.ldb;
                t.ldc = g.ldc;
                t.M = (int16_t)mh;
                t.N = (int16_t)nw;
                t.K = K;
                t.ta = (uint8_t)g.transA;
                t.tb = (uint8_t)g.transB;
                t.variant = (uint8_t)best;
                t.flags = readc ? kFlagReadC : 0;
                t.alpha = (float)g.alpha;
                t.beta = (float)g.beta;
                tasks.push_back(t);
                const double bytes = 4.0 * ((double)mh * K + (double)K * nw + (double)mh * nw * (readc ? 2 : 1));
                cost.push_back(ws_task_cost(vv, mh, nw, K, g.transA, g.transB, readc) + kWsByteSlots * bytes);
            }
        }
    }

    iaat_plan_s *plan = new (std::nothrow) iaat_plan_s;
    if (!plan)
        return fail(IAAT_ERR_OOM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&plan->device);
    if (e != cudaSuccess) {
        delete plan;
        return cuda_fail(e, "cudaGetDevice");
    }
    iaat_status_t ps = prepare_device(plan->device, 8);
    if (ps != IAAT_OK) {
        delete plan;
        return ps;
    }
    plan->ws = true;
    plan->esz = 4;
    plan->dtype = IAAT_F32;
    plan->precision = IAAT_PREC_DEFAULT;
    const int64_t nt = (int64_t)tasks.size();
    const int sms = sm_count(plan->device);
    const int grid = (int)std::min<int64_t>(nt, (int64_t)sms);
    const int nwarps = grid * kWsWarps;

    // Largest-cost-first assignment, each task to the least loaded warp;
    // equal loads go to the warp that comes first in the order warp 0 of
    // every CTA, then warp 1 of every CTA, ..., so small batches spread over
    // the SMs before they share one.
    std::vector<int32_t> wbeg((size_t)nwarps + 1, 0);
    std::vector<WsTask> flat((size_t)nt);
    if (nt > 0) {
        std::vector<int32_t> order((size_t)nt);
        for (int64_t k = 0; k < nt; ++k)
            order[(size_t)k] = (int32_t)k;
        std::stable_sort(order.begin(), order.end(), [&cost](int32_t a, int32_t b) { return cost[a] > cost[b]; });
        using Slot = std::pair<double, int32_t>;   // (load, rank of the warp)
        std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> heap;
        for (int r = 0; r < nwarps; ++r)
            heap.push(Slot(0.0, r));
        std::vector<int32_t> owner((size_t)nt);
        std::vector<int32_t> per((size_t)nwarps, 0);
        for (int32_t k : order) {
            Slot s = heap.top();
            heap.pop();
            const int r = s.second;
            const int w = (r % grid) * kWsWarps + r / grid;   // CTA r % grid, warp r / grid
            owner[(size_t)k] = w;
            ++per[(size_t)w];
            s.first += cost[(size_t)k];
            heap.push(s);
        }
        for (int w = 0; w < nwarps; ++w)
            wbeg[(size_t)w + 1] = wbeg[(size_t)w] + per[(size_t)w];
        std::vector<int32_t> fill(wbeg.begin(), wbeg.end() - 1);
        for (int32_t k : order)
            flat[(size_t)fill[(size_t)owner[(size_t)k]]++] = tasks[(size_t)k];
        if (opts && opts->inject_fault == 1)
            flat[0].variant = 0xff;   // a record the kernel must refuse
    }
    const size_t tb = (size_t)std::max<int64_t>(nt, 1) * sizeof(WsTask);
    const size_t wb = (((size_t)nwarps + 1) * sizeof(int32_t) + 255) & ~(size_t)255;
    if ((e = cudaMalloc(&plan->d_ws, tb + wb + 256)) != cudaSuccess) {
        plan->d_ws = nullptr;
        iaat_plan_destroy(plan);
        return fail(IAAT_ERR_OOM, "cudaMalloc of the plan: %s", cudaGetErrorString(e));
    }
    if ((nt > 0 && (e = cudaMemcpy(plan->d_ws, flat.data(), (size_t)nt * sizeof(WsTask), cudaMemcpyHostToDevice)) !=
                       cudaSuccess) ||
        (e = cudaMemcpy(plan->d_ws + tb, wbeg.data(), ((size_t)nwarps + 1) * sizeof(int32_t),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(plan->d_ws + tb + wb, 0, sizeof(int32_t))) != cudaSuccess) {
        iaat_plan_destroy(plan);
        return cuda_fail(e, "upload the warp tasks");
    }
    plan->wsp.tasks = reinterpret_cast<const WsTask *>(plan->d_ws);
    plan->wsp.wbeg = reinterpret_cast<const int32_t *>(plan->d_ws + tb);
    plan->wsp.err = reinterpret_cast<int32_t *>(plan->d_ws + tb + wb);
    plan->wsp.nwarps = nwarps;
    plan->d_err = plan->wsp.err;
    plan->ntasks = nt;
    plan->ngroups = nt > 0 ? nwarps : 0;
    plan->grid = grid;
    info.tasks = nt;
    info.groups = plan->ngroups;
    info.blocks = nt;
    info.plan_bytes = (int64_t)(tb + wb + 256);
    info.grid = grid;
    info.kernels = nt > 0 ? 1 : 0;
    info.kernel_family = 2;
    plan->info = info;
    *out = plan;
    return IAAT_OK;
}

// ----------------------------------------- pack-stream tensor-core planner
// Tensor-core plans run the pack-stream kernel (tc2.cuh).  Every instance is
// one task, or is cut into row / column pieces (each with the whole K) when
// it exceeds one MMA tile (128 rows, kT2Cols columns of C) or its raw
// operands would take more than half a group's staging ring.  Tasks are sorted by K (largest first) and
// placed into packs of up to kT2MaxTasks consecutive tasks (t2_layout: their
// rows fill at most the 128 rows of the tile, their columns at most kT2Cols,
// their staging at most half the ring),
// so that instances of similar K share one MMA pass.  Each pack becomes a
// program (header, task records with the staging offsets, bulk copies), and
// the packs are dealt to the warp groups, largest first, each to the least
// loaded group.
struct T2Task {
    TaskDesc d;
    TaskStages st;
};

// Rows and columns of the tasks [t0, t0 + n) of a pack.  Tasks of more than
// 32 rows take rows one after another from the start of quarter `rot` (or of
// quarter 0 when they would not fit there); tasks of up to 32 rows each go
// into one 32-row quarter (the rows of one epilogue warp), the quarter whose
// warp has the fewest accumulator columns to read so far, ties going to the
// first quarter from `rot` on.  Rotating `rot` from pack to pack spreads the
// epilogue work over the four SM sub-partitions (warp q of every group runs
// on sub-partition q).  Columns are handed out quarter by quarter, each
// task's rounded up to 16, so that the columns a warp reads are one
// contiguous run.  Returns false when the tasks do not fit (rows, or more
// than kT2Cols columns); *ncols: the MMA N.
static bool t2_layout(const std::vector<T2Task> &tasks, int64_t t0, int64_t n, int rot, int *row0, int *col0,
                      int *ncols)
{
    int big_rows = 0;
    for (int64_t k = 0; k < n; ++k)
        if (tasks[(size_t)(t0 + k)].d.M > 32)
            big_rows += tasks[(size_t)(t0 + k)].d.M;
    if (big_rows > kTcPackRows)
        return false;
    const int big_start = 32 * rot + big_rows <= kTcPackRows ? 32 * rot : 0;
    int big_end = big_start;
    for (int64_t k = 0; k < n; ++k)
        if (tasks[(size_t)(t0 + k)].d.M > 32) {
            row0[k] = big_end;
            big_end += tasks[(size_t)(t0 + k)].d.M;
        }
    int fill[4], load[4] = {0, 0, 0, 0}, quarter[kT2MaxTasks];
    for (int q = 0; q < 4; ++q) {
        // free rows of quarter q: all of it, or what the large tasks leave
        const int lo = 32 * q, hi = 32 * q + 32;
        fill[q] = (big_end <= lo || big_start >= hi) ? lo : (big_end < hi && big_start <= lo ? big_end : hi);
    }
    for (int64_t k = 0; k < n; ++k) {
        const TaskDesc &d = tasks[(size_t)(t0 + k)].d;
        const int w = std::max(16, (d.N + 15) & ~15);
        if (d.M > 32) {
            quarter[k] = row0[k] / 32;
            for (int q = row0[k] / 32; q <= (row0[k] + d.M - 1) / 32; ++q)
                load[q] += w;
        }
    }
    for (int64_t k = 0; k < n; ++k) {
        const TaskDesc &d = tasks[(size_t)(t0 + k)].d;
        if (d.M > 32)
            continue;
        int best = -1;
        for (int u = 0; u < 4; ++u) {
            const int q = (rot + u) & 3;
            if (fill[q] + d.M <= 32 * q + 32 && (best < 0 || load[q] < load[best]))
                best = q;
        }
        if (best < 0)
            return false;
        row0[k] = fill[best];
        fill[best] += d.M;
        load[best] += std::max(16, (d.N + 15) & ~15);
        quarter[k] = best;
    }
    int col = 0;
    for (int q = 0; q < 4; ++q)
        for (int64_t k = 0; k < n; ++k)
            if (quarter[k] == q) {
                col0[k] = col;
                col += std::max(16, (tasks[(size_t)(t0 + k)].d.N + 15) & ~15);
            }
    *ncols = std::max(16, col);
    return col <= kT2Cols;
}

static iaat_status_t plan_create_tc2(const iaat_gemm_desc_t *descs, int64_t count, iaat_precision_t precision,
                                     const iaat_plan_options_t *opts, iaat_plan_t *out, const int64_t *index_map)
{
    // A pack takes at most half a group's ring, so two are always in flight
    // (a group gives a pack's staging back before it waits for the next, so
    // an empty ring always takes the next pack).
    const uint32_t ring = (uint32_t)tc2_ring_bytes((int)precision);
    const uint32_t pack_cap = (ring / 2) & ~15u;
    const uint32_t task_cap = pack_cap - (uint32_t)(sizeof(Tc2Hdr) + sizeof(Tc2Rec));
    const int kstep = precision == IAAT_PREC_TF32 ? 8 : 16;
    std::vector<T2Task> tasks;
    tasks.reserve((size_t)count);
    iaat_plan_info_t info{};
    info.instances = count;
    info.dtype = IAAT_F32;
    info.precision = precision;
    for (int64_t i = 0; i < count; ++i) {
        const iaat_gemm_desc_t &g = descs[i];
        const int64_t gi = index_map ? index_map[i] : i;
        iaat_status_t st = check_instance(gi, g.M, g.N, g.K, g.lda, g.ldb, g.ldc, g.transA, g.transB, g.A, g.B, g.C,
                                          g.alpha, 4);
        if (st != IAAT_OK)
            return st;
        const int M = g.M, N = g.N;
        if (M == 0 || N == 0)
            continue;
        const int Keff = (g.alpha == 0.0) ? 0 : g.K;
        if (Keff == 0 && g.beta == 1.0)
            continue;
        int pm = 1, pn = 1;
        if (!choose_split(g, 4, Keff, task_cap, kTcPackRows, kT2Cols, pm, pn))
            return fail(IAAT_ERR_UNSUPPORTED, "instance %lld: operands do not fit a pipeline stage (M=%d N=%d K=%d)",
                        (long long)gi, M, N, g.K);
        info.active += 1;
        info.flops += 2 * (int64_t)M * N * Keff;
        info.algorithmic_bytes +=
            ((int64_t)M * Keff + (int64_t)Keff * N + (int64_t)M * N + (g.beta != 0.0 ? (int64_t)M * N : 0)) * 4;
        for (int a = 0; a < pm; ++a) {
            int r0, h;
            piece_range(M, pm, a, r0, h);
            for (int b = 0; b < pn; ++b) {
                int c0, w;
                piece_range(N, pn, b, c0, w);
                T2Task t;
                t.d = make_piece(g, 4, Keff, r0, h, c0, w);
                t.st = plan_task(t.d, 4);
                tasks.push_back(t);
            }
        }
    }
    std::stable_sort(tasks.begin(), tasks.end(), [](const T2Task &x, const T2Task &y) { return x.d.K > y.d.K; });

    // packs: [first task, end) ranges over the sorted tasks, each as many
    // consecutive tasks as t2_layout places, at most kT2MaxTasks and pack_cap
    // bytes of staging
    std::vector<int64_t> pbeg;
    {
        int row0[kT2MaxTasks], col0[kT2MaxTasks], ncols = 0;
        int64_t first = 0;
        uint32_t bytes = (uint32_t)sizeof(Tc2Hdr);
        pbeg.push_back(0);
        for (size_t k = 0; k < tasks.size(); ++k) {
            const uint32_t b = tasks[k].st.total() + (uint32_t)sizeof(Tc2Rec);
            const int64_t n = (int64_t)k - first + 1;
            if ((int64_t)k > first && (n > kT2MaxTasks || bytes + b > pack_cap ||
                                       !t2_layout(tasks, first, n, (int)(pbeg.size() - 1) & 3, row0, col0, &ncols))) {
                pbeg.push_back((int64_t)k);
                first = (int64_t)k;
                bytes = (uint32_t)sizeof(Tc2Hdr);
            }
            bytes += b;
        }
        if (tasks.empty())
            pbeg.clear();
        pbeg.push_back((int64_t)tasks.size());
    }
    const int64_t npacks = (int64_t)pbeg.size() - 1;

    // pack programs
    std::vector<char> prog;
    std::vector<int64_t> poff((size_t)std::max<int64_t>(npacks, 1), 0);
    std::vector<double> pcost((size_t)std::max<int64_t>(npacks, 0));
    std::vector<CopyCmd> cmds;
    for (int64_t p = 0; p < npacks; ++p) {
        const int64_t t0 = pbeg[(size_t)p], nt = pbeg[(size_t)p + 1] - t0;
        Tc2Hdr h{};
        h.ntasks = (int32_t)nt;
        std::vector<Tc2Rec> recs((size_t)nt);
        cmds.clear();
        uint32_t off = (uint32_t)(sizeof(Tc2Hdr) + nt * sizeof(Tc2Rec));
        h.rec_bytes = off;
        uint32_t tx = off;
        int row0[kT2MaxTasks], col0[kT2MaxTasks], ncols = 0, kmax = 0;
        if (!t2_layout(tasks, t0, nt, (int)(p & 3), row0, col0, &ncols))
            return fail(IAAT_ERR_INVALID_VALUE, "pack %lld: its tasks do not fit the tile", (long long)p);
        double conv = 0.0;
        for (int64_t k = 0; k < nt; ++k) {
            const TaskDesc &d = tasks[(size_t)(t0 + k)].d;
            const TaskStages &s = tasks[(size_t)(t0 + k)].st;
            Tc2Rec &r = recs[(size_t)k];
            r.C = d.C;
            r.ldc = d.ldc;
            r.offA = (int32_t)(off + ((uint32_t)(uintptr_t)d.A & 15u));
            r.offB = (int32_t)(off + s.a.bytes + ((uint32_t)(uintptr_t)d.B & 15u));
            r.offC = (int32_t)(off + s.a.bytes + s.b.bytes + ((uint32_t)(uintptr_t)d.C & 15u));
            r.csA = (int32_t)s.a.cs;
            r.csB = (int32_t)s.b.cs;
            r.csC = (int32_t)s.c.cs;
            r.K = d.K;
            r.M = d.M;
            r.N = d.N;
            r.ta = d.ta;
            r.tb = d.tb;
            r.row0 = (uint8_t)row0[k];
            r.col0 = (uint8_t)col0[k];
            r.flags = d.flags;
            r.alpha = (float)d.alpha;
            r.beta = (float)d.beta;
            kmax = std::max(kmax, (int)d.K);
            int ha, wa, hb, wb;
            stored_dims(d, ha, wa, hb, wb);
            const bool prod = d.K > 0;
            emit_copies(s.a, d.A, prod ? ha : 0, prod ? wa : 0, d.lda, 4, off, 0, cmds);
            emit_copies(s.b, d.B, prod ? hb : 0, prod ? wb : 0, d.ldb, 4, off + s.a.bytes, 0, cmds);
            emit_copies(s.c, d.C, d.M, d.N, d.ldc, 4, off + s.a.bytes + s.b.bytes, 0, cmds);
            tx += s.a.tx + s.b.tx + s.c.tx;
            off += s.total();
            conv += (double)(d.M + d.N) * ((d.K + kT2KC - 1) / kT2KC);
        }
        h.ncmd = (int32_t)cmds.size();
        h.kpack = kmax > 0 ? (kmax + kstep - 1) / kstep * kstep : 0;
        h.nt = ncols;
        h.item_bytes = off;
        h.tx_bytes = tx;
        if (off > pack_cap || off > ring)
            return fail(IAAT_ERR_UNSUPPORTED, "pack %lld needs %u bytes of staging", (long long)p, off);
        // every access the kernel derives from the program stays inside the
        // pack's staging item, its tile and its operand buffers
        {
            uint64_t sum = h.rec_bytes;
            for (const CopyCmd &c : cmds) {
                const uint32_t b = c.meta & 0xffffffu;
                if (c.dst < h.rec_bytes || c.dst + b > off || ((c.dst | b | (uint32_t)(uintptr_t)c.src) & 15u))
                    return fail(IAAT_ERR_INVALID_VALUE, "pack %lld: copy outside its staging item", (long long)p);
                sum += b;
            }
            if (sum != tx || h.nt > kT2Cols || (h.nt & 15))
                return fail(IAAT_ERR_INVALID_VALUE, "pack %lld: inconsistent program", (long long)p);
            auto inside = [&](int32_t o, int32_t cs, int rows, int cols) {
                if (rows <= 0 || cols <= 0)
                    return true;
                const int64_t last = (int64_t)o + (int64_t)(cols - 1) * cs + (int64_t)rows * 4;
                return o >= (int32_t)h.rec_bytes && last <= (int64_t)off;
            };
            for (int64_t k = 0; k < nt; ++k) {
                const Tc2Rec &r = recs[(size_t)k];
                const int K = r.K, M = r.M, N = r.N;
                const bool okA = inside(r.offA, r.csA, r.ta ? K : M, r.ta ? M : K);
                const bool okB = inside(r.offB, r.csB, r.tb ? N : K, r.tb ? K : N);
                const bool okC = !(r.flags & kFlagReadC) || inside(r.offC, r.csC, M, N);
                bool overlap = false;   // rows and column runs of the pack's tasks are disjoint
                for (int64_t k2 = 0; k2 < k; ++k2) {
                    const Tc2Rec &o = recs[(size_t)k2];
                    overlap = overlap || (r.row0 < o.row0 + o.M && o.row0 < r.row0 + M) ||
                              (r.col0 < o.col0 + ((o.N + 15) & ~15) && o.col0 < r.col0 + ((N + 15) & ~15));
                }
                if (!okA || !okB || !okC || overlap || r.row0 + M > 128 || r.col0 + ((N + 15) & ~15) > h.nt)
                    return fail(IAAT_ERR_INVALID_VALUE, "pack %lld: task %lld outside its staging or tile",
                                (long long)p, (long long)k);
            }
        }
        poff[(size_t)p] = (int64_t)prog.size();
        auto put = [&prog](const void *x, size_t n) {
            const char *c = static_cast<const char *>(x);
            prog.insert(prog.end(), c, c + n);
        };
        put(&h, sizeof h);
        put(recs.data(), recs.size() * sizeof(Tc2Rec));
        prog.resize(prog.size() + (kT2MaxTasks - recs.size()) * sizeof(Tc2Rec), 0);   // commands at kT2CmdOff
        put(cmds.data(), cmds.size() * sizeof(CopyCmd));
        // one pack: its bytes at the HBM rate plus its conversion and epilogue work
        pcost[(size_t)p] = (double)tx + 64.0 * conv + 2048.0;
    }
    // the issuing warp prefetches a fixed window of kT2Window bytes of each
    // program before it knows the program's size: pad the programs so that
    // the window of the last one stays inside them
    prog.resize(prog.size() + kT2Window, 0);
    if (opts && opts->inject_fault == 1 && npacks > 0)
        reinterpret_cast<Tc2Hdr *>(prog.data() + poff[0])->ntasks = kT2MaxTasks + 1;

    iaat_plan_s *plan = new (std::nothrow) iaat_plan_s;
    if (!plan)
        return fail(IAAT_ERR_OOM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&plan->device);
    if (e != cudaSuccess) {
        delete plan;
        return cuda_fail(e, "cudaGetDevice");
    }
    iaat_status_t ps = prepare_device(plan->device, 8 + (int)precision);
    if (ps != IAAT_OK) {
        delete plan;
        return ps;
    }
    plan->tc2 = true;
    plan->esz = 4;
    plan->dtype = IAAT_F32;
    plan->precision = precision;
    const int sms = sm_count(plan->device);
    const int grid = (int)std::min<int64_t>((npacks + kT2Groups - 1) / kT2Groups, (int64_t)sms);
    const int ngr = grid * kT2Groups;

    // deal the packs to the groups: largest first, each to the least loaded
    // group; equal loads go to group 0 of every CTA first, then group 1, ...
    std::vector<int32_t> gbeg((size_t)ngr + 1, 0);
    std::vector<int64_t> poff_sorted((size_t)std::max<int64_t>(npacks, 1), 0);
    if (npacks > 0) {
        std::vector<int32_t> order((size_t)npacks);
        for (int64_t k = 0; k < npacks; ++k)
            order[(size_t)k] = (int32_t)k;
        std::stable_sort(order.begin(), order.end(), [&pcost](int32_t a, int32_t b) { return pcost[a] > pcost[b]; });
        using Slot = std::pair<double, int32_t>;
        std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> heap;
        for (int r = 0; r < ngr; ++r)
            heap.push(Slot(0.0, r));
        std::vector<int32_t> owner((size_t)npacks), per((size_t)ngr, 0);
        for (int32_t k : order) {
            Slot sl = heap.top();
            heap.pop();
            const int r = sl.second;
            const int gid = (r % grid) * kT2Groups + r / grid;
            owner[(size_t)k] = gid;
            ++per[(size_t)gid];
            sl.first += pcost[(size_t)k];
            heap.push(sl);
        }
        for (int gid = 0; gid < ngr; ++gid)
            gbeg[(size_t)gid + 1] = gbeg[(size_t)gid] + per[(size_t)gid];
        std::vector<int32_t> fill(gbeg.begin(), gbeg.end() - 1);
        for (int32_t k : order)
            poff_sorted[(size_t)fill[(size_t)owner[(size_t)k]]++] = poff[(size_t)k];
        // every header names the programs of the next two packs of its group,
        // so the issuing warp never waits for a global load
        for (int gid = 0; gid < ngr; ++gid)
            for (int32_t k = gbeg[(size_t)gid]; k < gbeg[(size_t)gid + 1]; ++k) {
                Tc2Hdr *h = reinterpret_cast<Tc2Hdr *>(prog.data() + poff_sorted[(size_t)k]);
                h->next[0] = k + 1 < gbeg[(size_t)gid + 1] ? poff_sorted[(size_t)k + 1] : -1;
                h->next[1] = k + 2 < gbeg[(size_t)gid + 1] ? poff_sorted[(size_t)k + 2] : -1;
            }
    }
    const size_t pb = std::max<size_t>(16, prog.size());
    const size_t ob = poff_sorted.size() * sizeof(int64_t), gb = gbeg.size() * sizeof(int32_t);
    if ((e = cudaMalloc(&plan->d_prog, pb)) != cudaSuccess || (e = cudaMalloc(&plan->d_poff, ob)) != cudaSuccess ||
        (e = cudaMalloc(&plan->d_gbeg, gb)) != cudaSuccess || (e = cudaMalloc(&plan->d_err, sizeof(int32_t))) != cudaSuccess) {
        iaat_plan_destroy(plan);
        return fail(IAAT_ERR_OOM, "cudaMalloc of the plan: %s", cudaGetErrorString(e));
    }
    if ((!prog.empty() && (e = cudaMemcpy(plan->d_prog, prog.data(), prog.size(), cudaMemcpyHostToDevice)) != cudaSuccess) ||
        (e = cudaMemcpy(plan->d_poff, poff_sorted.data(), ob, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(plan->d_gbeg, gbeg.data(), gb, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(plan->d_err, 0, sizeof(int32_t))) != cudaSuccess) {
        iaat_plan_destroy(plan);
        return cuda_fail(e, "upload the pack programs");
    }
    plan->t2p.prog = plan->d_prog;
    plan->t2p.poff = plan->d_poff;
    plan->t2p.gbeg = plan->d_gbeg;
    plan->t2p.err = plan->d_err;
    plan->t2p.ngroups = ngr;
    plan->ntasks = (int64_t)tasks.size();
    plan->ngroups = npacks > 0 ? ngr : 0;
    plan->grid = grid;
    info.tasks = plan->ntasks;
    info.groups = npacks;
    info.blocks = npacks;
    info.plan_bytes = (int64_t)(pb + ob + gb + sizeof(int32_t));
    info.grid = grid;
    info.kernels = npacks > 0 ? 1 : 0;
    info.kernel_family = 2;
    plan->info = info;
    *out = plan;
    return IAAT_OK;
}

// The planner behind iaat_plan_create and iaat_plan_create_complex.  cscal:
// complex plans only, (re alpha, im alpha, re beta, im beta) per instance,
// already rounded to the component type; the descriptors then carry alpha
// and beta as markers (see make_tasks).  index_map: the caller's index of
// each descriptor, for error messages (NULL: the position itself).
// ------------------------------------------ warp-tile tensor-core planner
// Tensor-core plans with option kernel = 3 run the warp-tile kernel (tw.cuh).
// Every instance is cut into blocks of at most kTwBlockM x kTwBlockN of C
// (rows and columns into near-equal ranges), one warp task each with the instance's whole K;
// the K range is staged in pieces of kseg values (a multiple of 16), the
// largest that keep every item of the task within half of a warp's ring.  The
// tasks are dealt to the warps largest estimated cost first, each to the
// least loaded warp (warp 0 of every CTA first, then warp 1, ...).
static double tw_task_cost(const TwTask &t)
{
    // issue slots of one warp, roughly: per task set-up; per 16-value chunk
    // the row of op(A) per lane, the (row, core row) items of op(B), the MMA
    // issue and its wait; the epilogue per column; the copies per granule slot
    const int K = t.K, nw = t.N;
    const int chunks = K > 0 ? (K + 15) / 16 : 0;
    const double bsteps = std::ceil((double)nw * 2 / 32.0);
    double c = 260.0 + chunks * (90.0 + 50.0 * bsteps + 120.0) + 8.0 * nw + 60.0;
    const double slots = (K > 0 ? (double)tw_ab_item_bytes(t, K) : 0.0) +
                         ((t.flags & kFlagReadC) ? (double)tw_c_item_bytes(t) : 0.0);
    return c + 16.0 * std::ceil(slots / 16.0 / 32.0);
}

// Stage an operand block as one span (one bulk copy, issued by one lane)
// when that takes at most twice the ring bytes of staging it run by run
// (each run by the lanes' own copies) and at most a quarter of the ring.
static bool tw_span(int runs, int len, int64_t ld, uint32_t cap)
{
    const uint32_t sb = tw_op_bytes(runs, len, ld, true);
    return sb <= 2 * tw_op_bytes(runs, len, ld, false) && sb <= cap / 2;
}

static iaat_status_t plan_create_tw(const iaat_gemm_desc_t *descs, int64_t count, iaat_precision_t precision,
                                    const iaat_plan_options_t *opts, iaat_plan_t *out, const int64_t *index_map)
{
    const uint32_t cap = (uint32_t)tw_ring_bytes((int)precision) / 2;
    std::vector<TwTask> tasks;
    std::vector<double> cost;
    tasks.reserve((size_t)count * 2);
    cost.reserve((size_t)count * 2);
    iaat_plan_info_t info{};
    info.instances = count;
    info.dtype = IAAT_F32;
    info.precision = precision;
    for (int64_t i = 0; i < count; ++i) {
        const iaat_gemm_desc_t &g = descs[i];
        const int64_t gi = index_map ? index_map[i] : i;
        iaat_status_t st = check_instance(gi, g.M, g.N, g.K, g.lda, g.ldb, g.ldc, g.transA, g.transB, g.A, g.B, g.C,
                                          g.alpha, 4);
        if (st != IAAT_OK)
            return st;
        const int M = g.M, N = g.N;
        if (M == 0 || N == 0)
            continue;
        const int K = (g.alpha == 0.0) ? 0 : g.K;
        if (K == 0 && g.beta == 1.0)
            continue;   // C = 1*C: nothing to do
        const bool readc = g.beta != 0.0;
        info.active += 1;
        info.flops += 2 * (int64_t)M * N * K;
        info.algorithmic_bytes += ((int64_t)M * K + (int64_t)K * N + (int64_t)M * N + (readc ? (int64_t)M * N : 0)) * 4;
        const int nbm = (M + kTwBlockM - 1) / kTwBlockM, nbn = (N + kTwBlockN - 1) / kTwBlockN;
        for (int bj = 0; bj < nbn; ++bj) {
            int c0, nw;
            piece_range(N, nbn, bj, c0, nw);
            for (int bi = 0; bi < nbm; ++bi) {
                int r0, mh;
                piece_range(M, nbm, bi, r0, mh);
                TwTask t{};
                if (K > 0) {
                    t.A = static_cast<const char *>(g.A) + (size_t)(g.transA ? (int64_t)r0 * g.lda : (int64_t)r0) * 4;
                    t.B = static_cast<const char *>(g.B) + (size_t)(g.transB ? (int64_t)c0 : (int64_t)c0 * g.ldb) * 4;
                }
                t.C = static_cast<char *>(g.C) + (size_t)((int64_t)r0 + (int64_t)c0 * g.ldc) * 4;
                t.lda = g.lda;
                t.ldb = g.ldb;
                t.ldc = g.ldc;
                t.K = K;
                t.M = (int16_t)mh;
                t.N = (int16_t)nw;
                t.ta = (uint8_t)g.transA;
                t.tb = (uint8_t)g.transB;
                t.alpha = (float)g.alpha;
                t.beta = (float)g.beta;
                // the K range per item (kseg, a multiple of 16): the largest
                // that keeps every item of the task within half the ring; the
                // span-or-runs choice of op(A) and op(B) depends on it
                // (transposed operands' runs are the item's K range long)
                int kseg = K > 0 ? std::min(((K + 15) / 16) * 16, 16 * 255) : 16;
                for (int pass = 0; pass < 2; ++pass) {
                    const int kl = std::min(K, kseg);
                    t.flags = (uint8_t)((readc ? kFlagReadC : 0) | (tw_span(nw, mh, g.ldc, cap) ? kTwSpanC : 0));
                    if (K > 0) {
                        if (g.transA ? tw_span(mh, kl, g.lda, cap) : tw_span(kl, mh, g.lda, cap))
                            t.flags |= kTwSpanA;
                        if (g.transB ? tw_span(kl, nw, g.ldb, cap) : tw_span(nw, kl, g.ldb, cap))
                            t.flags |= kTwSpanB;
                        while (kseg > 16 && tw_ab_item_bytes(t, std::min(K, kseg)) > cap)
                            kseg -= 16;
                    }
                }
                t.kseg16 = (uint8_t)(kseg / 16);
                if (tw_ab_item_bytes(t, std::min(K, kseg)) > cap || tw_c_item_bytes(t) > cap)
                    return fail(IAAT_ERR_UNSUPPORTED, "instance %lld: a block does not fit the staging ring",
                                (long long)gi);
                tasks.push_back(t);
                cost.push_back(tw_task_cost(t));
            }
        }
    }

    iaat_plan_s *plan = new (std::nothrow) iaat_plan_s;
    if (!plan)
        return fail(IAAT_ERR_OOM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&plan->device);
    if (e != cudaSuccess) {
        delete plan;
        return cuda_fail(e, "cudaGetDevice");
    }
    iaat_status_t ps = prepare_device(plan->device, 12 + (int)precision);
    if (ps != IAAT_OK) {
        delete plan;
        return ps;
    }
    plan->tw = true;
    plan->esz = 4;
    plan->dtype = IAAT_F32;
    plan->precision = precision;
    const int64_t nt = (int64_t)tasks.size();
    const int sms = sm_count(plan->device);
    const int grid = (int)std::min<int64_t>(nt, (int64_t)sms);
    const int nwarps = grid * kTwWarps;

    std::vector<int32_t> wbeg((size_t)nwarps + 1, 0);
    std::vector<TwTask> flat((size_t)nt);
    if (nt > 0) {
        std::vector<int32_t> order((size_t)nt);
        for (int64_t k = 0; k < nt; ++k)
            order[(size_t)k] = (int32_t)k;
        std::stable_sort(order.begin(), order.end(), [&cost](int32_t a, int32_t b) { return cost[a] > cost[b]; });
        using Slot = std::pair<double, int32_t>;   // (load, rank of the warp)
        std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> heap;
        for (int r = 0; r < nwarps; ++r)
            heap.push(Slot(0.0, r));
        std::vector<int32_t> owner((size_t)nt);
        std::vector<int32_t> per((size_t)nwarps, 0);
        for (int32_t k : order) {
            Slot s = heap.top();
            heap.pop();
            const int r = s.second;
            const int w = (r % grid) * kTwWarps + r / grid;   // CTA r % grid, warp r / grid
            owner[(size_t)k] = w;
            ++per[(size_t)w];
            s.first += cost[(size_t)k];
            heap.push(s);
        }
        for (int w = 0; w < nwarps; ++w)
            wbeg[(size_t)w + 1] = wbeg[(size_t)w] + per[(size_t)w];
        std::vector<int32_t> fill(wbeg.begin(), wbeg.end() - 1);
        for (int32_t k : order)
            flat[(size_t)fill[(size_t)owner[(size_t)k]]++] = tasks[(size_t)k];
        if (opts && opts->inject_fault == 1)
            flat[0].M = 33;   // a record the kernel must refuse
    }
    const size_t tb = (size_t)std::max<int64_t>(nt, 1) * sizeof(TwTask);
    const size_t wb = (((size_t)nwarps + 1) * sizeof(int32_t) + 255) & ~(size_t)255;
    if ((e = cudaMalloc(&plan->d_tw, tb + wb + 256)) != cudaSuccess) {
        plan->d_tw = nullptr;
        iaat_plan_destroy(plan);
        return fail(IAAT_ERR_OOM, "cudaMalloc of the plan: %s", cudaGetErrorString(e));
    }
    if ((nt > 0 && (e = cudaMemcpy(plan->d_tw, flat.data(), (size_t)nt * sizeof(TwTask), cudaMemcpyHostToDevice)) !=
                       cudaSuccess) ||
        (e = cudaMemcpy(plan->d_tw + tb, wbeg.data(), ((size_t)nwarps + 1) * sizeof(int32_t),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(plan->d_tw + tb + wb, 0, sizeof(int32_t))) != cudaSuccess) {
        iaat_plan_destroy(plan);
        return cuda_fail(e, "upload the warp tasks");
    }
    plan->twp.tasks = reinterpret_cast<const TwTask *>(plan->d_tw);
    plan->twp.wbeg = reinterpret_cast<const int32_t *>(plan->d_tw + tb);
    plan->twp.err = reinterpret_cast<int32_t *>(plan->d_tw + tb + wb);
    plan->twp.nwarps = nwarps;
    plan->d_err = plan->twp.err;
    plan->ntasks = nt;
    plan->ngroups = nt > 0 ? nwarps : 0;
    plan->grid = grid;
    info.tasks = nt;
    info.groups = plan->ngroups;
    info.blocks = nt;
    info.plan_bytes = (int64_t)(tb + wb + 256);
    info.grid = grid;
    info.kernels = nt > 0 ? 1 : 0;
    info.kernel_family = 3;
    plan->info = info;
    *out = plan;
    return IAAT_OK;
}


// ------------------------------------------ warp-direct CUDA-core plans
// (wd.cuh) Every instance is cut into row blocks and, per row block of m
// rows, column blocks; the warp's lanes form g = floor(32 / m) column groups.
// Instances with K up to wd_k1 take blocks of at most 32 rows and
// wd_max_cols columns, the others at most 16 rows and half the columns (their
// longer op(A) rows and op(B) columns fit the same staging area).  The blocks
// are dealt to the warps largest estimated cost first, each to the least
// loaded warp.
static double wd_task_cost(const WdTask &t, int esz)
{
    // issue slots of one warp, roughly: record and set-up; the staging
    // copies (op(A) and op(B) per lane group of 32, C0 per column step); per
    // column step the k-loop (one FMA and a quarter or half of a 16-byte
    // shared load per k) and the epilogue; per extra K chunk a wait
    const int K = t.K, k2 = wd_k2(esz);
    const double per_k = esz == 4 ? 1.25 : 1.5;
    const int chunks = K > k2 ? (K + k2 - 1) / k2 : 1;
    const double copies = std::ceil((double)K * (t.m + t.n) / 32.0) * 6.0 +
                          ((t.flags & kWdReadC) ? t.iters * 5.0 : 0.0);
    return 120.0 + copies + t.iters * (per_k * K + 12.0 + 6.0 * (chunks - 1)) + 60.0 * (chunks - 1);
}

static iaat_status_t plan_create_wd(const iaat_gemm_desc_t *descs, int64_t count, int esz,
                                    const iaat_plan_options_t *opts, iaat_plan_t *out, const int64_t *index_map)
{
    std::vector<WdTask> tasks;
    std::vector<double> cost;
    tasks.reserve((size_t)count * 2);
    cost.reserve((size_t)count * 2);
    iaat_plan_info_t info{};
    info.instances = count;
    info.dtype = esz == 4 ? IAAT_F32 : IAAT_F64;
    info.precision = IAAT_PREC_DEFAULT;
    const int k1 = wd_k1(esz), cmax = wd_max_cols(esz);
    for (int64_t i = 0; i < count; ++i) {
        const iaat_gemm_desc_t &g = descs[i];
        const int64_t gi = index_map ? index_map[i] : i;
        iaat_status_t st = check_instance(gi, g.M, g.N, g.K, g.lda, g.ldb, g.ldc, g.transA, g.transB, g.A, g.B, g.C,
                                          g.alpha, esz);
        if (st != IAAT_OK)
            return st;
        const int M = g.M, N = g.N;
        if (M == 0 || N == 0)
            continue;
        const int K = (g.alpha == 0.0) ? 0 : g.K;
        if (K == 0 && g.beta == 1.0)
            continue;   // C = 1*C: nothing to do
        const bool readc = g.beta != 0.0;
        info.active += 1;
        info.flops += 2 * (int64_t)M * N * K;
        info.algorithmic_bytes +=
            ((int64_t)M * K + (int64_t)K * N + (int64_t)M * N + (readc ? (int64_t)M * N : 0)) * esz;
        const double alpha = esz == 4 ? (double)(float)g.alpha : g.alpha;
        const double beta = esz == 4 ? (double)(float)g.beta : g.beta;
        const bool wide = K > k1;
        const int rcap = wide ? kWdRows2 : kWdMaxRows, ncap = wide ? cmax / 2 : cmax;
        const int nbm = (M + rcap - 1) / rcap;
        for (int bi = 0; bi < nbm; ++bi) {
            int r0, mh;
            piece_range(M, nbm, bi, r0, mh);
            const int gmax = 32 / mh;
            const int nbn = (N + ncap - 1) / ncap;
            for (int bj = 0; bj < nbn; ++bj) {
                int c0, nw;
                piece_range(N, nbn, bj, c0, nw);
                WdTask t{};
                if (K > 0) {
                    t.A = static_cast<const char *>(g.A) + (size_t)(g.transA ? (int64_t)r0 * g.lda : (int64_t)r0) * esz;
                    t.B = static_cast<const char *>(g.B) + (size_t)(g.transB ? (int64_t)c0 : (int64_t)c0 * g.ldb) * esz;
                }
                t.C = static_cast<char *>(g.C) + (size_t)((int64_t)r0 + (int64_t)c0 * g.ldc) * esz;
                t.lda = g.lda;
                t.ldb = g.ldb;
                t.ldc = g.ldc;
                t.K = K;
                t.m = (uint8_t)mh;
                t.g = (uint8_t)std::min(gmax, nw);
                t.iters = (uint8_t)((nw + t.g - 1) / t.g);
                t.n = (uint16_t)nw;
                t.magic = (uint16_t)((32768 + mh - 1) / mh);
                t.flags = (uint8_t)((g.transA ? kWdTransA : 0) | (g.transB ? kWdTransB : 0) | (readc ? kWdReadC : 0));
                if (esz == 4) {
                    t.ab.f[0] = (float)alpha;
                    t.ab.f[1] = (float)beta;
                } else {
                    t.ab.d[0] = alpha;
                    t.ab.d[1] = beta;
                }
                tasks.push_back(t);
                cost.push_back(wd_task_cost(t, esz));
            }
        }
    }

    iaat_plan_s *plan = new (std::nothrow) iaat_plan_s;
    if (!plan)
        return fail(IAAT_ERR_OOM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&plan->device);
    if (e != cudaSuccess) {
        delete plan;
        return cuda_fail(e, "cudaGetDevice");
    }
    iaat_status_t ps = prepare_device(plan->device, esz == 4 ? 17 : 18);
    if (ps != IAAT_OK) {
        delete plan;
        return ps;
    }
    plan->wd = true;
    plan->esz = esz;
    plan->dtype = esz == 4 ? IAAT_F32 : IAAT_F64;
    plan->precision = IAAT_PREC_DEFAULT;
    const int64_t nt = (int64_t)tasks.size();
    const int sms = sm_count(plan->device);
    const int grid = (int)std::min<int64_t>((nt + kWdWarps - 1) / kWdWarps, (int64_t)sms * kWdCtasPerSm);
    const int nwarps = grid * kWdWarps;

    std::vector<int32_t> wbeg((size_t)nwarps + 1, 0);
    std::vector<WdTask> flat((size_t)nt);
    if (nt > 0) {
        std::vector<int32_t> order((size_t)nt);
        for (int64_t k = 0; k < nt; ++k)
            order[(size_t)k] = (int32_t)k;
        std::stable_sort(order.begin(), order.end(), [&cost](int32_t a, int32_t b) { return cost[a] > cost[b]; });
        using Slot = std::pair<double, int32_t>;   // (load, rank of the warp)
        std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> heap;
        for (int r = 0; r < nwarps; ++r)
            heap.push(Slot(0.0, r));
        std::vector<int32_t> owner((size_t)nt);
        std::vector<int32_t> per((size_t)nwarps, 0);
        for (int32_t k : order) {
            Slot sl = heap.top();
            heap.pop();
            const int r = sl.second;
            const int w = (r % grid) * kWdWarps + r / grid;   // CTA r % grid, warp r / grid
            owner[(size_t)k] = w;
            ++per[(size_t)w];
            sl.first += cost[(size_t)k];
            heap.push(sl);
        }
        for (int w = 0; w < nwarps; ++w)
            wbeg[(size_t)w + 1] = wbeg[(size_t)w] + per[(size_t)w];
        std::vector<int32_t> fill(wbeg.begin(), wbeg.end() - 1);
        for (int32_t k : order)
            flat[(size_t)fill[(size_t)owner[(size_t)k]]++] = tasks[(size_t)k];
        if (opts && opts->inject_fault == 1)
            flat[0].m = 33;   // a record the kernel must refuse
    }
    // every warp's first task again, at a fixed place: the kernel fetches it
    // without waiting for the warp's task range
    std::vector<WdTask> first((size_t)std::max(nwarps, 1));
    for (int w = 0; w < nwarps; ++w)
        if (wbeg[(size_t)w] < wbeg[(size_t)w + 1])
            first[(size_t)w] = flat[(size_t)wbeg[(size_t)w]];
    const size_t tb = (size_t)std::max<int64_t>(nt, 1) * sizeof(WdTask);
    const size_t fb = first.size() * sizeof(WdTask);
    const size_t wb = (((size_t)nwarps + 1) * sizeof(int32_t) + 255) & ~(size_t)255;
    if ((e = cudaMalloc(&plan->d_wd, tb + fb + wb + 256)) != cudaSuccess) {
        plan->d_wd = nullptr;
        iaat_plan_destroy(plan);
        return fail(IAAT_ERR_OOM, "cudaMalloc of the plan: %s", cudaGetErrorString(e));
    }
    if ((nt > 0 && (e = cudaMemcpy(plan->d_wd, flat.data(), (size_t)nt * sizeof(WdTask), cudaMemcpyHostToDevice)) !=
                       cudaSuccess) ||
        (e = cudaMemcpy(plan->d_wd + tb, first.data(), fb, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(plan->d_wd + tb + fb, wbeg.data(), ((size_t)nwarps + 1) * sizeof(int32_t),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(plan->d_wd + tb + fb + wb, 0, sizeof(int32_t))) != cudaSuccess) {
        iaat_plan_destroy(plan);
        return cuda_fail(e, "upload the warp tasks");
    }
    plan->wdp.tasks = reinterpret_cast<const WdTask *>(plan->d_wd);
    plan->wdp.first = reinterpret_cast<const WdTask *>(plan->d_wd + tb);
    plan->wdp.wbeg = reinterpret_cast<const int32_t *>(plan->d_wd + tb + fb);
    plan->wdp.err = reinterpret_cast<int32_t *>(plan->d_wd + tb + fb + wb);
    plan->wdp.nwarps = nwarps;
    plan->d_err = plan->wdp.err;
    plan->ntasks = nt;
    plan->ngroups = nt > 0 ? nwarps : 0;
    plan->grid = grid;
    info.tasks = nt;
    info.groups = plan->ngroups;
    info.blocks = nt;
    info.plan_bytes = (int64_t)(tb + fb + wb + 256);
    info.grid = grid;
    info.kernels = nt > 0 ? 1 : 0;
    info.kernel_family = 4;
    plan->info = info;
    *out = plan;
    return IAAT_OK;
}

// Options that pin the stage programs' tiling or stages (a forced variant
// or stage size, an injected fault) keep a plan on the stage programs alone.
static bool opts_force_free(const iaat_plan_options_t *o)
{
    return !o || (o->force_variant <= 0 && o->max_group_tasks <= 0 && o->inject_fault == 0);
}

// Append plan b after the last plan of a's chain (one iaat_gemm_grouped
// launches them in order) and add b's statistics to a's.
static void chain_plan(iaat_plan_t a, iaat_plan_t b)
{
    iaat_plan_t last = a;
    while (last->sub)
        last = last->sub;
    last->sub = b;
    iaat_plan_info_t &x = a->info;
    const iaat_plan_info_t &y = b->info;
    x.active += y.active;
    x.tasks += y.tasks;
    x.groups += y.groups;
    x.blocks += y.blocks;
    x.flops += y.flops;
    x.algorithmic_bytes += y.algorithmic_bytes;
    x.plan_bytes += y.plan_bytes;
    x.grid = std::max(x.grid, y.grid);
    x.kernels += y.kernels;
}

static iaat_status_t plan_create_impl(const iaat_gemm_desc_t *descs, int64_t count, int dt,
                                      iaat_precision_t precision, const iaat_plan_options_t *opts,
                                      const double *cscal, iaat_plan_t *out, const int64_t *index_map = nullptr,
                                      bool split_large = true)
{
    const int esz = dtype_esz(dt);
    const bool tc = precision != IAAT_PREC_DEFAULT;
    const bool cplx = is_complex(dt);
    const uint32_t cap = tc     ? (uint32_t)tc_group_cap((int)precision)
                         : cplx ? (uint32_t)cplx_max_group_bytes()
                                : (uint32_t)(esz == 4 ? max_group_bytes<4>() : max_group_bytes<8>());
    int max_tasks = kMaxGroupTasks;
    if (!cplx) {
        const int tuned = dt == IAAT_F64 ? tuning().group_tasks_f64 : tuning().group_tasks[(int)precision];
        if (tuned > 0)
            max_tasks = tuned;
    }
    int force_variant = -1;
    int ctas_per_sm = 1;
    if (opts) {
        if (opts->max_group_tasks > 0)
            max_tasks = std::min(opts->max_group_tasks, kMaxGroupTasks);
        if (opts->force_variant > 0) {
            int nv;
            variants(dt, &nv);
            if (opts->force_variant > nv)
                return fail(IAAT_ERR_INVALID_VALUE, "force_variant %d out of range", opts->force_variant);
            force_variant = opts->force_variant - 1;
        }
        if (opts->ctas_per_sm > 0)
            ctas_per_sm = 1;   // the kernel takes all shared memory: one CTA per SM
    }
    (void)ctas_per_sm;
    int kernel = opts ? opts->kernel : 0;
    if (kernel < 0 || kernel > 4)
        return fail(IAAT_ERR_INVALID_VALUE, "kernel %d out of range", kernel);
    if (kernel == 4 && (tc || cplx))
        return fail(IAAT_ERR_INVALID_VALUE,
                    "kernel 4 (warp-direct CUDA-core kernel) takes FP32 or FP64 plans of the default precision");
    if (kernel == 0 && dt == IAAT_F32)
        kernel = tuning().kernel[(int)precision];   // the autotuner's choice (0: stage programs)
    if (kernel == 4)
        return plan_create_wd(descs, count, esz, opts, out, index_map);
    if (kernel == 3 && !tc)
        return fail(IAAT_ERR_INVALID_VALUE, "kernel 3 (warp-tile tensor-core kernel) needs a tensor-core precision");
    if (tc && kernel == 3)
        return plan_create_tw(descs, count, precision, opts, out, index_map);
    if (dt == IAAT_F32 && !tc && kernel == 2)
        return plan_create_ws(descs, count, opts, force_variant, out, index_map);
    if (tc && kernel == 2)
        return plan_create_tc2(descs, count, precision, opts, out, index_map);

    // A default FP32 plan on the stage programs sends the instances that a
    // stage cannot hold whole -- the ones the stage programs would cut into
    // row / column pieces, each re-reading the shared operand -- to a kernel
    // that stages K in pieces instead: the warp-tile kernel for tensor-core
    // precisions (same-size 64^3 batches 2.6x faster there), the warp-stream
    // kernel for FFMA (80^3 1.45x faster); that plan runs after this one on
    // the same stream.  Only when they carry at least a quarter of the batch's bytes:
    // a second launch for a few of them costs more than their pieces (the
    // uneven batch, 0.1 % of its instances and 1.5 % of its bytes: 0.77 ->
    // 0.80 ms when split).
    if (dt == IAAT_F32 && split_large && (!opts || opts->kernel == 0) && opts_force_free(opts)) {
        std::vector<iaat_gemm_desc_t> dst, dlg;
        std::vector<int64_t> ist, ilg;
        double all_bytes = 0.0, large_bytes = 0.0;
        for (int64_t i = 0; i < count; ++i) {
            const iaat_gemm_desc_t &g = descs[i];
            const int64_t gi = index_map ? index_map[i] : i;
            const iaat_status_t st = check_instance(gi, g.M, g.N, g.K, g.lda, g.ldb, g.ldc, g.transA, g.transB, g.A,
                                                    g.B, g.C, g.alpha, 4);
            if (st != IAAT_OK)
                return st;
            const int Keff = g.alpha == 0.0 ? 0 : g.K;
            int pm = 1, pn = 1;
            const bool whole = g.M == 0 || g.N == 0 || (Keff == 0 && g.beta == 1.0) ||
                               (choose_split(g, 4, Keff, cap, tc ? kTcPackRows : kPieceRows,
                                             tc ? kTcPackCols : kPieceCols, pm, pn) &&
                                pm * pn == 1);
            (whole ? dst : dlg).push_back(g);
            (whole ? ist : ilg).push_back(gi);
            if (g.M > 0 && g.N > 0) {
                const double bytes = 4.0 * ((double)g.M * Keff + (double)Keff * g.N + 2.0 * g.M * g.N);
                all_bytes += bytes;
                if (!whole)
                    large_bytes += bytes;
            }
        }
        if (!dlg.empty() && large_bytes >= 0.25 * all_bytes) {
            iaat_plan_t a = nullptr, b = nullptr;
            iaat_status_t st = plan_create_impl(dst.data(), (int64_t)dst.size(), dt, precision, opts, nullptr, &a,
                                                ist.data(), false);
            if (st != IAAT_OK)
                return st;
            iaat_plan_options_t o = opts ? *opts : iaat_plan_options_t{};
            o.inject_fault = 0;
            st = tc ? plan_create_tw(dlg.data(), (int64_t)dlg.size(), precision, &o, &b, ilg.data())
                    : plan_create_ws(dlg.data(), (int64_t)dlg.size(), &o, -1, &b, ilg.data());
            if (st != IAAT_OK) {
                iaat_plan_destroy(a);
                return st;
            }
            chain_plan(a, b);
            a->info.instances = count;
            if (dst.empty())
                a->info.kernel_family = tc ? 3 : 2;
            *out = a;
            return IAAT_OK;
        }
    }

    std::vector<HostTask> tasks;
    tasks.reserve((size_t)count);
    iaat_plan_info_t info{};
    info.instances = count;
    info.dtype = dt;
    info.precision = precision;
    int64_t nblocks = 0;
    for (int64_t i = 0; i < count; ++i) {
        const iaat_gemm_desc_t &g = descs[i];
        const int64_t gi = index_map ? index_map[i] : i;
        iaat_status_t st = check_instance(gi, g.M, g.N, g.K, g.lda, g.ldb, g.ldc, g.transA, g.transB, g.A, g.B, g.C,
                                          g.alpha, esz);
        if (st != IAAT_OK)
            return st;
        const size_t before = tasks.size();
        // complex plans index their scalar table by position (never remapped)
        st = make_tasks(cplx ? i : gi, g, dt, tc, force_variant, cap, tasks, &nblocks);
        if (st != IAAT_OK)
            return st;
        if (tasks.size() > before) {
            info.active += 1;
            const int64_t M = g.M, N = g.N, K = (g.alpha == 0.0) ? 0 : g.K;
            info.flops += (cplx ? 8 : 2) * M * N * g.K * (g.alpha == 0.0 ? 0 : 1);
            info.algorithmic_bytes += (M * K + K * N + M * N + (g.beta != 0.0 ? M * N : 0)) * esz;
        }
    }
    std::vector<TaskDesc> flat;
    std::vector<int32_t> gbeg;
    std::vector<PackInfo> packs;
    std::vector<int32_t> pbeg;
    make_groups(tasks, cap, max_tasks, flat, gbeg);
    if (tc) {
        make_packs(flat, gbeg, packs, pbeg);
        nblocks = (int64_t)packs.size();
    }

    iaat_plan_s *plan = new (std::nothrow) iaat_plan_s;
    if (!plan)
        return fail(IAAT_ERR_OOM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&plan->device);
    if (e != cudaSuccess) {
        delete plan;
        return cuda_fail(e, "cudaGetDevice");
    }
    iaat_status_t ps = prepare_device(plan->device, kernel_kind(dt, precision));
    if (ps != IAAT_OK) {
        delete plan;
        return ps;
    }
    plan->esz = esz;
    plan->dtype = (iaat_dtype_t)dt;
    plan->precision = precision;
    plan->ntasks = (int64_t)flat.size();
    plan->ngroups = (int64_t)gbeg.size() - 1;
    const int sms = sm_count(plan->device);
    plan->grid = (int)std::min<int64_t>(plan->ngroups, (int64_t)sms);
    uint32_t ring_off = 0, ring_size = 0;
    if (tc)
        tc_ring((int)precision, &ring_off, &ring_size);
    else if (cplx)
        cplx_ring(&ring_off, &ring_size);
    else
        fma_ring(esz, &ring_off, &ring_size);
    // complex plans: the scalar table, 4 components per instance in the
    // component type (16 or 32 bytes), uploaded before the programs that
    // point into it are built
    size_t scal_bytes = 0;
    const uint32_t scal_stride = (uint32_t)(2 * esz);
    if (cplx) {
        scal_bytes = std::max<size_t>(16, (size_t)count * scal_stride);
        std::vector<char> host(scal_bytes, 0);
        for (int64_t i = 0; i < count; ++i)
            for (int c = 0; c < 4; ++c) {
                if (dt == IAAT_C32) {
                    const float v = (float)cscal[4 * i + c];
                    std::memcpy(host.data() + i * scal_stride + c * 4, &v, 4);
                } else {
                    std::memcpy(host.data() + i * scal_stride + c * 8, &cscal[4 * i + c], 8);
                }
            }
        if ((e = cudaMalloc(&plan->d_scal, scal_bytes)) != cudaSuccess) {
            iaat_plan_destroy(plan);
            return fail(IAAT_ERR_OOM, "cudaMalloc of the scalar table: %s", cudaGetErrorString(e));
        }
        if ((e = cudaMemcpy(plan->d_scal, host.data(), scal_bytes, cudaMemcpyHostToDevice)) != cudaSuccess) {
            iaat_plan_destroy(plan);
            return cuda_fail(e, "upload the scalar table");
        }
    }
    std::vector<char> prog;
    std::vector<int64_t> poff;
    iaat_status_t bs = build_programs(flat, gbeg, packs, pbeg, esz, tc, plan->grid, ring_off, ring_size,
                                      cplx ? plan->d_scal : nullptr, scal_stride, prog, poff);
    if (bs != IAAT_OK) {
        iaat_plan_destroy(plan);
        return bs;
    }
    if (opts && opts->inject_fault == 1 && !prog.empty()) {
        // the first stage claims more tasks than a stage can hold
        StageProg *h = reinterpret_cast<StageProg *>(prog.data() + poff[0]);
        h->nt = (uint8_t)(kMaxGroupTasks + 1);
    }
    const size_t pb = std::max<size_t>(16, prog.size()), ob = poff.size() * sizeof(int64_t);
    if ((e = cudaMalloc(&plan->d_prog, pb)) != cudaSuccess || (e = cudaMalloc(&plan->d_poff, ob)) != cudaSuccess ||
        (e = cudaMalloc(&plan->d_err, sizeof(int32_t))) != cudaSuccess) {
        iaat_plan_destroy(plan);
        return fail(IAAT_ERR_OOM, "cudaMalloc of the plan: %s", cudaGetErrorString(e));
    }
    if ((!prog.empty() && (e = cudaMemcpy(plan->d_prog, prog.data(), prog.size(), cudaMemcpyHostToDevice)) != cudaSuccess) ||
        (e = cudaMemcpy(plan->d_poff, poff.data(), ob, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(plan->d_err, 0, sizeof(int32_t))) != cudaSuccess) {
        iaat_plan_destroy(plan);
        return cuda_fail(e, "upload the stage programs");
    }
    info.tasks = plan->ntasks;
    info.groups = plan->ngroups;
    info.blocks = nblocks;
    info.plan_bytes = (int64_t)(pb + ob + sizeof(int32_t) + scal_bytes);
    info.grid = plan->grid;
    info.kernels = plan->ngroups > 0 ? 1 : 0;
    info.kernel_family = 1;
    plan->info = info;
    *out = plan;
    return IAAT_OK;
}

extern "C" iaat_status_t iaat_plan_create(const iaat_gemm_desc_t *descs, int64_t count, iaat_dtype_t dtype,
                                          iaat_precision_t precision, const iaat_plan_options_t *opts,
                                          iaat_plan_t *out)
{
    if (!out)
        return fail(IAAT_ERR_INVALID_VALUE, "out is NULL");
    *out = nullptr;
    if (count < 0 || (count > 0 && !descs))
        return fail(IAAT_ERR_INVALID_VALUE, "bad descriptor array");
    if (dtype != IAAT_F32 && dtype != IAAT_F64)
        return fail(IAAT_ERR_INVALID_VALUE, "unknown dtype %d (complex batches: iaat_plan_create_complex)",
                    (int)dtype);
    if (precision < IAAT_PREC_DEFAULT || precision > IAAT_PREC_6XBF16)
        return fail(IAAT_ERR_INVALID_VALUE, "unknown precision %d", (int)precision);
    if (precision != IAAT_PREC_DEFAULT && dtype == IAAT_F64)
        return fail(IAAT_ERR_UNSUPPORTED, "FP64 plans run on the FP64 pipes only");
    if (opts && opts->route_k_below < 0)
        return fail(IAAT_ERR_INVALID_VALUE, "route_k_below %d is negative", opts->route_k_below);
    if (opts && opts->route_mnk_below < 0)
        return fail(IAAT_ERR_INVALID_VALUE, "route_mnk_below %d is negative", opts->route_mnk_below);
    if (opts && (opts->route_kernel < 0 || opts->route_kernel == 3 || opts->route_kernel > 4))
        return fail(IAAT_ERR_INVALID_VALUE, "route_kernel %d is not a CUDA-core kernel family (0, 1, 2, 4)",
                    opts->route_kernel);
    if (precision == IAAT_PREC_DEFAULT || !opts || (opts->route_k_below == 0 && opts->route_mnk_below == 0))
        return plan_create_impl(descs, count, dtype, precision, opts, nullptr, out);

    // Routed tensor-core plan: instances with K below route_k_below (or
    // alpha == 0, which reads neither A nor B) go to an FP32 CUDA-core plan
    // that the same iaat_gemm_grouped call launches after the tensor-core
    // one.  Every instance is validated first so errors name the caller's
    // index; each part then keeps those indices through index_map.
    for (int64_t i = 0; i < count; ++i) {
        const iaat_gemm_desc_t &g = descs[i];
        const iaat_status_t st = check_instance(i, g.M, g.N, g.K, g.lda, g.ldb, g.ldc, g.transA, g.transB, g.A, g.B,
                                                g.C, g.alpha, 4);
        if (st != IAAT_OK)
            return st;
    }
    std::vector<iaat_gemm_desc_t> dtc, dfma;
    std::vector<int64_t> itc, ifma;
    for (int64_t i = 0; i < count; ++i) {
        const int keff = descs[i].alpha == 0.0 ? 0 : descs[i].K;
        const bool small = keff < opts->route_k_below ||
                           (int64_t)descs[i].M * descs[i].N * keff < (int64_t)opts->route_mnk_below;
        (small ? dfma : dtc).push_back(descs[i]);
        (small ? ifma : itc).push_back(i);
    }
    iaat_plan_options_t o = *opts;
    o.route_k_below = 0;
    o.route_mnk_below = 0;
    iaat_plan_t main_plan = nullptr, sub = nullptr;
    iaat_status_t st = plan_create_impl(dtc.data(), (int64_t)dtc.size(), IAAT_F32, precision, &o, nullptr, &main_plan,
                                        itc.data());
    if (st != IAAT_OK)
        return st;
    o.inject_fault = 0;
    if (opts->route_kernel != 0)
        o.kernel = opts->route_kernel;
    else if (o.kernel == 3)
        o.kernel = 0;   // the CUDA-core part has no warp-tile kernel: its default plan
    st = plan_create_impl(dfma.data(), (int64_t)dfma.size(), IAAT_F32, IAAT_PREC_DEFAULT, &o, nullptr, &sub,
                          ifma.data());
    if (st != IAAT_OK) {
        iaat_plan_destroy(main_plan);
        return st;
    }
    chain_plan(main_plan, sub);
    main_plan->info.instances = count;
    *out = main_plan;
    return IAAT_OK;
}

extern "C" iaat_status_t iaat_plan_create_complex(const iaat_cgemm_desc_t *descs, int64_t count, iaat_dtype_t dtype,
                                                  const iaat_plan_options_t *opts, iaat_plan_t *out)
{
    if (!out)
        return fail(IAAT_ERR_INVALID_VALUE, "out is NULL");
    *out = nullptr;
    if (count < 0 || (count > 0 && !descs))
        return fail(IAAT_ERR_INVALID_VALUE, "bad descriptor array");
    if (dtype != IAAT_C32 && dtype != IAAT_C64)
        return fail(IAAT_ERR_INVALID_VALUE, "iaat_plan_create_complex takes IAAT_C32 or IAAT_C64 (dtype %d)",
                    (int)dtype);
    std::vector<iaat_gemm_desc_t> proxy((size_t)count);
    std::vector<double> scal((size_t)count * 4);
    for (int64_t i = 0; i < count; ++i) {
        const iaat_cgemm_desc_t &c = descs[i];
        double v[4] = {c.alpha_re, c.alpha_im, c.beta_re, c.beta_im};
        if (dtype == IAAT_C32)
            for (double &x : v)
                x = (double)(float)x;
        std::memcpy(&scal[4 * i], v, sizeof v);
        const double alpha = (v[0] != 0.0 || v[1] != 0.0) ? 1.0 : 0.0;
        const double beta = (v[2] == 0.0 && v[3] == 0.0) ? 0.0 : (v[2] == 1.0 && v[3] == 0.0) ? 1.0 : 2.0;
        proxy[i] = iaat_gemm_desc_t{c.M, c.N, c.K, c.lda, c.ldb, c.ldc, c.transA, c.transB, alpha, beta, c.A, c.B, c.C};
    }
    return plan_create_impl(proxy.data(), count, dtype, IAAT_PREC_DEFAULT, opts, scal.data(), out);
}

extern "C" iaat_status_t iaat_gemm_grouped(iaat_plan_t plan, void *stream)
{
    if (!plan)
        return fail(IAAT_ERR_INVALID_VALUE, "plan is NULL");
    if (plan->ngroups == 0)
        return plan->sub ? iaat_gemm_grouped(plan->sub, stream) : IAAT_OK;
    if (plan->ws || plan->tc2 || plan->tw || plan->wd) {
        const cudaStream_t s = static_cast<cudaStream_t>(stream);
        const cudaError_t e = plan->ws    ? launch_ws(plan->wsp, plan->grid, s)
                              : plan->wd ? launch_wd(plan->esz, plan->wdp, plan->grid, s)
                              : plan->tw ? launch_tw((int)plan->precision, plan->twp, plan->grid, s)
                                         : launch_tc2((int)plan->precision, plan->t2p, plan->grid, s);
        if (e != cudaSuccess)
            return cuda_fail(e, "kernel launch");
        if (plan->sub)   // routed small-K instances, after the tensor-core launch on the same stream
            return iaat_gemm_grouped(plan->sub, stream);
        return IAAT_OK;
    }
    KParams kp;
    std::memset(&kp, 0, sizeof kp);
    kp.p.prog = plan->d_prog;
    kp.p.poff = plan->d_poff;
    kp.p.ngroups = (int32_t)plan->ngroups;
    kp.p.err = plan->d_err;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = is_complex(plan->dtype)              ? launch_cplx(plan->dtype, kp, plan->grid, s)
                    : plan->precision != IAAT_PREC_DEFAULT ? launch_tc((int)plan->precision, kp, plan->grid, s)
                                                           : launch_fma(plan->esz == 4 ? 0 : 1, kp, plan->grid, s);
    if (e != cudaSuccess)
        return cuda_fail(e, "kernel launch");
    if (plan->sub)   // routed small-K instances, after the tensor-core launch on the same stream
        return iaat_gemm_grouped(plan->sub, stream);
    return IAAT_OK;
}

static iaat_status_t read_and_clear(int32_t *d_err, cudaStream_t s)
{
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaStreamSynchronize");
    int32_t v = 0;
    if ((e = cudaMemcpy(&v, d_err, sizeof v, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "read error word");
    if (v != 0) {
        int32_t z = 0;
        cudaMemcpy(d_err, &z, sizeof z, cudaMemcpyHostToDevice);
        return fail(IAAT_ERR_DEVICE_TIMEOUT, "device reported error bits 0x%x (1: stage never arrived, "
                                             "2: stage never released, 4: bad plan)", v);
    }
    return IAAT_OK;
}

extern "C" iaat_status_t iaat_plan_check(iaat_plan_t plan, void *stream)
{
    if (plan) {
        iaat_status_t st = read_and_clear(plan->d_err, static_cast<cudaStream_t>(stream));
        if (plan->sub) {
            const iaat_status_t s2 = iaat_plan_check(plan->sub, stream);
            if (st == IAAT_OK)
                st = s2;
        }
        return st;
    }
    int32_t *w = nullptr;
    cudaError_t e = single_call_err_ptr(&w);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGetSymbolAddress");
    int32_t *w2 = nullptr;
    if ((e = noalloc_err_ptr(&w2)) != cudaSuccess)
        return cuda_fail(e, "cudaGetDevice");
    // both words are read and cleared; the first error found is returned
    const iaat_status_t st1 = w2 ? read_and_clear(w2, static_cast<cudaStream_t>(stream)) : IAAT_OK;
    const iaat_status_t st2 = read_and_clear(w, static_cast<cudaStream_t>(stream));
    return st1 != IAAT_OK ? st1 : st2;
}

extern "C" iaat_status_t iaat_plan_info(iaat_plan_t plan, iaat_plan_info_t *info)
{
    if (!plan || !info)
        return fail(IAAT_ERR_INVALID_VALUE, "NULL argument");
    *info = plan->info;
    return IAAT_OK;
}

extern "C" iaat_status_t iaat_plan_destroy(iaat_plan_t plan)
{
    if (!plan)
        return IAAT_OK;
    if (plan->sub)
        iaat_plan_destroy(plan->sub);
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != plan->device)
        cudaSetDevice(plan->device);
    cudaDeviceSynchronize();
    if (plan->d_prog)
        cudaFree(plan->d_prog);
    if (plan->d_poff)
        cudaFree(plan->d_poff);
    if (plan->d_err && !plan->ws && !plan->tw && !plan->wd)
        cudaFree(plan->d_err);
    if (plan->d_wd)
        cudaFree(plan->d_wd);
    if (plan->d_ws)
        cudaFree(plan->d_ws);
    if (plan->d_tw)
        cudaFree(plan->d_tw);
    if (plan->d_gbeg)
        cudaFree(plan->d_gbeg);
    if (plan->d_scal)
        cudaFree(plan->d_scal);
    if (cur >= 0 && cur != plan->device)
        cudaSetDevice(cur);
    delete plan;
    return IAAT_OK;
}

// ---------------------------------------------------- single GEMM call

static iaat_status_t single_gemm(int esz, int ta, int tb, int M, int N, int K, double alpha, const void *A,
                                 int lda, const void *B, int ldb, double beta, void *C, int ldc, void *stream)
{
    iaat_status_t st = check_instance(0, M, N, K, lda, ldb, ldc, ta, tb, A, B, C, alpha, esz);
    if (st != IAAT_OK)
        return st;
    iaat_gemm_desc_t g{M, N, K, lda, ldb, ldc, ta, tb, alpha, beta, A, B, C};
    std::vector<HostTask> tasks;
    int64_t nb = 0;
    // one instance per call: an FP64 instance is cut into pieces of about
    // 16 x 16 of C, as many as the parameter block holds, so that they run on
    // that many SMs -- one SM's DFMA rate (about 8 GFLOP/s) would otherwise
    // set the latency (measured: 80^3 from 92 to 36 us).  FP32 is not cut: at
    // 60x that rate the extra CTAs and operand re-reads cost more than they
    // save (48^3: 8 -> 15 us when cut).
    int piece = 0;
    if (esz == 8) {
        piece = 16;
        while (piece < kPieceRows && (int64_t)((M + piece - 1) / piece) * ((N + piece - 1) / piece) > kInline)
            piece *= 2;
    }
    st = make_tasks(0, g, esz == 4 ? IAAT_F32 : IAAT_F64, false, -1, (uint32_t)(esz == 4 ? max_group_bytes<4>() : max_group_bytes<8>()), tasks,
                    &nb, piece);
    if (st != IAAT_OK)
        return st;
    if (tasks.empty())
        return IAAT_OK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGetDevice");
    st = prepare_device(dev, kernel_kind(esz == 4 ? IAAT_F32 : IAAT_F64, IAAT_PREC_DEFAULT));
    if (st != IAAT_OK)
        return st;
    int32_t *w = nullptr;
    if ((e = single_call_err_ptr(&w)) != cudaSuccess)
        return cuda_fail(e, "cudaGetSymbolAddress");
    // The pieces travel in the kernel's parameter block, kInline per launch:
    // an instance cut into more pieces (e.g. 512000 x 1 x 1) takes several
    // launches on the stream, one after another, and no device memory.
    for (size_t t0 = 0; t0 < tasks.size(); t0 += kInline) {
        const size_t n = std::min(tasks.size() - t0, (size_t)kInline);
        KParams kp;
        std::memset(&kp, 0, sizeof kp);
        for (size_t i = 0; i < n; ++i) {
            kp.inline_tasks[i] = tasks[t0 + i].d;
            kp.inline_gbeg[i] = (int32_t)i;
        }
        kp.inline_gbeg[n] = (int32_t)n;
        kp.p.tasks = nullptr;
        kp.p.gbeg = nullptr;
        kp.p.ngroups = (int32_t)n;
        kp.p.err = w;
        e = launch_fma(esz == 4 ? 0 : 1, kp, (int)n, static_cast<cudaStream_t>(stream));
        if (e != cudaSuccess)
            return cuda_fail(e, "kernel launch");
    }
    return IAAT_OK;
}

extern "C" iaat_status_t iaat_sgemm(int transA, int transB, int M, int N, int K, float alpha, const float *A,
                                    int lda, const float *B, int ldb, float beta, float *C, int ldc, void *stream)
{
    return single_gemm(4, transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, stream);
}

extern "C" iaat_status_t iaat_dgemm(int transA, int transB, int M, int N, int K, double alpha, const double *A,
                                    int lda, const double *B, int ldb, double beta, double *C, int ldc,
                                    void *stream)
{
    return single_gemm(8, transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, stream);
}

// ------------------------------------------- single complex GEMM call
// One CGEMM / ZGEMM instance per call.  Complex tasks carry their scalars in
// a table, so these calls plan on the host like a plan does, but into the
// kernel's fixed single-call scratch (no allocation): the instance is cut
// into pieces of about piece x piece of C, each its own stage, so that the
// pieces run on as many SMs (one SM's DFMA rate would otherwise set the
// latency), and the scalars, program offsets and stage programs are copied
// into the scratch on the caller's stream before the launch.
static std::mutex g_cplx_single_mutex;
constexpr int kCplxSinglePieces = 152;   // pieces (stages) of one call at most, before pieces grow

static iaat_status_t single_complex(int dt, int ta, int tb, int M, int N, int K, const double *alpha, const void *A,
                                    int lda, const void *B, int ldb, const double *beta, void *C, int ldc, void *stream)
{
    const int esz = dtype_esz(dt);
    if (!alpha || !beta)
        return fail(IAAT_ERR_INVALID_VALUE, "alpha or beta is NULL");
    double v[4] = {alpha[0], alpha[1], beta[0], beta[1]};
    if (dt == IAAT_C32)
        for (double &x : v)
            x = (double)(float)x;
    const double am = (v[0] != 0.0 || v[1] != 0.0) ? 1.0 : 0.0;
    const double bm = (v[2] == 0.0 && v[3] == 0.0) ? 0.0 : (v[2] == 1.0 && v[3] == 0.0) ? 1.0 : 2.0;
    iaat_status_t st = check_instance(0, M, N, K, lda, ldb, ldc, ta, tb, A, B, C, am, esz);
    if (st != IAAT_OK)
        return st;
    iaat_gemm_desc_t g{M, N, K, lda, ldb, ldc, ta, tb, am, bm, A, B, C};
    const uint32_t cap = (uint32_t)cplx_max_group_bytes();
    int piece = dt == IAAT_C64 ? 16 : 32;
    while (piece < kPieceRows && (int64_t)((M + piece - 1) / piece) * ((N + piece - 1) / piece) > kCplxSinglePieces)
        piece *= 2;
    std::vector<HostTask> tasks;
    int64_t nb = 0;
    st = make_tasks(0, g, dt, false, -1, cap, tasks, &nb, piece);
    if (st != IAAT_OK)
        return st;
    if (tasks.empty())
        return IAAT_OK;
    std::vector<TaskDesc> flat;
    std::vector<int32_t> gbeg;
    make_groups(tasks, cap, 1, flat, gbeg);   // one piece per stage
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGetDevice");
    st = prepare_device(dev, kernel_kind(dt, IAAT_PREC_DEFAULT));
    if (st != IAAT_OK)
        return st;
    const int ng = (int)gbeg.size() - 1;
    const int grid = std::min(ng, sm_count(dev));
    std::lock_guard<std::mutex> lk(g_cplx_single_mutex);
    char *scr = nullptr;
    size_t scr_bytes = 0;
    if ((e = cplx_single_scratch(&scr, &scr_bytes)) != cudaSuccess)
        return cuda_fail(e, "cudaGetSymbolAddress of the single-call scratch");
    uint32_t ring_off = 0, ring_bytes = 0;
    cplx_ring(&ring_off, &ring_bytes);
    std::vector<char> prog;
    std::vector<int64_t> poff;
    const uint32_t stride = (uint32_t)(2 * esz);
    st = build_programs(flat, gbeg, std::vector<PackInfo>(), std::vector<int32_t>(), esz, false, grid, ring_off,
                        ring_bytes, scr, stride, prog, poff);
    if (st != IAAT_OK)
        return st;
    const size_t poff_at = 256, prog_at = poff_at + ((poff.size() * sizeof(int64_t) + 255) & ~(size_t)255);
    if (prog_at + prog.size() > scr_bytes)
        return fail(IAAT_ERR_UNSUPPORTED, "the call's stage programs (%zu bytes) exceed the single-call scratch",
                    prog.size());
    char sc[32];
    for (int c = 0; c < 4; ++c) {
        if (dt == IAAT_C32) {
            const float f = (float)v[c];
            std::memcpy(sc + 4 * c, &f, 4);
        } else {
            std::memcpy(sc + 8 * c, &v[c], 8);
        }
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // pageable sources: each copy has taken its bytes when it returns
    if ((e = cudaMemcpyAsync(scr, sc, stride, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(scr + poff_at, poff.data(), poff.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(scr + prog_at, prog.data(), prog.size(), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_fail(e, "copy into the single-call scratch");
    KParams kp;
    std::memset(&kp, 0, sizeof kp);
    kp.p.prog = scr + prog_at;
    kp.p.poff = reinterpret_cast<const int64_t *>(scr + poff_at);
    kp.p.ngroups = (int32_t)ng;
    int32_t *w = nullptr;
    if ((e = single_call_err_ptr(&w)) != cudaSuccess)
        return cuda_fail(e, "cudaGetSymbolAddress");
    kp.p.err = w;
    if ((e = launch_cplx(dt, kp, grid, s)) != cudaSuccess)
        return cuda_fail(e, "kernel launch");
    return IAAT_OK;
}

extern "C" iaat_status_t iaat_cgemm(int transA, int transB, int M, int N, int K, const float *alpha, const void *A,
                                    int lda, const void *B, int ldb, const float *beta, void *C, int ldc, void *stream)
{
    if (!alpha || !beta)
        return fail(IAAT_ERR_INVALID_VALUE, "alpha or beta is NULL");
    const double a[2] = {alpha[0], alpha[1]}, b[2] = {beta[0], beta[1]};
    return single_complex(IAAT_C32, transA, transB, M, N, K, a, A, lda, B, ldb, b, C, ldc, stream);
}

extern "C" iaat_status_t iaat_zgemm(int transA, int transB, int M, int N, int K, const double *alpha, const void *A,
                                    int lda, const void *B, int ldb, const double *beta, void *C, int ldc, void *stream)
{
    return single_complex(IAAT_C64, transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, stream);
}

extern "C" iaat_status_t iaat_fma_peak(iaat_dtype_t dtype, double *gflops)
{
    if ((dtype != IAAT_F32 && dtype != IAAT_F64) || !gflops)
        return fail(IAAT_ERR_INVALID_VALUE, "bad argument");
    cudaError_t e = measure_fma_peak(dtype == IAAT_F32 ? 0 : 1, gflops);
    if (e != cudaSuccess)
        return cuda_fail(e, "FMA peak probe");
    return IAAT_OK;
}

// ------------------------------------------- allocation-free planning
// The planning of iaat_plan_create, written into fixed arrays supplied by
// the caller instead of growing containers, for the entry point that must
// not allocate (iaat_gemm_grouped_noalloc).  Same validation, tiling,
// piece splitting, ordering and stage cutting as the regular planner.
iaat_status_t iaat::noalloc_plan(const iaat_gemm_desc_t *descs, int64_t count, int esz, int max_tasks,
                                 TaskDesc *tasks, uint32_t *bytes, double *cost, int32_t *order, TaskDesc *out,
                                 int32_t *gbeg, int64_t *ntasks_out, int64_t *ngroups_out)
{
    const uint32_t cap = (uint32_t)(esz == 4 ? max_group_bytes<4>() : max_group_bytes<8>());
    int64_t nt = 0;
    for (int64_t i = 0; i < count; ++i) {
        const iaat_gemm_desc_t &g = descs[i];
        iaat_status_t st = check_instance(i, g.M, g.N, g.K, g.lda, g.ldb, g.ldc, g.transA, g.transB, g.A, g.B, g.C,
                                          g.alpha, esz);
        if (st != IAAT_OK)
            return st;
        const int M = g.M, N = g.N;
        if (M == 0 || N == 0)
            continue;
        const int Keff = (g.alpha == 0.0) ? 0 : g.K;
        if (Keff == 0 && g.beta == 1.0)
            continue;
        int pm = 1, pn = 1;
        if (!choose_split(g, esz, Keff, cap, kPieceRows, kPieceCols, pm, pn))
            return fail(IAAT_ERR_UNSUPPORTED, "instance %lld: operands do not fit a pipeline stage (M=%d N=%d K=%d)",
                        (long long)i, M, N, g.K);
        if (nt + (int64_t)pm * pn > max_tasks)
            return fail(IAAT_ERR_INVALID_VALUE,
                        "instance %lld: the batch needs more than %d tasks, the limit of the allocation-free "
                        "entry point", (long long)i, max_tasks);
        for (int pi = 0; pi < pm; ++pi) {
            int r0, h;
            piece_range(M, pm, pi, r0, h);
            for (int pj = 0; pj < pn; ++pj) {
                int c0, w;
                piece_range(N, pn, pj, c0, w);
                TaskDesc d = make_piece(g, esz, Keff, r0, h, c0, w);
                const int dt = esz == 4 ? IAAT_F32 : IAAT_F64;
                const TileChoice t = choose_tiling(dt, h, w, Keff, -1, true, stage_min_blocks(d, dt, cap));
                d.variant = (uint8_t)t.variant;
                d.nbm = (uint8_t)t.nbm;
                d.nbn = (uint8_t)t.nbn;
                const TaskStages sg = plan_task(d, esz);
                tasks[nt] = d;
                bytes[nt] = sg.total();
                cost[nt] = (double)(sg.a.tx + sg.b.tx + sg.c.tx) + tuning().cost_per_slot * t.cost;
                ++nt;
            }
        }
    }
    // largest cost first, ties in input order (the regular planner's stable order)
    for (int64_t k = 0; k < nt; ++k)
        order[k] = (int32_t)k;
    std::sort(order, order + nt, [cost](int32_t a, int32_t b) {
        return cost[a] > cost[b] || (cost[a] == cost[b] && a < b);
    });
    int group_tasks = kMaxGroupTasks;
    {
        const int tuned = esz == 8 ? tuning().group_tasks_f64 : tuning().group_tasks[0];
        if (tuned > 0)
            group_tasks = tuned;
    }
    int64_t ng = 0;
    uint32_t used = 0;
    int in_group = 0;
    const uint32_t target = cap;   // the regular planner's stage size
    for (int64_t k = 0; k < nt; ++k) {
        const int32_t t = order[k];
        if (in_group == 0 || in_group >= group_tasks || used + bytes[t] > target) {
            gbeg[ng++] = (int32_t)k;
            used = 0;
            in_group = 0;
        }
        out[k] = tasks[t];
        used += bytes[t];
        ++in_group;
    }
    gbeg[ng] = (int32_t)nt;
    *ntasks_out = nt;
    *ngroups_out = ng;
    return IAAT_OK;
}

iaat_status_t iaat::noalloc_fail(iaat_status_t st, const char *msg) { return fail(st, "%s", msg); }

iaat_status_t iaat::noalloc_prepare(int dev)
{
    return prepare_device(dev, 0) == IAAT_OK && prepare_device(dev, 1) == IAAT_OK ? IAAT_OK : IAAT_ERR_CUDA;
}

int iaat::noalloc_sm_count(int dev) { return sm_count(dev); }

// Error reporting and validation for the other translation units (the pack
// step of pack.cu).
iaat_status_t iaat::host_fail(iaat_status_t st, const char *msg) { return fail(st, "%s", msg); }

iaat_status_t iaat::validate_instance(int64_t idx, const iaat_gemm_desc_t &g, int esz)
{
    return check_instance(idx, g.M, g.N, g.K, g.lda, g.ldb, g.ldc, g.transA, g.transB, g.A, g.B, g.C, g.alpha, esz);
}
