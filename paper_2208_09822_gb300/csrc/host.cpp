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

static const Variant *variants(int esz, int *n)
{
    if (esz == 4) {
        *n = kNumVariantsF32;
        return kVariantsF32;
    }
    *n = kNumVariantsF64;
    return kVariantsF64;
}

namespace iaat {
// The tiler's cost model without the tuned per-variant scale (the
// autotuner calibrates against it).
double model_block_cost(const Variant &v, int esz, int K);
}

static double block_cost(const Variant &v, int esz, int K) { return iaat::model_block_cost(v, esz, K); }

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

static TileChoice choose_tiling(int esz, int M, int N, int K, int force_variant)
{
    int nv;
    const Variant *vs = variants(esz, &nv);
    TileChoice best{0, 1, 1, 1e300};
    for (int v = 0; v < nv; ++v) {
        if (force_variant >= 0 && v != force_variant)
            continue;
        const int bm = vs[v].lm * vs[v].mr, bn = vs[v].ln * vs[v].nr;
        const int nbm = std::max(1, (M + bm - 1) / bm), nbn = std::max(1, (N + bn - 1) / bn);
        if (nbm > 255 || nbn > 255)
            continue;
        const double c = (double)nbm * nbn * block_cost(vs[v], esz, K) * tuning().variant_scale(esz, v);
        if (c < best.cost)
            best = TileChoice{v, nbm, nbn, c};
    }
    return best;
}

extern "C" int64_t iaat_tile(iaat_dtype_t dtype, int transA, int transB, int M, int N, int K, int32_t *blocks,
                             int64_t cap)
{
    (void)transA;
    (void)transB;
    if ((dtype != IAAT_F32 && dtype != IAAT_F64) || M < 0 || N < 0 || K < 0 || cap < 0 || (cap > 0 && !blocks))
        return -1;
    if (M == 0 || N == 0)
        return 0;
    const int esz = dtype == IAAT_F32 ? 4 : 8;
    const TileChoice t = choose_tiling(esz, M, N, K, -1);
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
    TaskDesc *d_tasks = nullptr;
    int32_t *d_gbeg = nullptr;
    int32_t *d_err = nullptr;
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
bool g_prepared[64][5];

// kind: 0 = FP32 FFMA, 1 = FP64 DFMA, 2.. = tcgen05 precision (kind - 1)
iaat_status_t prepare_device(int dev, int kind)
{
    std::lock_guard<std::mutex> lk(g_prep_mutex);
    if (dev < 0 || dev >= 64)
        return fail(IAAT_ERR_CUDA, "device index %d out of range", dev);
    if (!g_prepared[dev][kind]) {
        cudaError_t e = kind < 2 ? prepare_fma(kind) : prepare_tc(kind - 1);
        if (e != cudaSuccess)
            return cuda_fail(e, "cudaFuncSetAttribute");
        g_prepared[dev][kind] = true;
    }
    return IAAT_OK;
}

int kernel_kind(int esz, iaat_precision_t prec) { return prec != IAAT_PREC_DEFAULT ? 1 + (int)prec : (esz == 4 ? 0 : 1); }

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

// Build the tasks of one instance (one, or several column pieces when its
// operands do not fit one stage).
iaat_status_t make_tasks(int64_t idx, const iaat_gemm_desc_t &g, int esz, int force_variant, uint32_t cap,
                         std::vector<HostTask> &out, int64_t *blocks_out)
{
    const int M = g.M, N = g.N;
    if (M == 0 || N == 0)
        return IAAT_OK;
    const int Keff = (g.alpha == 0.0) ? 0 : g.K;
    if (Keff == 0 && g.beta == 1.0)
        return IAAT_OK;   // C = 1*C: nothing to do
    for (int pieces = 1; pieces <= N; ++pieces) {
        const int width = (N + pieces - 1) / pieces;
        const int np = (N + width - 1) / width;
        std::vector<HostTask> tmp;
        bool fits = true;
        for (int p = 0; p < np && fits; ++p) {
            const int c0 = p * width;
            const int nw = std::min(width, N - c0);
            TaskDesc d{};
            d.A = static_cast<const char *>(g.A);
            d.B = g.B ? static_cast<const char *>(g.B) +
                            (size_t)(g.transB ? (int64_t)c0 : (int64_t)c0 * g.ldb) * esz
                      : nullptr;
            d.C = static_cast<char *>(g.C) + (size_t)((int64_t)c0 * g.ldc) * esz;
            d.lda = g.lda;
            d.ldb = g.ldb;
            d.ldc = g.ldc;
            d.M = (int16_t)M;
            d.N = (int16_t)nw;
            d.K = (int16_t)Keff;
            d.ta = (uint8_t)g.transA;
            d.tb = (uint8_t)g.transB;
            d.flags = (g.beta != 0.0) ? kFlagReadC : 0;
            d.alpha = g.alpha;
            d.beta = g.beta;
            if (esz == 4) {
                d.alpha = (double)(float)g.alpha;
                d.beta = (double)(float)g.beta;
            }
            const TileChoice t = choose_tiling(esz, M, nw, Keff, force_variant);
            d.variant = (uint8_t)t.variant;
            d.nbm = (uint8_t)t.nbm;
            d.nbn = (uint8_t)t.nbn;
            const TaskStages st = plan_task(d, esz);
            const uint32_t bytes = st.total();
            if (bytes > cap) {
                fits = false;
                break;
            }
            tmp.push_back(HostTask{d, bytes, (double)(st.a.tx + st.b.tx + st.c.tx) + tuning().cost_per_slot * t.cost});
        }
        if (fits) {
            for (auto &t : tmp) {
                *blocks_out += (int64_t)t.d.nbm * t.d.nbn;
                out.push_back(t);
            }
            return IAAT_OK;
        }
    }
    return fail(IAAT_ERR_UNSUPPORTED, "instance %lld: operands do not fit a pipeline stage", (long long)idx);
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
// stack them into packs of at most 128 rows and 128 columns (one MMA tile
// each).  A task's pack index, row offset and column offset travel in its
// variant / nbm / nbn fields.  Returns the number of packs.
int64_t make_packs(std::vector<TaskDesc> &flat, const std::vector<int32_t> &gbeg)
{
    int64_t npacks = 0;
    for (size_t g = 0; g + 1 < gbeg.size(); ++g) {
        auto b = flat.begin() + gbeg[g], e = flat.begin() + gbeg[g + 1];
        std::stable_sort(b, e, [](const TaskDesc &x, const TaskDesc &y) { return x.K > y.K; });
        int pack = 0, rows = 0, cols = 0;
        for (auto it = b; it != e; ++it) {
            if (rows > 0 && (rows + it->M > kTcPackRows || cols + it->N > kTcPackCols)) {
                ++pack;
                rows = 0;
                cols = 0;
            }
            it->variant = (uint8_t)pack;
            it->nbm = (uint8_t)rows;
            it->nbn = (uint8_t)cols;
            rows += it->M;
            cols += it->N;
        }
        npacks += pack + 1;
    }
    return npacks;
}

}  // namespace

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
        return fail(IAAT_ERR_INVALID_VALUE, "unknown dtype %d", (int)dtype);
    if (precision < IAAT_PREC_DEFAULT || precision > IAAT_PREC_FP16)
        return fail(IAAT_ERR_INVALID_VALUE, "unknown precision %d", (int)precision);
    if (precision != IAAT_PREC_DEFAULT && dtype == IAAT_F64)
        return fail(IAAT_ERR_UNSUPPORTED, "FP64 plans run on the FP64 pipes only");
    const int esz = dtype == IAAT_F32 ? 4 : 8;
    const bool tc = precision != IAAT_PREC_DEFAULT;
    const uint32_t cap = tc ? (uint32_t)tc_group_cap((int)precision)
                            : (uint32_t)(esz == 4 ? max_group_bytes<4>() : max_group_bytes<8>());
    int max_tasks = kMaxGroupTasks;
    {
        const int tuned = dtype == IAAT_F64 ? tuning().group_tasks_f64 : tuning().group_tasks[(int)precision];
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
            variants(esz, &nv);
            if (opts->force_variant > nv)
                return fail(IAAT_ERR_INVALID_VALUE, "force_variant %d out of range", opts->force_variant);
            force_variant = opts->force_variant - 1;
        }
        if (opts->ctas_per_sm > 0)
            ctas_per_sm = 1;   // the kernel takes all shared memory: one CTA per SM
    }
    (void)ctas_per_sm;

    std::vector<HostTask> tasks;
    tasks.reserve((size_t)count);
    iaat_plan_info_t info{};
    info.instances = count;
    info.dtype = dtype;
    info.precision = precision;
    int64_t nblocks = 0;
    for (int64_t i = 0; i < count; ++i) {
        const iaat_gemm_desc_t &g = descs[i];
        iaat_status_t st = check_instance(i, g.M, g.N, g.K, g.lda, g.ldb, g.ldc, g.transA, g.transB, g.A, g.B, g.C,
                                          g.alpha, esz);
        if (st != IAAT_OK)
            return st;
        const size_t before = tasks.size();
        st = make_tasks(i, g, esz, force_variant, cap, tasks, &nblocks);
        if (st != IAAT_OK)
            return st;
        if (tasks.size() > before) {
            info.active += 1;
            const int64_t M = g.M, N = g.N, K = (g.alpha == 0.0) ? 0 : g.K;
            info.flops += 2 * M * N * g.K * (g.alpha == 0.0 ? 0 : 1);
            info.algorithmic_bytes += (M * K + K * N + M * N + (g.beta != 0.0 ? M * N : 0)) * esz;
        }
    }
    std::vector<TaskDesc> flat;
    std::vector<int32_t> gbeg;
    make_groups(tasks, cap, max_tasks, flat, gbeg);
    if (tc)
        nblocks = make_packs(flat, gbeg);
    if (opts && opts->inject_fault == 1 && gbeg.size() >= 2)
        gbeg[1] = gbeg[0] + kMaxGroupTasks + 1;   // a stage the kernel must reject

    iaat_plan_s *plan = new (std::nothrow) iaat_plan_s;
    if (!plan)
        return fail(IAAT_ERR_OOM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&plan->device);
    if (e != cudaSuccess) {
        delete plan;
        return cuda_fail(e, "cudaGetDevice");
    }
    iaat_status_t ps = prepare_device(plan->device, kernel_kind(esz, precision));
    if (ps != IAAT_OK) {
        delete plan;
        return ps;
    }
    plan->esz = esz;
    plan->dtype = dtype;
    plan->precision = precision;
    plan->ntasks = (int64_t)flat.size();
    plan->ngroups = (int64_t)gbeg.size() - 1;
    const size_t tb = std::max<size_t>(1, flat.size()) * sizeof(TaskDesc);
    const size_t gb = gbeg.size() * sizeof(int32_t);
    if ((e = cudaMalloc(&plan->d_tasks, tb)) != cudaSuccess || (e = cudaMalloc(&plan->d_gbeg, gb)) != cudaSuccess ||
        (e = cudaMalloc(&plan->d_err, sizeof(int32_t))) != cudaSuccess) {
        iaat_plan_destroy(plan);
        return fail(IAAT_ERR_OOM, "cudaMalloc of the plan: %s", cudaGetErrorString(e));
    }
    if (!flat.empty() && (e = cudaMemcpy(plan->d_tasks, flat.data(), flat.size() * sizeof(TaskDesc),
                                         cudaMemcpyHostToDevice)) != cudaSuccess) {
        iaat_plan_destroy(plan);
        return cuda_fail(e, "upload tasks");
    }
    if ((e = cudaMemcpy(plan->d_gbeg, gbeg.data(), gb, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(plan->d_err, 0, sizeof(int32_t))) != cudaSuccess) {
        iaat_plan_destroy(plan);
        return cuda_fail(e, "upload groups");
    }
    const int sms = sm_count(plan->device);
    plan->grid = (int)std::min<int64_t>(plan->ngroups, (int64_t)sms);
    info.tasks = plan->ntasks;
    info.groups = plan->ngroups;
    info.blocks = nblocks;
    info.plan_bytes = (int64_t)(tb + gb + sizeof(int32_t));
    info.grid = plan->grid;
    info.kernels = plan->ngroups > 0 ? 1 : 0;
    plan->info = info;
    *out = plan;
    return IAAT_OK;
}

extern "C" iaat_status_t iaat_gemm_grouped(iaat_plan_t plan, void *stream)
{
    if (!plan)
        return fail(IAAT_ERR_INVALID_VALUE, "plan is NULL");
    if (plan->ngroups == 0)
        return IAAT_OK;
    KParams kp;
    std::memset(&kp, 0, sizeof kp);
    kp.p.tasks = plan->d_tasks;
    kp.p.gbeg = plan->d_gbeg;
    kp.p.ngroups = (int32_t)plan->ngroups;
    kp.p.err = plan->d_err;
    cudaError_t e = plan->precision != IAAT_PREC_DEFAULT
                        ? launch_tc((int)plan->precision, kp, plan->grid, static_cast<cudaStream_t>(stream))
                        : launch_fma(plan->esz == 4 ? 0 : 1, kp, plan->grid, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess)
        return cuda_fail(e, "kernel launch");
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
    int32_t *w = nullptr;
    if (plan) {
        w = plan->d_err;
    } else {
        cudaError_t e = single_call_err_ptr(&w);
        if (e != cudaSuccess)
            return cuda_fail(e, "cudaGetSymbolAddress");
        int32_t *w2 = nullptr;
        if ((e = noalloc_err_ptr(&w2)) != cudaSuccess)
            return cuda_fail(e, "cudaGetDevice");
        if (w2) {
            const iaat_status_t st = read_and_clear(w2, static_cast<cudaStream_t>(stream));
            if (st != IAAT_OK)
                return st;
        }
    }
    return read_and_clear(w, static_cast<cudaStream_t>(stream));
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
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != plan->device)
        cudaSetDevice(plan->device);
    cudaDeviceSynchronize();
    if (plan->d_tasks)
        cudaFree(plan->d_tasks);
    if (plan->d_gbeg)
        cudaFree(plan->d_gbeg);
    if (plan->d_err)
        cudaFree(plan->d_err);
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
    st = make_tasks(0, g, esz, -1, (uint32_t)(esz == 4 ? max_group_bytes<4>() : max_group_bytes<8>()), tasks, &nb);
    if (st != IAAT_OK)
        return st;
    if (tasks.empty())
        return IAAT_OK;
    if (tasks.size() > (size_t)kInline)
        return fail(IAAT_ERR_UNSUPPORTED, "instance needs %zu pieces", tasks.size());
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGetDevice");
    st = prepare_device(dev, kernel_kind(esz, IAAT_PREC_DEFAULT));
    if (st != IAAT_OK)
        return st;
    KParams kp;
    std::memset(&kp, 0, sizeof kp);
    for (size_t i = 0; i < tasks.size(); ++i) {
        kp.inline_tasks[i] = tasks[i].d;
        kp.inline_gbeg[i] = (int32_t)i;
    }
    kp.inline_gbeg[tasks.size()] = (int32_t)tasks.size();
    kp.p.tasks = nullptr;
    kp.p.gbeg = nullptr;
    kp.p.ngroups = (int32_t)tasks.size();
    int32_t *w = nullptr;
    if ((e = single_call_err_ptr(&w)) != cudaSuccess)
        return cuda_fail(e, "cudaGetSymbolAddress");
    kp.p.err = w;
    e = launch_fma(esz == 4 ? 0 : 1, kp, (int)tasks.size(), static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess)
        return cuda_fail(e, "kernel launch");
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
// column splitting, ordering and stage cutting as the regular planner.
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
        bool placed = false;
        for (int pieces = 1; pieces <= N && !placed; ++pieces) {
            const int width = (N + pieces - 1) / pieces;
            const int np = (N + width - 1) / width;
            if (nt + np > max_tasks)
                return fail(IAAT_ERR_INVALID_VALUE,
                            "instance %lld: the batch needs more than %d tasks, the limit of the allocation-free "
                            "entry point", (long long)i, max_tasks);
            bool fits = true;
            for (int p = 0; p < np && fits; ++p) {
                const int c0 = p * width;
                const int nw = std::min(width, N - c0);
                TaskDesc d{};
                d.A = static_cast<const char *>(g.A);
                d.B = g.B ? static_cast<const char *>(g.B) +
                                (size_t)(g.transB ? (int64_t)c0 : (int64_t)c0 * g.ldb) * esz
                          : nullptr;
                d.C = static_cast<char *>(g.C) + (size_t)((int64_t)c0 * g.ldc) * esz;
                d.lda = g.lda;
                d.ldb = g.ldb;
                d.ldc = g.ldc;
                d.M = (int16_t)M;
                d.N = (int16_t)nw;
                d.K = (int16_t)Keff;
                d.ta = (uint8_t)g.transA;
                d.tb = (uint8_t)g.transB;
                d.flags = (g.beta != 0.0) ? kFlagReadC : 0;
                d.alpha = esz == 4 ? (double)(float)g.alpha : g.alpha;
                d.beta = esz == 4 ? (double)(float)g.beta : g.beta;
                const TileChoice t = choose_tiling(esz, M, nw, Keff, -1);
                d.variant = (uint8_t)t.variant;
                d.nbm = (uint8_t)t.nbm;
                d.nbn = (uint8_t)t.nbn;
                const TaskStages sg = plan_task(d, esz);
                if (sg.total() > cap) {
                    fits = false;
                    break;
                }
                tasks[nt + p] = d;
                bytes[nt + p] = sg.total();
                cost[nt + p] = (double)(sg.a.tx + sg.b.tx + sg.c.tx) + tuning().cost_per_slot * t.cost;
            }
            if (fits) {
                nt += np;
                placed = true;
            }
        }
        if (!placed)
            return fail(IAAT_ERR_UNSUPPORTED, "instance %lld: operands do not fit a pipeline stage", (long long)i);
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
