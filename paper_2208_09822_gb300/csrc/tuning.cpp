// Autotuning (the GPU counterpart of the paper's install-time tuning,
// Sec. III-A / Sec. IV) and its JSON cache.
//
// iaat_autotune measures, on the current GPU:
//  * for the CUDA-core kernels, every register-tile variant on a batch whose
//    shapes fill that variant's warp blocks exactly; the ratio of measured
//    time to the tiler's cost model becomes the variant's cost scale, so the
//    run-time tiler (Sec. V-A) ranks variants by what they really cost here;
//  * for every kernel, the stage size (tasks per pipeline stage) on an
//    uneven batch shaped like the workload the library targets;
//  * for FP32, on the same batch, which kernel family a default plan runs:
//    the stage-program kernels, the stream kernels, or (tensor-core
//    precisions) the warp-tile kernel; another family than the stage
//    programs only when it is at least 3 % faster.
// The result is written as JSON and read back by later processes through
// IAAT_TUNE_CACHE (or applied to the calling process at once).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/iaat.h"
#include "tuning.h"

namespace iaat {

namespace {
std::once_flag g_once;
std::mutex g_mutex;
Tuning g_tuning;

bool read_array(const std::string &txt, const char *key, float *dst, int n)
{
    std::string k = std::string("\"") + key + "\"";
    size_t p = txt.find(k);
    if (p == std::string::npos)
        return false;
    p = txt.find('[', p);
    if (p == std::string::npos)
        return false;
    const char *s = txt.c_str() + p + 1;
    std::vector<float> tmp(n);
    for (int i = 0; i < n; ++i) {
        char *end = nullptr;
        double v = std::strtod(s, &end);
        if (end == s || !(v > 0.0) || v > 1e6)
            return false;
        tmp[i] = (float)v;
        s = end;
        while (*s == ' ' || *s == ',' || *s == '\n' || *s == '\t' || *s == '\r')
            ++s;
    }
    std::copy(tmp.begin(), tmp.end(), dst);
    return true;
}

bool read_int(const std::string &txt, const char *key, int *dst, int lo, int hi)
{
    std::string k = std::string("\"") + key + "\"";
    size_t p = txt.find(k);
    if (p == std::string::npos)
        return false;
    p = txt.find(':', p);
    if (p == std::string::npos)
        return false;
    long v = std::strtol(txt.c_str() + p + 1, nullptr, 10);
    if (v < lo || v > hi)
        return false;
    *dst = (int)v;
    return true;
}

void apply_text(const std::string &txt, Tuning &t)
{
    bool a = read_array(txt, "variant_scale_f32", t.scale_f32, kNumVariantsF32);
    bool b = read_array(txt, "variant_scale_f64", t.scale_f64, kNumVariantsF64);
    for (int i = 0; i < 5; ++i) {
        static const char *keys[5] = {"group_tasks_ffma", "group_tasks_3xbf16", "group_tasks_tf32",
                                      "group_tasks_fp16", "group_tasks_6xbf16"};
        if (read_int(txt, keys[i], &t.group_tasks[i], 1, kMaxGroupTasks))
            a = true;
    }
    read_int(txt, "group_tasks_dfma", &t.group_tasks_f64, 1, kMaxGroupTasks);
    for (int i = 0; i < 5; ++i) {
        static const char *keys[5] = {"kernel_ffma", "kernel_3xbf16", "kernel_tf32", "kernel_fp16", "kernel_6xbf16"};
        int k = 0;
        // FFMA: stage programs, stream or warp-direct; tensor cores: stage
        // programs, stream or warp-tile
        if (read_int(txt, keys[i], &k, 1, 4) && (i == 0 ? k != 3 : k != 4))
            t.kernel[i] = k;
    }
    t.from_cache = a || b;
}

bool read_string(const std::string &txt, const char *key, std::string *dst)
{
    std::string k = std::string("\"") + key + "\"";
    size_t p = txt.find(k);
    if (p == std::string::npos)
        return false;
    p = txt.find(':', p + k.size());
    if (p == std::string::npos)
        return false;
    const size_t a = txt.find('"', p);
    if (a == std::string::npos)
        return false;
    const size_t b = txt.find('"', a + 1);
    if (b == std::string::npos)
        return false;
    *dst = txt.substr(a + 1, b - a - 1);
    return true;
}

// The GPU a cache is valid for: name, SM count, compute capability, driver
// and runtime versions of the current device.
struct DeviceKey {
    std::string name;
    int sms = 0, cc = 0, driver = 0, runtime = 0;
};

bool current_device_key(DeviceKey *k)
{
    int dev = 0;
    cudaDeviceProp prop{};
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess ||
        cudaDriverGetVersion(&k->driver) != cudaSuccess || cudaRuntimeGetVersion(&k->runtime) != cudaSuccess)
        return false;
    k->name = prop.name;
    k->sms = prop.multiProcessorCount;
    k->cc = prop.major * 10 + prop.minor;
    return true;
}

// A cache is applied only on the GPU it was measured on: a cache from
// another GPU, driver or CUDA runtime (or with no key) is ignored.
bool cache_matches(const std::string &txt)
{
    DeviceKey cur, c;
    if (!current_device_key(&cur))
        return false;
    return read_string(txt, "device", &c.name) && read_int(txt, "sm_count", &c.sms, 1, 1 << 20) &&
           read_int(txt, "compute_capability", &c.cc, 1, 1000) && read_int(txt, "driver_version", &c.driver, 1, 1 << 30) &&
           read_int(txt, "runtime_version", &c.runtime, 1, 1 << 30) && c.name == cur.name && c.sms == cur.sms &&
           c.cc == cur.cc && c.driver == cur.driver && c.runtime == cur.runtime;
}

void load()
{
    const char *path = std::getenv("IAAT_TUNE_CACHE");
    if (!path || !*path)
        return;
    FILE *f = std::fopen(path, "rb");
    if (!f)
        return;
    std::string txt;
    char buf[4096];
    size_t n;
    while ((n = std::fread(buf, 1, sizeof buf, f)) > 0)
        txt.append(buf, n);
    std::fclose(f);
    if (!cache_matches(txt))
        return;
    Tuning t;
    apply_text(txt, t);
    g_tuning = t;
}

// xorshift64* stream for the synthetic tuning batches
struct Rng {
    uint64_t s;
    explicit Rng(uint64_t seed) : s(seed * 0x9E3779B97F4A7C15ull + 1) {}
    uint64_t next()
    {
        s ^= s >> 12;
        s ^= s << 25;
        s ^= s >> 27;
        return s * 0x2545F4914F6CDD1Dull;
    }
    double uni() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
    int log_uniform(int lo, int hi)
    {
        double x = std::exp(std::log((double)lo) + uni() * (std::log((double)hi + 1) - std::log((double)lo)));
        return std::min(hi, (int)x);
    }
};

struct DeviceBatch {
    std::vector<iaat_gemm_desc_t> descs;
    void *pool = nullptr;
    ~DeviceBatch()
    {
        if (pool)
            cudaFree(pool);
    }
};

// Lay out `shapes` (M, N, K, case) in one device pool, entries in [-1, 1].
iaat_status_t make_batch(const std::vector<int> &shapes, int esz, Rng &rng, DeviceBatch &out)
{
    const size_t n = shapes.size() / 4;
    std::vector<size_t> offs(3 * n);
    size_t total = 0;
    auto place = [&](size_t elems) {
        size_t o = total;
        total += (elems * esz + 255) & ~(size_t)255;
        return o;
    };
    out.descs.resize(n);
    for (size_t i = 0; i < n; ++i) {
        const int M = shapes[4 * i], N = shapes[4 * i + 1], K = shapes[4 * i + 2], c = shapes[4 * i + 3];
        const int ta = (c >> 1) & 1, tb = c & 1;
        iaat_gemm_desc_t &d = out.descs[i];
        d.M = M; d.N = N; d.K = K;
        d.transA = ta; d.transB = tb;
        d.lda = std::max(1, ta ? K : M);
        d.ldb = std::max(1, tb ? N : K);
        d.ldc = std::max(1, M);
        d.alpha = 1.0; d.beta = 0.5;
        offs[3 * i] = place((size_t)M * K);
        offs[3 * i + 1] = place((size_t)K * N);
        offs[3 * i + 2] = place((size_t)M * N);
    }
    if (cudaMalloc(&out.pool, std::max<size_t>(total, 256)) != cudaSuccess)
        return IAAT_ERR_OOM;
    std::vector<unsigned char> host(total);
    for (size_t i = 0; i < total / esz; ++i) {
        const double v = 2.0 * rng.uni() - 1.0;
        if (esz == 4) {
            const float f = (float)v;
            std::memcpy(&host[i * 4], &f, 4);
        } else {
            std::memcpy(&host[i * 8], &v, 8);
        }
    }
    if (cudaMemcpy(out.pool, host.data(), total, cudaMemcpyHostToDevice) != cudaSuccess)
        return IAAT_ERR_CUDA;
    char *base = static_cast<char *>(out.pool);
    for (size_t i = 0; i < n; ++i) {
        out.descs[i].A = base + offs[3 * i];
        out.descs[i].B = base + offs[3 * i + 1];
        out.descs[i].C = base + offs[3 * i + 2];
    }
    return IAAT_OK;
}

// Median time (ms) of `reps` launches of a plan built with the options.
iaat_status_t time_plan(const DeviceBatch &b, iaat_dtype_t dt, iaat_precision_t prec, const iaat_plan_options_t &o,
                        cudaStream_t s, double *ms)
{
    iaat_plan_t plan = nullptr;
    iaat_status_t st = iaat_plan_create(b.descs.data(), (int64_t)b.descs.size(), dt, prec, &o, &plan);
    if (st != IAAT_OK)
        return st;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::vector<float> t;
    for (int r = 0; r < 7 && st == IAAT_OK; ++r) {
        cudaEventRecord(e0, s);
        st = iaat_gemm_grouped(plan, s);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float x = 0;
        cudaEventElapsedTime(&x, e0, e1);
        if (r >= 2)
            t.push_back(x);
    }
    if (st == IAAT_OK)
        st = iaat_plan_check(plan, s);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    iaat_plan_destroy(plan);
    if (st != IAAT_OK)
        return st;
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return IAAT_OK;
}
}  // namespace

const Tuning &tuning()
{
    std::call_once(g_once, load);
    return g_tuning;
}

// Cost of one warp block under the untuned model (defined in host.cpp).
double model_block_cost(const Variant &v, int esz, int K);

}  // namespace iaat

using namespace iaat;

extern "C" iaat_status_t iaat_autotune(iaat_dtype_t dtype, iaat_precision_t precision, const char *cache_path)
{
    if (dtype != IAAT_F32 && dtype != IAAT_F64)
        return IAAT_ERR_INVALID_VALUE;
    if (precision < IAAT_PREC_DEFAULT || precision > IAAT_PREC_6XBF16)
        return IAAT_ERR_INVALID_VALUE;
    if (dtype == IAAT_F64 && precision != IAAT_PREC_DEFAULT)
        return IAAT_ERR_UNSUPPORTED;
    tuning();   // make sure the cache (if any) was read before it is replaced
    const int esz = dtype == IAAT_F32 ? 4 : 8;
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
        return IAAT_ERR_CUDA;
    Rng rng(12345);
    Tuning t;
    {
        std::lock_guard<std::mutex> lk(g_mutex);
        t = g_tuning;
    }
    iaat_status_t st = IAAT_OK;
    int nv = 0;
    const Variant *vs = nullptr;
    if (precision == IAAT_PREC_DEFAULT) {
        nv = esz == 4 ? kNumVariantsF32 : kNumVariantsF64;
        vs = esz == 4 ? kVariantsF32 : kVariantsF64;
        std::vector<double> ratio(nv, 1.0);
        for (int v = 0; v < nv && st == IAAT_OK; ++v) {
            const int bm = vs[v].lm * vs[v].mr, bn = vs[v].ln * vs[v].nr;
            std::vector<int> shapes;
            double model = 0.0;
            const int count = std::max(2000, (int)(96e6 / ((double)(bm * 40 + 40 * bn + 2 * bm * bn) * esz)));
            for (int i = 0; i < count; ++i) {
                const int K = (i & 1) ? 16 : 48;
                static const int cases[3] = {0, 1, 3};   // NN, NT, TT: no TN-domain limit at these sizes
                shapes.insert(shapes.end(), {bm, bn, K, cases[i % 3]});
                model += model_block_cost(vs[v], esz, K);
            }
            DeviceBatch b;
            st = make_batch(shapes, esz, rng, b);
            if (st != IAAT_OK)
                break;
            iaat_plan_options_t o{};
            o.force_variant = v + 1;
            o.kernel = 1;   // the stage-program kernel, whose tiler the scales serve
            double ms = 0;
            st = time_plan(b, dtype, precision, o, s, &ms);
            ratio[v] = ms / model;
        }
        if (st == IAAT_OK) {
            double mean = 0;
            for (double r : ratio)
                mean += r;
            mean /= nv;
            for (int v = 0; v < nv; ++v) {
                if (esz == 4)
                    t.scale_f32[v] = (float)(ratio[v] / mean);
                else
                    t.scale_f64[v] = (float)(ratio[v] / mean);
            }
            std::lock_guard<std::mutex> lk(g_mutex);
            g_tuning = t;   // the group-size search below plans with the new scales
        }
    }
    // stage size on an uneven batch
    int best_group = 0, best_kernel = 0;
    if (st == IAAT_OK) {
        std::vector<int> shapes;
        const int count = 60000;
        for (int i = 0; i < count; ++i) {
            int M = rng.log_uniform(1, 80), N = rng.log_uniform(1, 80), K = rng.log_uniform(1, 80);
            int c = (int)(rng.next() & 3);
            if (dtype == IAAT_F64) {
                M = (rng.next() & 1) ? 64 : 32;
                N = rng.log_uniform(8, 80);
                K = rng.log_uniform(8, 80);
                c = (rng.next() & 1) ? 2 : 0;
            }
            if (c == 2 && (int64_t)M * N * K > 32768) {
                --i;
                continue;
            }
            shapes.insert(shapes.end(), {M, N, K, c});
        }
        DeviceBatch b;
        st = make_batch(shapes, esz, rng, b);
        double best = 1e30;
        for (int gt : {8, 16, 24, 32}) {
            if (st != IAAT_OK)
                break;
            iaat_plan_options_t o{};
            o.max_group_tasks = gt;
            o.kernel = 1;
            double ms = 0;
            st = time_plan(b, dtype, precision, o, s, &ms);
            if (st == IAAT_OK && ms < best) {
                best = ms;
                best_group = gt;
            }
        }
        // the kernel family of the default FP32 plans
        if (st == IAAT_OK && dtype == IAAT_F32) {
            best_kernel = 1;
            const double stage = best;
            for (int k : {2, precision == IAAT_PREC_DEFAULT ? 4 : 3}) {
                if (st != IAAT_OK)
                    break;
                iaat_plan_options_t o{};
                o.kernel = k;
                double ms = 0;
                st = time_plan(b, dtype, precision, o, s, &ms);
                if (st == IAAT_OK && ms < 0.97 * stage && ms < best) {
                    best = ms;
                    best_kernel = k;
                }
            }
        }
    }
    cudaStreamDestroy(s);
    if (st != IAAT_OK)
        return st;
    if (dtype == IAAT_F64)
        t.group_tasks_f64 = best_group;
    else
        t.group_tasks[(int)precision] = best_group;
    if (dtype == IAAT_F32)
        t.kernel[(int)precision] = best_kernel;
    t.from_cache = true;
    {
        std::lock_guard<std::mutex> lk(g_mutex);
        g_tuning = t;
    }
    const char *path = cache_path ? cache_path : std::getenv("IAAT_TUNE_CACHE");
    if (path && *path) {
        DeviceKey key;
        if (!current_device_key(&key))
            return IAAT_ERR_CUDA;
        FILE *f = std::fopen(path, "wb");
        if (!f)
            return IAAT_ERR_INVALID_VALUE;
        std::fprintf(f, "{\n  \"device\": \"%s\",\n  \"sm_count\": %d,\n  \"compute_capability\": %d,\n",
                     key.name.c_str(), key.sms, key.cc);
        std::fprintf(f, "  \"driver_version\": %d,\n  \"runtime_version\": %d,\n", key.driver, key.runtime);
        std::fprintf(f, "  \"variant_scale_f32\": [");
        for (int v = 0; v < kNumVariantsF32; ++v)
            std::fprintf(f, "%s%.4f", v ? ", " : "", t.scale_f32[v]);

        std::fprintf(f, "],\n  \"variant_scale_f64\": [");
        for (int v = 0; v < kNumVariantsF64; ++v)
            std::fprintf(f, "%s%.4f", v ? ", " : "", t.scale_f64[v]);
        std::fprintf(f, "],\n  \"group_tasks_ffma\": %d,\n  \"group_tasks_3xbf16\": %d,\n", t.group_tasks[0],
                     t.group_tasks[1]);
        std::fprintf(f, "  \"group_tasks_tf32\": %d,\n  \"group_tasks_fp16\": %d,\n  \"group_tasks_6xbf16\": %d,\n",
                     t.group_tasks[2], t.group_tasks[3], t.group_tasks[4]);
        std::fprintf(f, "  \"group_tasks_dfma\": %d,\n", t.group_tasks_f64);
        std::fprintf(f, "  \"kernel_ffma\": %d,\n  \"kernel_3xbf16\": %d,\n  \"kernel_tf32\": %d,\n", t.kernel[0],
                     t.kernel[1], t.kernel[2]);
        std::fprintf(f, "  \"kernel_fp16\": %d,\n  \"kernel_6xbf16\": %d\n}\n", t.kernel[3], t.kernel[4]);
        std::fclose(f);
    }
    return IAAT_OK;
}
