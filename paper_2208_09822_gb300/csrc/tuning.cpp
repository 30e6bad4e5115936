// Autotuning of the register-tile variants (the GPU counterpart of the
// install-time stage's tuning, Sec. III-A / Sec. IV) and its JSON cache.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/iaat.h"
#include "tuning.h"

namespace iaat {

namespace {
std::once_flag g_once;
Tuning g_tuning;

// Reads "key": [n, n, ...] from a small JSON text.
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
    for (int i = 0; i < n; ++i) {
        char *end = nullptr;
        double v = std::strtod(s, &end);
        if (end == s || !(v > 0.0) || v > 1e6)
            return false;
        dst[i] = (float)v;
        s = end;
        while (*s == ' ' || *s == ',' || *s == '\n' || *s == '\t')
            ++s;
    }
    return true;
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
    Tuning t;
    bool ok32 = read_array(txt, "variant_scale_f32", t.scale_f32, kNumVariantsF32);
    bool ok64 = read_array(txt, "variant_scale_f64", t.scale_f64, kNumVariantsF64);
    if (!ok32)
        for (float &s : t.scale_f32)
            s = 1.0f;
    if (!ok64)
        for (float &s : t.scale_f64)
            s = 1.0f;
    t.from_cache = ok32 || ok64;
    g_tuning = t;
}
}  // namespace

const Tuning &tuning()
{
    std::call_once(g_once, load);
    return g_tuning;
}

}  // namespace iaat

extern "C" iaat_status_t iaat_autotune(iaat_dtype_t dtype, iaat_precision_t precision, const char *cache_path)
{
    (void)dtype;
    (void)precision;
    (void)cache_path;
    return IAAT_ERR_UNSUPPORTED;
}
