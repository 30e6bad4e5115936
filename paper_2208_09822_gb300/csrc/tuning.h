// Cost-model weights of the run-time tiler, and their autotuned per-variant
// corrections (read from the JSON cache named by IAAT_TUNE_CACHE).
#pragma once
#include "common.cuh"

namespace iaat {

struct Tuning {
    double dfma_weight = 2.0;       // issue cost of a DFMA relative to an FFMA
    double repack_weight = 6.0;     // instructions per re-packed element sweep
    double epilogue_weight = 4.0;   // instructions per output element
    double block_overhead = 60.0;   // fixed cost of a warp block
    double cost_per_slot = 0.5;     // ordering key: bytes per issue slot
    float scale_f32[kNumVariantsF32];
    float scale_f64[kNumVariantsF64];
    int group_tasks[5] = {0, 0, 0, 0, 0};   // tasks per stage, by iaat_precision_t (0: default)
    int group_tasks_f64 = 0;             // same for FP64 (0: kMaxGroupTasks)
    // the kernel family a default FP32 plan (option kernel = 0) runs, by
    // iaat_precision_t: 1 stage programs, 2 stream, 3 warp-tile (tensor-core
    // precisions only), 4 warp-direct (FFMA only); 0: not tuned (stage programs)
    int kernel[5] = {0, 0, 0, 0, 0};
    bool from_cache = false;
    Tuning()
    {
        for (float &s : scale_f32)
            s = 1.0f;
        for (float &s : scale_f64)
            s = 1.0f;
    }
    double variant_scale(int esz, int v) const { return esz == 4 ? scale_f32[v] : scale_f64[v]; }
};

// The process-wide tuning (defaults, or the cache file when one is named).
const Tuning &tuning();

}  // namespace iaat
