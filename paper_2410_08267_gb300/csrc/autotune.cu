// Launch-shape autotuner for batched trajectory launches.
//
// The tile shape (threads per CTA x trajectories per thread) trades
// occupancy against instruction-level parallelism and tile padding; the best
// one depends on the GPU, the precision mode, the step count (which sets the
// shared-memory table size and hence how many CTAs fit on an SM) and the
// amount of work.  nu_autotune times each candidate shape on the caller's own
// batch of requests (one warm-up run, then the median of three timed runs of
// the trajectory kernel) and returns the fastest.  Results are cached in a
// JSON-lines file keyed by GPU name, precision, step-count bucket and
// trajectory-count bucket.  The tile shape changes the order of the
// floating-point reduction, so results from different shapes agree to
// rounding, not bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "nuprof_internal.h"

namespace {

struct Shape {
    int block, tpt, flags;
};
// threads per CTA, trajectories per thread (3: two, packed FP32x2), table source
const Shape kShapes[] = {{256, 1, 0}, {512, 1, 0}, {256, 2, 0}, {256, 1, NU_FLAG_GTAB},
                         {384, 1, NU_FLAG_GTAB}, {256, 3, NU_FLAG_GTAB}, {128, 3, NU_FLAG_GTAB},
                         {256, 3, 0}};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

int bucket_pow2(long long v)
{
    int b = 0;
    while ((1LL << b) < v && b < 62) ++b;
    return b;
}

std::string make_key(const char* gpu, int precision, int steps_bucket, int traj_bucket)
{
    char buf[512];
    std::snprintf(buf, sizeof(buf),
                  "{\"gpu\": \"%s\", \"precision\": %d, \"steps_log2\": %d, \"traj_log2\": %d",
                  gpu, precision, steps_bucket, traj_bucket);
    return std::string(buf);
}

int field_int(const std::string& line, const char* name, int* out)
{
    const std::string pat = std::string("\"") + name + "\": ";
    const size_t at = line.find(pat);
    if (at == std::string::npos) return 0;
    return std::sscanf(line.c_str() + at + pat.size(), "%d", out) == 1;
}

int field_float(const std::string& line, const char* name, float* out)
{
    const std::string pat = std::string("\"") + name + "\": ";
    const size_t at = line.find(pat);
    if (at == std::string::npos) return 0;
    return std::sscanf(line.c_str() + at + pat.size(), "%f", out) == 1;
}

// Last cached entry with this key, if any.
bool cache_lookup(const char* path, const std::string& key, nu_tune_result* out)
{
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char buf[1024];
    bool found = false;
    while (std::fgets(buf, sizeof(buf), f)) {
        std::string line(buf);
        if (line.compare(0, key.size(), key) != 0) continue;
        int block = 0, tpt = 0, flags = 0;
        float ms = 0.0f;
        if (field_int(line, "block", &block) && field_int(line, "tpt", &tpt) &&
            field_int(line, "flags", &flags) && field_float(line, "ms", &ms)) {
            out->block = block;
            out->tpt = tpt;
            out->flags = flags;
            out->best_ms = ms;
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

void cache_store(const char* path, const std::string& key, const nu_tune_result& r)
{
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s, \"block\": %d, \"tpt\": %d, \"flags\": %d, \"ms\": %.6f}\n", key.c_str(),
                 r.block, r.tpt, r.flags, r.best_ms);
    std::fclose(f);
}

}  // namespace

extern "C" int nu_autotune(nu_profile* const* hs, int n, void* stream, const char* cache_path,
                           nu_tune_result* out)
{
    if (!hs || n < 1 || !out) return NU_EINVAL;
    std::memset(out, 0, sizeof(*out));
    nu_plan_info info;
    long long traj = 0;
    int max_steps = 0, precision = -1;
    for (int i = 0; i < n; ++i) {
        // (the packed shape, tpt 3, is tried for mixed precision only)
        if (!hs[i] || nu_profile_info(hs[i], &info) != NU_OK) return NU_EINVAL;
        if (precision >= 0 && info.precision != precision) return NU_EINVAL;
        precision = info.precision;
        traj += info.n_traj;
        max_steps = std::max(max_steps, info.n_steps);
    }
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return NU_ECUDA;
    }
    const std::string key = make_key(prop.name, precision, bucket_pow2(max_steps), bucket_pow2(traj));
    if (cache_path && cache_lookup(cache_path, key, out)) {
        out->from_cache = 1;
        return NU_OK;
    }
    float best = 1e30f;
    int slot = 0;
    for (int c = 0; c < kNumShapes; ++c) {
        if (kShapes[c].tpt == 3 && precision != NU_MIXED) continue;
        nu_opts o;
        std::memset(&o, 0, sizeof(o));
        o.block = kShapes[c].block;
        o.tpt = kShapes[c].tpt;
        o.flags = NU_FLAG_TIMING | kShapes[c].flags;
        o.stream = stream;
        nu_batch* b = nullptr;
        int rc = nu_batch_create(hs, n, &o, &b);
        if (rc != NU_OK) return rc;
        float t[3] = {0, 0, 0};
        rc = nu_batch_run(b, stream);
        for (int r = 0; r < 3 && rc == NU_OK; ++r) {
            rc = nu_batch_run(b, stream);
            if (rc == NU_OK) rc = nu_batch_kernel_ms(b, &t[r]);
        }
        nu_batch_destroy(b);
        if (rc != NU_OK) return rc;
        std::sort(t, t + 3);
        out->cand_block[slot] = o.block;
        out->cand_tpt[slot] = o.tpt;
        out->cand_flags[slot] = kShapes[c].flags;
        out->cand_ms[slot] = t[1];
        ++slot;
        if (t[1] < best) {
            best = t[1];
            out->block = o.block;
            out->tpt = o.tpt;
            out->flags = kShapes[c].flags;
            out->best_ms = t[1];
        }
    }
    out->n_candidates = slot;
    if (cache_path) cache_store(cache_path, key, *out);
    return NU_OK;
}
