// Launch-plan choices and their autotuner (nmfkl_get_plan_choice,
// nmfkl_set_plan_choice, nmfkl_autotune in include/nmfkl.h).
//
// The choices pick among kernels that run the same Algorithm 2 on the same
// units: for units of at most 32/64/128/256 nonzeros in the list plan, the
// dense-tile warp kernels or the sub-warp group kernels over the compressed
// factor rows; which is faster depends on the fixed factor's density at the
// nonzeros and on r, so the autotuner measures both on the context's own data
// from its current state and caches the outcome per configuration.
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <string>
#include <vector>

using namespace nmfkl;

namespace {

constexpr int kShortClasses = 4;

void drop_step_graph(nmfkl_ctx *c) {
    if (c->step_graph) {
        cudaGraphExecDestroy(c->step_graph);
        c->step_graph = nullptr;
    }
}

// Density of the fixed factor of `side` at the nonzeros of V, from the
// current factors (the same measure the device-side plan choice uses).
bool current_density(nmfkl_ctx *c, int side, double *out) {
    const bool F = side == 0;
    if (!cuda_ok(c, cudaMemsetAsync(c->dens + side, 0, sizeof(unsigned long long), c->stream), "density reset"))
        return false;
    launch_compress(c->stream, F ? c->Wt : c->Ft, F ? c->n : c->m, c->ldr, c->p.r, F ? c->rowptr : c->colptr,
                    c->crow_cnt, c->crow_k, c->crow_a, c->dens + side);
    unsigned long long h = 0;
    if (!cuda_ok(c, cudaMemcpyAsync(&h, c->dens + side, sizeof(h), cudaMemcpyDeviceToHost, c->stream), "density") ||
        !cuda_ok(c, cudaStreamSynchronize(c->stream), "density sync"))
        return false;
    *out = c->nnz > 0 ? (double)h / ((double)c->nnz * c->p.r) : 0.0;
    return true;
}

// Units per short length class of a half (from the list plan's dense-tile
// alternatives, which hold every unit of at most 256 nonzeros).
void class_counts(const nmfkl_ctx *c, int side, int64_t out[kShortClasses]) {
    for (int k = 0; k < kShortClasses; ++k) out[k] = 0;
    for (const Bucket &b : c->plan_sparse[side])
        if (b.short_class >= 0 && !b.group) out[b.short_class] += b.count;
}

std::string cache_key(nmfkl_ctx *c, const double dens[2]) {
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, c->device);
    std::string name = prop.name;
    for (char &ch : name)
        if (ch == '"' || ch == '\\' || ch == ';') ch = '_';
    char buf[512];
    int64_t cnt[2][kShortClasses];
    class_counts(c, 0, cnt[0]);
    class_counts(c, 1, cnt[1]);
    std::snprintf(buf, sizeof(buf),
                  "dev=%s;r=%d;n=%lld;m=%lld;nnz=%lld;F=%lld,%lld,%lld,%lld;W=%lld,%lld,%lld,%lld;band=%d,%d",
                  name.c_str(), c->p.r, (long long)c->n, (long long)c->m, (long long)c->nnz, (long long)cnt[0][0],
                  (long long)cnt[0][1], (long long)cnt[0][2], (long long)cnt[0][3], (long long)cnt[1][0],
                  (long long)cnt[1][1], (long long)cnt[1][2], (long long)cnt[1][3], (int)std::floor(dens[0] * 10.0),
                  (int)std::floor(dens[1] * 10.0));
    return buf;
}

// Looks `key` up in the JSON-lines cache: one object per line,
// {"key": "...", "short_kernel": [[a,b,c,d],[e,f,g,h]], "ms": [16 numbers]}.
bool cache_lookup(const char *path, const std::string &key, int32_t choice[2][kShortClasses], double ms[16]) {
    std::ifstream in(path);
    if (!in) return false;
    std::string line;
    const std::string tag = "\"key\": \"" + key + "\"";
    while (std::getline(in, line)) {
        if (line.find(tag) == std::string::npos) continue;
        const size_t sk = line.find("\"short_kernel\": [[");
        const size_t sm = line.find("\"ms\": [");
        if (sk == std::string::npos || sm == std::string::npos) continue;
        int v[8];
        if (std::sscanf(line.c_str() + sk + 18, "%d,%d,%d,%d],[%d,%d,%d,%d", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5],
                        &v[6], &v[7]) != 8)
            continue;
        const char *q = line.c_str() + sm + 7;
        bool ok = true;
        for (int i = 0; i < 16 && ok; ++i) {
            char *end = nullptr;
            ms[i] = std::strtod(q, &end);
            if (end == q) ok = false;
            q = end;
            while (*q == ',' || *q == ' ') ++q;
        }
        if (!ok) continue;
        for (int i = 0; i < 8; ++i) {
            if (v[i] != 0 && v[i] != 1) ok = false;
            choice[i / 4][i % 4] = v[i];
        }
        if (ok) return true;
    }
    return false;
}

void cache_append(const char *path, const std::string &key, const int32_t choice[2][kShortClasses],
                  const double ms[16]) {
    std::FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "{\"key\": \"%s\", \"short_kernel\": [[%d,%d,%d,%d],[%d,%d,%d,%d]], \"ms\": [", key.c_str(),
                 choice[0][0], choice[0][1], choice[0][2], choice[0][3], choice[1][0], choice[1][1], choice[1][2],
                 choice[1][3]);
    for (int i = 0; i < 16; ++i) std::fprintf(f, "%s%.6g", i ? ", " : "", ms[i]);
    std::fprintf(f, "]}\n");
    std::fclose(f);
}

}  // namespace

extern "C" {

nmfkl_status nmfkl_get_plan_choice(const nmfkl_ctx *c, nmfkl_plan_choice *out) {
    if (!c || !out) return NMFKL_EINVAL;
    out->list_threshold = c->list_threshold;
    for (int s = 0; s < 2; ++s)
        for (int k = 0; k < kShortClasses; ++k) out->short_kernel[s][k] = c->short_choice[s][k];
    return NMFKL_OK;
}

nmfkl_status nmfkl_set_plan_choice(nmfkl_ctx *c, const nmfkl_plan_choice *in) {
    if (!c || !in) return NMFKL_EINVAL;
    if (!(in->list_threshold >= 0.0 && in->list_threshold <= 1.0)) return NMFKL_EINVAL;
    for (int s = 0; s < 2; ++s)
        for (int k = 0; k < kShortClasses; ++k)
            if (in->short_kernel[s][k] != 0 && in->short_kernel[s][k] != 1) return NMFKL_EINVAL;
    c->list_threshold = in->list_threshold;
    for (int s = 0; s < 2; ++s)
        for (int k = 0; k < kShortClasses; ++k) c->short_choice[s][k] = (int8_t)in->short_kernel[s][k];
    drop_step_graph(c);
    return NMFKL_OK;
}

nmfkl_status nmfkl_autotune(nmfkl_ctx *c, int64_t sweep, int32_t reps, const char *cache_path,
                            nmfkl_plan_choice *out, double *ms_out, int32_t *from_cache) {
    if (!c) return NMFKL_EINVAL;
    if (!c->have_data || reps < 1) {
        c->err = "autotune: needs data and reps >= 1";
        return NMFKL_EINVAL;
    }
    cudaSetDevice(c->device);
    TraceRange trace("nmfkl autotune");
    if (!cache_path) cache_path = std::getenv("NMFKL_TUNE_CACHE");
    if (from_cache) *from_cache = 0;
    double dens[2];
    if (!current_density(c, 0, &dens[0]) || !current_density(c, 1, &dens[1])) return NMFKL_ECUDA;
    const std::string key = cache_key(c, dens);
    int32_t choice[2][kShortClasses];
    double ms[16];
    for (double &x : ms) x = -1.0;
    bool cached = cache_path && cache_lookup(cache_path, key, choice, ms);
    if (!cached) {
        // fold the caller's pending kernel timings in and set them aside
        nmfkl_kernel_times(c, nullptr, nullptr, nullptr, 0, 0);
        const std::vector<KernelTimer> saved_timers = c->timers;
        const bool saved_timing = c->timing;
        const int32_t saved_list_mode = c->p.list_mode;
        int8_t saved_choice[2][kShortClasses];
        std::memcpy(saved_choice, c->short_choice, sizeof(saved_choice));
        // the factor each half updates, kept to be restored after every run
        const int64_t maxcols = std::max(c->n, c->m);
        float *backup = nullptr;
        if (!cuda_ok(c, cudaMalloc(&backup, sizeof(float) * (size_t)maxcols * c->ldr), "autotune backup"))
            return NMFKL_ENOMEM;
        nmfkl_status st = NMFKL_OK;
        c->p.list_mode = 2;  // the list plan, where the short alternatives live
        c->timing = true;
        for (int side = 0; side < 2 && st == NMFKL_OK; ++side) {
            float *X = side == 0 ? c->Ft : c->Wt;
            const size_t xbytes = sizeof(float) * (size_t)(side == 0 ? c->m : c->n) * c->ldr;
            if (!cuda_ok(c, cudaMemcpyAsync(backup, X, xbytes, cudaMemcpyDeviceToDevice, c->stream), "backup")) {
                st = NMFKL_ECUDA;
                break;
            }
            double t[kShortClasses][2] = {};
            bool has[kShortClasses][2] = {};
            for (const Bucket &b : c->plan_sparse[side])
                if (b.short_class >= 0) has[b.short_class][b.group ? 1 : 0] = true;
            for (int alt = 0; alt < 2 && st == NMFKL_OK; ++alt) {
                for (int k = 0; k < kShortClasses; ++k) c->short_choice[side][k] = (int8_t)alt;
                for (int rep = 0; rep < reps && st == NMFKL_OK; ++rep) {
                    c->timers.clear();
                    st = run_half(c, side, sweep);
                    if (st == NMFKL_OK) nmfkl_kernel_times(c, nullptr, nullptr, nullptr, 0, 0);
                    for (const Bucket &b : c->plan_sparse[side]) {
                        if (b.short_class < 0 || (b.group ? 1 : 0) != alt) continue;
                        const std::string name = bucket_timer_name(b, side);
                        for (const KernelTimer &kt : c->timers)
                            if (name == kt.name) t[b.short_class][alt] += kt.ms;
                    }
                    if (!cuda_ok(c, cudaMemcpyAsync(X, backup, xbytes, cudaMemcpyDeviceToDevice, c->stream),
                                 "restore"))
                        st = NMFKL_ECUDA;
                }
            }
            int64_t cnt[kShortClasses];
            class_counts(c, side, cnt);
            for (int k = 0; k < kShortClasses; ++k) {
                if (cnt[k] == 0) {
                    choice[side][k] = saved_choice[side][k];
                    continue;
                }
                ms[(side * 4 + k) * 2 + 0] = t[k][0] / reps;
                ms[(side * 4 + k) * 2 + 1] = has[k][1] ? t[k][1] / reps : -1.0;
                // a group kind the plan left out (shared memory) is not a candidate
                choice[side][k] = has[k][1] && t[k][1] < t[k][0] ? 1 : 0;
            }
        }
        cudaStreamSynchronize(c->stream);
        cudaFree(backup);
        c->p.list_mode = saved_list_mode;
        c->timing = saved_timing;
        c->timers = saved_timers;
        std::memcpy(c->short_choice, saved_choice, sizeof(saved_choice));
        if (st != NMFKL_OK) return st;
        if (cache_path) cache_append(cache_path, key, choice, ms);
    }
    for (int s = 0; s < 2; ++s)
        for (int k = 0; k < kShortClasses; ++k) c->short_choice[s][k] = (int8_t)choice[s][k];
    drop_step_graph(c);
    if (out) nmfkl_get_plan_choice(c, out);
    if (ms_out) std::memcpy(ms_out, ms, sizeof(ms));
    if (from_cache) *from_cache = cached ? 1 : 0;
    return NMFKL_OK;
}

}  // extern "C"
