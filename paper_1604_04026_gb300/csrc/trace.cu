// Observability of a factorization (nmfkl_set_metrics in include/nmfkl.h):
// with a metrics file set, every step (nmfkl_step, and each sweep of
// nmfkl_fit) appends one JSON line with Eq. 1 at the new factors, the step's
// device time, its throughput in coordinate updates and algorithmic bytes,
// the work per coordinate of Algorithm 2 (evaluations, Newton steps, cap hits)
// and the exact zeros of W and F (the measure of the paper's Table 2). The
// NVTX ranges around the host-side phases live in common.cuh.
#include "common.cuh"

#include <cstdio>

using namespace nmfkl;

namespace {

// Zero entries among the first r of each row of a unit-major factor: one warp
// per row, counts added per warp.
__global__ void count_zeros_kernel(const float *X, int64_t rows, int ldr, int r, unsigned long long *out) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    unsigned cnt = 0;
    for (int64_t row = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); row < rows; row += warps)
        for (int k = lane; k < r; k += 32) cnt += X[row * ldr + k] == 0.f ? 1u : 0u;
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0 && cnt) atomicAdd(out, (unsigned long long)cnt);
}

bool read_counters(nmfkl_ctx *c, unsigned long long h[4]) {
    return cuda_ok(c, cudaMemcpyAsync(h, c->counters, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                      c->stream),
                   "metrics counters") &&
           cuda_ok(c, cudaStreamSynchronize(c->stream), "metrics sync");
}

void close_metrics(nmfkl_ctx *c) {
    if (c->metrics) std::fclose(c->metrics);
    c->metrics = nullptr;
}

}  // namespace

namespace nmfkl {

// Called by the step after its work (timed between c->mev[0] and c->mev[1])
// has completed and its flags were read.
nmfkl_status write_metrics(nmfkl_ctx *c, int64_t sweep, double kl) {
    if (!c->metrics) return NMFKL_OK;
    float ms = 0.f;
    if (!cuda_ok(c, cudaEventElapsedTime(&ms, c->mev[0], c->mev[1]), "metrics time")) return NMFKL_ECUDA;
    if (!cuda_ok(c, cudaMemsetAsync(c->zeros_dev, 0, 2 * sizeof(unsigned long long), c->stream), "zeros reset"))
        return NMFKL_ECUDA;
    int dev_sms = 0;
    cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, c->device);
    const int grid = 4 * (dev_sms > 0 ? dev_sms : 1);
    count_zeros_kernel<<<grid, 256, 0, c->stream>>>(c->Wt, c->n, c->ldr, c->p.r, c->zeros_dev);
    count_zeros_kernel<<<grid, 256, 0, c->stream>>>(c->Ft, c->m, c->ldr, c->p.r, c->zeros_dev + 1);
    if (!cuda_ok(c, cudaGetLastError(), "count zeros")) return NMFKL_ECUDA;
    unsigned long long z[2] = {0, 0}, cnt[4] = {0, 0, 0, 0};
    if (!cuda_ok(c, cudaMemcpyAsync(z, c->zeros_dev, sizeof(z), cudaMemcpyDeviceToHost, c->stream), "zeros") ||
        !read_counters(c, cnt))
        return NMFKL_ECUDA;
    const double coords = (double)(cnt[0] - c->mprev[0]);
    const double evals = (double)(cnt[1] - c->mprev[1]), steps = (double)(cnt[2] - c->mprev[2]);
    const unsigned long long caps = cnt[3] - c->mprev[3];
    for (int i = 0; i < 4; ++i) c->mprev[i] = cnt[i];
    const double r = c->p.r, s = ms / 1e3;
    // one step: both halves; each nonzero's index, value and factor row, each
    // unit's r-vector read and written and its offset (per half)
    const double bytes = 2.0 * (double)c->nnz * (8.0 + 4.0 * r) + (double)(c->n + c->m) * (8.0 * r + 8.0);
    auto plan = [&](int side) { return c->used_sparse[side] == 1 ? "list" : (c->used_sparse[side] == 0 ? "dense" : "?"); };
    std::fprintf(c->metrics,
                 "{\"sweep\": %lld, \"kl\": %.17g, \"ms\": %.6g, \"updates_per_s\": %.6g, \"gb_per_s\": %.6g, "
                 "\"evals_per_coord\": %.6g, \"steps_per_coord\": %.6g, \"cap_hits\": %llu, "
                 "\"zeros_W_pct\": %.6g, \"zeros_F_pct\": %.6g, \"plan\": [\"%s\", \"%s\"], "
                 "\"density\": [%.6g, %.6g]}\n",
                 (long long)sweep, kl, (double)ms, s > 0 ? 2.0 * (double)c->nnz * r / s : 0.0,
                 s > 0 ? bytes / s / 1e9 : 0.0, coords > 0 ? evals / coords : 0.0, coords > 0 ? steps / coords : 0.0,
                 caps, c->n > 0 ? 100.0 * (double)z[0] / ((double)c->n * r) : 0.0,
                 c->m > 0 ? 100.0 * (double)z[1] / ((double)c->m * r) : 0.0, plan(0), plan(1), c->density[0],
                 c->density[1]);
    std::fflush(c->metrics);
    return NMFKL_OK;
}

void free_metrics(nmfkl_ctx *c) {
    close_metrics(c);
    if (c->mev[0]) cudaEventDestroy(c->mev[0]);
    if (c->mev[1]) cudaEventDestroy(c->mev[1]);
    c->mev[0] = c->mev[1] = nullptr;
    cudaFree(c->zeros_dev);
    c->zeros_dev = nullptr;
}

}  // namespace nmfkl

extern "C" {

nmfkl_status nmfkl_set_metrics(nmfkl_ctx *c, const char *path) {
    if (!c) return NMFKL_EINVAL;
    cudaSetDevice(c->device);
    close_metrics(c);
    if (!path || !*path) return NMFKL_OK;
    if (!c->mev[0] && (!cuda_ok(c, cudaEventCreate(&c->mev[0]), "metrics event") ||
                       !cuda_ok(c, cudaEventCreate(&c->mev[1]), "metrics event")))
        return NMFKL_ECUDA;
    if (!c->zeros_dev &&
        !cuda_ok(c, cudaMalloc(&c->zeros_dev, 2 * sizeof(unsigned long long)), "metrics zeros"))
        return NMFKL_ENOMEM;
    if (!read_counters(c, c->mprev)) return NMFKL_ECUDA;
    c->metrics = std::fopen(path, "a");
    if (!c->metrics) {
        c->err = std::string("cannot open metrics file ") + path;
        return NMFKL_EINVAL;
    }
    return NMFKL_OK;
}

}  // extern "C"
