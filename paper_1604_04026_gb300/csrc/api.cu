// C-ABI entry points of libnmfkl (declared in include/nmfkl.h).
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <thread>

namespace nmfkl {

int64_t dpart_required(int ldr);

bool cuda_ok(nmfkl_ctx *c, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return true;
    if (c) c->err = std::string(what) + ": " + cudaGetErrorString(e);
    return false;
}

int timer_begin(nmfkl_ctx *c, const char *name) {
    if (!c->timing) return -1;
    int idx = -1;
    for (size_t i = 0; i < c->timers.size(); ++i)
        if (std::strcmp(c->timers[i].name, name) == 0) idx = (int)i;
    if (idx < 0) {
        c->timers.push_back(KernelTimer{name, 0, 0.0});
        idx = (int)c->timers.size() - 1;
    }
    cudaEvent_t a, b;
    if (!c->ev_pool.empty()) {
        a = c->ev_pool.back();
        c->ev_pool.pop_back();
    } else {
        cudaEventCreate(&a);
    }
    if (!c->ev_pool.empty()) {
        b = c->ev_pool.back();
        c->ev_pool.pop_back();
    } else {
        cudaEventCreate(&b);
    }
    cudaEventRecord(a, c->stream);
    c->pending.push_back({idx, a, b});
    return (int)c->pending.size() - 1;
}

void timer_end(nmfkl_ctx *c, int token) {
    if (token < 0) return;
    cudaEventRecord(c->pending[token].b, c->stream);
}

}  // namespace nmfkl

using namespace nmfkl;

namespace {

template <class T>
bool dev_alloc(nmfkl_ctx *c, T **p, int64_t count, const char *what) {
    *p = nullptr;
    if (count <= 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, sizeof(T) * (size_t)count);
    if (e != cudaSuccess) {
        c->err = std::string("cudaMalloc ") + what + ": " + cudaGetErrorString(e);
        cudaGetLastError();
        return false;
    }
    return true;
}

void free_data(nmfkl_ctx *c) {
    if (c->step_graph) {  // the captured step holds the plans' launches
        cudaGraphExecDestroy(c->step_graph);
        c->step_graph = nullptr;
    }
    cudaFree(c->colptr); cudaFree(c->rowptr); cudaFree(c->rowidx); cudaFree(c->colidx);
    cudaFree(c->val); cudaFree(c->rval); cudaFree(c->scratch);
    c->colptr = c->rowptr = nullptr;
    c->rowidx = c->colidx = nullptr;
    c->val = c->rval = nullptr;
    c->scratch = nullptr;
    c->scratch_floats = 0;
    free_plan(c);
    c->have_data = false;
}

// Host-side check of one compressed layout, split over threads by unit range.
// Returns 0 if valid, else 1 (offsets), 2 (indices), 4 (values).
int check_range(int64_t u0, int64_t u1, int64_t extent, const int64_t *ptr, const int32_t *idx,
                const float *val) {
    for (int64_t u = u0; u < u1; ++u) {
        if (ptr[u + 1] < ptr[u]) return 1;
        int64_t prev = -1;
        for (int64_t p = ptr[u]; p < ptr[u + 1]; ++p) {
            if (idx[p] <= prev || idx[p] >= extent) return 2;
            prev = idx[p];
            if (!(val[p] > 0.f) || !std::isfinite(val[p])) return 4;
        }
    }
    return 0;
}

bool check_host(nmfkl_ctx *c, int64_t units, int64_t extent, int64_t nnz, const int64_t *ptr,
                const int32_t *idx, const float *val, const char *what) {
    if (ptr[0] != 0 || ptr[units] != nnz) {
        c->err = std::string(what) + ": offsets must start at 0 and end at nnz";
        return false;
    }
    // offsets must be monotone before any thread indexes with them
    for (int64_t u = 0; u < units; ++u)
        if (ptr[u + 1] < ptr[u] || ptr[u + 1] > nnz) {
            c->err = std::string(what) + ": offsets decrease or exceed nnz";
            return false;
        }
    int nt = (int)std::min<int64_t>(std::max(1u, std::thread::hardware_concurrency()), 32);
    if (nnz < (1 << 20)) nt = 1;
    std::vector<int> res(nt, 0);
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t)
        th.emplace_back([&, t] { res[t] = check_range(units * t / nt, units * (t + 1) / nt, extent, ptr, idx, val); });
    for (auto &x : th) x.join();
    int bad = 0;
    for (int v : res) bad |= v;
    if (bad & 2) c->err = std::string(what) + ": index out of range or not strictly increasing";
    else if (bad & 4) c->err = std::string(what) + ": values must be finite and > 0";
    else if (bad) c->err = std::string(what) + ": offsets decrease";
    return bad == 0;
}

}  // namespace

extern "C" {

void nmfkl_default_params(nmfkl_params *p, int32_t r) {
    std::memset(p, 0, sizeof(*p));
    p->r = r;
    p->eps_grad = 1e-6;
    p->eps_div = 1e-6;
    p->eps_x = 0.1;
    p->max_inner = 16;
    p->seed = 0;
}

const char *nmfkl_status_string(nmfkl_status s) {
    switch (s) {
        case NMFKL_OK: return "ok";
        case NMFKL_EINVAL: return "invalid argument";
        case NMFKL_ENOMEM: return "out of memory";
        case NMFKL_ECUDA: return "CUDA error";
        case NMFKL_ENUMERIC: return "non-finite objective";
        case NMFKL_ETIMEOUT: return "device wait timed out";
        case NMFKL_EBUSY: return "busy";
        case NMFKL_ENOTCONV: return "not converged";
        case NMFKL_ECANCELED: return "canceled";
    }
    return "unknown status";
}

nmfkl_status nmfkl_create(const nmfkl_params *p, int64_t n, int64_t m, int32_t device, void *stream,
                          nmfkl_ctx **out) {
    if (!out) return NMFKL_EINVAL;
    *out = nullptr;
    if (!p || p->r < 1 || p->r > kMaxR || n < 1 || m < 1 || n > INT32_MAX || m > INT32_MAX ||
        !(p->eps_x >= 0) || p->max_inner < 0 || !(p->eps_div >= 0) || !(p->eps_grad >= 0) ||
        p->alpha_W < 0 || p->alpha_F < 0 || p->beta_W < 0 || p->beta_F < 0 || p->list_mode < 0 ||
        p->list_mode > 2 || p->div_mode < 0 || p->div_mode > 1)
        return NMFKL_EINVAL;
    nmfkl_ctx *c = new (std::nothrow) nmfkl_ctx();
    if (!c) return NMFKL_ENOMEM;
    c->p = *p;
    c->n = n;
    c->m = m;
    c->ldr = (p->r + 3) / 4 * 4;
    c->device = device;
    c->stream = (cudaStream_t)stream;
    if (!cuda_ok(c, cudaSetDevice(device), "cudaSetDevice") ||
        !cuda_ok(c, cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device), "SM count") ||
        !cuda_ok(c, kernel_attributes(device), "kernel attributes")) {
        delete c;
        return NMFKL_ECUDA;
    }
    c->dpart_len = dpart_required(c->ldr);
    bool ok = dev_alloc(c, &c->Wt, n * c->ldr, "W") && dev_alloc(c, &c->Ft, m * c->ldr, "F") &&
              dev_alloc(c, &c->sumW, c->ldr, "sumW") && dev_alloc(c, &c->sumF, c->ldr, "sumF") &&
              dev_alloc(c, &c->dpart, c->dpart_len, "partials") && dev_alloc(c, &c->dscalar, 8, "scalars") &&
              dev_alloc(c, &c->counters, 8, "counters") && dev_alloc(c, &c->queues, 2 * kQueuesPerSide, "queues") &&
              dev_alloc(c, &c->err_flag, 1, "error flag") && dev_alloc(c, &c->dsum[0], c->ldr, "sumW64") &&
              dev_alloc(c, &c->dsum[1], c->ldr, "sumF64") && dev_alloc(c, &c->unit_obj, n, "row objective") &&
              dev_alloc(c, &c->dens, 2, "density") && dev_alloc(c, &c->plan_sel, 4, "plan choice") &&
              dev_alloc(c, &c->dens_out, 2, "density out") && dev_alloc(c, &c->sweep_dev, 1, "sweep index") &&
              dev_alloc(c, &c->crow_cnt, std::max(n, m), "compressed row counts") &&
              dev_alloc(c, &c->crow_k, std::max(n, m) * c->ldr, "compressed row indices") &&
              dev_alloc(c, &c->crow_a, std::max(n, m) * c->ldr, "compressed row values");
    if (ok && cudaMallocHost((void **)&c->h_sweep, sizeof(int64_t)) != cudaSuccess) {
        cudaGetLastError();
        c->h_sweep = nullptr;
        ok = false;
    }
    if (!ok) {
        nmfkl_destroy(c);
        return NMFKL_ENOMEM;
    }
    if (!cuda_ok(c, cudaMemset(c->plan_sel, 0, 4 * sizeof(int32_t)), "zero plan choice") ||
        !cuda_ok(c, cudaMemset(c->Wt, 0, sizeof(float) * n * c->ldr), "zero W") ||
        !cuda_ok(c, cudaMemset(c->Ft, 0, sizeof(float) * m * c->ldr), "zero F") ||
        !cuda_ok(c, cudaMemset(c->counters, 0, sizeof(unsigned long long) * 8), "zero counters") ||
        !cuda_ok(c, cudaMemset(c->err_flag, 0, sizeof(int32_t)), "zero flag")) {
        nmfkl_destroy(c);
        return NMFKL_ECUDA;
    }
    *out = c;
    return NMFKL_OK;
}

void nmfkl_destroy(nmfkl_ctx *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    free_data(c);
    free_fold(c);
    if (c->step_graph) cudaGraphExecDestroy(c->step_graph);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    cudaFree(c->plan_sel); cudaFree(c->dens_out); cudaFree(c->sweep_dev);
    if (c->h_sweep) cudaFreeHost(c->h_sweep);
    cudaFree(c->Wt); cudaFree(c->Ft); cudaFree(c->sumW); cudaFree(c->sumF); cudaFree(c->dpart);
    cudaFree(c->dscalar); cudaFree(c->counters); cudaFree(c->queues); cudaFree(c->err_flag);
    cudaFree(c->tbuf);
    cudaFree(c->dsum[0]); cudaFree(c->dsum[1]); cudaFree(c->unit_obj); cudaFree(c->dens);
    cudaFree(c->crow_cnt); cudaFree(c->crow_k); cudaFree(c->crow_a);
    for (auto &pd : c->pending) { cudaEventDestroy(pd.a); cudaEventDestroy(pd.b); }
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    free_metrics(c);
    delete c;
}

const char *nmfkl_last_error(const nmfkl_ctx *c) { return c ? c->err.c_str() : "null context"; }

nmfkl_status nmfkl_set_data(nmfkl_ctx *c, int64_t nnz, const int64_t *colptr, const int32_t *rowidx,
                            const float *val, const int64_t *rowptr, const int32_t *colidx, const float *rval,
                            int32_t mem_kind) {
    if (!c) return NMFKL_EINVAL;
    TraceRange trace("nmfkl set_data");
    if (nnz < 0 || nnz > INT32_MAX * 8LL || !colptr || (nnz > 0 && (!rowidx || !val)) ||
        (mem_kind != 0 && mem_kind != 1)) {
        c->err = "set_data: bad arguments";
        return NMFKL_EINVAL;
    }
    cudaSetDevice(c->device);
    free_data(c);
    const int64_t n = c->n, m = c->m;
    std::vector<int64_t> h_rowptr;
    std::vector<int32_t> h_colidx;
    std::vector<float> h_rval;
    // Host inputs with both layouts are validated on the device after the copy
    // (one warp per unit); the host CSR build below indexes by row, so a lone
    // CSC is checked on the host first.
    const bool check_on_device = mem_kind == 1 || rowptr != nullptr;
    if (mem_kind == 0) {
        if (!rowptr && !check_host(c, m, n, nnz, colptr, rowidx, val, "CSC")) return NMFKL_EINVAL;
        if (!rowptr) {
            // CSR by a counting sort of the CSC (order within rows stays sorted)
            h_rowptr.assign(n + 1, 0);
            h_colidx.resize(nnz);
            h_rval.resize(nnz);
            for (int64_t p = 0; p < nnz; ++p) h_rowptr[rowidx[p] + 1]++;
            for (int64_t i = 0; i < n; ++i) h_rowptr[i + 1] += h_rowptr[i];
            std::vector<int64_t> fill(h_rowptr.begin(), h_rowptr.end() - 1);
            for (int64_t j = 0; j < m; ++j)
                for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p) {
                    const int64_t q = fill[rowidx[p]]++;
                    h_colidx[q] = (int32_t)j;
                    h_rval[q] = val[p];
                }
            rowptr = h_rowptr.data();
            colidx = h_colidx.data();
            rval = h_rval.data();
        } else if (nnz > 0 && (!colidx || !rval)) {
            c->err = "set_data: CSR arrays missing";
            return NMFKL_EINVAL;
        }
    } else if (!rowptr || (nnz > 0 && (!colidx || !rval))) {
        c->err = "set_data: device inputs need both CSC and CSR";
        return NMFKL_EINVAL;
    }
    bool ok = dev_alloc(c, &c->colptr, m + 1, "colptr") && dev_alloc(c, &c->rowidx, nnz, "rowidx") &&
              dev_alloc(c, &c->val, nnz, "val") && dev_alloc(c, &c->rowptr, n + 1, "rowptr") &&
              dev_alloc(c, &c->colidx, nnz, "colidx") && dev_alloc(c, &c->rval, nnz, "rval");
    if (!ok) {
        free_data(c);
        return NMFKL_ENOMEM;
    }
    const cudaMemcpyKind kind = mem_kind == 0 ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    ok = cuda_ok(c, cudaMemcpy(c->colptr, colptr, 8 * (m + 1), kind), "copy colptr") &&
         cuda_ok(c, cudaMemcpy(c->rowptr, rowptr, 8 * (n + 1), kind), "copy rowptr");
    if (ok && nnz > 0)
        ok = cuda_ok(c, cudaMemcpy(c->rowidx, rowidx, 4 * nnz, kind), "copy rowidx") &&
             cuda_ok(c, cudaMemcpy(c->val, val, 4 * nnz, kind), "copy val") &&
             cuda_ok(c, cudaMemcpy(c->colidx, colidx, 4 * nnz, kind), "copy colidx") &&
             cuda_ok(c, cudaMemcpy(c->rval, rval, 4 * nnz, kind), "copy rval");
    if (!ok) {
        free_data(c);
        return NMFKL_ECUDA;
    }
    c->nnz = nnz;
    if (check_on_device) {
        int32_t *flag = c->err_flag;
        int32_t h = 0;
        ok = cuda_ok(c, cudaMemsetAsync(flag, 0, 4, c->stream), "flag") &&
             launch_validate(c, m, n, nnz, c->colptr, c->rowidx, c->val, flag) == NMFKL_OK &&
             launch_validate(c, n, m, nnz, c->rowptr, c->colidx, c->rval, flag) == NMFKL_OK &&
             cuda_ok(c, cudaMemcpyAsync(&h, flag, 4, cudaMemcpyDeviceToHost, c->stream), "flag copy") &&
             cuda_ok(c, cudaStreamSynchronize(c->stream), "validate sync");
        if (!ok) {
            free_data(c);
            return NMFKL_ECUDA;
        }
        int64_t first[2] = {0, 0}, last[2] = {0, 0};
        cudaMemcpy(&first[0], c->colptr, 8, cudaMemcpyDeviceToHost);
        cudaMemcpy(&first[1], c->rowptr, 8, cudaMemcpyDeviceToHost);
        cudaMemcpy(&last[0], c->colptr + m, 8, cudaMemcpyDeviceToHost);
        cudaMemcpy(&last[1], c->rowptr + n, 8, cudaMemcpyDeviceToHost);
        cudaMemsetAsync(flag, 0, 4, c->stream);
        if (h != 0 || first[0] != 0 || first[1] != 0 || last[0] != nnz || last[1] != nnz) {
            c->err = "set_data: device input failed validation (offsets, sorted in-range indices, values > 0)";
            free_data(c);
            return NMFKL_EINVAL;
        }
    }
    nmfkl_status st = plan_side(c, 0);
    if (st == NMFKL_OK) st = plan_side(c, 1);
    if (st != NMFKL_OK) {
        free_data(c);
        return st;
    }
    if (c->scratch_floats > 0 && !dev_alloc(c, &c->scratch, c->scratch_floats, "scratch")) {
        free_data(c);
        return NMFKL_ENOMEM;
    }
    // tiles only ever hold finite factor values; start them at 0
    if (c->scratch_floats > 0 &&
        !cuda_ok(c, cudaMemset(c->scratch, 0, sizeof(float) * (size_t)c->scratch_floats), "zero scratch")) {
        free_data(c);
        return NMFKL_ECUDA;
    }
    c->have_data = true;
    return NMFKL_OK;
}

nmfkl_status nmfkl_init(nmfkl_ctx *c, const float *W0, const float *F0, int32_t mem_kind) {
    if (!c || (mem_kind != 0 && mem_kind != 1)) return NMFKL_EINVAL;
    cudaSetDevice(c->device);
    const int64_t need = std::max(c->n, c->m) * (int64_t)c->p.r;
    if (c->tbuf_floats < need) {
        cudaFree(c->tbuf);
        c->tbuf = nullptr;
        c->tbuf_floats = 0;
        if (!dev_alloc(c, &c->tbuf, need, "transpose buffer")) return NMFKL_ENOMEM;
        c->tbuf_floats = need;
    }
    struct Item { const float *src; float *dst; int64_t cols; int which; } items[2] = {
        {W0, c->Wt, c->n, 0}, {F0, c->Ft, c->m, 1}};
    for (auto &it : items) {
        nmfkl_status st;
        if (!it.src) {
            st = launch_uniform_init(c, it.which, it.dst, it.cols);
        } else {
            const float *src = it.src;
            if (mem_kind == 0) {
                if (!cuda_ok(c, cudaMemcpyAsync(c->tbuf, it.src, sizeof(float) * it.cols * c->p.r,
                                                cudaMemcpyHostToDevice, c->stream), "copy init"))
                    return NMFKL_ECUDA;
                src = c->tbuf;
            }
            st = launch_to_unit_major(c, src, it.dst, it.cols);
            if (st == NMFKL_OK && mem_kind == 0 &&
                !cuda_ok(c, cudaStreamSynchronize(c->stream), "init sync"))
                st = NMFKL_ECUDA;
        }
        if (st != NMFKL_OK) return st;
    }
    return NMFKL_OK;
}

// Clears the device error flag before a half, step or fit.
static nmfkl_status clear_flags(nmfkl_ctx *c) {
    return cuda_ok(c, cudaMemsetAsync(c->err_flag, 0, sizeof(int32_t), c->stream), "clear error flag") ? NMFKL_OK
                                                                                                     : NMFKL_ECUDA;
}

// Reads the device error flag (synchronizes the stream) and maps its bits to
// a status: a bounded wait that gave up first (the results of that half are
// not meaningful), then a NaN written to a factor, then a unit its kernel
// refused.
static nmfkl_status read_flags(nmfkl_ctx *c) {
    int32_t flag = 0;
    int32_t sel[2] = {0, 0};
    double dens[2] = {0.0, 0.0};
    if (!cuda_ok(c, cudaMemcpyAsync(&flag, c->err_flag, sizeof(flag), cudaMemcpyDeviceToHost, c->stream),
                 "copy error flag") ||
        !cuda_ok(c, cudaMemcpyAsync(sel, c->plan_sel, sizeof(sel), cudaMemcpyDeviceToHost, c->stream),
                 "copy plan choice") ||
        !cuda_ok(c, cudaMemcpyAsync(dens, c->dens_out, sizeof(dens), cudaMemcpyDeviceToHost, c->stream),
                 "copy density") ||
        !cuda_ok(c, cudaStreamSynchronize(c->stream), "error flag sync"))
        return NMFKL_ECUDA;
    if (c->p.list_mode == 0) {
        for (int side = 0; side < 2; ++side) {
            c->used_sparse[side] = sel[side];
            c->density[side] = dens[side];
        }
    }
    if (flag & kErrTimeout) {
        c->err = "a bounded wait on a thread-block cluster peer gave up";
        return NMFKL_ETIMEOUT;
    }
    if (flag & kErrNaN) {
        c->err = "NaN produced in a sweep";
        return NMFKL_ENUMERIC;
    }
    if (flag & kErrLength) {
        c->err = "a unit was longer than its planned kernel holds";
        return NMFKL_EINVAL;
    }
    return NMFKL_OK;
}

static nmfkl_status sweep_side(nmfkl_ctx *c, int side, int64_t sweep) {
    if (!c) return NMFKL_EINVAL;
    if (!c->have_data) {
        c->err = "no data: call nmfkl_set_data first";
        return NMFKL_EINVAL;
    }
    cudaSetDevice(c->device);
    nmfkl_status st = clear_flags(c);
    if (st == NMFKL_OK) st = run_half(c, side, sweep);
    if (st == NMFKL_OK) st = read_flags(c);
    return st;
}

nmfkl_status nmfkl_sweep_F(nmfkl_ctx *c, int64_t sweep) { return sweep_side(c, 0, sweep); }
nmfkl_status nmfkl_sweep_W(nmfkl_ctx *c, int64_t sweep) { return sweep_side(c, 1, sweep); }

nmfkl_status nmfkl_objective(nmfkl_ctx *c, double *kl, double *reg) {
    if (!c) return NMFKL_EINVAL;
    if (!c->have_data) {
        c->err = "no data: call nmfkl_set_data first";
        return NMFKL_EINVAL;
    }
    cudaSetDevice(c->device);
    return launch_objective(c, kl, reg);
}

}  // extern "C"

namespace {

// One pass of the hot path enqueued on the context stream (no host
// synchronization): the F half, the W half and the fused objective.
nmfkl_status enqueue_step(nmfkl_ctx *c, int64_t sweep, const int64_t *sweep_dev) {
    nmfkl_status st = run_half(c, 0, sweep, sweep_dev);
    if (st == NMFKL_OK) st = run_half(c, 1, sweep, sweep_dev);
    if (st == NMFKL_OK) st = enqueue_fused_objective(c);
    return st;
}

// Captures enqueue_step once into a CUDA graph whose kernels read the sweep
// index from device memory; rebuilt when the plans change.
nmfkl_status build_step_graph(nmfkl_ctx *c) {
    if (!c->cap_stream && !cuda_ok(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking),
                                   "capture stream"))
        return NMFKL_ECUDA;
    cudaStream_t saved = c->stream;
    const bool saved_timing = c->timing;
    c->stream = c->cap_stream;
    c->timing = false;
    cudaGraph_t g = nullptr;
    nmfkl_status st = NMFKL_OK;
    if (!cuda_ok(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture")) {
        st = NMFKL_ECUDA;
    } else {
        st = enqueue_step(c, 0, c->sweep_dev);
        const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
        if (st == NMFKL_OK && !cuda_ok(c, e, "end capture")) st = NMFKL_ECUDA;
    }
    c->stream = saved;
    c->timing = saved_timing;
    if (st == NMFKL_OK && !cuda_ok(c, cudaGraphInstantiate(&c->step_graph, g, 0), "instantiate step graph")) {
        c->step_graph = nullptr;
        st = NMFKL_ECUDA;
    }
    if (g) cudaGraphDestroy(g);
    return st;
}

// One step: the captured graph (or, with kernel timing on, the same launches
// issued one by one so that each can be bracketed by events), then the
// objective, the device flags and the plans chosen, read back in one
// synchronization. Flags take precedence over a non-finite objective.
nmfkl_status step_impl(nmfkl_ctx *c, int64_t sweep, double *kl) {
    TraceRange trace("nmfkl step");
    nmfkl_status st = clear_flags(c);
    if (st != NMFKL_OK) return st;
    if (c->metrics && !cuda_ok(c, cudaEventRecord(c->mev[0], c->stream), "metrics event")) return NMFKL_ECUDA;
    if (c->timing) {
        st = enqueue_step(c, sweep, nullptr);
    } else {
        if (!c->step_graph) st = build_step_graph(c);
        if (st == NMFKL_OK) {
            *c->h_sweep = sweep;
            if (!cuda_ok(c, cudaMemcpyAsync(c->sweep_dev, c->h_sweep, sizeof(int64_t), cudaMemcpyHostToDevice,
                                            c->stream),
                         "sweep index") ||
                !cuda_ok(c, cudaGraphLaunch(c->step_graph, c->stream), "step graph launch"))
                st = NMFKL_ECUDA;
        }
    }
    if (st != NMFKL_OK) return st;
    if (c->metrics && !cuda_ok(c, cudaEventRecord(c->mev[1], c->stream), "metrics event")) return NMFKL_ECUDA;
    double h = 0.0;
    if (!cuda_ok(c, cudaMemcpyAsync(&h, c->dscalar, sizeof(h), cudaMemcpyDeviceToHost, c->stream), "copy objective"))
        return NMFKL_ECUDA;
    st = read_flags(c);  // synchronizes
    if (st != NMFKL_OK) return st;
    if (kl) *kl = h;
    if (!std::isfinite(h)) {
        c->err = "objective is not finite";
        return NMFKL_ENUMERIC;
    }
    return write_metrics(c, sweep, h);
}

}  // namespace

extern "C" {

nmfkl_status nmfkl_fit(nmfkl_ctx *c, int64_t sweep0, int32_t max_sweeps, double rel_tol, double *kl_trace,
                       int32_t *sweeps_done) {
    if (!c || max_sweeps < 0 || !(rel_tol >= 0)) return NMFKL_EINVAL;
    if (!c->have_data) {
        c->err = "no data: call nmfkl_set_data first";
        return NMFKL_EINVAL;
    }
    cudaSetDevice(c->device);
    TraceRange trace("nmfkl fit");
    double prev = 0.0;
    nmfkl_status st = launch_objective(c, &prev, nullptr);
    if (st != NMFKL_OK) return st;
    int32_t s = 0;
    bool conv = false;
    while (s < max_sweeps) {
        double kl = 0.0;
        st = step_impl(c, sweep0 + s, &kl);
        if (st != NMFKL_OK) {
            if (sweeps_done) *sweeps_done = s;
            return st;
        }
        if (kl_trace) kl_trace[s] = kl;
        ++s;
        if (rel_tol > 0 && std::fabs(prev - kl) <= rel_tol * std::fabs(prev)) {
            conv = true;
            break;
        }
        prev = kl;
    }
    if (sweeps_done) *sweeps_done = s;
    return (rel_tol > 0 && !conv) ? NMFKL_ENOTCONV : NMFKL_OK;
}

nmfkl_status nmfkl_step(nmfkl_ctx *c, int64_t sweep, double *kl) {
    if (!c) return NMFKL_EINVAL;
    if (!c->have_data) {
        c->err = "no data: call nmfkl_set_data first";
        return NMFKL_EINVAL;
    }
    cudaSetDevice(c->device);
    return step_impl(c, sweep, kl);
}

nmfkl_status nmfkl_sweep_range(nmfkl_ctx *c, int32_t side, int64_t sweep, int64_t u0, int64_t u1,
                               double *data_term) {
    if (!c || (side != 0 && side != 1)) return NMFKL_EINVAL;
    if (!c->have_data) {
        c->err = "no data: call nmfkl_set_data first";
        return NMFKL_EINVAL;
    }
    const int64_t units = side == 0 ? c->m : c->n;
    if (u0 < 0 || u1 < u0 || u1 > units) {
        c->err = "sweep_range: need 0 <= u0 <= u1 <= units";
        return NMFKL_EINVAL;
    }
    cudaSetDevice(c->device);
    nmfkl_status st = clear_flags(c);
    if (st == NMFKL_OK && u1 > u0) st = run_half(c, side, sweep, nullptr, u0, u1);
    double h = 0.0;
    if (st == NMFKL_OK && side == 1 && u1 > u0) {
        st = launch_range_sum(c, c->unit_obj + u0, u1 - u0, c->dscalar + 1);
        if (st == NMFKL_OK &&
            !cuda_ok(c, cudaMemcpyAsync(&h, c->dscalar + 1, sizeof(h), cudaMemcpyDeviceToHost, c->stream),
                     "copy data term"))
            st = NMFKL_ECUDA;
    }
    if (st == NMFKL_OK) st = read_flags(c);  // synchronizes
    if (st == NMFKL_OK && data_term) *data_term = h;
    return st;
}

nmfkl_status nmfkl_linear_term(nmfkl_ctx *c, double *out) {
    if (!c || !out) return NMFKL_EINVAL;
    cudaSetDevice(c->device);
    nmfkl_status st = launch_colsum(c, c->Wt, c->n, c->sumW, c->dsum[0]);
    if (st == NMFKL_OK) st = launch_colsum(c, c->Ft, c->m, c->sumF, c->dsum[1]);
    if (st != NMFKL_OK) return st;
    std::vector<double> sw(c->p.r), sf(c->p.r);
    if (!cuda_ok(c, cudaMemcpyAsync(sw.data(), c->dsum[0], sizeof(double) * c->p.r, cudaMemcpyDeviceToHost, c->stream),
                 "copy sumW") ||
        !cuda_ok(c, cudaMemcpyAsync(sf.data(), c->dsum[1], sizeof(double) * c->p.r, cudaMemcpyDeviceToHost, c->stream),
                 "copy sumF") ||
        !cuda_ok(c, cudaStreamSynchronize(c->stream), "linear term sync"))
        return NMFKL_ECUDA;
    double s = 0.0;
    for (int k = 0; k < c->p.r; ++k) s += sw[k] * sf[k];
    *out = s;
    return NMFKL_OK;
}

nmfkl_status nmfkl_factor_unit_major(nmfkl_ctx *c, int32_t side, float **ptr, int64_t *units, int32_t *ld) {
    if (!c || !ptr || (side != 0 && side != 1)) return NMFKL_EINVAL;
    *ptr = side == 0 ? c->Ft : c->Wt;
    if (units) *units = side == 0 ? c->m : c->n;
    if (ld) *ld = c->ldr;
    return NMFKL_OK;
}

nmfkl_status nmfkl_set_wait_limit(nmfkl_ctx *c, int64_t cycles) {
    if (!c || cycles < 0) return NMFKL_EINVAL;
    c->wait_cycles = cycles > 0 ? (long long)cycles : kDefaultWaitCycles;
    if (c->step_graph) {  // the limit is baked into the captured launches
        cudaGraphExecDestroy(c->step_graph);
        c->step_graph = nullptr;
    }
    return NMFKL_OK;
}

// Grows the fold-in input buffers to hold m_new columns and nnz nonzeros.
static nmfkl_status fold_reserve(nmfkl_ctx *c, int64_t m_new, int64_t nnz) {
    if (!c->fold) {
        c->fold = new (std::nothrow) FoldState();
        if (!c->fold) return NMFKL_ENOMEM;
    }
    FoldState &f = *c->fold;
    if (m_new > f.cap_m) {
        const int64_t cap = std::max<int64_t>(m_new, 2 * f.cap_m);
        cudaFree(f.colptr); cudaFree(f.ids); cudaFree(f.Ft); cudaFree(f.Fout); cudaFree(f.lists);
        cudaFree(f.sweeps); cudaFree(f.obj);
        f.colptr = f.ids = nullptr;
        f.Ft = f.Fout = nullptr;
        f.lists = f.sweeps = nullptr;
        f.obj = nullptr;
        f.cap_m = 0;
        if (!(dev_alloc(c, &f.colptr, cap + 1, "fold-in colptr") && dev_alloc(c, &f.ids, cap, "fold-in ids") &&
              dev_alloc(c, &f.Ft, cap * c->ldr, "fold-in F") && dev_alloc(c, &f.Fout, cap * c->p.r, "fold-in out") &&
              dev_alloc(c, &f.lists, cap * kFoldKinds, "fold-in lists") &&
              dev_alloc(c, &f.sweeps, cap, "fold-in sweeps") && dev_alloc(c, &f.obj, cap, "fold-in objective")))
            return NMFKL_ENOMEM;
        if (!cuda_ok(c, cudaMemset(f.Ft, 0, sizeof(float) * cap * c->ldr), "zero fold-in F")) return NMFKL_ECUDA;
        f.cap_m = cap;
        if (f.graph) {
            cudaGraphExecDestroy(f.graph);
            f.graph = nullptr;
        }
    }
    if (!f.ctl && !dev_alloc(c, &f.ctl, 2 * kFoldKinds + 1, "fold-in control")) return NMFKL_ENOMEM;
    if (nnz > f.cap_nnz) {
        const int64_t cap = std::max<int64_t>(nnz, 2 * f.cap_nnz);
        cudaFree(f.rowidx); cudaFree(f.val);
        f.rowidx = nullptr;
        f.val = nullptr;
        f.cap_nnz = 0;
        if (!(dev_alloc(c, &f.rowidx, cap, "fold-in rowidx") && dev_alloc(c, &f.val, cap, "fold-in val")))
            return NMFKL_ENOMEM;
        f.cap_nnz = cap;
        if (f.graph) {
            cudaGraphExecDestroy(f.graph);
            f.graph = nullptr;
        }
    }
    return NMFKL_OK;
}

}  // extern "C"

namespace nmfkl {

// nmfkl_foldin; with `segs`, the starting F is drawn per segment of columns
// (each from Uniform[0,1) as if the segment were a batch of its own, or
// copied from the segment's host F0), so that a segment's result does not
// depend on the batch it shares (the serving loop merges requests this way).
nmfkl_status foldin_impl(nmfkl_ctx *c, int64_t m_new, int64_t nnz, const int64_t *colptr, const int32_t *rowidx,
                         const float *val, const int64_t *doc_ids, const float *F0,
                         const std::vector<FoldSegment> *segs, float *F_out, double rel_tol, int32_t max_sweeps,
                         int32_t *sweeps_done, double *doc_obj, int32_t launch_mode, int32_t mem_kind) {
    TraceRange trace("nmfkl foldin");
    if (!c) return NMFKL_EINVAL;
    if (m_new < 0 || m_new > INT32_MAX || nnz < 0 || !colptr || (nnz > 0 && (!rowidx || !val)) || !F_out ||
        !(rel_tol >= 0) || max_sweeps < 0 || launch_mode < 0 || launch_mode > 2 || (mem_kind != 0 && mem_kind != 1)) {
        c->err = "foldin: bad arguments";
        return NMFKL_EINVAL;
    }
    cudaSetDevice(c->device);
    const int64_t r = c->p.r;
    if (mem_kind == 0) {
        if (!check_host(c, m_new, c->n, nnz, colptr, rowidx, val, "fold-in CSC")) return NMFKL_EINVAL;
        for (int64_t j = 0; j < m_new; ++j)
            if (foldin_kind_for_length(colptr[j + 1] - colptr[j]) < 0) {
                c->err = "foldin: a column has more than 8192 nonzeros";
                return NMFKL_EINVAL;
            }
    }
    nmfkl_status st = fold_reserve(c, m_new, nnz);
    if (st != NMFKL_OK) return st;
    FoldState &f = *c->fold;
    const cudaMemcpyKind in_kind = mem_kind == 0 ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const cudaMemcpyKind out_kind = mem_kind == 0 ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    bool ok = cuda_ok(c, cudaMemcpyAsync(f.colptr, colptr, 8 * (m_new + 1), in_kind, c->stream), "copy fold-in colptr");
    if (ok && nnz > 0)
        ok = cuda_ok(c, cudaMemcpyAsync(f.rowidx, rowidx, 4 * nnz, in_kind, c->stream), "copy fold-in rowidx") &&
             cuda_ok(c, cudaMemcpyAsync(f.val, val, 4 * nnz, in_kind, c->stream), "copy fold-in val");
    if (ok && doc_ids && m_new > 0)
        ok = cuda_ok(c, cudaMemcpyAsync(f.ids, doc_ids, 8 * m_new, in_kind, c->stream), "copy fold-in ids");
    if (!ok) return NMFKL_ECUDA;
    if (mem_kind == 1) {
        int32_t h = 0;
        int64_t last = 0;
        ok = cuda_ok(c, cudaMemsetAsync(c->err_flag, 0, 4, c->stream), "flag") &&
             launch_validate(c, m_new, c->n, nnz, f.colptr, f.rowidx, f.val, c->err_flag) == NMFKL_OK &&
             cuda_ok(c, cudaMemcpyAsync(&h, c->err_flag, 4, cudaMemcpyDeviceToHost, c->stream), "flag copy") &&
             cuda_ok(c, cudaMemcpyAsync(&last, f.colptr + m_new, 8, cudaMemcpyDeviceToHost, c->stream), "nnz copy") &&
             cuda_ok(c, cudaStreamSynchronize(c->stream), "validate sync") &&
             cuda_ok(c, cudaMemsetAsync(c->err_flag, 0, 4, c->stream), "flag");
        if (!ok) return NMFKL_ECUDA;
        if (h != 0 || last != nnz) {
            c->err = "foldin: device input failed validation (offsets, sorted in-range indices, values > 0)";
            return NMFKL_EINVAL;
        }
    }
    // starting F, unit-major
    if (segs) {
        for (const FoldSegment &g : *segs) {
            if (g.m <= 0) continue;
            if (!g.F0) {
                uniform_init_raw(c->stream, f.Ft + g.col0 * c->ldr, c->p.r, g.m, c->ldr, c->p.seed, 2);
                continue;
            }
            if (c->tbuf_floats < r * g.m) {
                cudaFree(c->tbuf);
                c->tbuf = nullptr;
                c->tbuf_floats = 0;
                if (!dev_alloc(c, &c->tbuf, r * g.m, "transpose buffer")) return NMFKL_ENOMEM;
                c->tbuf_floats = r * g.m;
            }
            if (!cuda_ok(c, cudaMemcpyAsync(c->tbuf, g.F0, sizeof(float) * r * g.m, cudaMemcpyHostToDevice, c->stream),
                         "copy segment F0"))
                return NMFKL_ECUDA;
            st = launch_to_unit_major(c, c->tbuf, f.Ft + g.col0 * c->ldr, g.m);
            if (st != NMFKL_OK) return st;
            if (!cuda_ok(c, cudaStreamSynchronize(c->stream), "segment F0 sync")) return NMFKL_ECUDA;
        }
    } else if (m_new > 0) {
        if (!F0) {
            uniform_init_raw(c->stream, f.Ft, c->p.r, m_new, c->ldr, c->p.seed, 2);
        } else {
            if (c->tbuf_floats < r * m_new) {
                cudaFree(c->tbuf);
                c->tbuf = nullptr;
                c->tbuf_floats = 0;
                if (!dev_alloc(c, &c->tbuf, r * m_new, "transpose buffer")) return NMFKL_ENOMEM;
                c->tbuf_floats = r * m_new;
            }
            if (!cuda_ok(c, cudaMemcpyAsync(c->tbuf, F0, sizeof(float) * r * m_new, in_kind, c->stream), "copy F0"))
                return NMFKL_ECUDA;
            st = launch_to_unit_major(c, c->tbuf, f.Ft, m_new);
            if (st != NMFKL_OK) return st;
        }
    }
    st = launch_mode == 2 ? foldin_per_doc(c, m_new, rel_tol, max_sweeps)
                          : foldin_run(c, m_new, doc_ids != nullptr, rel_tol, max_sweeps, launch_mode == 0);
    if (st != NMFKL_OK) return st;
    int32_t err = 0;
    ok = cuda_ok(c, cudaMemcpyAsync(&err, f.ctl + 2 * kFoldKinds, 4, cudaMemcpyDeviceToHost, c->stream), "fold-in flags");
    if (ok && m_new > 0) {
        ok = cuda_ok(c, cudaMemcpyAsync(F_out, f.Fout, sizeof(float) * r * m_new, out_kind, c->stream), "copy F_out");
        if (ok && sweeps_done)
            ok = cuda_ok(c, cudaMemcpyAsync(sweeps_done, f.sweeps, 4 * m_new, out_kind, c->stream), "copy sweeps");
        if (ok && doc_obj)
            ok = cuda_ok(c, cudaMemcpyAsync(doc_obj, f.obj, 8 * m_new, out_kind, c->stream), "copy objectives");
    }
    if (!ok || !cuda_ok(c, cudaStreamSynchronize(c->stream), "fold-in sync")) return NMFKL_ECUDA;
    if (err & 4) {
        c->err = "foldin: a column has more than 8192 nonzeros";
        return NMFKL_EINVAL;
    }
    if (err & 1) {
        c->err = "foldin: NaN produced";
        return NMFKL_ENUMERIC;
    }
    return NMFKL_OK;
}

}  // namespace nmfkl

extern "C" {

nmfkl_status nmfkl_foldin(nmfkl_ctx *c, int64_t m_new, int64_t nnz, const int64_t *colptr, const int32_t *rowidx,
                          const float *val, const int64_t *doc_ids, const float *F0, float *F_out, double rel_tol,
                          int32_t max_sweeps, int32_t *sweeps_done, double *doc_obj, int32_t launch_mode,
                          int32_t mem_kind) {
    return foldin_impl(c, m_new, nnz, colptr, rowidx, val, doc_ids, F0, nullptr, F_out, rel_tol, max_sweeps,
                       sweeps_done, doc_obj, launch_mode, mem_kind);
}

int32_t nmfkl_plan_info(const nmfkl_ctx *c, nmfkl_bucket_info *out, int32_t cap) {
    if (!c) return -1;
    int32_t i = 0;
    for (int side = 0; side < 2; ++side)
        for (int lp = 0; lp < 2; ++lp)
        for (const auto &b : lp ? c->plan_sparse[side] : c->plan[side]) {
            if (out && i < cap) {
                out[i].kernel = bucket_name(b);
                out[i].side = side;
                out[i].count = b.count;
                out[i].nnz = b.nnz;
                out[i].max_len = b.max_len;
                out[i].grid = b.grid;
                out[i].block = b.block;
                out[i].smem = (int64_t)b.smem;
                out[i].ran_last = (c->used_sparse[side] == lp &&
                                   (b.short_class < 0 || (b.group ? 1 : 0) == short_kernel(c, side, b.short_class)))
                                      ? 1
                                      : 0;
                out[i].list_plan = lp;
            }
            ++i;
        }
    return i;
}

static nmfkl_status get_factor(nmfkl_ctx *c, const float *Xt, int64_t cols, float *out, int32_t mem_kind) {
    if (!c || !out || (mem_kind != 0 && mem_kind != 1)) return NMFKL_EINVAL;
    cudaSetDevice(c->device);
    const int64_t need = cols * (int64_t)c->p.r;
    float *dst = out;
    if (mem_kind == 0) {
        if (c->tbuf_floats < need) {
            cudaFree(c->tbuf);
            c->tbuf = nullptr;
            c->tbuf_floats = 0;
            if (!dev_alloc(c, &c->tbuf, need, "transpose buffer")) return NMFKL_ENOMEM;
            c->tbuf_floats = need;
        }
        dst = c->tbuf;
    }
    nmfkl_status st = launch_from_unit_major(c, Xt, dst, cols);
    if (st != NMFKL_OK) return st;
    if (mem_kind == 0) {
        if (!cuda_ok(c, cudaMemcpyAsync(out, c->tbuf, sizeof(float) * need, cudaMemcpyDeviceToHost, c->stream),
                     "copy factor"))
            return NMFKL_ECUDA;
        if (!cuda_ok(c, cudaStreamSynchronize(c->stream), "get sync")) return NMFKL_ECUDA;
    }
    return NMFKL_OK;
}

nmfkl_status nmfkl_get_W(nmfkl_ctx *c, float *out, int32_t mem_kind) {
    return c ? get_factor(c, c->Wt, c->n, out, mem_kind) : NMFKL_EINVAL;
}
nmfkl_status nmfkl_get_F(nmfkl_ctx *c, float *out, int32_t mem_kind) {
    return c ? get_factor(c, c->Ft, c->m, out, mem_kind) : NMFKL_EINVAL;
}

// Checkpoint blob: header of eight 64-bit words, then W and F row-major.
namespace {
constexpr uint64_t kStateMagic = 0x3154534c4b464d4eull;  // "NMFKLST1" little-endian
constexpr uint64_t kStateVersion = 1;
constexpr int64_t kStateHeader = 64;
}  // namespace

int64_t nmfkl_state_bytes(const nmfkl_ctx *c) {
    if (!c) return -1;
    return kStateHeader + (int64_t)sizeof(float) * c->p.r * (c->n + c->m);
}

nmfkl_status nmfkl_get_state(nmfkl_ctx *c, int64_t next_sweep, void *buf, int64_t bytes) {
    if (!c || !buf || bytes < nmfkl_state_bytes(c) || next_sweep < 0) return NMFKL_EINVAL;
    uint64_t h[8] = {kStateMagic, kStateVersion, (uint64_t)c->p.r, (uint64_t)c->n,
                     (uint64_t)c->m, c->p.seed, (uint64_t)next_sweep, 0};
    unsigned char *b = static_cast<unsigned char *>(buf);
    std::memcpy(b, h, sizeof(h));
    float *W = reinterpret_cast<float *>(b + kStateHeader);
    float *F = W + (int64_t)c->p.r * c->n;
    nmfkl_status st = get_factor(c, c->Wt, c->n, W, 0);
    if (st == NMFKL_OK) st = get_factor(c, c->Ft, c->m, F, 0);
    return st;
}

nmfkl_status nmfkl_set_state(nmfkl_ctx *c, const void *buf, int64_t bytes, int64_t *next_sweep) {
    if (!c || !buf || bytes != nmfkl_state_bytes(c)) return NMFKL_EINVAL;
    uint64_t h[8];
    std::memcpy(h, buf, sizeof(h));
    if (h[0] != kStateMagic || h[1] != kStateVersion || h[2] != (uint64_t)c->p.r || h[3] != (uint64_t)c->n ||
        h[4] != (uint64_t)c->m || h[5] != c->p.seed || h[6] > (uint64_t)INT64_MAX) {
        c->err = "set_state: header does not match this context";
        return NMFKL_EINVAL;
    }
    const unsigned char *b = static_cast<const unsigned char *>(buf);
    const float *W = reinterpret_cast<const float *>(b + kStateHeader);
    const float *F = W + (int64_t)c->p.r * c->n;
    nmfkl_status st = nmfkl_init(c, W, F, 0);
    if (st == NMFKL_OK && next_sweep) *next_sweep = (int64_t)h[6];
    return st;
}

nmfkl_status nmfkl_get_counters(nmfkl_ctx *c, nmfkl_counters *out, int32_t reset) {
    if (!c || !out) return NMFKL_EINVAL;
    cudaSetDevice(c->device);
    unsigned long long h[4];
    if (!cuda_ok(c, cudaMemcpyAsync(h, c->counters, sizeof(h), cudaMemcpyDeviceToHost, c->stream), "counters") ||
        !cuda_ok(c, cudaStreamSynchronize(c->stream), "counters sync"))
        return NMFKL_ECUDA;
    out->coords = (int64_t)h[0];
    out->evals = (int64_t)h[1];
    out->steps = (int64_t)h[2];
    out->cap_hits = (int64_t)h[3];
    if (reset && !cuda_ok(c, cudaMemsetAsync(c->counters, 0, sizeof(h), c->stream), "reset counters"))
        return NMFKL_ECUDA;
    return NMFKL_OK;
}

nmfkl_status nmfkl_set_timing(nmfkl_ctx *c, int32_t enable) {
    if (!c) return NMFKL_EINVAL;
    c->timing = enable != 0;
    return NMFKL_OK;
}

int32_t nmfkl_kernel_times(nmfkl_ctx *c, const char **names, int64_t *launches, double *ms, int32_t cap,
                           int32_t reset) {
    if (!c) return -1;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    for (auto &pd : c->pending) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, pd.a, pd.b) == cudaSuccess) {
            c->timers[pd.timer].ms += t;
            c->timers[pd.timer].launches += 1;
        }
        c->ev_pool.push_back(pd.a);
        c->ev_pool.push_back(pd.b);
    }
    c->pending.clear();
    const int32_t nf = (int32_t)c->timers.size();
    for (int32_t i = 0; i < nf && i < cap; ++i) {
        if (names) names[i] = c->timers[i].name;
        if (launches) launches[i] = c->timers[i].launches;
        if (ms) ms[i] = c->timers[i].ms;
    }
    if (reset) {
        for (auto &t : c->timers) {
            t.launches = 0;
            t.ms = 0.0;
        }
    }
    return nf;
}

nmfkl_status nmfkl_debug_perm(nmfkl_ctx *c, int64_t sweep, int32_t side, int64_t count, const int64_t *cols,
                              int32_t *out) {
    if (!c || count < 0 || (count > 0 && (!cols || !out)) || (side != 0 && side != 1)) return NMFKL_EINVAL;
    cudaSetDevice(c->device);
    nmfkl_status st = launch_debug_perm(c, sweep, side, count, cols, out);
    if (st != NMFKL_OK) return st;
    return cuda_ok(c, cudaStreamSynchronize(c->stream), "debug_perm sync") ? NMFKL_OK : NMFKL_ECUDA;
}

}  // extern "C"
