// Serving loop (nmfkl_server_* in include/nmfkl.h): fold-in requests for new
// documents under one resident model W, and small full factorizations,
// admitted as they arrive while earlier work is still on the GPU.
//
// Structure: `slots` worker threads, each owning a CUDA stream and a fold-in
// context holding its copy of W on the device. A worker takes work from the
// head of one FIFO queue when the memory budget admits it: either every
// fold-in request waiting at the head with the same stopping settings
// (merged into one batched fold-in launch, up to max_batch_docs /
// max_batch_nnz), or one factorization (its own context on the worker's
// stream). Batches and factorizations of different workers overlap on the
// device. A request's result never depends on what it shared a batch with:
// its columns keep their request-local unit ids (which key the coordinate
// orders) and their own starting draw.
#include "common.cuh"

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>

using namespace nmfkl;

namespace {

using Clock = std::chrono::steady_clock;

struct ServerReq {
    uint64_t ticket = 0;
    int32_t kind = 0;
    int64_t n = 0, m = 0, nnz = 0;
    std::vector<int64_t> colptr;
    std::vector<int32_t> rowidx;
    std::vector<float> val;
    int32_t r = 0;
    uint64_t seed = 0;
    double rel_tol = 0.0;
    int32_t max_sweeps = 0;
    float *F_out = nullptr, *W_out = nullptr;
    int32_t *sweeps_out = nullptr;
    double *obj_out = nullptr;
    int64_t bytes = 0;
    Clock::time_point t_submit, t_admit, t_done;
    bool done = false;
    nmfkl_status status = NMFKL_OK;
    int32_t batch = 0;
    std::string message;
};

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

// Device bytes a request holds while it runs (beyond the per-slot state).
int64_t request_bytes(const ServerReq &q, int32_t model_r) {
    if (q.kind == NMFKL_REQ_FOLDIN) {
        const int64_t ldr = (model_r + 3) / 4 * 4;
        return 8 * (q.m + 1) + 8 * q.nnz + 8 * q.m + 4 * ldr * q.m + 4 * model_r * q.m + 16 * q.m +
               4 * (int64_t)kFoldKinds * q.m;
    }
    const int64_t ldr = (q.r + 3) / 4 * 4;
    const int64_t data = 24 * q.nnz + 8 * (q.n + q.m + 2);
    const int64_t factors = 4 * ldr * (q.n + q.m) + 4 * (int64_t)q.r * std::max(q.n, q.m);
    // tiles: at most one slot of r x (bucket capacity) floats per resident group
    const int64_t tiles = 4 * (int64_t)q.r * std::min<int64_t>(2 * q.nnz + 8192, int64_t(1) << 24);
    return data + factors + tiles + (int64_t(8) << 20);
}

}  // namespace

struct nmfkl_server {
    nmfkl_server_cfg cfg{};
    nmfkl_params p{};
    int64_t n = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<ServerReq *> pending;
    std::unordered_map<uint64_t, ServerReq *> reqs;  // submitted, not yet collected
    int64_t mem_in_use = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::vector<std::thread> workers;
    std::vector<nmfkl_ctx *> fold_ctx;
    std::vector<cudaStream_t> streams;
    std::string err;
    int64_t batches = 0, batched_requests = 0;
};

namespace {

// Requests to run next, taken from the head of the queue (lock held): the
// fold-in requests at the head with the head's settings, while the budget
// and the batch limits allow, or the factorization at the head.
std::vector<ServerReq *> take_work(nmfkl_server *s) {
    std::vector<ServerReq *> out;
    if (s->pending.empty()) return out;
    ServerReq *h = s->pending.front();
    if (s->mem_in_use > 0 && s->mem_in_use + h->bytes > s->cfg.mem_budget) return out;
    if (h->kind == NMFKL_REQ_FIT) {
        out.push_back(h);
        s->pending.pop_front();
        s->mem_in_use += h->bytes;
        return out;
    }
    int64_t docs = 0, nnz = 0;
    while (!s->pending.empty()) {
        ServerReq *q = s->pending.front();
        if (q->kind != NMFKL_REQ_FOLDIN || q->rel_tol != h->rel_tol || q->max_sweeps != h->max_sweeps) break;
        if (!out.empty() && (docs + q->m > s->cfg.max_batch_docs || nnz + q->nnz > s->cfg.max_batch_nnz ||
                             s->mem_in_use + q->bytes > s->cfg.mem_budget))
            break;
        out.push_back(q);
        s->pending.pop_front();
        s->mem_in_use += q->bytes;
        docs += q->m;
        nnz += q->nnz;
    }
    return out;
}

nmfkl_status run_foldin_batch(nmfkl_ctx *c, std::vector<ServerReq *> &batch, std::string &msg) {
    int64_t m_tot = 0, nnz_tot = 0;
    for (auto *q : batch) {
        m_tot += q->m;
        nnz_tot += q->nnz;
    }
    std::vector<int64_t> colptr(m_tot + 1, 0), ids(m_tot);
    std::vector<int32_t> rowidx(nnz_tot);
    std::vector<float> val(nnz_tot);
    std::vector<FoldSegment> segs;
    int64_t col = 0, off = 0;
    for (auto *q : batch) {
        segs.push_back(FoldSegment{col, q->m, nullptr});
        for (int64_t j = 0; j < q->m; ++j) {
            colptr[col + j + 1] = off + q->colptr[j + 1];
            ids[col + j] = j;
        }
        if (q->nnz > 0) {
            std::memcpy(rowidx.data() + off, q->rowidx.data(), 4 * q->nnz);
            std::memcpy(val.data() + off, q->val.data(), 4 * q->nnz);
        }
        col += q->m;
        off += q->nnz;
    }
    const int32_t r = c->p.r;
    std::vector<float> F((size_t)r * m_tot);
    std::vector<int32_t> sweeps(m_tot);
    std::vector<double> obj(m_tot);
    const nmfkl_status st =
        foldin_impl(c, m_tot, nnz_tot, colptr.data(), rowidx.data(), val.data(), ids.data(), nullptr, &segs,
                    F.data(), batch.front()->rel_tol, batch.front()->max_sweeps, sweeps.data(), obj.data(), 0, 0);
    if (st != NMFKL_OK) {
        msg = nmfkl_last_error(c);
        return st;
    }
    col = 0;
    for (auto *q : batch) {
        for (int32_t k = 0; k < r && q->F_out; ++k)
            std::memcpy(q->F_out + (int64_t)k * q->m, F.data() + (int64_t)k * m_tot + col, 4 * q->m);
        if (q->sweeps_out) std::memcpy(q->sweeps_out, sweeps.data() + col, 4 * q->m);
        if (q->obj_out) std::memcpy(q->obj_out, obj.data() + col, 8 * q->m);
        col += q->m;
    }
    return NMFKL_OK;
}

nmfkl_status run_fit(nmfkl_server *s, cudaStream_t stream, ServerReq *q, std::string &msg) {
    nmfkl_params pp = s->p;
    pp.r = q->r;
    pp.seed = q->seed;
    nmfkl_ctx *c = nullptr;
    nmfkl_status st = nmfkl_create(&pp, q->n, q->m, s->cfg.device, stream, &c);
    if (st != NMFKL_OK) {
        msg = "fit: context creation failed";
        return st;
    }
    st = nmfkl_set_data(c, q->nnz, q->colptr.data(), q->rowidx.data(), q->val.data(), nullptr, nullptr, nullptr, 0);
    if (st == NMFKL_OK) st = nmfkl_init(c, nullptr, nullptr, 0);
    int32_t done = 0;
    std::vector<double> trace(std::max(q->max_sweeps, 1));
    if (st == NMFKL_OK) {
        st = nmfkl_fit(c, 0, q->max_sweeps, q->rel_tol, trace.data(), &done);
        if (st == NMFKL_ENOTCONV) st = NMFKL_OK;  // max_sweeps is a legitimate stop for a request
    }
    if (st == NMFKL_OK && q->F_out) st = nmfkl_get_F(c, q->F_out, 0);
    if (st == NMFKL_OK && q->W_out) st = nmfkl_get_W(c, q->W_out, 0);
    if (st == NMFKL_OK) {
        if (q->sweeps_out) q->sweeps_out[0] = done;
        if (q->obj_out) {
            double kl = 0.0;
            if (done > 0) kl = trace[done - 1];
            else st = nmfkl_objective(c, &kl, nullptr);
            q->obj_out[0] = kl;
        }
    }
    if (st != NMFKL_OK) msg = nmfkl_last_error(c);
    nmfkl_destroy(c);
    return st;
}

void worker(nmfkl_server *s, int slot) {
    cudaSetDevice(s->cfg.device);
    for (;;) {
        std::vector<ServerReq *> work;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] {
                if (s->stop) return true;
                if (s->pending.empty()) return false;
                const ServerReq *h = s->pending.front();
                return s->mem_in_use == 0 || s->mem_in_use + h->bytes <= s->cfg.mem_budget;
            });
            if (s->stop) return;
            work = take_work(s);
            if (work.empty()) continue;
            const auto now = Clock::now();
            for (auto *q : work) {
                q->t_admit = now;
                q->batch = (int32_t)work.size();
            }
            if (work.front()->kind == NMFKL_REQ_FOLDIN) {
                s->batches += 1;
                s->batched_requests += (int64_t)work.size();
            }
        }
        // more work may be admissible for the other workers
        s->cv_work.notify_all();
        nmfkl_status st;
        std::string msg;
        if (work.front()->kind == NMFKL_REQ_FOLDIN) {
            TraceRange trace("serve fold-in batch");
            st = run_foldin_batch(s->fold_ctx[slot], work, msg);
        } else {
            TraceRange trace("serve fit");
            st = run_fit(s, s->streams[slot], work.front(), msg);
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            const auto now = Clock::now();
            for (auto *q : work) {
                q->status = st;
                q->message = msg;
                q->t_done = now;
                q->done = true;
                s->mem_in_use -= q->bytes;
            }
        }
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
}

void fill_result(const ServerReq *q, nmfkl_result *res) {
    if (!res) return;
    res->status = q->status;
    res->queued_ms = ms_between(q->t_submit, q->t_admit);
    res->run_ms = ms_between(q->t_admit, q->t_done);
    res->batch_requests = q->batch;
    std::snprintf(res->message, sizeof(res->message), "%s", q->message.c_str());
}

}  // namespace

extern "C" {

void nmfkl_server_default_cfg(nmfkl_server_cfg *cfg) {
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->device = 0;
    cfg->slots = 4;
    cfg->mem_budget = int64_t(16) << 30;
    cfg->max_pending = 4096;
    cfg->max_batch_docs = 20000;
    cfg->max_batch_nnz = int64_t(1) << 26;
}

nmfkl_status nmfkl_server_create(const nmfkl_server_cfg *cfg, const nmfkl_params *p, int64_t n, const float *W,
                                 nmfkl_server **out) {
    if (!out) return NMFKL_EINVAL;
    *out = nullptr;
    if (!cfg || !p || !W || n < 1 || cfg->slots < 1 || cfg->slots > 64 || cfg->mem_budget < 1 ||
        cfg->max_pending < 1 || cfg->max_batch_docs < 1 || cfg->max_batch_nnz < 1)
        return NMFKL_EINVAL;
    nmfkl_server *s = new (std::nothrow) nmfkl_server();
    if (!s) return NMFKL_ENOMEM;
    s->cfg = *cfg;
    s->p = *p;
    s->n = n;
    if (cudaSetDevice(cfg->device) != cudaSuccess) {
        delete s;
        return NMFKL_ECUDA;
    }
    nmfkl_status st = NMFKL_OK;
    std::vector<float> F1((size_t)p->r, 0.f);
    for (int i = 0; i < cfg->slots && st == NMFKL_OK; ++i) {
        cudaStream_t stream = nullptr;
        if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) {
            st = NMFKL_ECUDA;
            break;
        }
        s->streams.push_back(stream);
        nmfkl_ctx *c = nullptr;
        st = nmfkl_create(p, n, 1, cfg->device, stream, &c);
        if (st != NMFKL_OK) break;
        s->fold_ctx.push_back(c);
        st = nmfkl_init(c, W, F1.data(), 0);
    }
    if (st != NMFKL_OK) {
        nmfkl_server_destroy(s);
        return st;
    }
    for (int i = 0; i < cfg->slots; ++i) s->workers.emplace_back(worker, s, i);
    *out = s;
    return NMFKL_OK;
}

nmfkl_status nmfkl_server_submit(nmfkl_server *s, const nmfkl_request *req, uint64_t *ticket) {
    if (!s || !req || !ticket) return NMFKL_EINVAL;
    const bool fold = req->kind == NMFKL_REQ_FOLDIN;
    if ((req->kind != NMFKL_REQ_FOLDIN && req->kind != NMFKL_REQ_FIT) || req->m < 0 || req->nnz < 0 ||
        !req->colptr || (req->nnz > 0 && (!req->rowidx || !req->val)) || !(req->rel_tol >= 0) ||
        req->max_sweeps < 0 || (fold && req->n != s->n) ||
        (!fold && (req->n < 1 || req->m < 1 || req->r < 1 || req->r > kMaxR)))
        return NMFKL_EINVAL;
    if (req->colptr[0] != 0 || req->colptr[req->m] != req->nnz) return NMFKL_EINVAL;
    ServerReq *q = new (std::nothrow) ServerReq();
    if (!q) return NMFKL_ENOMEM;
    q->kind = req->kind;
    q->n = req->n;
    q->m = req->m;
    q->nnz = req->nnz;
    q->colptr.assign(req->colptr, req->colptr + req->m + 1);
    q->rowidx.assign(req->rowidx, req->rowidx + req->nnz);
    q->val.assign(req->val, req->val + req->nnz);
    q->r = fold ? s->p.r : req->r;
    q->seed = req->seed;
    q->rel_tol = req->rel_tol;
    q->max_sweeps = req->max_sweeps;
    q->F_out = req->F_out;
    q->W_out = req->W_out;
    q->sweeps_out = req->sweeps_out;
    q->obj_out = req->obj_out;
    q->bytes = request_bytes(*q, s->p.r);
    q->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (q->bytes > s->cfg.mem_budget) {
            s->err = "request needs more device memory than the budget";
            delete q;
            return NMFKL_EINVAL;
        }
        if ((int64_t)s->pending.size() >= s->cfg.max_pending) {
            delete q;
            return NMFKL_EBUSY;
        }
        q->ticket = s->next_ticket++;
        s->pending.push_back(q);
        s->reqs[q->ticket] = q;
        *ticket = q->ticket;
    }
    s->cv_work.notify_one();
    return NMFKL_OK;
}

nmfkl_status nmfkl_server_poll(nmfkl_server *s, uint64_t ticket, nmfkl_result *res) {
    if (!s) return NMFKL_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return NMFKL_EINVAL;
    if (!it->second->done) return NMFKL_EBUSY;
    fill_result(it->second, res);
    delete it->second;
    s->reqs.erase(it);
    return NMFKL_OK;
}

nmfkl_status nmfkl_server_wait(nmfkl_server *s, uint64_t ticket, nmfkl_result *res) {
    if (!s) return NMFKL_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return NMFKL_EINVAL;
    ServerReq *q = it->second;
    s->cv_done.wait(lk, [&] { return q->done; });
    fill_result(q, res);
    delete q;
    s->reqs.erase(ticket);
    return NMFKL_OK;
}

nmfkl_status nmfkl_server_cancel(nmfkl_server *s, uint64_t ticket) {
    if (!s) return NMFKL_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return NMFKL_EINVAL;
        ServerReq *q = it->second;
        // only a request still in the queue: a worker that took it owns it
        auto pos = std::find(s->pending.begin(), s->pending.end(), q);
        if (q->done || pos == s->pending.end()) return NMFKL_EBUSY;
        s->pending.erase(pos);
        q->t_admit = q->t_done = Clock::now();
        q->status = NMFKL_ECANCELED;
        q->message = "canceled before it ran";
        q->done = true;
    }
    s->cv_done.notify_all();
    // the new head of the queue may be admissible now
    s->cv_work.notify_all();
    return NMFKL_OK;
}

nmfkl_status nmfkl_server_stats(nmfkl_server *s, nmfkl_server_stats_t *out) {
    if (!s || !out) return NMFKL_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    out->pending = (int64_t)s->pending.size();
    out->mem_in_use = s->mem_in_use;
    out->batches = s->batches;
    out->batched_requests = s->batched_requests;
    return NMFKL_OK;
}

void nmfkl_server_destroy(nmfkl_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->workers) t.join();
    for (auto *c : s->fold_ctx) nmfkl_destroy(c);
    for (auto st : s->streams) cudaStreamDestroy(st);
    for (auto &kv : s->reqs) delete kv.second;
    delete s;
}

}  // extern "C"
