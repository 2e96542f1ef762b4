// Continuous-batching query server.
//
// The paper answers queries "asynchronously" as they arrive (Sec. 4.1,
// Queries); on one GPU throughput comes from answering many at once.  The
// server keeps a FIFO of pending requests per registered collection.  Worker
// threads (each with its own CUDA stream and query work space) repeatedly
// take the pending requests of one collection and answer them together with
// the exact query path, using k = the largest k of the batch: answers are
// totally ordered by (binary64 squared distance, id), so each request's
// answer is the prefix of length k_i, exactly what a call for that request
// alone returns.
//
// Admission: a batch takes device memory from the server's budget (its work
// spaces' estimated bytes) and gives it back when it completes; a worker
// admits as many pending requests as the budget has room for at that
// moment, at least one when nothing else is in flight, and otherwise waits
// for memory to free up.
//
// Persistent form (hk_server_opts.persistent): the tensor-core scans of all
// batches in flight -- the bulk of the work, from any registered collection
// with a 16-bit copy -- run in one resident launch (hk_tc.cu) that takes
// each batch's scan from a device-resident ring while it runs: a batch
// admitted while others are on the GPU joins the same launch, and its
// query blocks interleave with theirs; each query's bound U and candidate
// lists stay in device memory for the batch's lifetime.  The batches' other
// steps run on their workers' streams beside it.
//
// Every wait is bounded: hk_poll waits at most its timeout, a worker waits at
// most 120 s for a scan, and workers wake at least every few milliseconds
// to notice shutdown.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "hk_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kSideSMs = 8;   // SMs the resident scan leaves to the batches' other kernels

struct Request {
    uint64_t ticket;
    int coll;
    int k;
    std::vector<float> q;
    std::vector<int64_t> ids;
    std::vector<float> dist;
    Clock::time_point t_submit;
    int64_t latency_ns = 0;
    int status = 1;          // 1 pending/running, 0 done, < 0 error code
    std::string error;
};

struct Worker {
    cudaStream_t stream = nullptr;
    hk::Workspace ws, ws_retry;
    hk::DevBuf<float> Qd;
    float *Qh = nullptr;          // pinned
    int64_t *ids_h = nullptr;     // pinned
    float *dist_h = nullptr;      // pinned
    size_t cap_q = 0, cap_out = 0;
    std::thread th;
};

}  // namespace

struct hk_server {
    hk_server_opts opts{};
    hk::TcEngine *engine = nullptr;   // persistent form
    int64_t budget_used = 0;          // device bytes the batches in flight hold
    std::condition_variable cv_mem;   // budget freed
    std::vector<hk_index *> colls;
    std::vector<hk_query_opts> copts;  // per collection: its query configuration
    std::vector<char> has_copts;       // 1: copts applies, 0: the server's query_flags
    std::mutex mu;
    std::condition_variable cv_work;   // requests arrived / shutdown
    std::condition_variable cv_done;   // a request completed
    std::vector<std::deque<std::shared_ptr<Request>>> queues;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> table;
    uint64_t next_ticket = 1;
    size_t rr = 0;
    bool stop = false;
    std::vector<std::unique_ptr<Worker>> workers;
    int device = 0;
    // statistics
    int64_t batches = 0, served = 0, max_batch_seen = 0, errors = 0, budget_peak = 0;
    double busy_s = 0.0;
};

namespace {

// Whether a collection's batches take the precision form.  Called with
// sv->mu held.
bool coll_tc(const hk_server *sv, int coll) {
    const hk_index *idx = sv->colls[coll];
    const uint32_t f = sv->has_copts[coll] ? sv->copts[coll].flags : sv->opts.query_flags;
    return (f & HK_Q_BF16) && idx->has_bf16 && idx->n <= hk::kTcMaxLen;
}

// Device bytes of query work space per query of a batch on this index
// (pessimistic: the form's largest pools and candidate lists).
int64_t bytes_per_query(const hk_index *idx, int k, bool tc) {
    const int64_t L = idx->L, n = idx->n;
    const int64_t pool = tc ? hk::tc_list_cap(k) : 65536;
    return L * (1 + 4 + 8) + n * 4 * 2 + idx->S * 16 + 16 * 256 * 2 + pool * 16 +
           pool * 8 + 64 * (int64_t)k;
}

// Device bytes a batch of nq queries with this k holds while in flight
// (its work space and its retry work space).
int64_t batch_bytes(const hk_index *idx, int k, int nq, bool tc) {
    return bytes_per_query(idx, k, tc) * 2 * nq;
}

// Most requests a batch may take now: max_batch, and what the budget has
// room for beside the batches in flight (at least one when none is).
// Called with sv->mu held.
int batch_cap(hk_server *sv, int coll, int k) {
    const hk_index *idx = sv->colls[coll];
    int cap = sv->opts.max_batch > 0 ? sv->opts.max_batch : 1024;
    if (sv->opts.hbm_budget > 0) {
        const int64_t per = std::max<int64_t>(1, batch_bytes(idx, k, 1, coll_tc(sv, coll)));
        const int64_t room = sv->opts.hbm_budget - sv->budget_used;
        const int64_t fit = room > 0 ? room / per : 0;
        cap = (int)std::min<int64_t>(cap, fit);
        if (cap < 1 && sv->budget_used == 0) cap = 1;
    }
    return cap;
}

void ensure_host(Worker &w, size_t q_floats, size_t outs) {
    if (q_floats > w.cap_q) {
        if (w.Qh) cudaFreeHost(w.Qh);
        HK_CHECK_CUDA(cudaMallocHost((void **)&w.Qh, q_floats * sizeof(float)));
        w.cap_q = q_floats;
    }
    if (outs > w.cap_out) {
        if (w.ids_h) cudaFreeHost(w.ids_h);
        if (w.dist_h) cudaFreeHost(w.dist_h);
        HK_CHECK_CUDA(cudaMallocHost((void **)&w.ids_h, outs * sizeof(int64_t)));
        HK_CHECK_CUDA(cudaMallocHost((void **)&w.dist_h, outs * sizeof(float)));
        w.cap_out = outs;
    }
}

void worker_loop(hk_server *sv, Worker *w) {
    cudaSetDevice(sv->device);
    for (;;) {
        std::vector<std::shared_ptr<Request>> batch;
        int coll = -1;
        int64_t reserved = 0;
        hk_query_opts copt{};
        bool has_copt = false;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            for (;;) {
                if (sv->stop) return;
                // pick the next non-empty collection (round robin)
                const size_t nc = sv->queues.size();
                for (size_t i = 0; i < nc; ++i) {
                    const size_t c = (sv->rr + i) % nc;
                    if (!sv->queues[c].empty()) {
                        coll = (int)c;
                        sv->rr = c + 1;
                        break;
                    }
                }
                if (coll >= 0) break;
                sv->cv_work.wait_for(lk, std::chrono::milliseconds(5));
            }
            // optionally linger to fill the batch
            if (sv->opts.max_wait_us > 0) {
                const auto until = Clock::now() + std::chrono::microseconds(sv->opts.max_wait_us);
                const int kmax_guess = sv->queues[coll].front()->k;
                const int cap = batch_cap(sv, coll, kmax_guess);
                while ((int)sv->queues[coll].size() < cap && Clock::now() < until && !sv->stop)
                    sv->cv_work.wait_until(lk, until);
            }
            if (sv->queues[coll].empty()) continue;
            int kmax = 0;
            for (auto &r : sv->queues[coll]) kmax = std::max(kmax, r->k);
            const int cap = batch_cap(sv, coll, kmax);
            if (cap < 1) {
                // the budget is taken by batches in flight: wait for one to finish
                sv->cv_mem.wait_for(lk, std::chrono::milliseconds(5));
                continue;
            }
            while (!sv->queues[coll].empty() && (int)batch.size() < cap) {
                batch.push_back(sv->queues[coll].front());
                sv->queues[coll].pop_front();
            }
            has_copt = sv->has_copts[coll] != 0;
            if (has_copt) copt = sv->copts[coll];
            if (sv->opts.hbm_budget > 0) {
                reserved = batch_bytes(sv->colls[coll], kmax, (int)batch.size(), coll_tc(sv, coll));
                sv->budget_used += reserved;
                sv->budget_peak = std::max(sv->budget_peak, sv->budget_used);
            }
        }
        if (batch.empty()) continue;
        hk_index *idx = sv->colls[coll];
        const int nq = (int)batch.size(), n = idx->n;
        int k = 0;
        for (auto &r : batch) k = std::max(k, r->k);
        int rc = HK_OK;
        std::string msg;
        const auto t0 = Clock::now();
        try {
            ensure_host(*w, (size_t)nq * n, (size_t)nq * k);
            for (int i = 0; i < nq; ++i)
                std::memcpy(w->Qh + (size_t)i * n, batch[i]->q.data(), n * sizeof(float));
            w->Qd.reserve((size_t)nq * n, w->stream);
            HK_CHECK_CUDA(cudaMemcpyAsync(w->Qd.p, w->Qh, (size_t)nq * n * sizeof(float),
                                          cudaMemcpyHostToDevice, w->stream));
            hk_query_opts o;
            std::memset(&o, 0, sizeof(o));
            o.eapca_th = -1.0f;
            o.sax_th = -1.0f;
            o.flags = sv->opts.query_flags;
            if (has_copt) o = copt;   // the collection's own configuration
            // graph mode records a pass per index into that index's one graph
            // work space, which concurrent batches would share: not served
            o.flags &= ~(uint32_t)(HK_Q_TIMING | HK_Q_GRAPH);
            // the precision form where the collection has it (16-bit copy, n <= 256)
            if ((o.flags & HK_Q_BF16) && (!idx->has_bf16 || idx->n > hk::kTcMaxLen))
                o.flags &= ~(uint32_t)HK_Q_BF16;
            hk::run_query_ws(idx, w->ws, w->ws_retry, w->Qd.p, nq, k, o, w->stream, w->ids_h,
                             w->dist_h, nullptr);
        } catch (const hk::Error &e) {
            rc = e.code;
            msg = e.msg;
        } catch (...) {
            rc = HK_EINTERNAL;
            msg = "unexpected exception";
        }
        const auto t1 = Clock::now();
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            for (int i = 0; i < nq; ++i) {
                Request &r = *batch[i];
                if (rc == HK_OK) {
                    r.ids.assign(w->ids_h + (size_t)i * k, w->ids_h + (size_t)i * k + r.k);
                    r.dist.assign(w->dist_h + (size_t)i * k, w->dist_h + (size_t)i * k + r.k);
                    r.status = 0;
                } else {
                    r.status = rc;
                    r.error = msg;
                }
                r.latency_ns = std::chrono::duration_cast<std::chrono::nanoseconds>(t1 - r.t_submit).count();
            }
            sv->budget_used -= reserved;
            sv->batches += 1;
            sv->served += nq;
            sv->max_batch_seen = std::max<int64_t>(sv->max_batch_seen, nq);
            if (rc != HK_OK) sv->errors += 1;
            sv->busy_s += std::chrono::duration<double>(t1 - t0).count();
        }
        sv->cv_done.notify_all();
        sv->cv_mem.notify_all();
    }
}

}  // namespace

extern "C" {

int hk_server_create(const hk_server_opts *opts, hk_server **out) {
    try {
        hk::clear_last_error();
        if (!out) hk::fail(HK_EINVAL, "out is NULL");
        *out = nullptr;
        std::unique_ptr<hk_server> sv(new hk_server());
        if (opts) sv->opts = *opts;
        if (sv->opts.max_batch < 0 || sv->opts.max_wait_us < 0 || sv->opts.hbm_budget < 0 ||
            sv->opts.workers < 0)
            hk::fail(HK_EINVAL, "negative server option");
        if (sv->opts.persistent != 0 && sv->opts.persistent != 1) hk::fail(HK_EINVAL, "persistent must be 0 or 1");
        const int nw = sv->opts.workers > 0 ? sv->opts.workers : (sv->opts.persistent ? 3 : 2);
        HK_CHECK_CUDA(cudaGetDevice(&sv->device));
        if (sv->opts.persistent) sv->engine = hk::tc_engine_create(kSideSMs);
        for (int i = 0; i < nw; ++i) {
            auto w = std::make_unique<Worker>();
            HK_CHECK_CUDA(cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking));
            w->ws.engine = sv->engine;
            w->ws_retry.engine = sv->engine;
            sv->workers.push_back(std::move(w));
        }
        hk_server *raw = sv.get();
        for (auto &w : sv->workers) w->th = std::thread(worker_loop, raw, w.get());
        *out = sv.release();
        return HK_OK;
    } catch (const hk::Error &e) {
        hk::set_last_error(e.code, e.msg);
        return e.code;
    }
}

int hk_server_add(hk_server *sv, hk_index *idx, int32_t *coll_id) {
    return hk_server_add_opts(sv, idx, nullptr, coll_id);
}

int hk_server_add_opts(hk_server *sv, hk_index *idx, const hk_query_opts *opts, int32_t *coll_id) {
    try {
        hk::clear_last_error();
        if (!sv || !idx || !coll_id) hk::fail(HK_EINVAL, "NULL argument");
        if (opts) hk::check_query_opts(idx, *opts);
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->colls.push_back(idx);
        sv->queues.emplace_back();
        sv->copts.push_back(opts ? *opts : hk_query_opts{});
        sv->has_copts.push_back(opts ? 1 : 0);
        *coll_id = (int32_t)sv->colls.size() - 1;
        return HK_OK;
    } catch (const hk::Error &e) {
        hk::set_last_error(e.code, e.msg);
        return e.code;
    }
}

int hk_submit(hk_server *sv, int32_t coll_id, const float *q, int32_t k, uint64_t *ticket) {
    try {
        hk::clear_last_error();
        if (!sv || !q || !ticket) hk::fail(HK_EINVAL, "NULL argument");
        auto r = std::make_shared<Request>();
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            if (coll_id < 0 || coll_id >= (int)sv->colls.size())
                hk::fail(HK_EINVAL, "unknown collection %d", coll_id);
            const hk_index *idx = sv->colls[coll_id];
            if (k < 1 || k > HK_MAX_K || (int64_t)k > idx->N)
                hk::fail(HK_EINVAL, "k=%d must be in [1, min(N, %d)]", k, HK_MAX_K);
            r->q.assign(q, q + idx->n);
        }
        for (float v : r->q)
            if (!std::isfinite(v)) hk::fail(HK_EINVAL, "the query holds NaN or Inf");
        r->coll = coll_id;
        r->k = k;
        r->t_submit = Clock::now();
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            if (sv->stop) hk::fail(HK_EBUSY, "the server is shutting down");
            r->ticket = sv->next_ticket++;
            sv->table[r->ticket] = r;
            sv->queues[coll_id].push_back(r);
            *ticket = r->ticket;
        }
        sv->cv_work.notify_one();
        return HK_OK;
    } catch (const hk::Error &e) {
        hk::set_last_error(e.code, e.msg);
        return e.code;
    }
}

int hk_poll(hk_server *sv, uint64_t ticket, int64_t *ids, float *dist, int32_t timeout_us,
            int64_t *latency_ns) {
    try {
        hk::clear_last_error();
        if (!sv || !ids || !dist) hk::fail(HK_EINVAL, "NULL argument");
        std::unique_lock<std::mutex> lk(sv->mu);
        auto it = sv->table.find(ticket);
        if (it == sv->table.end()) hk::fail(HK_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
        std::shared_ptr<Request> r = it->second;
        const auto until = Clock::now() + std::chrono::microseconds(std::max(0, timeout_us));
        while (r->status == 1) {
            if (sv->cv_done.wait_until(lk, until) == std::cv_status::timeout && r->status == 1)
                return HK_ETIMEOUT;   // not an error: the ticket stays valid
        }
        sv->table.erase(it);
        if (r->status != 0) hk::fail(r->status, "request failed: %s", r->error.c_str());
        std::memcpy(ids, r->ids.data(), r->ids.size() * sizeof(int64_t));
        std::memcpy(dist, r->dist.data(), r->dist.size() * sizeof(float));
        if (latency_ns) *latency_ns = r->latency_ns;
        return HK_OK;
    } catch (const hk::Error &e) {
        hk::set_last_error(e.code, e.msg);
        return e.code;
    }
}

int hk_server_stats_get(hk_server *sv, hk_server_stats *out) {
    if (!sv || !out) return HK_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    std::memset(out, 0, sizeof(*out));
    out->batches = sv->batches;
    out->served = sv->served;
    out->max_batch = sv->max_batch_seen;
    out->errors = sv->errors;
    int64_t pending = 0;
    for (auto &q : sv->queues) pending += (int64_t)q.size();
    out->pending = pending;
    out->busy_ns = (int64_t)(sv->busy_s * 1e9);
    out->budget_peak = sv->budget_peak;
    if (sv->engine) {
        hk::TcEngineStats es;
        hk::tc_engine_stats(sv->engine, &es);
        out->scan_launches = es.launches;
        out->scan_jobs = es.jobs;
        out->scan_jobs_inflight = es.jobs_inflight;
        out->scan_max_collections = es.max_colls_per_launch;
    }
    return HK_OK;
}

int hk_server_destroy(hk_server *sv) {
    if (!sv) return HK_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    for (auto &w : sv->workers)
        if (w->th.joinable()) w->th.join();
    for (auto &w : sv->workers) {
        if (w->stream) cudaStreamSynchronize(w->stream);
        if (w->Qh) cudaFreeHost(w->Qh);
        if (w->ids_h) cudaFreeHost(w->ids_h);
        if (w->dist_h) cudaFreeHost(w->dist_h);
        if (w->stream) cudaStreamDestroy(w->stream);
    }
    hk::tc_engine_destroy(sv->engine);
    {
        // requests never served fail with HK_EBUSY
        std::lock_guard<std::mutex> lk(sv->mu);
        for (auto &kv : sv->table)
            if (kv.second->status == 1) kv.second->status = HK_EBUSY;
    }
    sv->cv_done.notify_all();
    delete sv;
    return HK_OK;
}

}  // extern "C"
