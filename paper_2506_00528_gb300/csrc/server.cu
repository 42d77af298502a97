// Continuous-batching request loop over a resident database.
//
// Requests (host float32 query rows, a k) are queued by evp_server_submit.
// A host worker thread owns a small set of slots; each slot is one batch in
// flight on the GPU: a stream, pinned host staging, a device workspace and a
// completion event.  Whenever a slot is free the worker coalesces the
// oldest pending request with every other pending request of the same k,
// in arrival order, up to the slot's query capacity, and launches the whole
// path for them with one evp_db_search_host call (H2D copy, encode, scan,
// rerank, D2H copy).  Requests that arrive while batches run are admitted
// into the next free slot at once, so batches overlap on the device.  A
// request's result depends only on its own queries and k: the shortlist
// length is a function of k, batches never mix values of k, and every
// kernel treats queries independently.
//
// Admission is by memory: the number of slots is the largest count whose
// workspaces fit in the configured device budget (at least one; creation
// fails with EVP_ERR_NO_MEMORY if not even one fits), and a request larger
// than a slot's capacity is rejected at submission.
#include "evp_internal.cuh"

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t id;
    const float* Q;
    int64_t nq;
    int32_t k;
    int64_t* ids_out;
    float* scores_out;
    Clock::time_point arrival;
    double latency_us = 0.0;
    int32_t status = EVP_OK;
    bool done = false;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done_ev = nullptr;
    float* q_h = nullptr;        // pinned [cap][d]
    int64_t* ids_h = nullptr;    // pinned [cap][max_k]
    float* sc_h = nullptr;       // pinned [cap][max_k]
    int32_t* status_h = nullptr; // pinned [1]
    int32_t* status_d = nullptr; // device [1]
    void* ws = nullptr;          // device workspace
    size_t ws_bytes = 0;
    std::vector<Request*> reqs;
    int32_t k = 0;
    bool busy = false;
};

}  // namespace

struct evp_server {
    evp_db_t db = nullptr;
    evp_server_config cfg{};
    int d = 0;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> pending;
    std::unordered_map<int64_t, Request*> reqs;
    std::vector<double> lat_us;
    int64_t next_id = 1;
    int64_t batches = 0, queries_done = 0;
    bool stop = false;
    bool paused = false;
    std::thread worker;
};

namespace {

int32_t shortlist_for(const evp_server* s, int32_t k) {
    int64_t n = (int64_t)s->cfg.shortlist_factor * k;
    n = std::min<int64_t>(n, EVP_MAX_K);
    n = std::max<int64_t>(n, k);
    return (int32_t)n;
}

void free_slot(Slot& sl) {
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.done_ev) cudaEventDestroy(sl.done_ev);
    if (sl.q_h) cudaFreeHost(sl.q_h);
    if (sl.ids_h) cudaFreeHost(sl.ids_h);
    if (sl.sc_h) cudaFreeHost(sl.sc_h);
    if (sl.status_h) cudaFreeHost(sl.status_h);
    if (sl.status_d) cudaFree(sl.status_d);
    if (sl.ws) cudaFree(sl.ws);
    sl = Slot();
}

// Launch one batch on a free slot (called with the lock held).
void launch_batch(evp_server* s, Slot& sl, std::vector<Request*>& batch, int32_t k) {
    int64_t nq = 0;
    for (Request* r : batch) {
        std::memcpy(sl.q_h + nq * s->d, r->Q, (size_t)r->nq * s->d * sizeof(float));
        nq += r->nq;
    }
    sl.reqs = batch;
    sl.k = k;
    sl.busy = true;
    int32_t rc = cudaMemsetAsync(sl.status_d, 0, sizeof(int32_t), sl.stream) == cudaSuccess
                     ? EVP_OK
                     : EVP_ERR_CUDA;
    if (rc == EVP_OK)
        rc = evp_db_search_host(s->db, sl.q_h, nq, shortlist_for(s, k), k, sl.ids_h, sl.sc_h,
                                sl.ws, sl.ws_bytes, sl.status_d, sl.stream);
    if (rc == EVP_OK &&
        cudaMemcpyAsync(sl.status_h, sl.status_d, sizeof(int32_t), cudaMemcpyDeviceToHost,
                        sl.stream) != cudaSuccess)
        rc = EVP_ERR_CUDA;
    if (rc == EVP_OK && cudaEventRecord(sl.done_ev, sl.stream) != cudaSuccess) rc = EVP_ERR_CUDA;
    if (rc != EVP_OK) {
        // nothing usable is in flight on this slot: fail its requests now
        cudaStreamSynchronize(sl.stream);
        const Clock::time_point now = Clock::now();
        for (Request* r : sl.reqs) {
            r->status = rc;
            r->done = true;
            r->latency_us = std::chrono::duration<double, std::micro>(now - r->arrival).count();
        }
        sl.reqs.clear();
        sl.busy = false;
        s->cv_done.notify_all();
    }
    ++s->batches;
}

void complete_slot(evp_server* s, Slot& sl) {
    const Clock::time_point now = Clock::now();
    int64_t row = 0;
    const int32_t st = *sl.status_h;
    for (Request* r : sl.reqs) {
        for (int64_t q = 0; q < r->nq; ++q) {
            std::memcpy(r->ids_out + q * r->k, sl.ids_h + (row + q) * sl.k, (size_t)r->k * 8);
            std::memcpy(r->scores_out + q * r->k, sl.sc_h + (row + q) * sl.k, (size_t)r->k * 4);
        }
        row += r->nq;
        r->status = st;
        r->done = true;
        r->latency_us = std::chrono::duration<double, std::micro>(now - r->arrival).count();
        s->lat_us.push_back(r->latency_us);
        s->queries_done += r->nq;
    }
    sl.reqs.clear();
    sl.busy = false;
}

void worker_loop(evp_server* s) {
    cudaSetDevice(s->cfg.device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        bool progressed = false;
        for (Slot& sl : s->slots) {
            if (sl.busy && cudaEventQuery(sl.done_ev) == cudaSuccess) {
                complete_slot(s, sl);
                progressed = true;
            }
        }
        if (progressed) s->cv_done.notify_all();
        for (Slot& sl : s->slots) {
            if (sl.busy || s->pending.empty() || s->paused) continue;
            const int32_t k = s->pending.front()->k;
            std::vector<Request*> batch;
            int64_t nq = 0;
            for (auto it = s->pending.begin(); it != s->pending.end();) {
                Request* r = *it;
                if (r->k == k && nq + r->nq <= s->cfg.max_batch_queries) {
                    batch.push_back(r);
                    nq += r->nq;
                    it = s->pending.erase(it);
                } else {
                    ++it;
                }
            }
            launch_batch(s, sl, batch, k);
            progressed = true;
        }
        bool any_busy = false;
        for (Slot& sl : s->slots) any_busy |= sl.busy;
        if (s->stop && !any_busy && s->pending.empty()) break;
        if (!progressed) {
            if (any_busy)
                s->cv_work.wait_for(lk, std::chrono::microseconds(20));
            else
                s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
        }
    }
}

}  // namespace

extern "C" {

int32_t evp_server_create(evp_db_t db, const evp_server_config* cfg, evp_server_t* out) {
    if (!out) return EVP_ERR_INVALID;
    *out = nullptr;
    if (!db || !cfg || cfg->max_batch_queries < 1 || cfg->max_k < 1 || cfg->max_k > EVP_MAX_K ||
        cfg->shortlist_factor < 1 || cfg->max_slots < 1)
        return EVP_ERR_INVALID;
    evp_server* s = new (std::nothrow) evp_server();
    if (!s) return EVP_ERR_NO_MEMORY;
    s->db = db;
    s->cfg = *cfg;
    s->d = evp_db_dim(db);
    if (cudaSetDevice(cfg->device) != cudaSuccess) {
        delete s;
        return EVP_ERR_CUDA;
    }
    const int64_t cap = cfg->max_batch_queries;
    // the largest workspace any class of k needs for a full slot
    size_t ws = 0;
    for (int32_t k = 1; k <= cfg->max_k; ++k)
        ws = std::max(ws, evp_db_search_host_workspace(db, cap, shortlist_for(s, k), k));
    const size_t slot_bytes = ws + 256;
    int64_t nslots = cfg->mem_budget_bytes > 0 ? (int64_t)(cfg->mem_budget_bytes / slot_bytes) : 1;
    nslots = std::min<int64_t>(nslots, cfg->max_slots);
    if (nslots < 1) {
        delete s;
        return EVP_ERR_NO_MEMORY;
    }
    s->slots.resize((size_t)nslots);
    for (Slot& sl : s->slots) {
        bool ok = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&sl.done_ev, cudaEventDisableTiming) == cudaSuccess &&
                  cudaMallocHost(&sl.q_h, (size_t)cap * s->d * 4) == cudaSuccess &&
                  cudaMallocHost(&sl.ids_h, (size_t)cap * cfg->max_k * 8) == cudaSuccess &&
                  cudaMallocHost(&sl.sc_h, (size_t)cap * cfg->max_k * 4) == cudaSuccess &&
                  cudaMallocHost(&sl.status_h, sizeof(int32_t)) == cudaSuccess &&
                  cudaMalloc(&sl.status_d, sizeof(int32_t)) == cudaSuccess &&
                  cudaMalloc(&sl.ws, ws) == cudaSuccess;
        sl.ws_bytes = ws;
        if (!ok) {
            cudaGetLastError();
            for (Slot& x : s->slots) free_slot(x);
            delete s;
            return EVP_ERR_NO_MEMORY;
        }
    }
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return EVP_OK;
}

int32_t evp_server_slots(evp_server_t s) { return s ? (int32_t)s->slots.size() : 0; }

int32_t evp_server_submit(evp_server_t s, const float* Q_host, int64_t nq, int32_t k,
                          int64_t* ids_host, float* scores_host, int64_t* request_id) {
    if (!s || !Q_host || !ids_host || !scores_host || !request_id || nq < 1 || k < 1 ||
        k > s->cfg.max_k)
        return EVP_ERR_INVALID;
    if (nq > s->cfg.max_batch_queries) return EVP_ERR_NO_MEMORY;
    Request* r = new (std::nothrow) Request();
    if (!r) return EVP_ERR_NO_MEMORY;
    r->Q = Q_host;
    r->nq = nq;
    r->k = k;
    r->ids_out = ids_host;
    r->scores_out = scores_host;
    r->arrival = Clock::now();
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (s->stop) {
            delete r;
            return EVP_ERR_INVALID;
        }
        r->id = s->next_id++;
        s->reqs[r->id] = r;
        s->pending.push_back(r);
        *request_id = r->id;
    }
    s->cv_work.notify_one();
    return EVP_OK;
}

int32_t evp_server_wait(evp_server_t s, int64_t request_id, int64_t timeout_us,
                        int32_t* request_status, double* latency_us) {
    if (!s) return EVP_ERR_INVALID;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(request_id);
    if (it == s->reqs.end()) return EVP_ERR_INVALID;
    Request* r = it->second;
    const auto deadline = Clock::now() + std::chrono::microseconds(std::max<int64_t>(0, timeout_us));
    while (!r->done) {
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !r->done)
            return EVP_ERR_TIMEOUT;
    }
    if (request_status) *request_status = r->status;
    if (latency_us) *latency_us = r->latency_us;
    s->reqs.erase(it);
    delete r;
    return EVP_OK;
}

int32_t evp_server_stats(evp_server_t s, evp_server_stats_t* out) {
    if (!s || !out) return EVP_ERR_INVALID;
    std::lock_guard<std::mutex> g(s->mu);
    std::vector<double> v = s->lat_us;
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) -> double {
        if (v.empty()) return 0.0;
        const size_t i = (size_t)std::min<double>((double)v.size() - 1, p * (double)(v.size() - 1) + 0.5);
        return v[i];
    };
    out->requests = (int64_t)v.size();
    out->queries = s->queries_done;
    out->batches = s->batches;
    out->p50_us = pct(0.50);
    out->p99_us = pct(0.99);
    out->max_us = v.empty() ? 0.0 : v.back();
    out->pending = (int64_t)s->pending.size();
    return EVP_OK;
}

int32_t evp_server_pause(evp_server_t s, int32_t paused) {
    if (!s) return EVP_ERR_INVALID;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->paused = paused != 0;
    }
    s->cv_work.notify_all();
    return EVP_OK;
}

int32_t evp_server_reset_stats(evp_server_t s) {
    if (!s) return EVP_ERR_INVALID;
    std::lock_guard<std::mutex> g(s->mu);
    s->lat_us.clear();
    s->queries_done = 0;
    s->batches = 0;
    return EVP_OK;
}

int32_t evp_server_destroy(evp_server_t s) {
    if (!s) return EVP_ERR_INVALID;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
        s->paused = false;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (Slot& sl : s->slots) free_slot(sl);
    for (auto& kv : s->reqs) delete kv.second;
    delete s;
    return EVP_OK;
}

}  // extern "C"
