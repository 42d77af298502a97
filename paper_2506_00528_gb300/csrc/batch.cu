// Batched form: many query batches, of uneven sizes and against several
// resident databases, planned once and run as one CUDA graph.
//
// evp_batch_plan_create validates a list of batch descriptors, picks the
// scan path of every batch from the autotuner's table (timing the paths on
// first sight of a (database, query-count bucket, k) class, see
// evp_autotune), sizes one workspace per batch and allocates them together.
// evp_batch_run enqueues every batch on the caller's stream, spreading
// independent batches over a few forked streams so that small batches share
// the GPU; with EVP_BATCH_GRAPH the first run is captured into a CUDA graph
// and later runs replay it with a single launch.  Each batch's results are
// exactly those of the matching evp_db_search / evp_db_knn call.
#include "evp_internal.cuh"

#include <algorithm>
#include <chrono>
#include <mutex>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

namespace {

constexpr int BRANCHES = 4;  // forked streams inside one run

struct TuneKey {
    const void* db;
    int64_t nq_bucket;
    int32_t k;
    bool operator==(const TuneKey& o) const {
        return db == o.db && nq_bucket == o.nq_bucket && k == o.k;
    }
};
struct TuneHash {
    size_t operator()(const TuneKey& t) const {
        return std::hash<const void*>()(t.db) ^ (std::hash<int64_t>()(t.nq_bucket) * 31) ^
               (std::hash<int32_t>()(t.k) * 131);
    }
};

std::mutex g_tune_mu;
std::unordered_map<TuneKey, int32_t, TuneHash> g_tune;

int64_t bucket(int64_t nq) {
    int64_t b = 1;
    while (b < nq) b <<= 1;
    return b;
}

}  // namespace

struct evp_batch_plan {
    std::vector<evp_batch_desc> batches;
    std::vector<int32_t> paths;
    std::vector<size_t> ws_off, ws_size;
    void* ws = nullptr;
    size_t ws_total = 0;
    int32_t flags = 0;
    cudaStream_t branch[BRANCHES] = {};
    cudaEvent_t fork_ev = nullptr, join_ev[BRANCHES] = {};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" {

int32_t evp_autotune(evp_db_t db, int64_t nq, int32_t k, int32_t* path_out, float* popc_ms,
                     float* mma_ms, void* stream) {
    if (!db || nq < 1 || k < 1 || !path_out) return EVP_ERR_INVALID;
    const TuneKey key{db, bucket(nq), k};
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end() && !popc_ms && !mma_ms) {
            *path_out = it->second;
            return EVP_OK;
        }
    }
    const int64_t ns = evp_db_rows(db);
    const int32_t d = evp_db_dim(db);
    if ((int64_t)k > ns) return EVP_ERR_INVALID;
    const int64_t tq = std::min<int64_t>(bucket(nq), ns);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // trial queries: the database's own first rows (the timing does not
    // depend on the query values)
    const uint64_t* Q = evp_db_codes(db);
    const bool packed = k <= evp::MMA_K_MAX && evp::mma_packed_supported(ns, d, k);
    size_t wsz[4] = {0, 0, 0, 0};
    wsz[EVP_PATH_POPC] = evp_db_knn_workspace(db, tq, k, EVP_PATH_POPC);
    if (k <= evp::MMA_K_MAX) wsz[EVP_PATH_MMA] = evp_db_knn_workspace(db, tq, k, EVP_PATH_MMA);
    if (packed) wsz[EVP_PATH_MMA_PACKED] = evp_db_knn_workspace(db, tq, k, EVP_PATH_MMA_PACKED);
    const size_t ws_bytes = std::max({wsz[1], wsz[2], wsz[3]});
    void* ws = nullptr;
    int64_t* ids = nullptr;
    int32_t* dist = nullptr;
    if (cudaMalloc(&ws, ws_bytes) != cudaSuccess || cudaMalloc(&ids, (size_t)tq * k * 8) != cudaSuccess ||
        cudaMalloc(&dist, (size_t)tq * k * 4) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(ws);
        cudaFree(ids);
        cudaFree(dist);
        return EVP_ERR_NO_MEMORY;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float t[4] = {0.f, 1e30f, 1e30f, 1e30f};
    int32_t rc = EVP_OK;
    for (int path = EVP_PATH_POPC; path <= EVP_PATH_MMA_PACKED && rc == EVP_OK; ++path) {
        if (path != EVP_PATH_POPC && k > evp::MMA_K_MAX) break;
        if (path == EVP_PATH_MMA_PACKED && !packed) break;
        // one warm-up, then the timed run
        for (int rep = 0; rep < 2 && rc == EVP_OK; ++rep) {
            cudaEventRecord(e0, s);
            rc = evp_db_knn(db, Q, tq, k, ids, dist, ws, wsz[path], nullptr, stream, path);
            cudaEventRecord(e1, s);
        }
        if (rc == EVP_OK && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&t[path], e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(ws);
    cudaFree(ids);
    cudaFree(dist);
    if (rc != EVP_OK) return rc;
    int32_t best = EVP_PATH_POPC;
    for (int path = EVP_PATH_MMA; path <= EVP_PATH_MMA_PACKED; ++path)
        if (t[path] < t[best]) best = path;
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_tune[key] = best;
    }
    *path_out = best;
    if (popc_ms) *popc_ms = t[EVP_PATH_POPC];
    if (mma_ms) *mma_ms = std::min(t[EVP_PATH_MMA], t[EVP_PATH_MMA_PACKED]);
    return EVP_OK;
}

int32_t evp_autotune_clear(void) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune.clear();
    return EVP_OK;
}

int32_t evp_batch_plan_create(const evp_batch_desc* batches, int32_t nb, int32_t flags,
                              void* stream, evp_batch_plan_t* out) {
    if (!out) return EVP_ERR_INVALID;
    *out = nullptr;
    if (!batches || nb < 1 || (flags & ~(EVP_BATCH_GRAPH | EVP_BATCH_NO_TUNE)) != 0)
        return EVP_ERR_INVALID;
    evp_batch_plan* p = new (std::nothrow) evp_batch_plan();
    if (!p) return EVP_ERR_NO_MEMORY;
    p->flags = flags;
    p->batches.assign(batches, batches + nb);
    size_t off = 0;
    for (const evp_batch_desc& b : p->batches) {
        const bool search = b.Q != nullptr;
        if (!b.db || b.nq < 0 || b.k < 1 || !b.ids || (!search && (!b.Qc || !b.dist)) ||
            (search && (!b.scores || b.n_shortlist < b.k))) {
            delete p;
            return EVP_ERR_INVALID;
        }
        int32_t path = EVP_PATH_AUTO;
        const int32_t scan_k = search ? b.n_shortlist : b.k;
        if (!(flags & EVP_BATCH_NO_TUNE) && b.nq > 0) {
            const int32_t rc = evp_autotune(b.db, b.nq, scan_k, &path, nullptr, nullptr, stream);
            if (rc != EVP_OK) {
                delete p;
                return rc;
            }
        }
        p->paths.push_back(path);
        size_t need = 0;
        if (b.nq > 0)
            need = search ? evp_db_search_path_workspace(b.db, b.nq, b.n_shortlist, b.k, path)
                          : evp_db_knn_workspace(b.db, b.nq, b.k, path);
        need = (need + 255) / 256 * 256;
        p->ws_off.push_back(off);
        p->ws_size.push_back(need);
        off += need;
    }
    p->ws_total = std::max<size_t>(off, 256);
    bool ok = cudaMalloc(&p->ws, p->ws_total) == cudaSuccess &&
              cudaEventCreateWithFlags(&p->fork_ev, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; i < BRANCHES && ok; ++i)
        ok = cudaStreamCreateWithFlags(&p->branch[i], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&p->join_ev[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        evp_batch_plan_destroy(p);
        return EVP_ERR_NO_MEMORY;
    }
    *out = p;
    return EVP_OK;
}

int32_t evp_batch_plan_path(evp_batch_plan_t p, int32_t i) {
    if (!p || i < 0 || i >= (int32_t)p->batches.size()) return -1;
    return p->paths[i];
}

size_t evp_batch_plan_workspace(evp_batch_plan_t p) { return p ? p->ws_total : 0; }

}  // extern "C"

namespace {

// Enqueue every batch: batches are dealt round-robin to the forked
// branches, which join back into `s` at the end.
int32_t enqueue_all(evp_batch_plan* p, int32_t* dev_status, cudaStream_t s) {
    if (cudaEventRecord(p->fork_ev, s) != cudaSuccess) return EVP_ERR_CUDA;
    for (int i = 0; i < BRANCHES; ++i)
        if (cudaStreamWaitEvent(p->branch[i], p->fork_ev, 0) != cudaSuccess) return EVP_ERR_CUDA;
    for (size_t i = 0; i < p->batches.size(); ++i) {
        const evp_batch_desc& b = p->batches[i];
        if (b.nq == 0) continue;
        cudaStream_t bs = p->branch[i % BRANCHES];
        void* ws = static_cast<uint8_t*>(p->ws) + p->ws_off[i];
        int32_t rc;
        if (b.Q)
            rc = evp_db_search_path(b.db, b.Q, b.nq, b.n_shortlist, b.k, b.ids, b.scores, ws,
                                    p->ws_size[i], dev_status, bs, p->paths[i]);
        else
            rc = evp_db_knn(b.db, b.Qc, b.nq, b.k, b.ids, b.dist, ws, p->ws_size[i], dev_status,
                            bs, p->paths[i]);
        if (rc != EVP_OK) return rc;
    }
    for (int i = 0; i < BRANCHES; ++i) {
        if (cudaEventRecord(p->join_ev[i], p->branch[i]) != cudaSuccess) return EVP_ERR_CUDA;
        if (cudaStreamWaitEvent(s, p->join_ev[i], 0) != cudaSuccess) return EVP_ERR_CUDA;
    }
    return EVP_OK;
}

}  // namespace

extern "C" {

int32_t evp_batch_run(evp_batch_plan_t p, int32_t* dev_status, void* stream) {
    if (!p) return EVP_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!(p->flags & EVP_BATCH_GRAPH)) return enqueue_all(p, dev_status, s);
    if (!p->exec) {
        // legacy default stream cannot be captured
        if (s == nullptr) return EVP_ERR_INVALID;
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return EVP_ERR_CUDA;
        const int32_t rc = enqueue_all(p, dev_status, s);
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(s, &g);
        if (rc != EVP_OK || ec != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return rc != EVP_OK ? rc : EVP_ERR_CUDA;
        }
        if (cudaGraphInstantiate(&p->exec, g, 0) != cudaSuccess) {
            cudaGraphDestroy(g);
            cudaGetLastError();
            return EVP_ERR_CUDA;
        }
        p->graph = g;
    }
    return cudaGraphLaunch(p->exec, s) == cudaSuccess ? EVP_OK : EVP_ERR_CUDA;
}

int32_t evp_batch_plan_destroy(evp_batch_plan_t p) {
    if (!p) return EVP_ERR_INVALID;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    for (int i = 0; i < BRANCHES; ++i) {
        if (p->branch[i]) cudaStreamDestroy(p->branch[i]);
        if (p->join_ev[i]) cudaEventDestroy(p->join_ev[i]);
    }
    if (p->fork_ev) cudaEventDestroy(p->fork_ev);
    if (p->ws) cudaFree(p->ws);
    delete p;
    return EVP_OK;
}

}  // extern "C"
