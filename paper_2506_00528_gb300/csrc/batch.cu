// Batched form: many query batches, of uneven sizes and against several
// resident databases, planned once and replayed.
//
// evp_batch_plan_create validates a list of batch descriptors and picks each
// batch's scan path from the autotuner (timing the paths on first sight of a
// (GPU, d, x, query-count bucket, k, row-count bucket) class, see
// evp_autotune).  Every batch whose path is the fp4 tensor-core scan and
// whose database holds its tensor copy joins the fused scan: one persistent
// launch over the work items (query unit, database slice) of all of them,
// preceded by one launch that prepares every batch's queries and followed by
// one multi-batch final merge (evp_batch_plan_fused counts them).  The tile
// shape of the fused scan -- database tiles per work item, balanced across
// batches of different d -- is chosen by timing a few shapes on the plan's
// own batches and kept with the tuner's decisions.  The other batches run
// their own calls on a few forked streams beside it.  With EVP_BATCH_GRAPH
// the first run is captured into a CUDA graph and later runs replay it.
// Each batch's results are exactly those of the matching evp_db_search /
// evp_db_knn call.  The tuner's table can be written to and read from a
// text file (evp_autotune_save / evp_autotune_load), so a deployment tunes
// once per GPU model.
#include "evp_internal.cuh"

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

namespace {

constexpr int BRANCHES = 4;               // forked streams inside one run
// Tile shapes tried for the fused scan, in k-chunk tiles per work item (an
// item of a batch with kc 128-byte K chunks per row covers shape / kc
// database tiles of MMA_TILE_ROWS rows); 0 = each batch sliced in whole waves of the
// persistent grid, as its own call would be.  Items must stay large: each
// ends with a sort of its heaps and a k-key list per query, and every
// list is merged at the end.
constexpr int FUSED_SHAPES[] = {0, 1536, 3072, 6144};
constexpr int FUSED_DEFAULT = 0;

int64_t bucket(int64_t n) {
    int64_t b = 1;
    while (b < n) b <<= 1;
    return b;
}

std::string gpu_name() {
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return "unknown";
    }
    std::string s(prop.name);
    for (char& c : s)
        if (c == ' ' || c == '\t' || c == '|') c = '_';
    return s;
}

// Tuner table: key "gpu|kind|a|b|c|d|e" -> value.  kind "path": (d, x,
// query-count bucket, k, row-count bucket) -> scan path; kind "fused":
// (batches, total-query bucket, 0, 0, 0) -> k-chunk tiles per work item.
std::mutex g_tune_mu;
std::unordered_map<std::string, int32_t> g_tune;

std::string tune_key(const char* kind, int64_t a, int64_t b, int64_t c, int64_t d, int64_t e) {
    char buf[160];
    std::snprintf(buf, sizeof(buf), "%s|%s|%lld|%lld|%lld|%lld|%lld", gpu_name().c_str(), kind,
                  (long long)a, (long long)b, (long long)c, (long long)d, (long long)e);
    return buf;
}

bool tune_get(const std::string& key, int32_t* v) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tune.find(key);
    if (it == g_tune.end()) return false;
    *v = it->second;
    return true;
}

void tune_put(const std::string& key, int32_t v) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune[key] = v;
}

}  // namespace

extern "C" {

int32_t evp_autotune(evp_db_t db, int64_t nq, int32_t k, int32_t* path_out, float* popc_ms,
                     float* mma_ms, void* stream) {
    if (!db || nq < 1 || k < 1 || !path_out) return EVP_ERR_INVALID;
    const int64_t ns = evp_db_rows(db);
    const int32_t d = evp_db_dim(db);
    if ((int64_t)k > ns) return EVP_ERR_INVALID;
    const std::string key = tune_key("path", d, evp::db_x(db), bucket(nq), k, bucket(ns));
    if (!popc_ms && !mma_ms && tune_get(key, path_out)) return EVP_OK;
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
    tune_put(key, best);
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

int32_t evp_autotune_save(const char* path) {
    if (!path) return EVP_ERR_INVALID;
    FILE* f = std::fopen(path, "w");
    if (!f) return EVP_ERR_INVALID;
    std::lock_guard<std::mutex> g(g_tune_mu);
    std::fprintf(f, "# evp autotune table: key value\n");
    for (const auto& kv : g_tune) std::fprintf(f, "%s %d\n", kv.first.c_str(), kv.second);
    const bool ok = std::fclose(f) == 0;
    return ok ? EVP_OK : EVP_ERR_INVALID;
}

int32_t evp_autotune_load(const char* path) {
    if (!path) return EVP_ERR_INVALID;
    FILE* f = std::fopen(path, "r");
    if (!f) return EVP_ERR_INVALID;
    char line[512];
    int32_t rc = EVP_OK;
    std::vector<std::pair<std::string, int32_t>> got;
    while (std::fgets(line, sizeof(line), f)) {
        if (line[0] == '#' || line[0] == '\n') continue;
        char key[400];
        int v = 0;
        if (std::sscanf(line, "%399s %d", key, &v) != 2 || std::strchr(key, '|') == nullptr) {
            rc = EVP_ERR_INVALID;
            break;
        }
        got.emplace_back(key, v);
    }
    std::fclose(f);
    if (rc != EVP_OK) return rc;
    std::lock_guard<std::mutex> g(g_tune_mu);
    for (auto& kv : got) g_tune[kv.first] = kv.second;
    return EVP_OK;
}

}  // extern "C"

struct evp_batch_plan {
    std::vector<evp_batch_desc> batches;
    std::vector<int32_t> paths;          // scan path of each batch
    std::vector<char> fused;             // 1: scanned by the fused launch
    std::vector<int32_t> tiles;          // fused: database tiles per work item
    std::vector<size_t> ws_off, ws_size;
    void* ws = nullptr;
    size_t ws_total = 0;
    int32_t flags = 0;
    int32_t shape = 0;                   // fused: k-chunk tiles per work item
    evp::MmaMultiPlan* multi = nullptr;
    cudaStream_t branch[BRANCHES] = {};
    cudaEvent_t fork_ev = nullptr, join_ev[BRANCHES] = {};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Layout of a fused batch's workspace region: for a search, the query codes
// and the shortlist, then the scan's workspace.
struct FusedLayout {
    size_t codes, sl_ids, sl_dist, scan, total;
};

int32_t scan_k_of(const evp_batch_desc& b) { return b.Q ? b.n_shortlist : b.k; }

int kchunks_of(const evp_batch_desc& b) { return evp::mma_kp(evp_db_dim(b.db)) / 128; }

int tiles_for(const evp_batch_desc& b, int shape) {
    return shape == 0 ? 0 : std::max(1, shape / kchunks_of(b));
}

FusedLayout fused_layout(const evp_batch_desc& b, int tiles) {
    FusedLayout L{};
    const int d = evp_db_dim(b.db), W = (d + 63) / 64;
    if (b.Q) {
        L.codes = align256((size_t)b.nq * 2 * W * 8);
        L.sl_ids = align256((size_t)b.nq * b.n_shortlist * 8);
        L.sl_dist = align256((size_t)b.nq * b.n_shortlist * 4);
    }
    L.scan = align256(evp::mma_multi_ws(b.nq, evp_db_rows(b.db), d, scan_k_of(b), tiles));
    L.total = L.codes + L.sl_ids + L.sl_dist + L.scan;
    return L;
}

// (Re)build the fused scan for the given shape.
int32_t build_multi(evp_batch_plan* p, int shape) {
    if (p->multi) {
        evp::mma_multi_destroy(p->multi);
        p->multi = nullptr;
    }
    std::vector<evp::MmaBatchSpec> specs;
    for (size_t i = 0; i < p->batches.size(); ++i) {
        if (!p->fused[i]) continue;
        const evp_batch_desc& b = p->batches[i];
        const int tiles = tiles_for(b, shape);
        const FusedLayout L = fused_layout(b, tiles);
        uint8_t* w = static_cast<uint8_t*>(p->ws) + p->ws_off[i];
        evp::MmaBatchSpec s{};
        s.Q = b.Q ? reinterpret_cast<const uint64_t*>(w) : b.Qc;
        s.nq = b.nq;
        s.S8 = evp::db_tensor_copy(b.db);
        s.ns = evp_db_rows(b.db);
        s.d = evp_db_dim(b.db);
        s.x = evp::db_x(b.db);
        s.k = scan_k_of(b);
        s.ids = b.Q ? reinterpret_cast<int64_t*>(w + L.codes) : b.ids;
        s.dist = b.Q ? reinterpret_cast<int32_t*>(w + L.codes + L.sl_ids) : b.dist;
        s.ws = w + L.codes + L.sl_ids + L.sl_dist;
        s.tiles_per_item = tiles;
        // reported shape: database tiles per item (whole-wave slices included)
        p->tiles[i] = (int32_t)(evp::plan_mma_scan(b.nq, s.ns, s.d, s.k, false, tiles).rows_per_slice /
                                evp::MMA_TILE_ROWS);
        specs.push_back(s);
    }
    p->shape = shape;
    if (specs.empty()) return EVP_OK;
    return evp::mma_multi_create(specs.data(), (int)specs.size(), &p->multi);
}

int32_t enqueue_all(evp_batch_plan* p, int32_t* dev_status, cudaStream_t s);

}  // namespace

extern "C" {

int32_t evp_batch_plan_create(const evp_batch_desc* batches, int32_t nb, int32_t flags,
                              void* stream, evp_batch_plan_t* out) {
    if (!out) return EVP_ERR_INVALID;
    *out = nullptr;
    if (!batches || nb < 1 ||
        (flags & ~(EVP_BATCH_GRAPH | EVP_BATCH_NO_TUNE | EVP_BATCH_SEPARATE)) != 0)
        return EVP_ERR_INVALID;
    evp_batch_plan* p = new (std::nothrow) evp_batch_plan();
    if (!p) return EVP_ERR_NO_MEMORY;
    p->flags = flags;
    p->batches.assign(batches, batches + nb);
    const bool tune = !(flags & EVP_BATCH_NO_TUNE);
    int nfused = 0;
    int64_t fused_q = 0;
    for (const evp_batch_desc& b : p->batches) {
        const bool search = b.Q != nullptr;
        if (!b.db || b.nq < 0 || b.k < 1 || !b.ids || (!search && (!b.Qc || !b.dist)) ||
            (search && (!b.scores || b.n_shortlist < b.k))) {
            delete p;
            return EVP_ERR_INVALID;
        }
        int32_t path = EVP_PATH_AUTO;
        const int32_t scan_k = scan_k_of(b);
        if (tune && b.nq > 0) {
            const int32_t rc = evp_autotune(b.db, b.nq, scan_k, &path, nullptr, nullptr, stream);
            if (rc != EVP_OK) {
                delete p;
                return rc;
            }
        }
        const bool copy = evp::db_tensor_copy(b.db) != nullptr;
        const int resolved = path == EVP_PATH_AUTO && b.nq > 0
                                 ? evp::auto_path(b.nq, evp_db_rows(b.db), evp_db_dim(b.db), scan_k, copy)
                                 : path;
        const bool fuse = !(flags & EVP_BATCH_SEPARATE) && b.nq > 0 && copy &&
                          resolved == EVP_PATH_MMA && scan_k <= evp::MMA_K_MAX &&
                          (!search || evp::db_float_rows(b.db) != nullptr) &&
                          (int64_t)scan_k <= evp_db_rows(b.db) && nfused < 64;
        p->paths.push_back(path);
        p->fused.push_back(fuse ? 1 : 0);
        p->tiles.push_back(0);
        size_t need = 0;
        if (fuse) {
            // the largest workspace over the shapes the tuner may pick
            for (int shape : FUSED_SHAPES) need = std::max(need, fused_layout(b, tiles_for(b, shape)).total);
            ++nfused;
            fused_q += b.nq;
        } else if (b.nq > 0) {
            need = search ? evp_db_search_path_workspace(b.db, b.nq, b.n_shortlist, b.k, path)
                          : evp_db_knn_workspace(b.db, b.nq, b.k, path);
        }
        need = align256(need);
        p->ws_off.push_back(p->ws_total);
        p->ws_size.push_back(need);
        p->ws_total += need;
    }
    p->ws_total = std::max<size_t>(p->ws_total, 256);
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
    // tile shape of the fused scan: cached, or timed on these batches
    int32_t rc = EVP_OK;
    if (nfused > 0) {
        const std::string key = tune_key("fused", nfused, bucket(fused_q), 0, 0, 0);
        int32_t shape = FUSED_DEFAULT;
        if (tune && !tune_get(key, &shape)) {
            cudaStream_t s = static_cast<cudaStream_t>(stream);
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            float best = 1e30f;
            for (int cand : FUSED_SHAPES) {
                if ((rc = build_multi(p, cand)) != EVP_OK) break;
                float t = 1e30f;
                for (int rep = 0; rep < 2 && rc == EVP_OK; ++rep) {
                    cudaEventRecord(e0, s);
                    rc = enqueue_all(p, nullptr, s);
                    cudaEventRecord(e1, s);
                }
                if (rc == EVP_OK && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
                if (t < best) {
                    best = t;
                    shape = cand;
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (rc == EVP_OK) tune_put(key, shape);
        }
        if (rc == EVP_OK) rc = build_multi(p, shape);
    }
    if (rc != EVP_OK) {
        evp_batch_plan_destroy(p);
        return rc;
    }
    *out = p;
    return EVP_OK;
}

int32_t evp_batch_plan_path(evp_batch_plan_t p, int32_t i) {
    if (!p || i < 0 || i >= (int32_t)p->batches.size()) return -1;
    return p->paths[i];
}

int32_t evp_batch_plan_fused(evp_batch_plan_t p) {
    if (!p) return -1;
    int n = 0;
    for (char f : p->fused) n += f ? 1 : 0;
    return n;
}

int32_t evp_batch_plan_tile(evp_batch_plan_t p, int32_t i) {
    if (!p || i < 0 || i >= (int32_t)p->batches.size()) return -1;
    return p->fused[i] ? p->tiles[i] : 0;
}

size_t evp_batch_plan_workspace(evp_batch_plan_t p) { return p ? p->ws_total : 0; }

}  // extern "C"

namespace {

// Enqueue every batch: the fused scan (with the encodes and reranks of its
// search batches) on `s`, the other batches dealt round-robin to the forked
// branches, which join back into `s` at the end.
int32_t enqueue_all(evp_batch_plan* p, int32_t* dev_status, cudaStream_t s) {
    if (cudaEventRecord(p->fork_ev, s) != cudaSuccess) return EVP_ERR_CUDA;
    for (int i = 0; i < BRANCHES; ++i)
        if (cudaStreamWaitEvent(p->branch[i], p->fork_ev, 0) != cudaSuccess) return EVP_ERR_CUDA;
    int branch = 0;
    for (size_t i = 0; i < p->batches.size(); ++i) {
        const evp_batch_desc& b = p->batches[i];
        if (b.nq == 0 || p->fused[i]) continue;
        cudaStream_t bs = p->branch[branch++ % BRANCHES];
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
    if (p->multi) {
        for (size_t i = 0; i < p->batches.size(); ++i) {
            const evp_batch_desc& b = p->batches[i];
            if (!p->fused[i] || !b.Q) continue;
            uint64_t* codes = reinterpret_cast<uint64_t*>(static_cast<uint8_t*>(p->ws) + p->ws_off[i]);
            if (evp::launch_encode(b.Q, b.nq, evp_db_dim(b.db), evp::db_x(b.db), codes, dev_status,
                                   s) != cudaSuccess)
                return EVP_ERR_CUDA;
        }
        const int32_t rc = evp::mma_multi_run(p->multi, dev_status, s);
        if (rc != EVP_OK) return rc;
        for (size_t i = 0; i < p->batches.size(); ++i) {
            const evp_batch_desc& b = p->batches[i];
            if (!p->fused[i] || !b.Q) continue;
            const FusedLayout L = fused_layout(b, 0);   // the shortlist's offset does not depend on the shape
            const int64_t* sl = reinterpret_cast<const int64_t*>(static_cast<uint8_t*>(p->ws) +
                                                                 p->ws_off[i] + L.codes);
            if (evp::launch_rerank(b.Q, b.nq, evp::db_float_rows(b.db), evp_db_rows(b.db),
                                   evp_db_dim(b.db), sl, b.n_shortlist, b.k, b.ids, b.scores,
                                   dev_status, s) != cudaSuccess)
                return EVP_ERR_CUDA;
        }
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
    if (p->multi) evp::mma_multi_destroy(p->multi);
    if (p->ws) cudaFree(p->ws);
    delete p;
    return EVP_OK;
}

}  // extern "C"
