// C ABI entry points of libevp (declared in include/evp.h): argument
// checks on the host, then kernel launches on the caller's stream.
#include "evp_internal.cuh"

#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

namespace evp {

EncodeTiledFn encode_tiled_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

int num_sms() {
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    if (cached[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
            v = 148;
        cached[dev] = v;
    }
    return cached[dev];
}

// ---- testing support: a stalled copy producer ------------------------------
namespace {
std::atomic<int> g_stall_mma{-1}, g_stall_packed{-1};
}  // namespace

int take_stall_mma() { return g_stall_mma.exchange(-1); }
int take_stall_packed() { return g_stall_packed.exchange(-1); }

// ---- kernel timing ------------------------------------------------------
namespace {

struct TimingRecord {
    const char* name;
    cudaEvent_t start, stop;
};

struct TimingState {
    std::mutex mu;
    bool enabled = false;
    std::vector<TimingRecord> records;
    std::vector<cudaEvent_t> spare;
};

TimingState& timing() {
    static TimingState* t = new TimingState();  // never destroyed: safe at exit
    return *t;
}

cudaEvent_t take_event(TimingState& t) {
    if (!t.spare.empty()) {
        cudaEvent_t e = t.spare.back();
        t.spare.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

}  // namespace

TimedLaunch::TimedLaunch(const char* name, cudaStream_t stream)
    : name_(name), stream_(stream), slot_(-1) {
    TimingState& t = timing();
    std::lock_guard<std::mutex> g(t.mu);
    if (!t.enabled) return;
    TimingRecord r{name, take_event(t), take_event(t)};
    if (!r.start || !r.stop) return;
    if (cudaEventRecord(r.start, stream) != cudaSuccess) return;
    slot_ = (int)t.records.size();
    t.records.push_back(r);
}

TimedLaunch::~TimedLaunch() {
    if (slot_ < 0) return;
    TimingState& t = timing();
    std::lock_guard<std::mutex> g(t.mu);
    if (slot_ < (int)t.records.size()) cudaEventRecord(t.records[slot_].stop, stream_);
}

}  // namespace evp

using namespace evp;

extern "C" {

const char* evp_status_string(int32_t status) {
    switch (status) {
        case EVP_OK: return "EVP_OK";
        case EVP_ERR_INVALID: return "EVP_ERR_INVALID: invalid argument";
        case EVP_ERR_NONFINITE: return "EVP_ERR_NONFINITE: NaN or infinity in a float input";
        case EVP_ERR_NO_MEMORY: return "EVP_ERR_NO_MEMORY: workspace too small or allocation refused";
        case EVP_ERR_TIMEOUT: return "EVP_ERR_TIMEOUT: a bounded device wait gave up";
        case EVP_ERR_CUDA: return "EVP_ERR_CUDA: a CUDA runtime call failed";
        case EVP_ERR_UNSUPPORTED: return "EVP_ERR_UNSUPPORTED: outside this build's limits";
        case EVP_ERR_RANGE: return "EVP_ERR_RANGE: index outside its array";
        default: return "EVP_ERR_UNKNOWN";
    }
}

int32_t evp_version(void) { return 100; }

int32_t evp_words(int32_t d) { return d < 1 ? 0 : (d + 63) / 64; }

int32_t evp_default_x(int32_t d) { return d < 1 ? 0 : (2 * d + 1) / 3; }

int32_t evp_encode(const float* U, int64_t n, int32_t d, int32_t x, uint64_t* T,
                   int32_t* dev_status, void* stream) {
    if (n < 0 || d < 1 || x < 1 || x > d) return EVP_ERR_INVALID;
    if (d > EVP_MAX_D_ENCODE) return EVP_ERR_UNSUPPORTED;
    if (n == 0) return EVP_OK;
    if (!U || !T) return EVP_ERR_INVALID;
    cudaError_t e = launch_encode(U, n, d, x, T, dev_status, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? EVP_OK : EVP_ERR_CUDA;
}

}  // extern "C"

int evp::auto_path(int64_t nq, int64_t ns, int d, int k, bool resident_copy) {
    if (k <= MMA_K_MAX && mma_packed_supported(ns, d, k)) {
        if (nq <= EVP_AUTO_POPC_MAX_NQ) return EVP_PATH_POPC;
        return nq <= auto_packed_max_nq(resident_copy) ? EVP_PATH_MMA_PACKED : EVP_PATH_MMA;
    }
    return (nq >= auto_mma_min_nq(resident_copy) && k <= MMA_K_MAX) ? EVP_PATH_MMA
                                                                     : EVP_PATH_POPC;
}

namespace {

int resolve_path(int64_t nq, int64_t ns, int32_t d, int32_t k, int32_t path) {
    return path == EVP_PATH_AUTO ? auto_path(nq, ns, d, k, false) : path;
}

}  // namespace

size_t evp::knn_ws_bound(int64_t nq, int64_t ns, int d, int k, int path, bool convert_db) {
    if (nq <= 0) return 0;
    size_t best = 0;
    // popcount path (AUTO takes it for one query): its workspace does not depend on nq
    if (path == EVP_PATH_POPC || path == EVP_PATH_AUTO)
        best = plan_popc_scan(std::min<int64_t>(nq, 16), ns, d, k).ws_bytes;
    // packed tensor path: one pass's workspace, whatever nq
    const bool packed = k <= MMA_K_MAX && mma_packed_supported(ns, d, k);
    if ((path == EVP_PATH_MMA_PACKED && packed) ||
        (path == EVP_PATH_AUTO && packed && nq > EVP_AUTO_POPC_MAX_NQ))
        best = std::max(best, mma_packed_workspace(ns, d, k));
    // tensor path, taken by AUTO from nq0 queries up: the slice count depends
    // on the number of query tiles, so the lists can need more room at fewer
    // queries; the largest call in each tile count is the last one
    const int64_t nq0 = path == EVP_PATH_MMA ? 1
                        : packed             ? auto_packed_max_nq(!convert_db) + 1
                                             : auto_mma_min_nq(!convert_db);
    if ((path == EVP_PATH_MMA || path == EVP_PATH_AUTO) && k <= MMA_K_MAX && nq >= nq0) {
        const int64_t qa = mma_active_queries(k);
        for (int64_t t = (nq0 + qa - 1) / qa; t <= (nq + qa - 1) / qa; ++t)
            best = std::max(best,
                            plan_mma_scan(std::min(nq, t * qa), ns, d, k, convert_db, 0, true).ws_bytes);
    }
    return best;
}

namespace {

int32_t check_knn_args(int64_t nq, int64_t ns, int32_t d, int32_t x, int32_t k, int32_t path) {
    if (nq < 0 || ns < 1 || ns >= (int64_t(1) << 31) || d < 1 || x < 1 || x > d || k < 1 ||
        (int64_t)k > ns || path < EVP_PATH_AUTO || path > EVP_PATH_MMA_PACKED)
        return EVP_ERR_INVALID;
    if (d > EVP_MAX_D_SCAN || k > EVP_MAX_K) return EVP_ERR_UNSUPPORTED;
    const int rp = resolve_path(nq, ns, d, k, path);
    if (rp == EVP_PATH_MMA && k > MMA_K_MAX) return EVP_ERR_UNSUPPORTED;
    if (rp == EVP_PATH_MMA_PACKED && !mma_packed_supported(ns, d, k)) return EVP_ERR_UNSUPPORTED;
    return EVP_OK;
}

}  // namespace

extern "C" {

size_t ternary_knn_path_workspace(int64_t nq, int64_t ns, int32_t d, int32_t k, int32_t path) {
    if (nq <= 0 || ns <= 0 || d < 1 || k < 1) return 0;
    return knn_ws_bound(nq, ns, d, k, path, /*convert_db=*/true);
}

size_t ternary_knn_workspace(int64_t nq, int64_t ns, int32_t d, int32_t k) {
    return ternary_knn_path_workspace(nq, ns, d, k, EVP_PATH_AUTO);
}

int32_t ternary_knn_path(const uint64_t* Q, int64_t nq, const uint64_t* S, int64_t ns,
                         int32_t d, int32_t x, int32_t k, int64_t* ids, int32_t* dist, void* ws,
                         size_t ws_bytes, int32_t* dev_status, void* stream, int32_t path) {
    const int32_t rc = check_knn_args(nq, ns, d, x, k, path);
    if (rc != EVP_OK) return rc;
    if (nq == 0) return EVP_OK;
    if (!Q || !S || !ids || !dist || !ws) return EVP_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(S) & 15) != 0 || (reinterpret_cast<uintptr_t>(ws) & 255) != 0)
        return EVP_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int rp = resolve_path(nq, ns, d, k, path);
    if (rp == EVP_PATH_MMA)
        return run_mma_knn(Q, nq, nullptr, S, ns, d, x, k, ids, dist, ws, ws_bytes, dev_status, s);
    if (rp == EVP_PATH_MMA_PACKED)
        return run_mma_packed_knn(Q, nq, S, ns, d, x, k, ids, dist, ws, ws_bytes, dev_status, s);
    return run_popc_knn(Q, nq, S, ns, d, x, k, ids, dist, ws, ws_bytes, dev_status, s);
}

int32_t ternary_knn(const uint64_t* Q, int64_t nq, const uint64_t* S, int64_t ns, int32_t d,
                    int32_t x, int32_t k, int64_t* ids, int32_t* dist, void* ws, size_t ws_bytes,
                    int32_t* dev_status, void* stream) {
    return ternary_knn_path(Q, nq, S, ns, d, x, k, ids, dist, ws, ws_bytes, dev_status, stream,
                            EVP_PATH_AUTO);
}

int32_t evp_quantize_i8(const float* Q, int64_t nq, int32_t d, int8_t* Q8, int32_t* dev_status,
                        void* stream) {
    if (nq < 0 || d < 1) return EVP_ERR_INVALID;
    if (nq == 0) return EVP_OK;
    if (!Q || !Q8) return EVP_ERR_INVALID;
    const cudaError_t e = launch_quantize_i8(Q, nq, d, Q8, dev_status,
                                             static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? EVP_OK : EVP_ERR_CUDA;
}

int32_t evp_pack_sparse(const uint64_t* T, int64_t n, int32_t d, int32_t x, uint16_t* E,
                        int32_t* dev_status, void* stream) {
    if (n < 0 || d < 1 || d > 32768 || x < 1 || x > d) return EVP_ERR_INVALID;
    if (n == 0) return EVP_OK;
    if (!T || !E) return EVP_ERR_INVALID;
    const cudaError_t e = launch_pack_sparse(T, n, d, x, E, dev_status,
                                             static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? EVP_OK : EVP_ERR_CUDA;
}

size_t ternary_knn_sparse_workspace(int64_t nq, int64_t ns, int32_t d, int32_t x, int32_t k) {
    if (nq < 0 || ns < 1 || !evp::sparse_supported(d, x, k)) return 0;
    return evp::sparse_workspace(nq, ns, d, k);
}

int32_t ternary_knn_sparse(const uint64_t* Q, int64_t nq, const uint16_t* E, int64_t ns,
                           int32_t d, int32_t x, int32_t k, int64_t* ids, int32_t* dist, void* ws,
                           size_t ws_bytes, int32_t* dev_status, void* stream) {
    if (nq < 0 || ns < 1 || ns >= (int64_t(1) << 31) || d < 1 || x < 1 || x > d || k < 1 ||
        (int64_t)k > ns)
        return EVP_ERR_INVALID;
    if (!evp::sparse_supported(d, x, k)) return EVP_ERR_UNSUPPORTED;
    if (nq == 0) return EVP_OK;
    if (!Q || !E || !ids || !dist || !ws || (reinterpret_cast<uintptr_t>(E) & 15) != 0)
        return EVP_ERR_INVALID;
    return evp::run_sparse_knn(Q, nq, E, ns, d, x, k, ids, dist, ws, ws_bytes, dev_status,
                               static_cast<cudaStream_t>(stream));
}

size_t ternary_knn_i8q_workspace(int64_t nq, int64_t ns, int32_t d, int32_t k) {
    if (nq < 0 || ns < 1 || d < 1 || k < 1 || !evp::mma_packed_supported(ns, d, k)) return 0;
    return evp::mma_packed_workspace(ns, d, k);
}

int32_t ternary_knn_i8q(const int8_t* Q8, int64_t nq, const uint64_t* S, int64_t ns, int32_t d,
                        int32_t x, int32_t k, int64_t* ids, int32_t* score, void* ws,
                        size_t ws_bytes, int32_t* dev_status, void* stream) {
    if (nq < 0 || ns < 1 || ns >= (int64_t(1) << 31) || d < 1 || x < 1 || x > d || k < 1 ||
        (int64_t)k > ns)
        return EVP_ERR_INVALID;
    if (!evp::mma_packed_supported(ns, d, k)) return EVP_ERR_UNSUPPORTED;
    if (nq == 0) return EVP_OK;
    if (!Q8 || !S || !ids || !score || !ws || (reinterpret_cast<uintptr_t>(S) & 15) != 0)
        return EVP_ERR_INVALID;
    return evp::run_i8q_knn(Q8, nq, S, ns, d, x, k, ids, score, ws, ws_bytes, dev_status,
                            static_cast<cudaStream_t>(stream));
}

size_t evp_merge_topk_workspace(int64_t nq, int32_t nlists, int32_t k) {
    if (nq <= 0 || nlists < 1 || k < 1) return 0;
    return merge_topk_workspace(nq, nlists, k);
}

int32_t evp_merge_topk(const int64_t* ids, const int32_t* dist, int64_t nq, int32_t nlists,
                       int32_t k, int64_t* out_ids, int32_t* out_dist, void* ws, size_t ws_bytes,
                       int32_t* dev_status, void* stream) {
    if (nq < 0 || nlists < 1 || k < 1) return EVP_ERR_INVALID;
    if (k > EVP_MAX_K || nlists > 1024) return EVP_ERR_UNSUPPORTED;
    if (nq == 0) return EVP_OK;
    if (!ids || !dist || !out_ids || !out_dist || !ws || (reinterpret_cast<uintptr_t>(ws) & 255))
        return EVP_ERR_INVALID;
    return run_merge_topk(ids, dist, nq, nlists, k, out_ids, out_dist, ws, ws_bytes, dev_status,
                          static_cast<cudaStream_t>(stream));
}

int32_t rerank(const float* Q, int64_t nq, const float* S, int64_t ns, int32_t d,
               const int64_t* shortlist, int32_t n, int32_t k, int64_t* ids, float* scores,
               int32_t* dev_status, void* stream) {
    if (nq < 0 || ns < 1 || d < 1 || n < 1 || k < 1 || k > n) return EVP_ERR_INVALID;
    if (d > EVP_MAX_D_RERANK || n > EVP_MAX_SHORTLIST) return EVP_ERR_UNSUPPORTED;
    if (nq == 0) return EVP_OK;
    if (!Q || !S || !shortlist || !ids || !scores) return EVP_ERR_INVALID;
    cudaError_t e = launch_rerank(Q, nq, S, ns, d, shortlist, n, k, ids, scores, dev_status,
                                  static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? EVP_OK : EVP_ERR_CUDA;
}

int32_t evp_test_stall_producer(int32_t path, int32_t fills) {
    if (path == EVP_PATH_MMA) evp::g_stall_mma.store(fills < 0 ? -1 : fills);
    else if (path == EVP_PATH_MMA_PACKED) evp::g_stall_packed.store(fills < 0 ? -1 : fills);
    else return EVP_ERR_INVALID;
    return EVP_OK;
}

int32_t evp_timing_enable(int32_t on) {
    TimingState& t = timing();
    std::lock_guard<std::mutex> g(t.mu);
    t.enabled = on != 0;
    return EVP_OK;
}

int32_t evp_timing_reset(void) {
    TimingState& t = timing();
    std::lock_guard<std::mutex> g(t.mu);
    for (auto& r : t.records) {
        cudaEventSynchronize(r.stop);
        t.spare.push_back(r.start);
        t.spare.push_back(r.stop);
    }
    t.records.clear();
    return EVP_OK;
}

int32_t evp_timing_read(const char* name, int64_t* launches, double* total_ms) {
    if (!name || !launches || !total_ms) return EVP_ERR_INVALID;
    TimingState& t = timing();
    std::lock_guard<std::mutex> g(t.mu);
    int64_t n = 0;
    double ms = 0.0;
    for (auto& r : t.records) {
        if (std::strcmp(r.name, name) != 0) continue;
        if (cudaEventSynchronize(r.stop) != cudaSuccess) return EVP_ERR_CUDA;
        float f = 0.f;
        if (cudaEventElapsedTime(&f, r.start, r.stop) != cudaSuccess) return EVP_ERR_CUDA;
        ms += f;
        ++n;
    }
    *launches = n;
    *total_ms = ms;
    return EVP_OK;
}

}  // extern "C"
