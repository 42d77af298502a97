// Resident database handle: the packed codes and float originals stay on
// the device across calls, together with the tensor-core operand copy of
// the codes, so a query batch runs encode -> scan -> rerank without
// re-preparing the database.
#include "evp_internal.cuh"

#include <new>

struct evp_db {
    const uint64_t* T;  // borrowed packed codes [ns][2W]
    const float* U;     // borrowed float rows [ns][d] (may be null)
    int64_t ns;
    int d, x, W, kp;
    uint8_t* S8;        // owned e2m1 copy [ns][kp] (null without EVP_DB_TENSOR_COPY)
};

using namespace evp;

namespace {

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

int resolve_db_path(const evp_db* db, int64_t nq, int32_t k, int32_t path) {
    return path == EVP_PATH_AUTO ? auto_path(nq, db->ns, db->d, k, db->S8 != nullptr) : path;
}

size_t db_knn_ws(const evp_db* db, int64_t nq, int32_t k, int32_t path) {
    return knn_ws_bound(nq, db->ns, db->d, k, path, db->S8 == nullptr);
}

struct SearchLayout {
    size_t codes, sl_ids, sl_dist, knn, total;
};

SearchLayout search_layout(const evp_db* db, int64_t nq, int32_t n_shortlist,
                           int32_t path = EVP_PATH_AUTO) {
    SearchLayout L;
    L.codes = align256((size_t)nq * 2 * db->W * 8);
    L.sl_ids = align256((size_t)nq * n_shortlist * 8);
    L.sl_dist = align256((size_t)nq * n_shortlist * 4);
    L.knn = align256(db_knn_ws(db, nq, n_shortlist, path));
    L.total = L.codes + L.sl_ids + L.sl_dist + L.knn;
    return L;
}

}  // namespace

namespace evp {
const uint8_t* db_tensor_copy(const evp_db* db) { return db ? db->S8 : nullptr; }
const float* db_float_rows(const evp_db* db) { return db ? db->U : nullptr; }
int db_x(const evp_db* db) { return db ? db->x : 0; }
}  // namespace evp

extern "C" {

int32_t evp_db_create(const uint64_t* T, const float* U, int64_t ns, int32_t d, int32_t x,
                      int32_t flags, void* stream, evp_db_t* out) {
    if (!out) return EVP_ERR_INVALID;
    *out = nullptr;
    if (!T || ns < 1 || ns >= (int64_t(1) << 31) || d < 1 || x < 1 || x > d ||
        (flags & ~EVP_DB_TENSOR_COPY) != 0)
        return EVP_ERR_INVALID;
    if (d > EVP_MAX_D_SCAN) return EVP_ERR_UNSUPPORTED;
    if ((reinterpret_cast<uintptr_t>(T) & 15) != 0) return EVP_ERR_INVALID;
    evp_db* db = new (std::nothrow) evp_db();
    if (!db) return EVP_ERR_NO_MEMORY;
    db->T = T;
    db->U = U;
    db->ns = ns;
    db->d = d;
    db->x = x;
    db->W = (d + 63) / 64;
    db->kp = mma_kp(d);
    db->S8 = nullptr;
    if (flags & EVP_DB_TENSOR_COPY) {
        void* p = nullptr;
        if (cudaMalloc(&p, (size_t)ns * db->kp) != cudaSuccess) {
            cudaGetLastError();
            delete db;
            return EVP_ERR_NO_MEMORY;
        }
        db->S8 = static_cast<uint8_t*>(p);
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        if (launch_unpack_fp4(T, ns, d, db->S8, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cudaFree(db->S8);
            delete db;
            return EVP_ERR_CUDA;
        }
    }
    *out = db;
    return EVP_OK;
}

int32_t evp_db_dim(evp_db_t db) { return db ? db->d : 0; }

int64_t evp_db_rows(evp_db_t db) { return db ? db->ns : 0; }

const uint64_t* evp_db_codes(evp_db_t db) { return db ? db->T : nullptr; }

int32_t evp_db_destroy(evp_db_t db) {
    if (!db) return EVP_ERR_INVALID;
    int32_t rc = EVP_OK;
    if (db->S8 && cudaFree(db->S8) != cudaSuccess) rc = EVP_ERR_CUDA;
    delete db;
    return rc;
}

size_t evp_db_knn_workspace(evp_db_t db, int64_t nq, int32_t k, int32_t path) {
    if (!db || nq <= 0 || k < 1) return 0;
    return db_knn_ws(db, nq, k, path);
}

int32_t evp_db_knn(evp_db_t db, const uint64_t* Q, int64_t nq, int32_t k, int64_t* ids,
                   int32_t* dist, void* ws, size_t ws_bytes, int32_t* dev_status, void* stream,
                   int32_t path) {
    if (!db) return EVP_ERR_INVALID;
    if (nq < 0 || k < 1 || (int64_t)k > db->ns || path < EVP_PATH_AUTO ||
        path > EVP_PATH_MMA_PACKED)
        return EVP_ERR_INVALID;
    if (k > EVP_MAX_K) return EVP_ERR_UNSUPPORTED;
    const int rp = resolve_db_path(db, nq, k, path);
    if (rp == EVP_PATH_MMA && k > MMA_K_MAX) return EVP_ERR_UNSUPPORTED;
    if (rp == EVP_PATH_MMA_PACKED && !mma_packed_supported(db->ns, db->d, k))
        return EVP_ERR_UNSUPPORTED;
    if (nq == 0) return EVP_OK;
    if (!Q || !ids || !dist || !ws || (reinterpret_cast<uintptr_t>(ws) & 255) != 0)
        return EVP_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (rp == EVP_PATH_MMA)
        return run_mma_knn(Q, nq, db->S8, db->T, db->ns, db->d, db->x, k, ids, dist, ws, ws_bytes,
                           dev_status, s);
    if (rp == EVP_PATH_MMA_PACKED)
        return run_mma_packed_knn(Q, nq, db->T, db->ns, db->d, db->x, k, ids, dist, ws, ws_bytes,
                                  dev_status, s);
    return run_popc_knn(Q, nq, db->T, db->ns, db->d, db->x, k, ids, dist, ws, ws_bytes,
                        dev_status, s);
}

size_t evp_db_search_path_workspace(evp_db_t db, int64_t nq, int32_t n_shortlist, int32_t k,
                                    int32_t path) {
    if (!db || nq <= 0 || n_shortlist < 1 || k < 1) return 0;
    return search_layout(db, nq, n_shortlist, path).total;
}

size_t evp_db_search_workspace(evp_db_t db, int64_t nq, int32_t n_shortlist, int32_t k) {
    return evp_db_search_path_workspace(db, nq, n_shortlist, k, EVP_PATH_AUTO);
}

int32_t evp_db_search_path(evp_db_t db, const float* Q, int64_t nq, int32_t n_shortlist,
                           int32_t k, int64_t* ids, float* scores, void* ws, size_t ws_bytes,
                           int32_t* dev_status, void* stream, int32_t path) {
    if (!db) return EVP_ERR_INVALID;
    if (nq < 0 || k < 1 || n_shortlist < k || (int64_t)n_shortlist > db->ns ||
        path < EVP_PATH_AUTO || path > EVP_PATH_MMA_PACKED)
        return EVP_ERR_INVALID;
    if (n_shortlist > EVP_MAX_K) return EVP_ERR_UNSUPPORTED;
    if (nq == 0) return EVP_OK;
    if (!db->U || !Q || !ids || !scores || !ws || (reinterpret_cast<uintptr_t>(ws) & 255) != 0)
        return EVP_ERR_INVALID;
    const SearchLayout L = search_layout(db, nq, n_shortlist, path);
    if (ws_bytes < L.total) return EVP_ERR_NO_MEMORY;
    uint8_t* w = static_cast<uint8_t*>(ws);
    uint64_t* codes = reinterpret_cast<uint64_t*>(w);
    int64_t* sl_ids = reinterpret_cast<int64_t*>(w + L.codes);
    int32_t* sl_dist = reinterpret_cast<int32_t*>(w + L.codes + L.sl_ids);
    void* knn_ws = w + L.codes + L.sl_ids + L.sl_dist;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (launch_encode(Q, nq, db->d, db->x, codes, dev_status, s) != cudaSuccess)
        return EVP_ERR_CUDA;
    const int32_t rc = evp_db_knn(db, codes, nq, n_shortlist, sl_ids, sl_dist, knn_ws, L.knn,
                                  dev_status, stream, path);
    if (rc != EVP_OK) return rc;
    if (launch_rerank(Q, nq, db->U, db->ns, db->d, sl_ids, n_shortlist, k, ids, scores,
                      dev_status, s) != cudaSuccess)
        return EVP_ERR_CUDA;
    return EVP_OK;
}

int32_t evp_db_search(evp_db_t db, const float* Q, int64_t nq, int32_t n_shortlist, int32_t k,
                      int64_t* ids, float* scores, void* ws, size_t ws_bytes, int32_t* dev_status,
                      void* stream) {
    return evp_db_search_path(db, Q, nq, n_shortlist, k, ids, scores, ws, ws_bytes, dev_status,
                              stream, EVP_PATH_AUTO);
}

size_t evp_db_search_host_workspace(evp_db_t db, int64_t nq, int32_t n_shortlist, int32_t k) {
    if (!db || nq <= 0 || n_shortlist < 1 || k < 1) return 0;
    return align256((size_t)nq * db->d * 4) + align256((size_t)nq * k * 8) +
           align256((size_t)nq * k * 4) + search_layout(db, nq, n_shortlist).total;
}

int32_t evp_db_search_host(evp_db_t db, const float* Q_host, int64_t nq, int32_t n_shortlist,
                           int32_t k, int64_t* ids_host, float* scores_host, void* ws,
                           size_t ws_bytes, int32_t* dev_status, void* stream) {
    if (!db) return EVP_ERR_INVALID;
    if (nq < 0 || k < 1 || n_shortlist < k) return EVP_ERR_INVALID;
    if (nq == 0) return EVP_OK;
    if (!Q_host || !ids_host || !scores_host || !ws) return EVP_ERR_INVALID;
    const size_t need = evp_db_search_host_workspace(db, nq, n_shortlist, k);
    if (ws_bytes < need) return EVP_ERR_NO_MEMORY;
    uint8_t* w = static_cast<uint8_t*>(ws);
    const size_t qb = align256((size_t)nq * db->d * 4);
    const size_t ib = align256((size_t)nq * k * 8);
    const size_t sb = align256((size_t)nq * k * 4);
    float* Qd = reinterpret_cast<float*>(w);
    int64_t* idd = reinterpret_cast<int64_t*>(w + qb);
    float* scd = reinterpret_cast<float*>(w + qb + ib);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(Qd, Q_host, (size_t)nq * db->d * 4, cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return EVP_ERR_CUDA;
    const int32_t rc = evp_db_search(db, Qd, nq, n_shortlist, k, idd, scd, w + qb + ib + sb,
                                     ws_bytes - (qb + ib + sb), dev_status, stream);
    if (rc != EVP_OK) return rc;
    if (cudaMemcpyAsync(ids_host, idd, (size_t)nq * k * 8, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(scores_host, scd, (size_t)nq * k * 4, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess)
        return EVP_ERR_CUDA;
    return EVP_OK;
}

}  // extern "C"
