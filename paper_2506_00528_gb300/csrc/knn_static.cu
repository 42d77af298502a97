// ternary_knn_static: the popcount kNN scan with its scratch in a fixed
// device array owned by this library, for callers that cannot allocate
// device memory.
//
// Who needs it: code that must not or cannot allocate device memory -- a
// latency-critical serving thread that must never enter the device
// allocator (which can block on device-wide synchronisation), a plugin that
// is handed raw device pointers by a host framework that owns all
// allocation, or a C caller that has no allocator of its own.  Those callers
// still pass their inputs and outputs; only the workspace comes from here.
//
// The scratch is one file-scope __device__ array of EVP_STATIC_SCRATCH_BYTES
// (16 MiB), present on every GPU that loads the library until the process
// exits.  Host code cannot use the array's name as a device address, so on
// the first call on each device the library asks the runtime for the
// array's device address (cudaGetSymbolAddress, with that device current)
// and caches it.  That first call on a device should therefore happen
// before any stream capture.  A device reset reloads the device code and
// invalidates the cached address; the entry point is not for use after one.
//
// Every call shares the one array: calls that overlap on the GPU (two
// streams, or two host threads) race on it and must be ordered by the
// caller.  The array keeps the previous call's contents; the per-query
// thresholds and list lengths that must start empty are re-initialised by
// the scan's own init kernel at every pass, and every list entry is written
// before it is read.
#include "evp_internal.cuh"

#include <mutex>


namespace {

static __device__ __align__(256) uint8_t g_static_scratch[EVP_STATIC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
void* g_scratch_ptr[MAX_DEVICES] = {nullptr};
std::mutex g_scratch_mu;

// Device address of the scratch array on the current device (set up once).
int32_t scratch_for_current_device(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return EVP_ERR_CUDA;
    std::lock_guard<std::mutex> g(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return EVP_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return EVP_OK;
}

}  // namespace

extern "C" {

int32_t ternary_knn_static(const uint64_t* Q, int64_t nq, const uint64_t* S, int64_t ns,
                           int32_t d, int32_t x, int32_t k, int64_t* ids, int32_t* dist,
                           int32_t* dev_status, void* stream) {
    if (nq < 0 || ns < 1 || ns >= (int64_t(1) << 31) || d < 1 || x < 1 || x > d || k < 1 ||
        (int64_t)k > ns)
        return EVP_ERR_INVALID;
    if (d > EVP_MAX_D_SCAN || k > EVP_MAX_K) return EVP_ERR_UNSUPPORTED;
    if (nq == 0) return EVP_OK;
    if (!Q || !S || !ids || !dist || (reinterpret_cast<uintptr_t>(S) & 15) != 0)
        return EVP_ERR_INVALID;
    const size_t need = evp::plan_popc_scan(nq, ns, d, k).ws_bytes;
    if (need > (size_t)EVP_STATIC_SCRATCH_BYTES) return EVP_ERR_NO_MEMORY;
    void* ws = nullptr;
    const int32_t rc = scratch_for_current_device(&ws);
    if (rc != EVP_OK) return rc;
    return evp::run_popc_knn(Q, nq, S, ns, d, x, k, ids, dist, ws, (size_t)EVP_STATIC_SCRATCH_BYTES,
                             dev_status, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
