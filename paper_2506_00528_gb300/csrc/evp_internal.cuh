// Internal helpers of libevp (CUDA side only): status reporting, PTX
// wrappers for mbarriers and TMA, bounded waits, and the launchers that
// api.cu calls.  Nothing here is part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "evp.h"

namespace evp {

constexpr uint64_t KEY_NONE = ~0ull;                // empty candidate slot
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;   // bounded device waits: 2 s

// First error wins: a status word only changes from EVP_OK.
__device__ __forceinline__ void report(int32_t* status, int32_t code) {
    if (status) atomicCAS(status, (int32_t)EVP_OK, code);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---- mbarrier ---------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity; give up after WAIT_LIMIT_NS.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (globaltimer_ns() - t0 > WAIT_LIMIT_NS) return false;
    }
    return true;
}

// ---- TMA --------------------------------------------------------------
// 2-D tiled load of one box into shared memory; completion is signalled on
// `bar` as transaction bytes.  c0 is the inner (contiguous) coordinate.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int32_t c0, int32_t c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
        : "memory");
}

// ---- warp-level sorted-key helpers -------------------------------------
// Ascending bitonic sort of buf[0, P) (P a power of two) by one warp.
__device__ __forceinline__ void warp_bitonic_sort(uint64_t* buf, int P) {
    const int lane = threadIdx.x & 31;
    for (int kk = 2; kk <= P; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < P; i += 32) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const uint64_t a = buf[i], b = buf[ixj];
                    const bool up = (i & kk) == 0;
                    if ((a > b) == up) {
                        buf[i] = b;
                        buf[ixj] = a;
                    }
                }
            }
            __syncwarp();
        }
    }
}

// Number of entries of the ascending array a[0, n) that are < key.
__device__ __forceinline__ int lower_bound_u64(const uint64_t* a, int n, uint64_t key) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// out[0, min(k, nL + nc)) = the smallest keys of L[0,nL) and C[0,nc), both
// ascending with all keys distinct.  One warp; out must not alias L or C.
// Returns the new length.
__device__ __forceinline__ int warp_merge_topk(const uint64_t* L, int nL, const uint64_t* C,
                                               int nc, uint64_t* out, int k) {
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < nL; i += 32) {
        const uint64_t key = L[i];
        const int r = i + lower_bound_u64(C, nc, key);
        if (r < k) out[r] = key;
    }
    for (int j = lane; j < nc; j += 32) {
        const uint64_t key = C[j];
        const int r = j + lower_bound_u64(L, nL, key);
        if (r < k) out[r] = key;
    }
    __syncwarp();
    const int total = nL + nc;
    return total < k ? total : k;
}

// ---- kernel timing (measurement support) ------------------------------
// Records start/stop events around a launch when timing is enabled.
struct TimedLaunch {
    TimedLaunch(const char* name, cudaStream_t stream);
    ~TimedLaunch();
    const char* name_;
    cudaStream_t stream_;
    int slot_;
};

// ---- launchers (defined in the .cu files, called from api.cu) ----------
int num_sms();

// cuTensorMapEncodeTiled through the runtime's driver entry point (the
// library does not link libcuda directly).  nullptr if unavailable.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled_fn();

cudaError_t launch_encode(const float* U, int64_t n, int d, int x, uint64_t* T,
                          int32_t* status, cudaStream_t stream);

struct ScanPlan {
    int nslices;        // CTAs of the scan, each a contiguous slice of rows
    int qb;             // queries per scan pass
    int groups;         // passes
    size_t list_bytes;  // per-pass list storage
    size_t meta_bytes;  // per-pass list lengths
    size_t hist_bytes;  // union-bound histograms and minima
    size_t ws_bytes;    // total workspace
};
ScanPlan plan_popc_scan(int64_t nq, int64_t ns, int d, int k);

int32_t run_popc_knn(const uint64_t* Q, int64_t nq, const uint64_t* S, int64_t ns, int d,
                     int x, int k, int64_t* ids, int32_t* dist, void* ws, size_t ws_bytes,
                     int32_t* status, cudaStream_t stream);

// Per-query merge of per-(query, slice) sorted key lists ([nq][nslices][2][k]
// with meta [nq][nslices] = (length, buffer)) into the k best.
int32_t launch_final_merge(const uint64_t* lists, const int32_t* meta, const uint64_t* tau,
                           const uint32_t* hist, const uint32_t* minhalf, int hist_bins,
                           int64_t nq, int nslices, int k, int64_t* ids, int32_t* dist,
                           cudaStream_t stream);

size_t merge_topk_workspace(int64_t nq, int nlists, int k);
int32_t run_merge_topk(const int64_t* ids, const int32_t* dist, int64_t nq, int nlists, int k,
                       int64_t* out_ids, int32_t* out_dist, void* ws, size_t ws_bytes,
                       int32_t* status, cudaStream_t stream);

struct MmaPlan {
    int kp;                 // K padded to a multiple of 128
    int qa;                 // active queries per 128-row tile
    int qtiles;             // query tiles (of qa queries)
    int nslices;            // database slices per query tile
    int cg;                 // CTAs per tensor-core instruction: 1, or 2 (a CTA pair)
    bool spread;            // <= 128 queries spread over every epilogue warp's lanes
    int workers;            // resident CTAs (cg = 1) or CTA pairs (cg = 2)
    int64_t rows_per_slice;
    size_t a_bytes, b_bytes, list_bytes, meta_bytes, tau_bytes, hist_bytes, ws_bytes;
};
constexpr int MMA_K_MAX = 1024;  // largest k of the tensor-core path
// Smallest query count for which the automatic choice takes the tensor-core
// scan: from 9 queries when the database's e4m3 copy is resident (the scan
// then reads 1 byte per element at HBM speed, faster than a 16-query
// popcount pass), from 17 when the copy must be built first.
inline int64_t auto_mma_min_nq(bool resident_copy) { return resident_copy ? 9 : 17; }
int mma_kp(int d);
// Workspace bytes that serve every kNN call with at most nq queries (and
// the same other arguments) on `path` (AUTO resolved per call).
size_t knn_ws_bound(int64_t nq, int64_t ns, int d, int k, int path, bool convert_db);
int mma_active_queries(int k);
MmaPlan plan_mma_scan(int64_t nq, int64_t ns, int d, int k, bool convert_db);
// spread_cg > 0: query rows placed as the tensor-core scan's small-batch
// spread over spread_cg CTAs expects (queries only).
cudaError_t launch_unpack_fp8(const uint64_t* T, int64_t n, int d, uint8_t* out,
                              cudaStream_t stream, int spread_cg = 0);
// S8: resident e4m3 copy of the database ([ns][kp]) or nullptr, in which case
// S is converted into the workspace first.
int32_t run_mma_knn(const uint64_t* Q, int64_t nq, const uint8_t* S8, const uint64_t* S,
                    int64_t ns, int d, int x, int k, int64_t* ids, int32_t* dist, void* ws,
                    size_t ws_bytes, int32_t* status, cudaStream_t stream);

cudaError_t launch_rerank(const float* Q, int64_t nq, const float* S, int64_t ns, int d,
                          const int64_t* shortlist, int n, int k, int64_t* ids, float* scores,
                          int32_t* status, cudaStream_t stream);

}  // namespace evp
