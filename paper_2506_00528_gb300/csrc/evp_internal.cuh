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

// Count `bytes` of transactions as done on a barrier of this CTA without a
// copy (accounts for a copy that was expected but will never be issued).
__device__ __forceinline__ void mbar_complete_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.complete_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(
                     smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// One arrival on a barrier of this CTA.
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
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

// ---- sorted-key and team helpers ------------------------------------
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

__device__ inline int next_pow2(int v) {
    int p = 32;
    while (p < v) p <<= 1;
    return p;
}

__device__ __forceinline__ void named_barrier(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// The smallest bin T with sum(hist[0..T]) >= k, scanning up from the
// smallest non-empty bin; 0xFFFFFFFF if fewer than k keys are counted.
// Team-wide (every thread gets the result); `scratch` holds TT/32 + 2 words.
template <typename Sync>
__device__ __forceinline__ uint32_t team_kth_bin(const uint32_t* hist, const uint32_t* minhalf,
                                                 int bins, uint32_t k, uint32_t* scratch, int t,
                                                 int TT, Sync& sync) {
    const int nw = TT / 32, wt = t >> 5, ln = t & 31;
    if (t == 0) {
        scratch[nw] = __ldcg(minhalf);
        scratch[nw + 1] = 0xFFFFFFFFu;
    }
    sync();
    const uint32_t lo = scratch[nw];
    uint32_t before = 0, T = 0xFFFFFFFFu;
    for (uint32_t h0 = lo; h0 < (uint32_t)bins; h0 += (uint32_t)TT) {
        const uint32_t h = h0 + (uint32_t)t;
        const uint32_t c = h < (uint32_t)bins ? __ldcg(&hist[h]) : 0u;
        uint32_t sum = c;  // inclusive scan over the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t n = __shfl_up_sync(0xffffffffu, sum, o);
            if (ln >= o) sum += n;
        }
        if (ln == 31) scratch[wt] = sum;
        sync();
        uint32_t off = 0, total = 0;
        for (int w = 0; w < nw; ++w) {
            const uint32_t v = scratch[w];
            if (w < wt) off += v;
            total += v;
        }
        sum += off;
        if (c > 0 && before + sum >= k && before + sum - c < k) scratch[nw + 1] = h;
        sync();
        T = scratch[nw + 1];
        before += total;
        if (T != 0xFFFFFFFFu || before >= k) break;
    }
    return T;
}

// ---- tcgen05 / TMEM ----------------------------------------------------
// Shared-memory matrix descriptor of a K-major SWIZZLE_128B tile whose
// 8-row core groups are 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4)  // start address
           | (1ull << 16)                       // leading byte offset (unused for SW128 K-major)
           | (64ull << 32)                      // stride byte offset 1024 >> 4
           | (1ull << 46)                       // descriptor version
           | (2ull << 61);                      // SWIZZLE_128B
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Bounded mbarrier wait that also gives up as soon as *abort is set.
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t parity,
                                                   const int* abort) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (*reinterpret_cast<const volatile int*>(abort)) return false;
        if (globaltimer_ns() - t0 > WAIT_LIMIT_NS) return false;
    }
    return true;
}

// Issue a 32-column TMEM load without waiting for it.
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
        "[%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
          "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
          "=r"(v[31])
        : "r"(taddr));
}

// Wait for the warp's outstanding TMEM loads; v is an in-out operand so that
// no use of the loaded registers can be scheduled before the wait.
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.wait::ld.sync.aligned;"
        : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]),
          "+r"(v[7]), "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]),
          "+r"(v[13]), "+r"(v[14]), "+r"(v[15]), "+r"(v[16]), "+r"(v[17]), "+r"(v[18]),
          "+r"(v[19]), "+r"(v[20]), "+r"(v[21]), "+r"(v[22]), "+r"(v[23]), "+r"(v[24]),
          "+r"(v[25]), "+r"(v[26]), "+r"(v[27]), "+r"(v[28]), "+r"(v[29]), "+r"(v[30]),
          "+r"(v[31])
        :
        : "memory");
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

// Testing support (evp_test_stall_producer): stage fills after which the
// next launch of a tensor-core scan stops its first CTA's copy producer;
// -1 = none.  take_* returns the armed value and disarms it.
int take_stall_mma();
int take_stall_packed();

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

// Per-query merge of per-(query, slice) sorted key lists ([nq][nslices][2][kl]
// with meta [nq][nslices] = (length, buffer)) into the k best; kl = list
// capacity (0: k; a scan with capped lists passes kl < k).  Histogram
// bins count Delta/2 (bin_shift < 0) or (key >> 32) >> bin_shift; the
// output distance is key >> 32, or dist_bias - (key >> 32) when dist_bias
// is not 0 (the score of the int8-query scan).
int32_t launch_final_merge(const uint64_t* lists, const int32_t* meta, const uint64_t* tau,
                           const uint32_t* hist, const uint32_t* minhalf, int hist_bins,
                           int64_t nq, int nslices, int k, int64_t* ids, int32_t* dist,
                           cudaStream_t stream, int bin_shift = -1, int dist_bias = 0,
                           int kl = 0);

// One batch of a multi-batch final merge: queries q0 .. q0 + nq - 1 of the
// launch are queries 0 .. nq - 1 of this batch (Delta keys).
struct FmBatch {
    const uint64_t* lists;
    const int32_t* meta;
    const uint64_t* tau;
    const uint32_t* hist;
    const uint32_t* minhalf;
    int hist_bins, nslices, k, kl, stage;  // kl: list capacity (<= k)
    int64_t q0;
    int64_t* ids;
    int32_t* dist;
};
// Shared-memory bytes of a final merge of nslices lists of k keys, and
// whether it stages the lists (*stage).
size_t final_merge_smem(int nslices, int k, int* stage);
// tab: device array of nb + 1 entries (the last only supplies q0 = total).
int32_t launch_final_merge_multi(const FmBatch* tab, int nb, int64_t total_q, size_t smem,
                                 cudaStream_t stream);

// int8 queries (the single-operand translation of Sec. 6).
cudaError_t launch_quantize_i8(const float* Q, int64_t n, int d, int8_t* Q8, int32_t* status,
                               cudaStream_t stream);

size_t merge_topk_workspace(int64_t nq, int nlists, int k);
int32_t run_merge_topk(const int64_t* ids, const int32_t* dist, int64_t nq, int nlists, int k,
                       int64_t* out_ids, int32_t* out_dist, void* ws, size_t ws_bytes,
                       int32_t* status, cudaStream_t stream);

struct MmaPlan {
    int kp;                 // bytes per row of the e2m1 operands (a multiple of 128)
    int kl;                 // keys kept per (query, slice): k, or 128 with capped lists
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
constexpr int MMA_TILE_ROWS = 240;  // database rows per tensor-core tile (the MMA's N)
// Smallest query count for which the automatic choice takes the tensor-core
// scan: from 9 queries when the database's e2m1 copy is resident (the scan
// then reads half a byte per element at HBM speed, faster than a 16-query
// popcount pass), from 17 when the copy must be built first.
inline int64_t auto_mma_min_nq(bool resident_copy) { return resident_copy ? 9 : 17; }
// Largest query count for which the automatic choice takes the packed
// tensor-core scan (where it applies): one 64-query pass costs about what
// the fp4 scan costs against a resident copy; without one, the fp4 scan
// must first expand the whole database.
inline int64_t auto_packed_max_nq(bool resident_copy) {
    return resident_copy ? EVP_AUTO_PACKED_MAX_NQ : EVP_AUTO_PACKED_MAX_NQ_NO_COPY;
}
int mma_kp(int d);
// Workspace bytes that serve every kNN call with at most nq queries (and
// the same other arguments) on `path` (AUTO resolved per call).
size_t knn_ws_bound(int64_t nq, int64_t ns, int d, int k, int path, bool convert_db);
int mma_active_queries(int k);
// tiles_per_item > 0: slices of about that many 240-row database tiles (the
// tile shape of the fused multi-batch scan) instead of whole waves.
// allow_cap: keep kl < k keys per (query, slice) -- kl the smallest power of
// two >= 16 with kl x nslices >= 4k, at most 128 (every query lane of a tile
// active) -- when the slices are many enough that a slice rarely holds more
// than kl / 2 of a query's k nearest (nslices x kl / 2 >= k); a repair pass
// then makes the result exact (run_mma_knn).
MmaPlan plan_mma_scan(int64_t nq, int64_t ns, int d, int k, bool convert_db,
                      int tiles_per_item = 0, bool allow_cap = false);

// Fused multi-batch tensor-core scan (the batched form): several kNN
// batches, each against a resident e2m1 database copy, scanned by one
// persistent launch over the work items of all of them, then merged by one
// multi-batch final merge.  The plan owns a small device table (tensor maps,
// per-batch arguments) written once at creation; workspaces are the
// caller's.
struct MmaBatchSpec {
    const uint64_t* Q;   // packed query codes [nq][2W]
    int64_t nq;
    const uint8_t* S8;   // resident e2m1 copy of the database [ns][kp], 256-byte aligned
    int64_t ns;
    int d, x, k;
    int64_t* ids;        // [nq][k]
    int32_t* dist;       // [nq][k]
    void* ws;            // mma_multi_ws(...) bytes, 256-byte aligned
    int tiles_per_item;  // tile shape: 240-row database tiles per work item
};
struct MmaMultiPlan;
size_t mma_multi_ws(int64_t nq, int64_t ns, int d, int k, int tiles_per_item);
int32_t mma_multi_create(const MmaBatchSpec* specs, int nb, MmaMultiPlan** out);
int32_t mma_multi_run(MmaMultiPlan* p, int32_t* status, cudaStream_t stream);
void mma_multi_destroy(MmaMultiPlan* p);
// spread_cg > 0: query rows placed as the tensor-core scan's small-batch
// spread over spread_cg CTAs expects (queries only).
cudaError_t launch_unpack_fp4(const uint64_t* T, int64_t n, int d, uint8_t* out,
                              cudaStream_t stream, int spread_cg = 0);
// S8: resident e2m1 copy of the database ([ns][kp]) or nullptr, in which case
// S is converted into the workspace first.
int32_t run_mma_knn(const uint64_t* Q, int64_t nq, const uint8_t* S8, const uint64_t* S,
                    int64_t ns, int d, int x, int k, int64_t* ids, int32_t* dist, void* ws,
                    size_t ws_bytes, int32_t* status, cudaStream_t stream);

// Packed tensor-core path (database rows as the MMA's M side, tiles
// unpacked on chip).  supported(): d, k and ns within its limits.
bool mma_packed_supported(int64_t ns, int d, int k);
size_t mma_packed_workspace(int64_t ns, int d, int k);
int32_t run_mma_packed_knn(const uint64_t* Q, int64_t nq, const uint64_t* S, int64_t ns, int d,
                           int x, int k, int64_t* ids, int32_t* dist, void* ws, size_t ws_bytes,
                           int32_t* status, cudaStream_t stream);

// int8-query scan (the single-operand translation of Sec. 6 with the
// masked-addition score of Sec. 5.1.2) on the packed tensor-core pipeline:
// same limits and workspace as the packed scan; score[q][j] is <q8, s>,
// ids ordered by (score descending, row ascending).
int32_t run_i8q_knn(const int8_t* Q8, int64_t nq, const uint64_t* S, int64_t ns, int d, int x,
                    int k, int64_t* ids, int32_t* score, void* ws, size_t ws_bytes,
                    int32_t* status, cudaStream_t stream);

// Sparse small-x codes (Sec. 6): pack from bitplanes, and the scan.
bool sparse_supported(int d, int x, int k);
size_t sparse_workspace(int64_t nq, int64_t ns, int d, int k);
cudaError_t launch_pack_sparse(const uint64_t* T, int64_t n, int d, int x, uint16_t* E,
                               int32_t* status, cudaStream_t stream);
int32_t run_sparse_knn(const uint64_t* Q, int64_t nq, const uint16_t* E, int64_t ns, int d,
                       int x, int k, int64_t* ids, int32_t* dist, void* ws, size_t ws_bytes,
                       int32_t* status, cudaStream_t stream);

// Internals of a resident database (db.cu): its e2m1 copy (null without
// EVP_DB_TENSOR_COPY), its float rows (may be null) and its x.
const uint8_t* db_tensor_copy(const evp_db* db);
const float* db_float_rows(const evp_db* db);
int db_x(const evp_db* db);

// Path the automatic rule takes for nq queries (resident_copy: the
// database's e2m1 copy is resident).
int auto_path(int64_t nq, int64_t ns, int d, int k, bool resident_copy);

cudaError_t launch_rerank(const float* Q, int64_t nq, const float* S, int64_t ns, int d,
                          const int64_t* shortlist, int n, int k, int64_t* ids, float* scores,
                          int32_t* status, cudaStream_t stream);

}  // namespace evp
