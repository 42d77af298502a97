// ternary_knn, tensor-core path: the exhaustive scan as a dense contraction
// on the 5th-generation tensor cores (tcgen05, kind::mxf4).
//
// b2sp(q, s) of Sec. 5.1.2 is the scalar product of two ternary vectors.
// Both operands are written as 4-bit e2m1 values (+1 = 0x2, -1 = 0xA, 0 =
// 0x0, two per byte, the lower K index in the low nibble), which represent
// {-1, 0, 1} exactly; the block-scaled fp4 instruction (kind::mxf4, K = 64
// per instruction) multiplies every 32-element block by a scale factor,
// here 2^0 everywhere (ue8m0 0x7F), and accumulates in float32, where every
// partial sum is an integer of magnitude <= d < 2^24, so D = Q S^T holds
// b2sp exactly.  Delta = 2x - 2 b2sp for codes with x non-zeros each.
// Packed fp4 moves half the bytes of an 8-bit operand per element and the
// instruction does twice the e4m3 work per clock; the dense int8 kind does
// not exist on this target.
//
// Kernel (persistent: one CTA per SM, or one CTA pair per two SMs, looping
// over work items = (query tile, database slice)):
//   warp 0      TMA producer: the work item's query tile (A, 128 rows, all
//               K, loaded once per item and kept in shared memory) and
//               K-chunks of 128 bytes (256 elements) of the database tile
//               (B, 240 x 128 B, or its half for a CTA pair), SWIZZLE_128B,
//               through a ring of mbarrier stages;
//   warp 1      allocates the 512 TMEM columns -- two accumulators of 240
//               columns and the scale factors (32 columns of 2^0, written
//               once by the epilogue warps) -- and issues tcgen05.mma
//               (M = 128 or, for a pair, 256; N = 240; K = 64) from one
//               thread into one of the accumulators, commits stage releases
//               and accumulator-ready signals with tcgen05.commit
//               (multicast to both CTAs of a pair);
//   warp 6      threshold helper: recomputes each query's union bound (below)
//               from the workspace histogram and publishes it in shared memory;
//   warps 2-5   epilogue: tcgen05.ld of the accumulator (thread = TMEM lane
//               = query), Delta from D, and a private max-heap of the kl
//               best (Delta/2 << 20 | row-in-slice) keys in shared memory.
//               A row is a candidate only if its D beats the heap root (rows
//               arrive in ascending index order, so an equal Delta never
//               displaces) and is not worse than the union bound: every key
//               any slice of the query inserts is counted in a per-query
//               Delta histogram in the workspace, and the k-th smallest
//               counted Delta bounds the answer for all slices.
//               The maxima of 32-column groups come from tcgen05.ld.red,
//               four loads per wait; a warp skips a group when no lane has a
//               candidate, and otherwise loads it again and examines only
//               the 4-column sub-groups in which some lane has one.
//               Candidates go to a per-thread staging buffer that the warp
//               inserts into the heaps together when a lane's buffer could
//               overflow, so heap updates of different lanes do not
//               serialise.
// The Delta matrix is never written to memory.  Per (query, slice) sorted
// lists of kl keys go to the workspace and the per-query merge of the
// popcount path combines them; with kl < k (capped lists) a check of every
// list's tail against the merged k-th key, and a rescan of the rare slice
// that may have held more, keep the result exact.  Every mbarrier wait is bounded (2 s); on expiry the CTA
// reports EVP_ERR_TIMEOUT, raises an abort flag in itself and its pair
// peer (every other wait then gives up at once), waits (bounded) for the
// copies and MMAs already issued to complete, and frees TMEM.
#include "evp_internal.cuh"

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

namespace evp {

namespace {

constexpr int MMA_M = 128;   // query rows per CTA (= TMEM lanes)
constexpr int MMA_N = MMA_TILE_ROWS;  // database rows per accumulator tile (240)
// Accumulator tiles in tensor memory: the epilogue examines one while the
// MMAs fill the other.  (Three tiles of 160 columns decouple the two sides
// further, but the issuing thread's own time per 4-instruction chunk, ~540
// clocks at any N, then exceeds the chunk's 320 clocks of tensor work: 240
// columns in two tiles measured faster.)
constexpr int NACC = 2;
constexpr int KSTEP = 32;    // bytes of K per instruction (64 fp4 elements)
constexpr int KCHUNK = 128;  // bytes of K per stage (256 elements)
constexpr int MMA_KCHUNK_MAX = 4;  // chunks per row: d <= 1024
constexpr int EPI_GROUPS = (MMA_N + 31) / 32;  // 32-column TMEM loads per tile
static_assert(MMA_N % 16 == 0 && MMA_N >= 32 && MMA_N <= 256, "N of the instruction");
constexpr uint32_t SF_COL = NACC * MMA_N;  // scale factors: A at column SF_COL, B 8 after (<= 8 each)
constexpr int HEAP_SLOTS = 128 * 128;  // heap capacity: active queries x k <= 128 x 128
constexpr int NUM_THREADS = 224;  // TMA, MMA, 4 epilogue warps, threshold helper
constexpr int EPI_WARPS = 4;
constexpr int A_STAGE_BYTES = MMA_M * KCHUNK;
constexpr int HEAP_BYTES = HEAP_SLOTS * 4;
constexpr int STAGE_SLOTS = 32;                     // per-thread candidate staging
constexpr int FLUSH_AT = 1;   // staged keys that trigger a flush at the end of a tile
constexpr int STAGING_BYTES = STAGE_SLOTS * MMA_M * 4;
// A 32-column group can stage up to 32 keys per lane right after a flush.
static_assert(STAGE_SLOTS >= 32, "staging must hold one full column group");
constexpr uint32_t TMEM_COLS = 512;
static_assert(SF_COL + 32 <= TMEM_COLS, "TMEM columns");
static_assert((NACC - 1) * MMA_N + EPI_GROUPS * 32 <= (int)TMEM_COLS,
              "the last tile's last 32-column load stays inside the allocation");
constexpr int LOCAL_BITS = 20;  // row-in-slice bits of a heap key
constexpr int64_t MAX_SLICE_ROWS = int64_t(1) << LOCAL_BITS;
constexpr int UBOUND_BYTES = MMA_M * 8;             // helper -> epilogue thresholds

// Shared memory outside the operand pool: alignment slack, heaps, staging,
// thresholds, barriers and flags.
constexpr int SMEM_FIXED = 1024 + HEAP_BYTES + STAGING_BYTES + UBOUND_BYTES + 256;
// Operand pool: the work item's query tile (kchunks x 16 KB, resident for
// all of the item's database tiles) followed by the database stages.
constexpr int POOL_BYTES = (232448 - SMEM_FIXED) / 1024 * 1024;
constexpr int MAX_STAGES = 8;

// CG = CTAs per tensor-core instruction.  CG = 1: M = 128, each CTA holds
// its query tile and stages the whole 240-row database tile.  CG = 2: a CTA
// pair (cluster of two) runs M = 256, N = 240 instructions issued by the
// even CTA; each CTA holds its own 128 query rows and stages one half (120
// rows) of the database tile, and holds the accumulator rows of its own
// queries in its TMEM.  The query tile is loaded once per work item: per
// database tile only the database rows move through L2 and shared memory.
template <int CG>
struct MmaCfg {
    static constexpr int B_ROWS = MMA_N / CG;  // database rows staged per CTA
    static constexpr int STAGE_BYTES = B_ROWS * KCHUNK;
    static constexpr size_t SMEM_BYTES = (size_t)SMEM_FIXED + POOL_BYTES;
    // database stages that fit beside a query tile of a_chunks chunks
    static constexpr int stages_for(int a_chunks) {
        return (POOL_BYTES - a_chunks * A_STAGE_BYTES) / STAGE_BYTES < MAX_STAGES
                   ? (POOL_BYTES - a_chunks * A_STAGE_BYTES) / STAGE_BYTES
                   : MAX_STAGES;
    }
    // Instruction descriptor of the block-scaled kinds: A = B = e2m1
    // (format 1 of kind::mxf4), both K-major, N = MMA_N, scale factors ue8m0
    // (bit 23), M = 128 x CG; scale-factor IDs 0.
    static constexpr uint32_t IDESC = (1u << 7) | (1u << 10) | ((uint32_t)(MMA_N >> 3) << 17) |
                                      (1u << 23) | ((uint32_t)((MMA_M * CG) >> 4) << 24);
};
static_assert(MmaCfg<1>::SMEM_BYTES <= 232448 && MmaCfg<2>::SMEM_BYTES <= 232448,
              "shared memory per CTA");
static_assert(MmaCfg<1>::stages_for(MMA_KCHUNK_MAX) >= 2 && MmaCfg<2>::stages_for(MMA_KCHUNK_MAX) >= 2,
              "at least two database stages beside the largest query tile");
static_assert(MmaCfg<1>::STAGE_BYTES % 1024 == 0 && MmaCfg<2>::STAGE_BYTES % 1024 == 0 &&
              A_STAGE_BYTES % 1024 == 0, "128-byte swizzle atoms stay 1024-byte aligned");

struct MmaArgs {
    int nq;
    int64_t ns;
    int kchunks;
    int x;
    int k;                 // keys kept per (query, slice): heap and list capacity
    int kunion;            // the query's k: the union bound is its kunion-th smallest counted key
    int64_t rows_per_slice;
    int qtiles, nslices;   // work items = qtiles * nslices
    int qa;                // active queries per 128-row tile (k <= HEAP_SLOTS / qa)
    int spread;            // a batch of <= 128 queries spread over every TMEM lane quadrant
                           // of both CTAs (see query_of_lane)
    uint64_t* lists;       // [nq][nslices][2][k], buffer 0 used
    int32_t* meta;         // [nq][nslices][2]
    uint64_t* tau_global;  // [nq] (unused by the tensor path)
    uint32_t* hist;        // [nq][hist_bins]: Delta/2 of every key any slice inserted
    uint32_t* minhalf;     // [nq]: smallest Delta/2 any slice inserted
    int hist_bins;         // 2x + 1
    int32_t* status;
    int stall_fills;       // testing: CTA 0's producer stops after this many fills (-1: never)
    // launch-wide (the multi-batch form reads them from the launch's own
    // arguments): query-tile chunks reserved in shared memory (the largest
    // kchunks of the launch) and the database stages beside them
    int a_chunks, nstages;
};

// Multi-batch form (the batched plan's fused scan): one persistent launch
// whose work items are the (query unit, database slice) items of several
// batches, each batch against its own resident database.  Items are
// numbered batch after batch; batch b owns items [item0[b], item0[b+1]).
// Each item reads its batch's arguments and tensor maps from this table in
// device memory (written once by the host before the first launch).
constexpr int MMA_MULTI_MAX = 64;
struct MmaMulti {  // 64-byte aligned through its tensor maps
    CUtensorMap mapA[MMA_MULTI_MAX];  // query operand of each batch
    CUtensorMap mapB[MMA_MULTI_MAX];  // database operand of each batch
    MmaArgs args[MMA_MULTI_MAX];
    int item0[MMA_MULTI_MAX + 1];
    int nbatches, nitems;
};

// Maximum of three floats in one instruction (no NaN among the inputs here).
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// D (+)= A B^T over one K step: e2m1 operands in shared memory, unit scale
// factors in tensor memory (sfa, sfb).
template <int CG>
__device__ __forceinline__ void mma_f4(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t sfa, uint32_t sfb, uint32_t accumulate) {
    if constexpr (CG == 1) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %6, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X "
            "[%0], %1, %2, %3, [%4], [%5], p;\n\t}" ::"r"(dtmem),
            "l"(adesc), "l"(bdesc), "r"(MmaCfg<1>::IDESC), "r"(sfa), "r"(sfb), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %6, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::mxf4.block_scale.scale_vec::2X "
            "[%0], %1, %2, %3, [%4], [%5], p;\n\t}" ::"r"(dtmem),
            "l"(adesc), "l"(bdesc), "r"(MmaCfg<2>::IDESC), "r"(sfa), "r"(sfb), "r"(accumulate)
            : "memory");
    }
}

// Write v to 32 consecutive columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_fill32(uint32_t taddr, uint32_t v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
        "%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(taddr),
        "r"(v)
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// One arrival on `bar` once every MMA issued so far has completed: on this
// CTA's barrier (CG = 1) or on the barrier at the same offset in both CTAs
// of the pair (CG = 2).
template <int CG>
__device__ __forceinline__ void mma_commit_all(uint64_t* bar) {
    if constexpr (CG == 1) {
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(bar))
            : "memory");
    } else {
        const uint16_t both = 3;
        asm volatile(
            "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster"
            ".b64 [%0], %1;" ::"r"(smem_u32(bar)),
            "h"(both)
            : "memory");
    }
}

// The same, arriving on this CTA's barrier only.
template <int CG>
__device__ __forceinline__ void mma_commit_self(uint64_t* bar) {
    if constexpr (CG == 1) {
        mma_commit_all<1>(bar);
    } else {
        asm volatile(
            "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(bar))
            : "memory");
    }
}

// The issuing thread's forms, on shared-memory addresses it keeps in
// registers (no address arithmetic between the instructions).
__device__ __forceinline__ bool mbar_try_wait_u32(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Non-blocking test of a phase (no suspension while it is incomplete).
__device__ __forceinline__ bool mbar_test_wait_u32(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

template <int CG>
__device__ __forceinline__ void mma_commit_all_u32(uint32_t bar) {
    if constexpr (CG == 1) {
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                     : "memory");
    } else {
        const uint16_t both = 3;
        asm volatile(
            "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster"
            ".b64 [%0], %1;" ::"r"(bar),
            "h"(both)
            : "memory");
    }
}

// 32 (or 16) accumulator columns of this lane and their maximum, in one
// tcgen05.ld.red; completed by tmem_wait_ld_max.
__device__ __forceinline__ void tmem_ldmax32_async(uint32_t taddr, uint32_t (&v)[32], float& mx) {
    asm volatile(
        "tcgen05.ld.red.sync.aligned.32x32b.x32.max.f32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
        "%32, [%33];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
          "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
          "=r"(v[31]), "=f"(mx)
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ldmax16_async(uint32_t taddr, uint32_t (&v)[32], float& mx) {
    asm volatile(
        "tcgen05.ld.red.sync.aligned.32x32b.x16.max.f32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, %16, [%17];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=f"(mx)
        : "r"(taddr));
}
// Orders later uses of v and mx after a tcgen05.wait::ld already issued
// (which waits for every load of the thread): no instruction of its own.
__device__ __forceinline__ void tmem_loaded(uint32_t (&v)[32], float& mx) {
    asm volatile(""
        : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]),
          "+r"(v[7]), "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]),
          "+r"(v[13]), "+r"(v[14]), "+r"(v[15]), "+r"(v[16]), "+r"(v[17]), "+r"(v[18]),
          "+r"(v[19]), "+r"(v[20]), "+r"(v[21]), "+r"(v[22]), "+r"(v[23]), "+r"(v[24]),
          "+r"(v[25]), "+r"(v[26]), "+r"(v[27]), "+r"(v[28]), "+r"(v[29]), "+r"(v[30]),
          "+r"(v[31]), "+f"(mx)
        :
        : "memory");
}
__device__ __forceinline__ void tmem_wait_ld_max(uint32_t (&v)[32], float& mx) {
    asm volatile(
        "tcgen05.wait::ld.sync.aligned;"
        : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]),
          "+r"(v[7]), "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]),
          "+r"(v[13]), "+r"(v[14]), "+r"(v[15]), "+r"(v[16]), "+r"(v[17]), "+r"(v[18]),
          "+r"(v[19]), "+r"(v[20]), "+r"(v[21]), "+r"(v[22]), "+r"(v[23]), "+r"(v[24]),
          "+r"(v[25]), "+r"(v[26]), "+r"(v[27]), "+r"(v[28]), "+r"(v[29]), "+r"(v[30]),
          "+r"(v[31]), "+f"(mx)
        :
        : "memory");
}

// ---- CTA-pair helpers (cluster of two) ----------------------------------
__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// shared::cluster address of the same shared-memory location in CTA `rank`.
__device__ __forceinline__ uint32_t peer_addr(const void* p, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
    return r;
}

// Arrival on a barrier of either CTA of the pair.  Release at CTA scope
// (the default) suffices: the only data it publishes are TMEM reads, which
// tcgen05.fence::before_thread_sync orders; a cluster-scope release would
// wait for every outstanding memory operation of the thread.
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar_cluster) {
    asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster) : "memory");
}

__device__ __forceinline__ void st_cluster_u32(uint32_t addr_cluster, uint32_t v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(addr_cluster), "r"(v) : "memory");
}

// Every thread of both CTAs: all shared-memory and barrier operations issued
// before are visible to the other CTA after.
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// 2-D tiled load into this CTA's shared memory, its bytes counted on the
// barrier at shared::cluster address `bar_cluster`, which may be in the
// other CTA of the pair.
__device__ __forceinline__ void tma_load_2d_pair(void* dst, const CUtensorMap* map,
                                                 uint32_t bar_cluster, int32_t c0, int32_t c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar_cluster), "r"(c0), "r"(c1)
        : "memory");
}

// Small batches (at most 128 queries, qa = 128) are spread over the lanes of
// all epilogue warps (and both CTAs of a pair) instead of filling the first
// lanes of one tile: query i sits in CTA i % CG, lane m = 32 (j % 4) + j / 4
// with j = i / CG.  The inverse maps a lane back to its query.
__host__ __device__ __forceinline__ int64_t lane_of_query(int64_t i, int cg) {
    const int64_t j = i / cg;
    return (i % cg) * 128 + (j % 4) * 32 + j / 4;
}
__device__ __forceinline__ int64_t query_of_lane(int m, int rank, int cg) {
    const int j = (m & 31) * 4 + (m >> 5);
    return (int64_t)j * cg + rank;
}

// 4-ary max-heap of u32 keys, element i of thread m at h[i * qa + m] (qa =
// active queries per tile); the children of i are 4i + 1 .. 4i + 4.  Half
// the depth of a binary heap: a sift-down is a chain of about four
// dependent shared-memory rounds (the four child loads are independent)
// instead of seven for the 100 keys of a typical k.
__device__ __forceinline__ void heap_sift_down(uint32_t* h, int qa, int m, int n, int i) {
    const uint32_t v = h[i * qa + m];
    while (true) {
        const int c = 4 * i + 1;
        if (c >= n) break;
        uint32_t cv = h[c * qa + m];
        int best = c;
#pragma unroll
        for (int u = 1; u < 4; ++u) {
            if (c + u < n) {
                const uint32_t x = h[(c + u) * qa + m];
                if (x > cv) {
                    cv = x;
                    best = c + u;
                }
            }
        }
        if (cv <= v) break;
        h[i * qa + m] = cv;
        i = best;
    }
    h[i * qa + m] = v;
}

__device__ __forceinline__ void heap_push(uint32_t* h, int qa, int m, int n, uint32_t key) {
    int i = n;
    while (i > 0) {
        const int p = (i - 1) >> 2;
        const uint32_t pv = h[p * qa + m];
        if (pv >= key) break;
        h[i * qa + m] = pv;
        i = p;
    }
    h[i * qa + m] = key;
}

// MULTI = false: one batch, arguments a and maps tmA/tmB.  MULTI = true:
// the items of every batch of `multi`; a supplies only the status word.
template <int CG, bool MULTI>
__global__ void __launch_bounds__(NUM_THREADS, 1)
scan_mma_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                const __grid_constant__ MmaArgs a, const MmaMulti* __restrict__ multi) {
    using C = MmaCfg<CG>;
    constexpr int STAGE_BYTES = C::STAGE_BYTES;
    // database stages (launch-wide: the stage ring runs on across items)
    const int nst = a.nstages;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw_addr = smem_u32(smem_raw);
    uint8_t* smem = smem_raw + (((raw_addr + 1023u) & ~1023u) - raw_addr);
    uint8_t* qtile = smem;  // the item's query rows, [a_chunks][128 rows][128 B], swizzled
    uint8_t* stages = smem + a.a_chunks * A_STAGE_BYTES;
    uint32_t* heap = reinterpret_cast<uint32_t*>(smem + POOL_BYTES);
    uint32_t* staging = reinterpret_cast<uint32_t*>(smem + POOL_BYTES + HEAP_BYTES);
    uint64_t* ubound = reinterpret_cast<uint64_t*>(smem + POOL_BYTES + HEAP_BYTES +
                                                   STAGING_BYTES);  // [MMA_M]: item << 32 | T
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + POOL_BYTES + HEAP_BYTES +
                                                 STAGING_BYTES + UBOUND_BYTES);
    uint64_t* full = bars;                       // [MAX_STAGES]
    uint64_t* empty = bars + MAX_STAGES;         // [MAX_STAGES]
    uint64_t* acc_full = bars + 2 * MAX_STAGES;            // [NACC]
    uint64_t* acc_empty = bars + 2 * MAX_STAGES + NACC;    // [NACC]
    uint64_t* done = bars + 2 * MAX_STAGES + 2 * NACC;     // [1]
    uint64_t* q_full = done + 1;    // [1] the item's query tile landed
    uint64_t* q_empty = done + 2;   // [1] the item's MMAs completed
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 3);
    int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
    int* cur_item = abort_flag + 1;   // item the epilogue is on
    int* epi_done = abort_flag + 2;   // epilogue finished (helper stops)
    int* fills = abort_flag + 3;      // stage fills this CTA's producer issued
    int* peer_fills = abort_flag + 4; // CG = 2: the same count of the other CTA
    int* qfills = abort_flag + 5;     // query tiles this CTA's producer loaded
    int* peer_qfills = abort_flag + 6;
    static_assert((2 * MAX_STAGES + 2 * NACC + 3) * 8 + 4 + 7 * 4 <= 256, "barriers and flags");

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // CTA pair: rank 0 issues the MMAs; both run every other role.
    const uint32_t rank = CG == 2 ? cluster_ctarank() : 0u;
    const bool leader = rank == 0;
    const int worker = (int)blockIdx.x / CG, nworkers = (int)gridDim.x / CG;
    const int nitems = MULTI ? multi->nitems : ((a.qtiles + CG - 1) / CG) * a.nslices;
    // Work item -> (batch, query unit, database slice); this CTA takes query
    // tile unit * CG + rank.  Consecutive items share a slice, so the CTAs of
    // one wave that work on the same slice read its rows from L2 rather than
    // HBM.
    struct Item {
        int b, qt, slice, ntiles;
        int64_t row0, row_end;
    };
    // (the address of a __grid_constant__ parameter is valid for the whole kernel)
    const MmaArgs* const a_param = &a;
    auto args_of = [&](int b) -> const MmaArgs& {
        if constexpr (MULTI) return multi->args[b];
        else return *a_param;
    };
    auto item_of = [&](int item) {
        Item w;
        w.b = 0;
        int li = item;
        if constexpr (MULTI) {
            int lo = 0, hi = multi->nbatches - 1;  // last batch with item0 <= item
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (multi->item0[mid] <= item) lo = mid;
                else hi = mid - 1;
            }
            w.b = lo;
            li = item - multi->item0[lo];
        }
        const MmaArgs& A = args_of(w.b);
        const int units = (A.qtiles + CG - 1) / CG;  // query tiles (CG = 1) or tile pairs per slice
        w.qt = (li % units) * CG + (int)rank;
        w.slice = li / units;
        w.row0 = (int64_t)w.slice * A.rows_per_slice;
        w.row_end = min(w.row0 + A.rows_per_slice, A.ns);
        w.ntiles = w.row_end > w.row0 ? (int)((w.row_end - w.row0 + MMA_N - 1) / MMA_N) : 0;
        return w;
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < nst; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < NACC; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], CG * EPI_WARPS);  // one arrival per epilogue warp
        }
        mbar_init(done, 1);
        mbar_init(q_full, 1);
        mbar_init(q_empty, 1);
        *abort_flag = 0;
        *cur_item = -1;
        *epi_done = 0;
        *fills = 0;
        *peer_fills = 0;
        *qfills = 0;
        *peer_qfills = 0;
        fence_mbar_init();
    }
    for (int i = threadIdx.x; i < MMA_M; i += NUM_THREADS) ubound[i] = ~0ull;
    if (warp == 1) {
        // CG = 2: one warp of each CTA of the pair allocates, collectively
        if constexpr (CG == 1) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(tmem_slot)),
                         "r"(TMEM_COLS)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        } else {
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(tmem_slot)),
                         "r"(TMEM_COLS)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
        }
    }
    tc_fence_before();
    __syncthreads();
    if constexpr (CG == 2) cluster_sync_all();  // the peer's barriers are initialised
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    // unit scale factors (ue8m0 2^0) in columns 480-511 of every lane, before any MMA
    if (warp >= 2 && warp < 2 + EPI_WARPS)
        tmem_fill32(tmem_base + ((uint32_t)((warp & 3) * 32) << 16) + SF_COL, 0x7F7F7F7Fu);
    tc_fence_before();
    __syncthreads();
    if constexpr (CG == 2) cluster_sync_all();  // both CTAs' scale factors are written
    tc_fence_after();
    // Raise the abort flag here and, for a pair, in the other CTA.
    auto raise_abort = [&]() {
        *(volatile int*)abort_flag = 1;
        if constexpr (CG == 2) st_cluster_u32(peer_addr(abort_flag, rank ^ 1u), 1u);
    };

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            // CG = 2: both CTAs' copies are counted on the leader's
            // barriers, which expect the bytes of the pair.
            int it = 0, s = 0, qi = 0;
            uint32_t ph = 0;
            bool ok = true;
            for (int item = worker; item < nitems && ok; item += nworkers, ++qi) {
                const Item w = item_of(item);
                const MmaArgs& a = args_of(w.b);
                const int kchunks = a.kchunks;
                const CUtensorMap* mapA = &tmA;
                const CUtensorMap* mapB = &tmB;
                if constexpr (MULTI) {
                    mapA = &multi->mapA[w.b];
                    mapB = &multi->mapB[w.b];
                }
                // a tile past the last query (odd tile count) loads tile 0; its rows are ignored
                const int32_t arow = w.qt < a.qtiles ? w.qt * a.qa : 0;
                // the item's query tile, once the previous item's MMAs have
                // read theirs
                if (!mbar_wait_or_abort(q_empty, (uint32_t)(qi & 1) ^ 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                const uint32_t qbytes = (uint32_t)(kchunks * A_STAGE_BYTES);
                if constexpr (CG == 1) {
                    mbar_arrive_expect_tx(q_full, qbytes);
                    for (int kc = 0; kc < kchunks; ++kc)
                        tma_load_2d(qtile + kc * A_STAGE_BYTES, mapA, q_full, kc * KCHUNK, arow);
                } else {
                    if (leader) mbar_arrive_expect_tx(q_full, 2 * qbytes);
                    const uint32_t qb = peer_addr(q_full, 0u);
                    for (int kc = 0; kc < kchunks; ++kc)
                        tma_load_2d_pair(qtile + kc * A_STAGE_BYTES, mapA, qb, kc * KCHUNK, arow);
                }
                *qfills = qi + 1;
                for (int t = 0; t < w.ntiles && ok; ++t) {
                    const int32_t brow = (int32_t)(w.row0 + (int64_t)t * MMA_N + rank * C::B_ROWS);
                    for (int kc = 0; kc < kchunks; ++kc, ++it) {
                        if (it == a.stall_fills && blockIdx.x == 0) {
                            // testing: a producer that stops issuing copies, so
                            // that the consumers' bounded waits expire
                            const uint64_t t0 = globaltimer_ns();
                            while (!*(volatile int*)abort_flag &&
                                   globaltimer_ns() - t0 < 2 * WAIT_LIMIT_NS)
                                __nanosleep(1000);
                            ok = false;
                            break;
                        }
                        if (!mbar_wait_or_abort(&empty[s], ph ^ 1u, abort_flag)) {
                            ok = false;
                            break;
                        }
                        uint8_t* st = stages + s * STAGE_BYTES;
                        if constexpr (CG == 1) {
                            mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
                            tma_load_2d(st, mapB, &full[s], kc * KCHUNK, brow);
                        } else {
                            if (leader) mbar_arrive_expect_tx(&full[s], 2 * STAGE_BYTES);
                            tma_load_2d_pair(st, mapB, peer_addr(&full[s], 0u), kc * KCHUNK, brow);
                        }
                        if (++s == nst) {
                            s = 0;
                            ph ^= 1u;
                        }
                    }
                }
            }
            if (ok) {
                // the MMAs have read every stage filled (and, for a pair, the
                // leader's releases of them have all arrived here)
                for (int j = max(0, it - nst); j < it && ok; ++j)
                    ok = mbar_wait_or_abort(&empty[j % nst], (uint32_t)((j / nst) & 1),
                                            abort_flag);
            }
            if (!ok) {
                if (!*(volatile int*)abort_flag) report(a.status, EVP_ERR_TIMEOUT);
                raise_abort();
            }
            *fills = it;
        }
    } else if (warp == 1) {
        if (lane == 0 && leader) {
            // ---------------- MMA issuer ----------------
            // CG = 2: the shared-memory descriptors name this CTA's stage;
            // the instruction reads the same offsets in the peer CTA (and
            // the scale factors at the same TMEM columns).
            const uint32_t sfa = tmem_base + SF_COL, sfb = tmem_base + SF_COL + 8u;
            // Ring positions kept as the values the instructions take: the
            // stage's barrier addresses and B descriptor, the accumulator's
            // TMEM address and barrier addresses (a descriptor's start
            // address is its low field, so offsets add to it directly).
            const uint32_t full0 = smem_u32(full), empty0 = smem_u32(empty);
            const uint32_t accf0 = smem_u32(acc_full), acce0 = smem_u32(acc_empty);
            const uint64_t adesc0 = sw128_desc(smem_u32(qtile)), bdesc0 = sw128_desc(smem_u32(stages));
            constexpr uint64_t A_CHUNK16 = A_STAGE_BYTES >> 4, B_STAGE16 = STAGE_BYTES >> 4;
            constexpr uint64_t KSTEP16 = KSTEP >> 4;
            int s = 0, ab = 0, qi = 0;
            uint32_t ph = 0, aph = 0;  // stage and accumulator ring phases
            uint32_t fb = full0, eb = empty0, afb = accf0, aeb = acce0, dt = tmem_base;
            uint64_t bd = bdesc0;
            bool ok = true;
            // One item's tiles with the chunk loop unrolled for its chunk
            // count: the issuing thread's control flow between MMAs costs
            // tensor time (the probe: a tile of three 4-instruction chunks
            // issued by a run-time loop takes 138 clocks per instruction at
            // N = 240, unrolled 120, the instruction's own), so a tile's
            // MMAs, waits and commits are straight-line code; a wait that is
            // not already complete goes to the bounded slow path.
            // The tensor pipe queues only a few instructions, so the issuing
            // thread's own work between a chunk's instructions (a barrier
            // test costs ~90 clocks) idles it unless that work overlaps
            // queued instructions: the barrier of the next chunk (and, in a
            // tile's last chunk, the next accumulator's) is tested between
            // the chunk's second and third instructions, without blocking;
            // only a test that failed is followed by a (bounded) wait, after
            // the chunk's commit.
            auto issue_item = [&](auto kch_c, int ntiles) {
                constexpr int KCH = decltype(kch_c)::value;
                constexpr int KSTEPS = KCHUNK / KSTEP;
                static_assert(KSTEPS == 4, "two instructions on either side of the look-ahead");
                if (!mbar_wait_or_abort(q_full, (uint32_t)(qi & 1), abort_flag)) return false;
                if (ntiles > 0) {
                    if (!mbar_try_wait_u32(aeb, aph ^ 1u) &&
                        !mbar_wait_or_abort(&acc_empty[ab], aph ^ 1u, abort_flag))
                        return false;
                    if (!mbar_try_wait_u32(fb, ph) && !mbar_wait_or_abort(&full[s], ph, abort_flag))
                        return false;
                    tc_fence_after();
                }
                for (int t = 0; t < ntiles; ++t) {
                    const bool more = t + 1 < ntiles;
                    bool acc_ready = true;  // the next tile's accumulator, tested in the last chunk
                    const bool awrap = ab + 1 == NACC;
                    const uint32_t naeb = awrap ? acce0 : aeb + 8u;
                    const uint32_t naph = aph ^ (awrap ? 1u : 0u);
#pragma unroll
                    for (int kc = 0; kc < KCH; ++kc) {
                        const bool next = kc + 1 < KCH || more;  // a chunk follows in this item
                        const bool wrap = s + 1 == nst;
                        const uint32_t nfb = wrap ? full0 : fb + 8u;
                        const uint32_t nph = ph ^ (wrap ? 1u : 0u);
                        const uint64_t a = adesc0 + (uint64_t)kc * A_CHUNK16;
                        mma_f4<CG>(dt, a, bd, sfa, sfb, kc > 0 ? 1u : 0u);
                        mma_f4<CG>(dt, a + KSTEP16, bd + KSTEP16, sfa, sfb, 1u);
                        bool stage_ready = true;
                        if (next) stage_ready = mbar_test_wait_u32(nfb, nph);
                        if (kc == KCH - 1 && more) acc_ready = mbar_test_wait_u32(naeb, naph ^ 1u);
                        mma_f4<CG>(dt, a + 2 * KSTEP16, bd + 2 * KSTEP16, sfa, sfb, 1u);
                        mma_f4<CG>(dt, a + 3 * KSTEP16, bd + 3 * KSTEP16, sfa, sfb, 1u);
                        mma_commit_all_u32<CG>(eb);
                        s = wrap ? 0 : s + 1;
                        ph = nph;
                        fb = nfb;
                        eb = wrap ? empty0 : eb + 8u;
                        bd = wrap ? bdesc0 : bd + B_STAGE16;
                        if (next && !stage_ready && !mbar_wait_or_abort(&full[s], ph, abort_flag))
                            return false;
                        if (kc < KCH - 1) tc_fence_after();
                    }
                    mma_commit_all_u32<CG>(afb);
                    ab = awrap ? 0 : ab + 1;
                    aph = naph;
                    afb = awrap ? accf0 : afb + 8u;
                    aeb = naeb;
                    dt = awrap ? tmem_base : dt + (uint32_t)MMA_N;
                    if (more && !acc_ready && !mbar_wait_or_abort(&acc_empty[ab], aph ^ 1u, abort_flag))
                        return false;
                    tc_fence_after();
                }
                // the query tile is free once the item's MMAs complete
                mma_commit_all<CG>(q_empty);
                ++qi;
                return true;
            };
            static_assert(MMA_KCHUNK_MAX == 4, "chunk counts 1-4 instantiated");
            for (int item = worker; item < nitems && ok; item += nworkers) {
              const Item w = item_of(item);
              switch (args_of(w.b).kchunks) {
                case 1: ok = issue_item(std::integral_constant<int, 1>{}, w.ntiles); break;
                case 2: ok = issue_item(std::integral_constant<int, 2>{}, w.ntiles); break;
                case 3: ok = issue_item(std::integral_constant<int, 3>{}, w.ntiles); break;
                default: ok = issue_item(std::integral_constant<int, 4>{}, w.ntiles); break;
              }
            }
            if (!ok) {
                if (!*(volatile int*)abort_flag) report(a.status, EVP_ERR_TIMEOUT);
                raise_abort();
            }
            // all issued MMAs complete before TMEM is released
            mma_commit_self<CG>(done);
            mbar_wait_bounded(done, 0);
        }
    } else if (warp < 6) {
        // ---------------- epilogue ----------------
        const int quarter = warp & 3;
        const int m = quarter * 32 + lane;  // TMEM lane = query row in the tile
        int ab = 0;        // accumulator ring position and phase (runs on across items)
        uint32_t aph = 0;
        bool ok = true;
        for (int item = worker; item < nitems && ok; item += nworkers) {
        const Item w = item_of(item);
        const MmaArgs& a = args_of(w.b);
        const int k = a.k, nslices = a.nslices;
        const int slice = w.slice, ntiles = w.ntiles;
        const int64_t row0 = w.row0, row_end = w.row_end;
        const int qa = a.qa;
        const int64_t qrow = a.spread ? query_of_lane(m, (int)rank, CG) : (int64_t)w.qt * qa + m;
        const bool valid_q = (a.spread || m < qa) && qrow < a.nq;
        uint32_t* hist = a.hist + (valid_q ? qrow : 0) * (int64_t)a.hist_bins;
        if (warp == 2 && lane == 0) *reinterpret_cast<volatile int*>(cur_item) = item;
        int hs = 0;
        float dtau = -INFINITY;   // own heap root: accept D > dtau (strict: rows arrive in order)
        float dglob = -INFINITY;  // union bound: accept D >= x - uthr
        uint32_t uthr = 0xFFFFFFFFu;     // k-th smallest Delta/2 over all slices' inserted keys
        uint32_t lmin = 0xFFFFFFFFu;     // smallest Delta/2 this thread inserted
        int sc = 0;  // staged candidates of this thread
        // Insert the staged candidates into the heap.  All lanes of the warp
        // flush together, so their heap updates run side by side instead of
        // one lane at a time.  Every inserted key is also counted in the
        // query's Delta/2 histogram shared by all slices.
        auto flush = [&]() {
            const int cmax = __reduce_max_sync(0xffffffffu, sc);
            const uint32_t old_min = lmin;
            for (int i = 0; i < cmax; ++i) {
                if (i < sc) {
                    const uint32_t key = staging[i * MMA_M + m];
                    bool ins = false;
                    if (hs < k) {
                        heap_push(heap, qa, m, hs, key);
                        ++hs;
                        ins = true;
                    } else if (key < heap[m]) {
                        heap[m] = key;
                        heap_sift_down(heap, qa, m, hs, 0);
                        ins = true;
                    }
                    if (ins) {
                        const uint32_t h = key >> LOCAL_BITS;
                        atomicAdd(&hist[h], 1u);
                        lmin = min(lmin, h);
                    }
                }
            }
            if (lmin < old_min) atomicMin(&a.minhalf[qrow], lmin);
            sc = 0;
            if (hs == k) dtau = (float)(a.x - (int)(heap[m] >> LOCAL_BITS));
        };
        for (int t = 0; t < ntiles; ++t) {
            // one lane waits, the warp follows it (keeps the warp converged)
            int got = 1;
            if (lane == 0) got = mbar_wait_or_abort(&acc_full[ab], aph, abort_flag);
            got = __shfl_sync(0xffffffffu, got, 0);
            if (!got) {
                ok = false;
                break;
            }
            tc_fence_after();
            {   // union bound published by the helper warp for this item
                const uint64_t ub = *reinterpret_cast<volatile uint64_t*>(&ubound[m]);
                const uint32_t T = (uint32_t)ub;
                if ((int)(ub >> 32) == item && T < uthr) {
                    uthr = T;
                    dglob = (float)(a.x - (int)uthr) - 0.5f;
                }
            }
            const int64_t tile_row = row0 + (int64_t)t * MMA_N;
            const uint32_t tbase = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(ab * MMA_N);
            // One 32-column group already in registers: stage the lanes'
            // candidates (flushing first if a lane's staging could overflow).
            // mx: the group's maximum, from the load itself.
            auto group = [&](const uint32_t (&v)[32], float mx, int c) {
                float thr = fmaxf(dtau, dglob);
                if (!__any_sync(0xffffffffu, valid_q && mx > thr)) return;
                // maxima of the 8 sub-groups of 4 columns
                float sm[8];
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    sm[i] = fmaxf(fmax3(__uint_as_float(v[4 * i]), __uint_as_float(v[4 * i + 1]),
                                        __uint_as_float(v[4 * i + 2])),
                                  __uint_as_float(v[4 * i + 3]));
                // columns of this group inside the tile and inside the
                // slice (the last tile is ragged)
                const int64_t left = min(row_end - (tile_row + c * 32), (int64_t)(MMA_N - 32 * c));
                const int lim = !valid_q ? 0 : (left >= 32 ? 32 : (left > 0 ? (int)left : 0));
                uint32_t my8 = 0;  // this lane's 4-column sub-groups with a candidate
#pragma unroll
                for (int i = 0; i < 8; ++i) my8 |= (sm[i] > thr && 4 * i < lim) ? 1u << i : 0u;
                // sub-groups in which any lane has a candidate (one reduction
                // instead of a vote per sub-group; still valid after a flush,
                // which only raises the threshold)
                const uint32_t all8 = __reduce_or_sync(0xffffffffu, my8);
                // flush first if this group could overflow a lane's staging
                if (__any_sync(0xffffffffu, sc + 4 * __popc(my8) > STAGE_SLOTS)) {
                    flush();
                    thr = fmaxf(dtau, dglob);
                }
                const uint32_t gbase = (uint32_t)(tile_row + c * 32 - row0);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    if (!((all8 >> i) & 1u)) continue;
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) {
                        const int j = 4 * i + jj;
                        const float dv = __uint_as_float(v[j]);
                        if (dv > thr && j < lim) {
                            // D is an integer below 2^22 in magnitude: adding
                            // 1.5 * 2^23 leaves it in the low mantissa bits
                            const int di = __float_as_int(dv + 12582912.0f) - 0x4B400000;
                            // clamped: a code without exactly x non-zeros must not
                            // index outside the histogram
                            const uint32_t half_delta = (uint32_t)min(max(a.x - di, 0), 2 * a.x);
                            staging[sc * MMA_M + m] = (half_delta << LOCAL_BITS) | (gbase + (uint32_t)j);
                            ++sc;
                        }
                    }
                }
            };
            // The groups' maxima are taken in batches of four loads and one
            // wait (the load latency, not the comparison, dominates a group
            // whose maximum clears nothing); a group in which some lane has
            // a candidate is loaded again and examined from one register
            // buffer.  A last group narrower than 32 columns is loaded 16
            // wide, so that its maximum covers only this tile's columns.
            auto load_group = [&](int c, uint32_t (&v)[32], float& mx) {
                if (MMA_N % 32 != 0 && c == EPI_GROUPS - 1)
                    tmem_ldmax16_async(tbase + (uint32_t)(c * 32), v, mx);
                else
                    tmem_ldmax32_async(tbase + (uint32_t)(c * 32), v, mx);
            };
            static_assert(MMA_N % 32 == 0 || MMA_N % 32 == 16, "last group 16 or 32 wide");
            constexpr int BATCH = 4;
#pragma unroll 1
            for (int c0 = 0; c0 < EPI_GROUPS; c0 += BATCH) {
                uint32_t b0[32], b1[32], b2[32], b3[32];
                float m0 = -INFINITY, m1 = -INFINITY, m2 = -INFINITY, m3 = -INFINITY;
                const int nb = min(BATCH, EPI_GROUPS - c0);  // warp-uniform
                __syncwarp();
                load_group(c0, b0, m0);
                if (nb > 1) load_group(c0 + 1, b1, m1);
                if (nb > 2) load_group(c0 + 2, b2, m2);
                if (nb > 3) load_group(c0 + 3, b3, m3);
                tmem_wait_ld_max(b0, m0);
                tmem_loaded(b1, m1);
                tmem_loaded(b2, m2);
                tmem_loaded(b3, m3);
                const float thr = fmaxf(dtau, dglob);
                const uint32_t flag = !valid_q ? 0u
                                               : (m0 > thr ? 1u : 0u) | (m1 > thr ? 2u : 0u) |
                                                     (m2 > thr ? 4u : 0u) | (m3 > thr ? 8u : 0u);
                uint32_t wflag = __reduce_or_sync(0xffffffffu, flag);
                while (wflag) {
                    const int i = __ffs(wflag) - 1;
                    wflag &= wflag - 1u;
                    uint32_t vx[32];
                    float mx;
                    __syncwarp();
                    load_group(c0 + i, vx, mx);
                    tmem_wait_ld_max(vx, mx);
                    group(vx, mx, c0 + i);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                // accumulator release: the leader's barrier (in the other CTA for rank 1)
                if (CG == 1 || rank == 0) mbar_arrive(&acc_empty[ab]);
                else mbar_arrive_cluster(peer_addr(&acc_empty[ab], 0u));
            }
            {
                const bool awrap = ab + 1 == NACC;
                ab = awrap ? 0 : ab + 1;
                aph ^= awrap ? 1u : 0u;
            }
            // heap updates run after the accumulator is released, overlapping
            // the next tile's MMAs
            if (__any_sync(0xffffffffu, sc > FLUSH_AT)) flush();
        }
        if (!ok) break;
        flush();
        if (valid_q) {
            // heap -> ascending order in place, then the (query, slice) list
            for (int n = hs - 1; n > 0; --n) {
                const uint32_t top = heap[m];
                heap[m] = heap[n * qa + m];
                heap[n * qa + m] = top;
                heap_sift_down(heap, qa, m, n, 0);
            }
            uint64_t* out = a.lists + ((qrow * nslices + slice) * 2) * k;
            uint64_t last = KEY_NONE;
            for (int j = 0; j < hs; ++j) {
                const uint32_t key = heap[j * qa + m];
                last = ((uint64_t)(2u * (key >> LOCAL_BITS)) << 32) |
                       (uint64_t)(row0 + (key & ((1u << LOCAL_BITS) - 1u)));
                out[j] = last;
            }
            int32_t* mt = a.meta + (qrow * nslices + slice) * 2;
            mt[0] = hs;
            mt[1] = 0;
            if (hs == k)
                atomicMin(reinterpret_cast<unsigned long long*>(&a.tau_global[qrow]),
                          (unsigned long long)last);
        }
        }  // item
        if (!ok && lane == 0) {
            if (!*(volatile int*)abort_flag) report(a.status, EVP_ERR_TIMEOUT);
            raise_abort();
        }
        __syncwarp();
        if (warp == 2 && lane == 0) *reinterpret_cast<volatile int*>(epi_done) = 1;
    } else {
        // ---------------- threshold helper ----------------
        // Union bound of each query of the current item: the smallest T with
        // count(Delta/2 <= T) >= k over the keys all slices of the query have
        // inserted (counted in the workspace histogram).  Those are real rows,
        // so no row with Delta/2 > T can be among the k nearest.  Computed
        // here, off the epilogue's critical path, and published in shared
        // memory tagged with the item.
        uint32_t best[MMA_M / 32];
        int seen = -1;
        while (!*reinterpret_cast<volatile int*>(epi_done) &&
               !*reinterpret_cast<volatile int*>(abort_flag)) {
            const int item = *reinterpret_cast<volatile int*>(cur_item);
            if (item < 0) {
                __nanosleep(1000);
                continue;
            }
            if (item != seen) {
#pragma unroll
                for (int j = 0; j < MMA_M / 32; ++j) best[j] = 0xFFFFFFFFu;
                seen = item;
            }
            const Item wi = item_of(item);
            const MmaArgs& a = args_of(wi.b);
            const int qt = wi.qt;
#pragma unroll 1
            for (int j = 0; j < MMA_M / 32; ++j) {
                const int mm = j * 32 + lane;
                const int64_t qrow =
                    a.spread ? query_of_lane(mm, (int)rank, CG) : (int64_t)qt * a.qa + mm;
                if ((!a.spread && mm >= a.qa) || qrow >= a.nq) continue;
                const uint32_t lo = __ldcg(&a.minhalf[qrow]);
                if (lo == 0xFFFFFFFFu) continue;
                const uint32_t* hist = a.hist + qrow * (int64_t)a.hist_bins;
                const uint32_t hi = min(best[j], (uint32_t)(a.hist_bins - 1));
                uint32_t cum = 0;
                bool found = false;
                for (uint32_t h0 = lo; h0 <= hi && !found; h0 += 16) {
                    uint32_t c16[16];
#pragma unroll
                    for (int u = 0; u < 16; ++u) c16[u] = (h0 + u <= hi) ? __ldcg(&hist[h0 + u]) : 0u;
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        cum += c16[u];
                        if (!found && cum >= (uint32_t)a.kunion && h0 + u < best[j]) {
                            best[j] = h0 + u;
                            found = true;
                        }
                    }
                }
                if (found)
                    *reinterpret_cast<volatile uint64_t*>(&ubound[mm]) =
                        ((uint64_t)(uint32_t)item << 32) | best[j];
            }
            // a refresh every ~8 us: more often costs the epilogue more (in
            // issue slots and L2 traffic) than the fresher bound saves
            __nanosleep(8000);
        }
    }

    tc_fence_before();
    __syncthreads();
    if constexpr (CG == 2) {
        // each CTA tells the other how many stage fills and query tiles its
        // producer issued
        if (threadIdx.x == 0) {
            st_cluster_u32(peer_addr(peer_fills, rank ^ 1u), (uint32_t)*fills);
            st_cluster_u32(peer_addr(peer_qfills, rank ^ 1u), (uint32_t)*qfills);
        }
        cluster_sync_all();
    }
    if (*(volatile int*)abort_flag && threadIdx.x == 0 && leader) {
        // After an abort, copies issued into either CTA's stages may still be
        // in flight; every copy of fill j signals the leader's full barrier
        // of stage j % nst.  A fill could only be issued once the fill nst
        // before it had completed, so only the last nst fills of the two
        // producers can be pending: wait (bounded) for each of them, first
        // completing the accounting of a fill that one CTA of the pair
        // issued and the other did not (its expected bytes never come, or
        // its arrival never happened).  The MMA issuer has already waited
        // for every MMA it issued.
        const int own = *fills;
        const int other = CG == 2 ? *peer_fills : own;
        const int hi = max(own, other);
        for (int j = max(0, hi - nst); j < hi; ++j) {
            const int s = j % nst;
            if constexpr (CG == 2) {
                if (j >= own) mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
                else if (j >= other) mbar_complete_tx(&full[s], STAGE_BYTES);
            }
            if (!mbar_wait_bounded(&full[s], (uint32_t)((j / nst) & 1))) break;
        }
        // The same for the query tiles: a producer loads tile j only after
        // the MMAs of item j - 1 completed, which waited for tile j - 1, so
        // only the last one can be pending.
        const int qown = *qfills;
        const int qother = CG == 2 ? *peer_qfills : qown;
        const int qhi = max(qown, qother);
        if (qhi > 0) {
            const int j = qhi - 1;
            const uint32_t qbytes =
                (uint32_t)(args_of(item_of(worker + j * nworkers).b).kchunks * A_STAGE_BYTES);
            if constexpr (CG == 2) {
                if (j >= qown) mbar_arrive_expect_tx(q_full, qbytes);
                else if (j >= qother) mbar_complete_tx(q_full, qbytes);
            }
            mbar_wait_bounded(q_full, (uint32_t)(j & 1));
        }
    }
    __syncthreads();
    if constexpr (CG == 2) cluster_sync_all();  // no copies or arrivals into the peer remain
    tc_fence_after();
    if (warp == 1) {
        if constexpr (CG == 1)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                         "r"(TMEM_COLS)
                         : "memory");
        else
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                         "r"(TMEM_COLS)
                         : "memory");
    }
}

// 32 elements of a code (bits of the + and - planes) -> 16 bytes of e2m1,
// element e in nibble e (+1 -> 0x2, -1 -> 0xA, 0 -> 0; a set + bit wins).
__device__ __forceinline__ uint4 e2m1_pack32(uint32_t pp, uint32_t mm) {
    uint32_t o[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        uint32_t word = 0;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int e = i * 8 + b;
            const uint32_t nib = ((pp >> e) & 1u) ? 0x2u : (((mm >> e) & 1u) ? 0xAu : 0u);
            word |= nib << (4 * b);
        }
        o[i] = word;
    }
    return make_uint4(o[0], o[1], o[2], o[3]);
}

// Packed codes -> e2m1 rows [n][Kp bytes] (Kp a multiple of 128; elements
// >= d are 0).  spread_cg > 0: row i goes to lane_of_query(i, spread_cg)
// instead of i.
__global__ void unpack_fp4_kernel(const uint64_t* __restrict__ T, int64_t n, int W, int Kp,
                                  int spread_cg, uint8_t* __restrict__ out) {
    const int groups = Kp / 16;  // 16 bytes = 32 elements per thread
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t row = idx / groups;
    if (row >= n) return;
    const int g = (int)(idx - row * groups);
    const int j0 = g * 32, w = j0 >> 6, sh = j0 & 63;
    uint32_t p = 0, q = 0;
    if (w < W) {
        p = (uint32_t)(T[row * 2 * W + w] >> sh);
        q = (uint32_t)(T[row * 2 * W + W + w] >> sh);
    }
    const int64_t orow = spread_cg > 0 ? lane_of_query(row, spread_cg) : row;
    reinterpret_cast<uint4*>(out + orow * (int64_t)Kp)[g] = e2m1_pack32(p, q);
}

// ---- exactness of a scan with capped lists ------------------------------
// With k > 128 the scan may keep only kl = 128 keys per (query, slice) list
// (every query lane of a tile then stays active).  The merged result is the
// k best of the lists; it is exact unless some slice holds more than kl of
// the keys below the result's k-th key T.  A slice can do so only if its
// list is full and the list's last key lies below T: those (query, slice)
// pairs are rescanned here, one CTA per query, by popcount on the packed
// codes with the scan's own Delta (2 clamp(x - b2sp, 0, 2x), so the keys
// equal the scan's), keeping the keys between the list's last key and the
// current k-th key; the result is re-selected from its k keys and those
// (block bitonic sort), T tightening as it goes.  Rows are randomly ordered
// with respect to a query, so with the slice counts the capped plan
// requires (at least 2k/kl slices) the rescan is rarely needed; it keeps
// the result exact when it is.
constexpr int RP_THREADS = 256;
constexpr int RP_BUF = 2048;           // keys appended between two selections
constexpr int RP_SORT = 4096;          // >= EVP_MMA_MAX_K + RP_BUF, a power of two
static_assert(MMA_K_MAX + RP_BUF <= RP_SORT, "repair sort buffer");
constexpr int RP_W_MAX = 16;

__device__ void rp_block_sort(uint64_t* b, int n) {
    for (int kk = 2; kk <= n; kk <<= 1)
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n; i += RP_THREADS) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const uint64_t a0 = b[i], a1 = b[ixj];
                    if ((a0 > a1) == ((i & kk) == 0)) {
                        b[i] = a1;
                        b[ixj] = a0;
                    }
                }
            }
            __syncthreads();
        }
}

__global__ void __launch_bounds__(RP_THREADS) repair_capped_kernel(
    const uint64_t* __restrict__ Q, const uint64_t* __restrict__ S, int64_t ns, int W, int x,
    const uint64_t* __restrict__ lists, const int32_t* __restrict__ meta, int nslices, int kl,
    int64_t rows_per_slice, int k, int64_t* __restrict__ ids, int32_t* __restrict__ dist,
    uint32_t* __restrict__ repaired) {
    extern __shared__ __align__(16) uint64_t rp_buf[];  // [RP_SORT]
    __shared__ uint64_t qw[2 * RP_W_MAX];
    __shared__ int cnt, any;
    const int64_t q = blockIdx.x;
    const int tid = threadIdx.x;
    for (int i = tid; i < 2 * W; i += RP_THREADS) qw[i] = Q[q * 2 * W + i];
    // the merged result as keys; T = its k-th key
    for (int i = tid; i < k; i += RP_THREADS) {
        const int64_t id = ids[q * k + i];
        rp_buf[i] = id < 0 ? KEY_NONE : ((uint64_t)(uint32_t)dist[q * k + i] << 32) | (uint64_t)id;
    }
    if (tid == 0) any = 0;
    __syncthreads();
    uint64_t T = rp_buf[k - 1];
    auto last_of = [&](int s, int* len) {
        const int64_t e = (q * nslices + s) * 2;
        *len = min(max(meta[e], 0), kl);
        return *len > 0 ? lists[(e + (meta[e + 1] & 1)) * kl + *len - 1] : 0ull;
    };
    // selection of the k best of rp_buf[0, k + cnt)
    auto select = [&]() {
        const int n = k + cnt;
        int P = 2;
        while (P < n) P <<= 1;
        for (int i = n + tid; i < P; i += RP_THREADS) rp_buf[i] = KEY_NONE;
        __syncthreads();
        rp_block_sort(rp_buf, P);
        T = rp_buf[k - 1];
        __syncthreads();
        if (tid == 0) cnt = 0;
        __syncthreads();
    };
    for (int s = 0; s < nslices; ++s) {
        int len;
        const uint64_t lo = last_of(s, &len);
        if (len < kl || (T != KEY_NONE && lo >= T)) continue;  // the list holds all its keys below T
        if (tid == 0) {
            cnt = 0;
            any = 1;
        }
        __syncthreads();
        const int64_t r0 = (int64_t)s * rows_per_slice;
        const int64_t r1 = min(r0 + rows_per_slice, ns);
        for (int64_t b0 = r0; b0 < r1; b0 += RP_THREADS) {
            const int64_t row = b0 + tid;
            if (row < r1) {
                const uint64_t* sr = S + row * 2 * W;
                int dot = 0;
                for (int w = 0; w < W; ++w) {
                    const uint64_t sp = sr[w], sm = sr[W + w];
                    dot += __popcll(qw[w] & sp) + __popcll(qw[W + w] & sm) -
                           __popcll(qw[w] & sm) - __popcll(qw[W + w] & sp);
                }
                const uint32_t half = (uint32_t)min(max(x - dot, 0), 2 * x);
                const uint64_t key = ((uint64_t)(2u * half) << 32) | (uint64_t)row;
                if (key > lo && key < T) rp_buf[k + atomicAdd(&cnt, 1)] = key;
            }
            __syncthreads();
            if (cnt > RP_BUF - RP_THREADS) select();  // the next round adds <= RP_THREADS
        }
        if (cnt > 0) select();
    }
    if (!any) return;
    for (int j = tid; j < k; j += RP_THREADS) {
        const uint64_t key = rp_buf[j];
        ids[q * k + j] = key == KEY_NONE ? -1 : (int64_t)(key & 0xffffffffull);
        dist[q * k + j] = key == KEY_NONE ? -1 : (int32_t)(key >> 32);
    }
    if (tid == 0 && repaired) atomicAdd(repaired, 1u);
}

__global__ void init_tau_n_kernel(uint64_t* tau, int n, uint32_t* hist, int64_t hist_words,
                                  uint32_t* minhalf) {
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = i0; i < n; i += stride) {
        tau[i] = KEY_NONE;
        minhalf[i] = 0xFFFFFFFFu;
    }
    for (int64_t i = i0; i < hist_words; i += stride) hist[i] = 0u;
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

// Bytes per row of the e2m1 operand copies: d elements, two per byte, padded
// to whole 128-byte K chunks.
int mma_kp(int d) { return (d + 2 * KCHUNK - 1) / (2 * KCHUNK) * KCHUNK; }

// Queries served per 128-row tile: all 128 while their heaps fit
// (k <= 128); for larger k fewer queries share the tile (the other rows of
// the tile are computed and ignored), so that active queries x k <= 128^2.
int mma_active_queries(int k) {
    int qa = MMA_M;
    while (qa > 16 && qa * k > HEAP_SLOTS) qa >>= 1;
    return qa;
}

// CTA pairs the device can keep resident at once (0: pairs unavailable, or
// single CTAs requested with EVP_MMA_CTA_PAIR=0 in the environment).
int mma_pair_workers() {
    const char* env = std::getenv("EVP_MMA_CTA_PAIR");
    if (env && env[0] == '0') return 0;
    static int cached[64];
    static bool known[64] = {false};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 0;
    }
    if (!known[dev]) {
        int n = 0;
        if (cudaFuncSetAttribute(scan_mma_kernel<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)MmaCfg<2>::SMEM_BYTES) == cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = 2;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3(2 * (unsigned)num_sms());
            cfg.blockDim = dim3(NUM_THREADS);
            cfg.dynamicSmemBytes = MmaCfg<2>::SMEM_BYTES;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            if (cudaOccupancyMaxActiveClusters(&n, scan_mma_kernel<2, false>, &cfg) != cudaSuccess) n = 0;
        }
        cudaGetLastError();
        cached[dev] = std::max(0, n);
        known[dev] = true;
    }
    return cached[dev];
}

MmaPlan plan_mma_scan(int64_t nq, int64_t ns, int d, int k, bool convert_db,
                      int tiles_per_item, bool allow_cap) {
    // kl keys per (query, slice) list and heap
    auto build = [&](int kl) {
        MmaPlan p{};
        p.kp = mma_kp(d);
        p.kl = kl;
        p.qa = mma_active_queries(kl);
        p.qtiles = (int)((nq + p.qa - 1) / p.qa);
        const int pairs = mma_pair_workers();
        p.cg = pairs > 0 ? 2 : 1;
        p.workers = pairs > 0 ? pairs : num_sms();
        // a single tile's worth of queries is spread over every epilogue warp
        // (and both CTAs of a pair), so that no warp carries all the candidates
        p.spread = p.qa == MMA_M && nq <= MMA_M;
        if (p.spread) p.qtiles = p.cg;
        const int units = (p.qtiles + p.cg - 1) / p.cg;
        const int64_t ntiles = (ns + MMA_N - 1) / MMA_N;
        const int64_t min_slices = (ns + MAX_SLICE_ROWS - 1) / MAX_SLICE_ROWS;
        // units * slices a multiple of the resident workers (whole waves of the
        // persistent grid), at least min_slices, at most one slice per tile
        const int64_t sms = p.workers;
        int64_t g = sms, b = std::max(1, units);
        while (b) {
            const int64_t r = g % b;
            g = b;
            b = r;
        }
        const int64_t step = sms / g;
        int64_t slices = step;
        while (slices < min_slices) slices += step;
        // a given tile shape (the fused multi-batch scan): slices of about
        // tiles_per_item database tiles each
        if (tiles_per_item > 0)
            slices = std::max(min_slices, (ntiles + tiles_per_item - 1) / tiles_per_item);
        slices = std::min(slices, std::max<int64_t>(1, ntiles));
        const int64_t tiles_per_slice = (ntiles + slices - 1) / slices;
        p.rows_per_slice = tiles_per_slice * MMA_N;
        p.nslices = (int)((ns + p.rows_per_slice - 1) / p.rows_per_slice);
        p.a_bytes = align256((size_t)p.qtiles * MMA_M * p.kp);
        p.b_bytes = convert_db ? align256((size_t)ns * p.kp) : 0;
        p.list_bytes = align256((size_t)nq * p.nslices * 2 * kl * 8);
        p.meta_bytes = align256((size_t)nq * p.nslices * 2 * 4);
        p.tau_bytes = align256((size_t)nq * 8);
        p.hist_bytes = align256((size_t)nq * (2 * d + 1) * 4) + align256((size_t)nq * 4);
        p.ws_bytes = p.a_bytes + p.b_bytes + p.list_bytes + p.meta_bytes + p.tau_bytes +
                     p.hist_bytes;
        return p;
    };
    // Capped lists: each slice keeps its kl best keys, kl the smallest power
    // of two >= 16 with kl x nslices >= 4k (a slice holds k / nslices of a
    // query's k nearest on average; the repair pass rescans the rare slice
    // that may have held more).  A smaller heap settles its threshold on
    // fewer rows and is cheaper to update, which is most of the scan's
    // epilogue work while the thresholds are loose.
    if (allow_cap && tiles_per_item == 0) {
        const MmaPlan c = build(std::min(k, MMA_M));  // slicing does not depend on kl <= 128
        int kl = 16;
        while (kl < MMA_M && (int64_t)kl * c.nslices < 4 * (int64_t)k) kl *= 2;
        if (kl < k && (int64_t)c.nslices * (kl / 2) >= k) return build(kl);
    }
    return build(k);
}

cudaError_t launch_unpack_fp4(const uint64_t* T, int64_t n, int d, uint8_t* out,
                              cudaStream_t stream, int spread_cg) {
    if (n <= 0) return cudaSuccess;
    const int W = (d + 63) / 64, Kp = mma_kp(d);
    const int64_t threads = n * (Kp / 16);
    TimedLaunch timer("unpack_fp4", stream);
    unpack_fp4_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, stream>>>(T, n, W, Kp,
                                                                               spread_cg, out);
    return cudaGetLastError();
}

int32_t run_mma_knn(const uint64_t* Q, int64_t nq, const uint8_t* S8, const uint64_t* S,
                    int64_t ns, int d, int x, int k, int64_t* ids, int32_t* dist, void* ws,
                    size_t ws_bytes, int32_t* status, cudaStream_t stream) {
    if (k > MMA_K_MAX) return EVP_ERR_UNSUPPORTED;
    const MmaPlan p = plan_mma_scan(nq, ns, d, k, S8 == nullptr, 0, S != nullptr);
    if (ws_bytes < p.ws_bytes) return EVP_ERR_NO_MEMORY;
    uint8_t* w = static_cast<uint8_t*>(ws);
    uint8_t* A8 = w;
    uint8_t* B8 = S8 ? const_cast<uint8_t*>(S8) : w + p.a_bytes;
    uint64_t* lists = reinterpret_cast<uint64_t*>(w + p.a_bytes + p.b_bytes);
    int32_t* meta = reinterpret_cast<int32_t*>(w + p.a_bytes + p.b_bytes + p.list_bytes);
    uint64_t* tau = reinterpret_cast<uint64_t*>(w + p.a_bytes + p.b_bytes + p.list_bytes +
                                                p.meta_bytes);
    uint32_t* hist = reinterpret_cast<uint32_t*>(reinterpret_cast<uint8_t*>(tau) + p.tau_bytes);
    const int hist_bins = 2 * x + 1;
    uint32_t* minhalf = reinterpret_cast<uint32_t*>(
        reinterpret_cast<uint8_t*>(hist) + align256((size_t)nq * (2 * d + 1) * 4));
    if ((reinterpret_cast<uintptr_t>(B8) & 255) != 0) return EVP_ERR_INVALID;

    if (p.spread && cudaMemsetAsync(A8, 0, p.a_bytes, stream) != cudaSuccess) return EVP_ERR_CUDA;
    if (launch_unpack_fp4(Q, nq, d, A8, stream, p.spread ? p.cg : 0) != cudaSuccess)
        return EVP_ERR_CUDA;
    if (!S8 && launch_unpack_fp4(S, ns, d, B8, stream) != cudaSuccess) return EVP_ERR_CUDA;
    {
        TimedLaunch timer("scan_init", stream);
        const int64_t hw = nq * (int64_t)hist_bins;
        const int64_t blocks = std::min<int64_t>((hw + 255) / 256, (int64_t)num_sms() * 8);
        init_tau_n_kernel<<<(unsigned)std::max<int64_t>(1, blocks), 256, 0, stream>>>(
            tau, (int)nq, hist, hw, minhalf);
    }

    EncodeTiledFn enc = encode_tiled_fn();
    if (!enc) return EVP_ERR_CUDA;
    CUtensorMap tmA, tmB;
    cuuint64_t gdimA[2] = {(cuuint64_t)p.kp, (cuuint64_t)(p.spread ? p.qtiles * MMA_M : nq)};
    cuuint64_t gdimB[2] = {(cuuint64_t)p.kp, (cuuint64_t)ns};
    cuuint64_t gstride[1] = {(cuuint64_t)p.kp};
    cuuint32_t boxA[2] = {(cuuint32_t)KCHUNK, (cuuint32_t)MMA_M};
    cuuint32_t boxB[2] = {(cuuint32_t)KCHUNK, (cuuint32_t)(MMA_N / p.cg)};
    cuuint32_t es[2] = {1, 1};
    if (enc(&tmA, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, A8, gdimA, gstride, boxA, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return EVP_ERR_CUDA;
    if (enc(&tmB, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, B8, gdimB, gstride, boxB, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return EVP_ERR_CUDA;

    MmaArgs args{};
    args.nq = (int)nq;
    args.ns = ns;
    args.kchunks = p.kp / KCHUNK;
    args.x = x;
    args.k = p.kl;
    args.kunion = k;
    args.rows_per_slice = p.rows_per_slice;
    args.qtiles = p.qtiles;
    args.qa = p.qa;
    args.spread = p.spread ? 1 : 0;
    args.nslices = p.nslices;
    args.lists = lists;
    args.meta = meta;
    args.tau_global = tau;
    args.hist = hist;
    args.minhalf = minhalf;
    args.hist_bins = hist_bins;
    args.status = status;
    args.stall_fills = take_stall_mma();
    args.a_chunks = args.kchunks;
    args.nstages = p.cg == 1 ? MmaCfg<1>::stages_for(args.a_chunks) : MmaCfg<2>::stages_for(args.a_chunks);
    const int items = (p.qtiles + p.cg - 1) / p.cg * p.nslices;
    if (p.cg == 1) {
        if (cudaFuncSetAttribute(scan_mma_kernel<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)MmaCfg<1>::SMEM_BYTES) != cudaSuccess)
            return EVP_ERR_CUDA;
        TimedLaunch timer("scan_mma", stream);
        scan_mma_kernel<1, false><<<std::min(items, p.workers), NUM_THREADS, MmaCfg<1>::SMEM_BYTES,
                                    stream>>>(tmA, tmB, args, nullptr);
    } else {
        // attribute already set by mma_pair_workers
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(2 * (unsigned)std::min(items, p.workers));
        cfg.blockDim = dim3(NUM_THREADS);
        cfg.dynamicSmemBytes = MmaCfg<2>::SMEM_BYTES;
        cfg.stream = stream;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        TimedLaunch timer("scan_mma", stream);
        if (cudaLaunchKernelEx(&cfg, scan_mma_kernel<2, false>, tmA, tmB, args,
                               static_cast<const MmaMulti*>(nullptr)) != cudaSuccess)
            return EVP_ERR_CUDA;
    }
    if (cudaGetLastError() != cudaSuccess) return EVP_ERR_CUDA;
    const int32_t rc = launch_final_merge(lists, meta, tau, hist, minhalf, hist_bins, nq,
                                          p.nslices, k, ids, dist, stream, -1, 0, p.kl);
    if (rc != EVP_OK || p.kl >= k) return rc;
    // capped lists: the exactness check and, where a slice may have left out
    // keys, its rescan
    TimedLaunch timer("scan_repair", stream);
    repair_capped_kernel<<<(unsigned)nq, RP_THREADS, RP_SORT * 8, stream>>>(
        Q, S, ns, (d + 63) / 64, x, lists, meta, p.nslices, p.kl, p.rows_per_slice, k, ids, dist,
        nullptr);
    return cudaGetLastError() == cudaSuccess ? EVP_OK : EVP_ERR_CUDA;
}


// ---- fused multi-batch scan -------------------------------------------------
namespace {

struct PrepBatch {
    const uint64_t* Q;    // packed query codes [nq][2W]
    int64_t nq, rows;     // queries, and rows of the e2m1 query operand written
    int W, Kp, spread_cg;
    uint8_t* A8;          // [rows][Kp bytes] e2m1 query operand
    uint64_t* tau;        // [nq]
    uint32_t* minhalf;    // [nq]
    uint32_t* hist;       // [hist_words]
    int64_t hist_words;
};

// One launch prepares every batch (blockIdx.y = batch): each row of the
// query operand is written once -- the unpacked query whose lane it is, or
// zeros for an unused lane of a spread batch -- and the thresholds, minima
// and histograms of the union bound start empty.
__global__ void multi_prep_kernel(const PrepBatch* __restrict__ tab) {
    const PrepBatch& p = tab[blockIdx.y];
    const int groups = p.Kp / 16;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t idx = i0; idx < p.rows * groups; idx += stride) {
        const int64_t R = idx / groups;
        const int g = (int)(idx - R * groups);
        const int64_t q = p.spread_cg > 0 ? query_of_lane((int)(R & 127), (int)(R >> 7), p.spread_cg) : R;
        const int j0 = g * 32, w = j0 >> 6, sh = j0 & 63;
        uint32_t pp = 0, mm = 0;
        if (q < p.nq && w < p.W) {
            pp = (uint32_t)(p.Q[q * 2 * p.W + w] >> sh);
            mm = (uint32_t)(p.Q[q * 2 * p.W + p.W + w] >> sh);
        }
        reinterpret_cast<uint4*>(p.A8 + R * (int64_t)p.Kp)[g] = e2m1_pack32(pp, mm);
    }
    for (int64_t i = i0; i < p.nq; i += stride) {
        p.tau[i] = KEY_NONE;
        p.minhalf[i] = 0xFFFFFFFFu;
    }
    for (int64_t i = i0; i < p.hist_words; i += stride) p.hist[i] = 0u;
}

struct MultiLayout {
    MmaPlan p;
    uint8_t* A8;
    uint64_t* lists;
    int32_t* meta;
    uint64_t* tau;
    uint32_t* hist;
    uint32_t* minhalf;
};

MultiLayout multi_layout(const MmaBatchSpec& b, int tiles_per_item) {
    MultiLayout L;
    L.p = plan_mma_scan(b.nq, b.ns, b.d, b.k, false, tiles_per_item);
    uint8_t* w = static_cast<uint8_t*>(b.ws);
    L.A8 = w;
    L.lists = reinterpret_cast<uint64_t*>(w + L.p.a_bytes);
    L.meta = reinterpret_cast<int32_t*>(w + L.p.a_bytes + L.p.list_bytes);
    L.tau = reinterpret_cast<uint64_t*>(w + L.p.a_bytes + L.p.list_bytes + L.p.meta_bytes);
    L.hist = reinterpret_cast<uint32_t*>(reinterpret_cast<uint8_t*>(L.tau) + L.p.tau_bytes);
    L.minhalf = reinterpret_cast<uint32_t*>(reinterpret_cast<uint8_t*>(L.hist) +
                                            align256((size_t)b.nq * (2 * b.d + 1) * 4));
    return L;
}

}  // namespace

struct MmaMultiPlan {
    int nb = 0, cg = 1, workers = 0;
    int a_chunks = 1;  // the largest chunk count of the batches
    int64_t total_q = 0;
    size_t fm_smem = 0;
    MmaMulti* table = nullptr;   // device
    PrepBatch* prep = nullptr;   // device [nb]
    FmBatch* fm = nullptr;       // device [nb + 1]
    int max_rows_groups = 0;
    int32_t* status_slot = nullptr;
};

size_t mma_multi_ws(int64_t nq, int64_t ns, int d, int k, int tiles_per_item) {
    return plan_mma_scan(nq, ns, d, k, false, tiles_per_item).ws_bytes;
}

int32_t mma_multi_create(const MmaBatchSpec* specs, int nb, MmaMultiPlan** out) {
    *out = nullptr;
    if (nb < 1 || nb > MMA_MULTI_MAX) return EVP_ERR_UNSUPPORTED;
    EncodeTiledFn enc = encode_tiled_fn();
    if (!enc) return EVP_ERR_CUDA;
    MmaMulti* h = new (std::nothrow) MmaMulti();
    if (!h) return EVP_ERR_NO_MEMORY;
    std::vector<PrepBatch> prep(nb);
    std::vector<FmBatch> fm(nb + 1);
    MmaMultiPlan* P = new (std::nothrow) MmaMultiPlan();
    if (!P) {
        delete h;
        return EVP_ERR_NO_MEMORY;
    }
    int items = 0;
    size_t fm_smem = 0;
    int64_t q0 = 0;
    int32_t rc = EVP_OK;
    for (int b = 0; b < nb && rc == EVP_OK; ++b) {
        const MmaBatchSpec& B = specs[b];
        if (!B.Q || B.nq < 1 || !B.S8 || B.k < 1 || B.k > MMA_K_MAX || !B.ids || !B.dist || !B.ws ||
            (reinterpret_cast<uintptr_t>(B.S8) & 255) != 0) {
            rc = EVP_ERR_INVALID;
            break;
        }
        const MultiLayout L = multi_layout(B, B.tiles_per_item);
        const MmaPlan& p = L.p;
        if (b == 0) {
            P->cg = p.cg;
            P->workers = p.workers;
        }
        const int64_t arows = p.spread ? (int64_t)p.qtiles * MMA_M : B.nq;
        CUtensorMap* tmA = &h->mapA[b];
        CUtensorMap* tmB = &h->mapB[b];
        cuuint64_t gdimA[2] = {(cuuint64_t)p.kp, (cuuint64_t)arows};
        cuuint64_t gdimB[2] = {(cuuint64_t)p.kp, (cuuint64_t)B.ns};
        cuuint64_t gstride[1] = {(cuuint64_t)p.kp};
        cuuint32_t boxA[2] = {(cuuint32_t)KCHUNK, (cuuint32_t)MMA_M};
        cuuint32_t boxB[2] = {(cuuint32_t)KCHUNK, (cuuint32_t)(MMA_N / p.cg)};
        cuuint32_t es[2] = {1, 1};
        if (enc(tmA, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, L.A8, gdimA, gstride, boxA, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
            enc(tmB, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t*>(B.S8), gdimB, gstride,
                boxB, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
            rc = EVP_ERR_CUDA;
            break;
        }
        MmaArgs& A = h->args[b];
        A = MmaArgs{};
        A.nq = (int)B.nq;
        A.ns = B.ns;
        A.kchunks = p.kp / KCHUNK;
        P->a_chunks = std::max(P->a_chunks, A.kchunks);
        A.x = B.x;
        A.k = B.k;
        A.kunion = B.k;
        A.rows_per_slice = p.rows_per_slice;
        A.qtiles = p.qtiles;
        A.qa = p.qa;
        A.spread = p.spread ? 1 : 0;
        A.nslices = p.nslices;
        A.lists = L.lists;
        A.meta = L.meta;
        A.tau_global = L.tau;
        A.hist = L.hist;
        A.minhalf = L.minhalf;
        A.hist_bins = 2 * B.x + 1;
        A.status = nullptr;
        A.stall_fills = -1;
        h->item0[b] = items;
        items += (p.qtiles + p.cg - 1) / p.cg * p.nslices;
        prep[b] = PrepBatch{B.Q, B.nq, arows, (B.d + 63) / 64, p.kp, p.spread ? p.cg : 0, L.A8,
                            L.tau, L.minhalf, L.hist, B.nq * (int64_t)A.hist_bins};
        int stage = 0;
        fm_smem = std::max(fm_smem, final_merge_smem(p.nslices, B.k, &stage));
        fm[b] = FmBatch{L.lists, L.meta, L.tau, L.hist, L.minhalf, A.hist_bins, p.nslices, B.k,
                        B.k, stage, q0, B.ids, B.dist};
        q0 += B.nq;
        P->max_rows_groups = std::max<int>(P->max_rows_groups, (int)std::min<int64_t>(
                                               arows * (p.kp / 16), 1 << 30));
    }
    if (rc == EVP_OK) {
        h->item0[nb] = items;
        h->nbatches = nb;
        h->nitems = items;
        fm[nb] = FmBatch{};
        fm[nb].q0 = q0;
        P->nb = nb;
        P->total_q = q0;
        P->fm_smem = fm_smem;
        if (cudaMalloc(&P->table, sizeof(MmaMulti)) != cudaSuccess ||
            cudaMalloc(&P->prep, sizeof(PrepBatch) * nb) != cudaSuccess ||
            cudaMalloc(&P->fm, sizeof(FmBatch) * (nb + 1)) != cudaSuccess) {
            cudaGetLastError();
            rc = EVP_ERR_NO_MEMORY;
        } else if (cudaMemcpy(P->table, h, sizeof(MmaMulti), cudaMemcpyHostToDevice) != cudaSuccess ||
                   cudaMemcpy(P->prep, prep.data(), sizeof(PrepBatch) * nb,
                              cudaMemcpyHostToDevice) != cudaSuccess ||
                   cudaMemcpy(P->fm, fm.data(), sizeof(FmBatch) * (nb + 1),
                              cudaMemcpyHostToDevice) != cudaSuccess) {
            rc = EVP_ERR_CUDA;
        }
    }
    delete h;
    if (rc != EVP_OK) {
        mma_multi_destroy(P);
        return rc;
    }
    *out = P;
    return EVP_OK;
}

int32_t mma_multi_run(MmaMultiPlan* P, int32_t* status, cudaStream_t stream) {
    if (!P) return EVP_ERR_INVALID;
    {
        TimedLaunch timer("unpack_fp4", stream);
        const int64_t bx = std::min<int64_t>((P->max_rows_groups + 255) / 256, (int64_t)num_sms() * 4);
        multi_prep_kernel<<<dim3((unsigned)std::max<int64_t>(1, bx), (unsigned)P->nb), 256, 0,
                            stream>>>(P->prep);
        if (cudaGetLastError() != cudaSuccess) return EVP_ERR_CUDA;
    }
    MmaArgs a{};      // the launch's status word (the table's arguments hold the rest)
    a.status = status;
    a.stall_fills = -1;
    a.a_chunks = P->a_chunks;
    a.nstages = P->cg == 1 ? MmaCfg<1>::stages_for(a.a_chunks) : MmaCfg<2>::stages_for(a.a_chunks);
    CUtensorMap dummy;
    std::memset(&dummy, 0, sizeof(dummy));
    if (P->cg == 1) {
        if (cudaFuncSetAttribute(scan_mma_kernel<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)MmaCfg<1>::SMEM_BYTES) != cudaSuccess)
            return EVP_ERR_CUDA;
        TimedLaunch timer("scan_mma", stream);
        scan_mma_kernel<1, true><<<P->workers, NUM_THREADS, MmaCfg<1>::SMEM_BYTES, stream>>>(
            dummy, dummy, a, P->table);
    } else {
        if (cudaFuncSetAttribute(scan_mma_kernel<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)MmaCfg<2>::SMEM_BYTES) != cudaSuccess)
            return EVP_ERR_CUDA;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(2 * (unsigned)P->workers);
        cfg.blockDim = dim3(NUM_THREADS);
        cfg.dynamicSmemBytes = MmaCfg<2>::SMEM_BYTES;
        cfg.stream = stream;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        TimedLaunch timer("scan_mma", stream);
        if (cudaLaunchKernelEx(&cfg, scan_mma_kernel<2, true>, dummy, dummy, a,
                               static_cast<const MmaMulti*>(P->table)) != cudaSuccess)
            return EVP_ERR_CUDA;
    }
    if (cudaGetLastError() != cudaSuccess) return EVP_ERR_CUDA;
    return launch_final_merge_multi(P->fm, P->nb, P->total_q, P->fm_smem, stream);
}

void mma_multi_destroy(MmaMultiPlan* P) {
    if (!P) return;
    if (P->table) cudaFree(P->table);
    if (P->prep) cudaFree(P->prep);
    if (P->fm) cudaFree(P->fm);
    delete P;
}

}  // namespace evp
