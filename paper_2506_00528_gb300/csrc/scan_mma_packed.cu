// ternary_knn, packed tensor-core path: the exhaustive scan of Sec. 5.3 as
// a dense contraction on the tensor cores (tcgen05, kind::f8f6f4) that
// reads the packed 2-bit codes straight from HBM and unpacks each tile on
// chip, for batches of up to 64 queries per pass.
//
// D = S Q^T with the database tile as the M side (128 rows = the 128 TMEM
// lanes) and the pass's queries as the N side (16, 32 or 64):
//   * database element of a code: +1 -> e4m3 0x40 (+2), -1 -> 0xC0 (-2),
//     0 -> 0x00; query element: +1 -> 0x38 (+1), -1 -> 0xB8 (-1).  Every
//     product is 0 or +-2 and float32 accumulation of at most 2d of them is
//     exact, so D = 2 b2sp (Sec. 5.1.2) and Delta = 2x - D for codes with
//     x non-zeros each;
//   * the K order of both operands is the same permutation of the
//     dimensions (a scalar product does not depend on the order of its
//     terms): within each 32-dimension half of a 64-bit word, K position
//     4j + b (j = 0..7, b = 0..3) holds dimension 8b + j.  Then the four
//     bytes of one 32-bit TMEM column are bits j, 8 + j, 16 + j and 24 + j
//     of the two bitplanes, and a column is two shifts and masks of a word
//     in which the non-zero bit of each dimension sits next to its sign bit.
//
// Kernel (one CTA per SM, persistent over a contiguous slice of 128-row
// tiles, 608 threads in five roles that meet only at mbarriers):
//   warp 17     TMA producer: tiles of packed rows (box 2W + 2 words wide,
//               the padding words read as 0 so that 16-byte row reads are
//               bank-conflict free) through a ring of mbarrier stages;
//   warps 0-7   unpack, two threads per database row (TMEM lane): each
//               copies its half of the row's 16-byte word pairs out of the
//               stage, releases the stage and writes the unpacked e4m3
//               columns with tcgen05.st into one of two A buffers (192
//               columns each) once the MMAs have read it;
//   warp 16     allocates the 512 TMEM columns and issues the MMAs from one
//               thread: A (the unpacked tile) from TMEM, B (the queries)
//               from shared memory (SWIZZLE_128B, written once at start),
//               D into one of two accumulators (QN columns each), one
//               commit per tile;
//   warps 8-15  epilogue, two threads per row (each half of the queries):
//               each warp reads its rows' accumulator columns and appends
//               rows that beat a query's threshold to candidate buffers of
//               its own, which it merges (bitonic sort + merge path) into
//               sorted lists of the k best of its own in the workspace (one
//               list per query and row quadrant of the CTA), so epilogue
//               warps never wait for one another;
//   warp 18     union-bound helper: per query, the k-th smallest Delta/2
//               over every row any list has taken, from a histogram in the
//               workspace that all CTAs share; the epilogue warps fold it
//               (and the other lists' thresholds) into their own.
// The per-query final merge of the popcount path combines the lists.
// Every mbarrier wait is bounded (2 s): on expiry the CTA reports
// EVP_ERR_TIMEOUT, raises its abort flag (every other wait then gives up at
// once), waits for the copies and MMAs it issued and frees TMEM.
#include "evp_internal.cuh"

#include <cuda_fp8.h>

#include <algorithm>
#include <type_traits>

namespace evp {

namespace {

constexpr int PK_ROWS = 128;                         // database rows per tile = TMEM lanes
constexpr int PK_UNPACK_WARPS = 8;                   // warps 0-7: two threads per row
constexpr int PK_EPI_WARP0 = 8;                      // warps 8-15: two threads per row
constexpr int PK_EPI_WARPS = 8;
constexpr int PK_LISTS_PER_CTA = 4;                  // one slice list per row quadrant
constexpr int PK_MMA_WARP = 16;
constexpr int PK_TMA_WARP = 17;
constexpr int PK_HELPER_WARP = 18;
constexpr int PK_THREADS = 19 * 32;
constexpr int PK_STAGE_LIST_K = 128;                 // merges stage the list in shared memory up to this k
constexpr int PK_K_MAX = 256;                        // largest k of this path
constexpr int PK_QN_MAX = 64;                        // queries per pass
constexpr int PK_W_MAX = 12;                         // words per bitplane: d <= 768
constexpr int PK_CAP = 64;                           // candidate slots per (epilogue warp, query)
constexpr int PK_MERGE_AT = PK_CAP - 32;             // merge at this count: a tile adds <= 32
constexpr int PK_LOCAL_BITS = 20;                    // row-in-slice bits of a candidate key
constexpr int64_t PK_MAX_TILES_PER_SLICE = (int64_t(1) << PK_LOCAL_BITS) / PK_ROWS;
constexpr int PK_MAX_STAGES = 6;
constexpr int PK_MIN_STAGES = 2;
constexpr int PK_SMEM_LIMIT = 232448;                // opt-in shared memory per block
constexpr uint32_t PK_TMEM_COLS = 512;
constexpr int PK_A_COLS = 16 * PK_W_MAX;             // 192: one unpacked tile (768 K bytes)
constexpr int PK_D_COL0 = 2 * PK_A_COLS;             // accumulators after the two A buffers
constexpr int PK_MAX_SLICES = 1024;                  // lists the final merge takes per query
static_assert(PK_D_COL0 + 2 * PK_QN_MAX <= (int)PK_TMEM_COLS, "TMEM columns");

struct PkArgs {
    const uint64_t* Q;     // this pass's query codes [nqg][2W]
    int nqg;
    int64_t ns;
    int W;                 // words per bitplane (even, <= PK_W_MAX)
    int x, k;
    int pitch;             // uint64 words per staged row (2W + 2)
    int stages;
    int64_t tiles_per_slice, ntiles;
    uint64_t* lists;       // [PK_QN_MAX][4 * CTAs][2][k]: one list per (query, CTA, row quadrant)
    int32_t* meta;         // [PK_QN_MAX][4 * CTAs][2]: (length, current buffer)
    uint64_t* tau_global;  // [PK_QN_MAX]
    uint32_t* hist;        // [PK_QN_MAX][hist_bins]
    uint32_t* minhalf;     // [PK_QN_MAX]
    int hist_bins;         // 2x + 1
    int32_t* status;
    int stall_fills;  // testing: CTA 0's producer stops after this many fills (-1: never)
    // int8-query mode (MODE 1): the pass's queries [nqg][d], the score key
    // bias - score (bias = 127 x >= every score) and the histogram bin shift
    const int8_t* Q8;
    int d;
    int bias;
    int hshift;
};

__host__ __device__ inline size_t pk_align(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct PkLayout {
    size_t stage_bytes, b_off, cand_off, scratch_off, tau_off, thr_off, ub_off, cnt_off, bar_off,
        misc_off, total;
};

// Per-(epilogue warp, query) state: warp e (0-7) serves the rows of
// quadrant e % 4 against queries [(e / 4) qn/2, (e / 4 + 1) qn/2); its
// entry j is at index e * qn/2 + j of each array.

// Shared-memory carve-up (offsets from a 1024-byte aligned base; `total`
// includes the alignment slack of the dynamic allocation).
// mode 1 (int8 queries) stages two query operands and 64-bit candidates.
__host__ __device__ inline PkLayout pk_layout(int W, int stages, int qn, int mode = 0) {
    PkLayout L;
    L.stage_bytes = pk_align((size_t)PK_ROWS * (2 * W + 2) * 8, 1024);
    L.b_off = L.stage_bytes * stages;
    const size_t states = (size_t)PK_EPI_WARPS * (qn / 2);
    // mode 0: ceil(W/4) K-chunks of qn x 128 B (e2m1, 256 elements a chunk);
    // mode 1: two operands of W/2 K-chunks (e4m3, 128 elements a chunk)
    L.cand_off = L.b_off + (mode ? (size_t)(W / 2) * qn * 128 * 2 : (size_t)((W + 3) / 4) * qn * 128);
    L.scratch_off = L.cand_off + states * PK_CAP * (mode ? 8 : 4);  // one staged list per epilogue warp
    L.tau_off = L.scratch_off + (size_t)PK_EPI_WARPS * PK_STAGE_LIST_K * 8;
    L.thr_off = L.tau_off + states * 8;
    L.ub_off = L.thr_off + states * 4;
    L.cnt_off = L.ub_off + (size_t)qn * 4;
    L.bar_off = pk_align(L.cnt_off + 4 * states * 4, 8);
    L.misc_off = L.bar_off + (size_t)(2 * stages + 7) * 8;
    L.total = L.misc_off + 16 + 1024;
    return L;
}

// Instruction descriptor: D = f32, A = B = e4m3, both K-major, M = 128, N = qn.
__host__ __device__ constexpr uint32_t pk_idesc(int qn) {
    return (1u << 4) | ((uint32_t)(qn >> 3) << 17) | ((uint32_t)(PK_ROWS >> 4) << 24);
}

// Block-scaled fp4 (kind::mxf4): A = B = e2m1 (format 1), both K-major,
// ue8m0 scale factors (bit 23), M = 128, N = qn.
__host__ __device__ constexpr uint32_t pk_idesc_f4(int qn) {
    return (1u << 7) | (1u << 10) | ((uint32_t)(qn >> 3) << 17) | (1u << 23) |
           ((uint32_t)(PK_ROWS >> 4) << 24);
}

// D (TMEM) += A (TMEM) * B (shared memory descriptor), e2m1 operands with
// the scale factors at TMEM addresses sfa, sfb.
__device__ __forceinline__ void mma_f4_tmem_a(uint32_t dtmem, uint32_t atmem, uint64_t bdesc,
                                              uint32_t idesc, uint32_t sfa, uint32_t sfb,
                                              uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %6, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], [%1], %2, %3, [%4], "
        "[%5], p;\n\t}" ::"r"(dtmem),
        "r"(atmem), "l"(bdesc), "r"(idesc), "r"(sfa), "r"(sfb), "r"(accumulate)
        : "memory");
}

// D (TMEM) += A (TMEM) * B (shared memory descriptor).
__device__ __forceinline__ void mma_f8_tmem_a(uint32_t dtmem, uint32_t atmem, uint64_t bdesc,
                                              uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n\t}" ::"r"(dtmem),
        "r"(atmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

// Store 16 consecutive 32-bit columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
        "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
        "r"(v[15])
        : "memory");
}

// Store 32 consecutive 32-bit columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
        "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(
            taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
        "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
        "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]),
        "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]),
        "r"(v[29]), "r"(v[30]), "r"(v[31])
        : "memory");
}

__device__ __forceinline__ void tmem_wait_st() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Load N (8, 16 or 32) consecutive 32-bit columns of this warp's lanes and
// wait for them.
template <int N>
__device__ __forceinline__ void tmem_ld_wait(uint32_t taddr, uint32_t (&v)[N]) {
    if constexpr (N == 32) {
        tmem_ld32_async(taddr, v);
        tmem_wait_ld(v);
    } else if constexpr (N == 16) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
            "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n\t"
            "tcgen05.wait::ld.sync.aligned;"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
              "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
              "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr)
            : "memory");
    } else {
        static_assert(N == 8, "8, 16 or 32 columns");
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t"
            "tcgen05.wait::ld.sync.aligned;"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
              "=r"(v[6]), "=r"(v[7])
            : "r"(taddr)
            : "memory");
    }
}

// TMEM columns of one 64-bit word pair of the bitplanes (64 dimensions per
// word, 16 columns each; see the K order above).  nz = v+ | v-, ng = v-.
// The database byte of a dimension is (nz << 6) | (ng << 7).
__device__ __forceinline__ void unpack_half(uint32_t nz, uint32_t ng, uint32_t* o) {
    constexpr uint32_t M = 0xC0C0C0C0u;
    const uint32_t rng = __funnelshift_l(ng, ng, 1);  // sign of dimension i at bit i + 1
    const uint32_t xe = (nz & 0x55555555u) | (rng & 0xAAAAAAAAu);
    const uint32_t xo = (nz & 0xAAAAAAAAu) | (rng & 0x55555555u);
    o[0] = (xe << 6) & M;
    o[1] = (xo << 5) & M;
    o[2] = (xe << 4) & M;
    o[3] = (xo << 3) & M;
    o[4] = (xe << 2) & M;
    o[5] = (xo << 1) & M;
    o[6] = xe & M;
    o[7] = __funnelshift_r(xo, xo, 1) & M;
}

__device__ __forceinline__ void unpack_word(uint64_t p, uint64_t m, uint32_t* o) {
    const uint64_t nz = p | m;
    unpack_half((uint32_t)nz, (uint32_t)m, o);
    unpack_half((uint32_t)(nz >> 32), (uint32_t)(m >> 32), o + 8);
}

// e2m1 TMEM columns of one 64-bit word pair (64 dimensions, 8 columns of 8
// nibbles).  The database element is +2 (0x4) or -2 (0xC): nibble bit 2 =
// non-zero, bit 3 = sign.  K order: column 4h + c (h = the word's 32-bit
// half), nibble i holds dimension 32h + c + 4i, so a column is two shifts
// and masks of each plane.
__device__ __forceinline__ void unpack_word_f4(uint64_t p, uint64_t m, uint32_t* o) {
    const uint64_t nz = p | m;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const uint32_t z = (uint32_t)(nz >> (32 * h)), g = (uint32_t)(m >> (32 * h));
#pragma unroll
        for (int c = 0; c < 4; ++c)
            o[4 * h + c] = (((z >> c) & 0x11111111u) << 2) | (((g >> c) & 0x11111111u) << 3);
    }
}

// Candidate key -> list key.  Mode 0: (Delta/2 << 20 | row - row0), a
// uint32, -> (Delta << 32 | row).  Mode 1: (score key << 20 | row - row0), a
// uint64, -> (score key << 32 | row).
template <int MODE, typename CandT>
__device__ __forceinline__ uint64_t pk_key64(CandT c, int64_t row0) {
    const uint64_t v = (uint64_t)(c >> PK_LOCAL_BITS);
    return ((MODE == 0 ? 2u * v : v) << 32) |
           (uint64_t)(row0 + (int64_t)(c & (CandT)((1u << PK_LOCAL_BITS) - 1u)));
}

template <int MODE, typename CandT>
__device__ __forceinline__ int lower_bound_cand(const CandT* C, int n, uint64_t key,
                                                int64_t row0) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (pk_key64<MODE>(C[mid], row0) < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Ascending bitonic sort of buf[0, P) (P a power of two) by one warp.
template <typename T>
__device__ __forceinline__ void warp_sort(T* buf, int P, int lane) {
    for (int kk = 2; kk <= P; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < P; i += 32) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const T x0 = buf[i], x1 = buf[ixj];
                    if ((x0 > x1) == ((i & kk) == 0)) {
                        buf[i] = x1;
                        buf[ixj] = x0;
                    }
                }
            }
            __syncwarp();
        }
    }
}

// Admission threshold on D for a query threshold key tau = (Delta << 32 |
// row): D > thr admits exactly Delta <= Delta(tau) (the exact key test
// follows on the rare candidates).  No threshold yet: -2^22, below every D
// and small enough that D - thr stays exact in float32.
// Mode 1: D = 2 score (even), and D > thr admits exactly the score keys
// bias - score <= the key of tau.
constexpr float PK_ADMIT_ALL = -4194304.0f;
template <int MODE>
__device__ __forceinline__ float pk_thr(uint64_t tau, int x, int bias) {
    if (tau == KEY_NONE) return PK_ADMIT_ALL;
    if (MODE == 0) return (float)(2 * x - (int)(tau >> 32)) - 0.5f;
    return (float)(2 * (bias - (int)(tau >> 32))) - 1.0f;
}

// List key bounding every key counted in histogram bins 0..T (the union
// bound): bins are Delta/2 (mode 0) or score key >> hshift (mode 1).
template <int MODE>
__device__ __forceinline__ uint64_t pk_bin_key(uint32_t T, int hshift) {
    if (MODE == 0) return (uint64_t)(2u * T + 1u) << 32;
    return ((uint64_t)(T + 1u) << hshift) << 32;
}

// MODE 0: packed query codes (ternary), Delta keys.  MODE 1: int8 queries,
// each split as q = 16 hi + lo with hi in [-8, 8] and lo in [-8, 7] (both
// exact in e4m3, 16 hi too), contracted as two operands into the same
// accumulator: D = 2 <q, s>, the masked-addition score of Sec. 5.1.2 times
// two, exact in float32.
template <int QN, int MODE>
__global__ void __launch_bounds__(PK_THREADS, 1)
scan_mma_packed_kernel(const __grid_constant__ CUtensorMap tmap, const PkArgs a) {
    using CandT = std::conditional_t<MODE == 0, uint32_t, uint64_t>;
    // mode 0: e2m1 operands (kind::mxf4, unit scale factors, K = 64 a step);
    // mode 1: e4m3 (kind::f8f6f4, K = 32 a step; the split int8 query parts
    // need e4m3's range)
    constexpr bool F4 = MODE == 0;
    constexpr uint32_t IDESC = F4 ? pk_idesc_f4(QN) : pk_idesc(QN);
    constexpr int ACOLS = F4 ? 8 * PK_W_MAX : PK_A_COLS;   // TMEM columns of one A buffer
    constexpr int DCOL0 = 2 * ACOLS;                        // accumulators after the A buffers
    constexpr uint32_t SFCOL = DCOL0 + 2 * PK_QN_MAX;       // mode 0: scale factors (32 columns)
    static_assert(!F4 || SFCOL + 32 <= PK_TMEM_COLS, "TMEM columns");
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw_addr = smem_u32(smem_raw);
    uint8_t* smem = smem_raw + (((raw_addr + 1023u) & ~1023u) - raw_addr);
    const int W = a.W, k = a.k, x = a.x, S = a.stages;
    const PkLayout L = pk_layout(W, S, QN, MODE);
    uint8_t* stages = smem;
    uint8_t* qop = smem + L.b_off;  // query operand, W/2 chunks of QN x 128 B
    constexpr int QH = QN / 2;  // queries per epilogue warp
    constexpr int NSTATE = PK_EPI_WARPS * QH;
    CandT* cand = reinterpret_cast<CandT*>(smem + L.cand_off);         // [NSTATE][PK_CAP]
    uint64_t* scratch = reinterpret_cast<uint64_t*>(smem + L.scratch_off);
    uint64_t* tau = reinterpret_cast<uint64_t*>(smem + L.tau_off);     // [NSTATE] thresholds
    float* thr_s = reinterpret_cast<float*>(smem + L.thr_off);         // [NSTATE] on D
    uint32_t* ub = reinterpret_cast<uint32_t*>(smem + L.ub_off);       // [QN] union bounds
    int* cnt = reinterpret_cast<int*>(smem + L.cnt_off);               // [NSTATE] candidates
    int* len = cnt + NSTATE;                                           // [NSTATE] list lengths
    int* cur = len + NSTATE;                                           // [NSTATE] list buffers
    uint32_t* lmin = reinterpret_cast<uint32_t*>(cur + NSTATE);        // [NSTATE] least Delta/2
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar_off);
    uint64_t* full = bars;                 // [S]  TMA -> unpack warps
    uint64_t* empty = bars + S;            // [S]  unpack warps -> TMA
    uint64_t* a_full = bars + 2 * S;       // [2]  unpack warps -> MMA (A buffer written)
    uint64_t* d_full = bars + 2 * S + 2;   // [2]  MMA -> epilogue and unpack warps (tile's
                                           //      MMAs complete: accumulator ready, A read)
    uint64_t* d_empty = bars + 2 * S + 4;  // [2]  epilogue -> MMA (accumulator read)
    uint64_t* done = bars + 2 * S + 6;     // [1]  every MMA issued has completed
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L.misc_off);
    int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
    int* epi_done = abort_flag + 1;        // epilogue warps finished (the helper stops at 8)

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nslices = gridDim.x, slice = blockIdx.x;
    const int64_t tile0 = (int64_t)slice * a.tiles_per_slice;
    const int64_t tile_end = min(tile0 + a.tiles_per_slice, a.ntiles);
    const int ntl = tile_end > tile0 ? (int)(tile_end - tile0) : 0;
    const int64_t row0 = tile0 * PK_ROWS;
    const int npairs = W / 2;
    const int ksteps = F4 ? W : 2 * W;  // K = 64 W elements: 64 per e2m1 step, 32 per e4m3 step
    const uint32_t tile_bytes = (uint32_t)(PK_ROWS * a.pitch * 8);

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], PK_UNPACK_WARPS);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&a_full[b], PK_UNPACK_WARPS);
            mbar_init(&d_full[b], 1);
            mbar_init(&d_empty[b], PK_EPI_WARPS);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        *epi_done = 0;
        fence_mbar_init();
    }
    // Query operand: 16-byte units of K-major SWIZZLE_128B rows (the 16-byte
    // unit u of row n of a 128-byte chunk sits at unit u ^ (n % 8)).
    if constexpr (F4) {
        // mode 0: e2m1 nibbles, +1 = 0x2, -1 = 0xA, 32 elements a 16-byte
        // unit; K position 64 w + 32 h + 8 c + i holds dimension
        // 64 w + 32 h + c + 4 i (the database's column order)
        const int units_per_row = 8 * ((W + 3) / 4);  // whole 128-byte chunks
        for (int i = tid; i < QN * units_per_row; i += PK_THREADS) {
            const int n = i / units_per_row, ku = i - n * units_per_row;
            const int kb0 = ku * 32;  // first K element of the unit
            uint32_t o[4] = {0u, 0u, 0u, 0u};
            const int w = kb0 >> 6;
            if (n < a.nqg && w < W) {
                const uint64_t p = a.Q[(int64_t)n * 2 * W + w];
                const uint64_t m = a.Q[(int64_t)n * 2 * W + W + w];
                const int h = (kb0 >> 5) & 1;
#pragma unroll
                for (int e = 0; e < 32; ++e) {
                    const int bit = 32 * h + (e >> 3) + 4 * (e & 7);
                    const uint32_t nib = ((p >> bit) & 1u) ? 0x2u : (((m >> bit) & 1u) ? 0xAu : 0u);
                    o[e >> 3] |= nib << (4 * (e & 7));
                }
            }
            const int c = kb0 >> 8, uc = (kb0 & 255) >> 5;
            uint8_t* dst = qop + (size_t)c * QN * 128 + (n >> 3) * 1024 + (n & 7) * 128 +
                           ((uc ^ (n & 7)) << 4);
            *reinterpret_cast<uint4*>(dst) = make_uint4(o[0], o[1], o[2], o[3]);
        }
        fence_proxy_async_smem();  // generic-proxy writes read by the tensor core
    } else {
        const int units_per_row = 4 * W;  // 64 W bytes / 16
        for (int i = tid; i < QN * units_per_row; i += PK_THREADS) {
            const int n = i / units_per_row, ku = i - n * units_per_row;
            const int kb0 = ku * 16;
            uint32_t o[4] = {0u, 0u, 0u, 0u}, o2[4] = {0u, 0u, 0u, 0u};
            if (n < a.nqg) {
                const int w = kb0 >> 6;
                if constexpr (MODE == 0) {
                    const uint64_t p = a.Q[(int64_t)n * 2 * W + w];
                    const uint64_t m = a.Q[(int64_t)n * 2 * W + W + w];
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const int s = (kb0 & 63) + e;  // K position within the word
                        const int bit = 32 * (s >> 5) + 8 * (s & 3) + ((s & 31) >> 2);
                        const uint32_t byte =
                            ((p >> bit) & 1u) ? 0x38u : (((m >> bit) & 1u) ? 0xB8u : 0u);
                        o[e >> 2] |= byte << (8 * (e & 3));
                    }
                } else {
                    const int8_t* q8 = a.Q8 + (int64_t)n * a.d;
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const int s = (kb0 & 63) + e;  // K position within the word
                        const int dim = 64 * w + 32 * (s >> 5) + 8 * (s & 3) + ((s & 31) >> 2);
                        const int v = dim < a.d ? (int)q8[dim] : 0;
                        const int hi = (v + 8) >> 4, lo = v - 16 * hi;
                        const uint32_t bh = __nv_cvt_float_to_fp8((float)(16 * hi), __NV_SATFINITE, __NV_E4M3);
                        const uint32_t bl = __nv_cvt_float_to_fp8((float)lo, __NV_SATFINITE, __NV_E4M3);
                        o[e >> 2] |= bh << (8 * (e & 3));
                        o2[e >> 2] |= bl << (8 * (e & 3));
                    }
                }
            }
            const int c = kb0 >> 7, uc = (kb0 & 127) >> 4;
            uint8_t* dst = qop + (size_t)c * QN * 128 + (n >> 3) * 1024 + (n & 7) * 128 +
                           ((uc ^ (n & 7)) << 4);
            *reinterpret_cast<uint4*>(dst) = make_uint4(o[0], o[1], o[2], o[3]);
            if constexpr (MODE == 1)   // the lo operand follows the hi one
                *reinterpret_cast<uint4*>(dst + (size_t)(W / 2) * QN * 128) =
                    make_uint4(o2[0], o2[1], o2[2], o2[3]);
        }
        fence_proxy_async_smem();  // generic-proxy writes read by the tensor core
    }
    for (int i = tid; i < NSTATE; i += PK_THREADS) {
        const int q = (i / QH >> 2) * QH + i % QH;
        tau[i] = KEY_NONE;
        thr_s[i] = q < a.nqg ? PK_ADMIT_ALL : INFINITY;  // padding queries never admit
        cnt[i] = 0;
        len[i] = 0;
        cur[i] = 0;
        lmin[i] = 0xFFFFFFFFu;
    }
    if (tid < QN) ub[tid] = 0xFFFFFFFFu;
    if (warp == PK_MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(PK_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    auto give_up = [&]() {
        if (!*(volatile int*)abort_flag) report(a.status, EVP_ERR_TIMEOUT);
        *(volatile int*)abort_flag = 1;
    };

    if (warp == PK_TMA_WARP) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            bool ok = true;
            int t = 0;
            for (; t < ntl; ++t) {
                const int s = t % S;
                if (t == a.stall_fills && blockIdx.x == 0) {
                    // testing: a producer that stops issuing copies, so that
                    // the consumers' bounded waits expire
                    const uint64_t t0 = globaltimer_ns();
                    while (!*(volatile int*)abort_flag && globaltimer_ns() - t0 < 2 * WAIT_LIMIT_NS)
                        __nanosleep(1000);
                    ok = false;
                    break;
                }
                if (t >= S &&
                    !mbar_wait_or_abort(&empty[s], (uint32_t)(((t / S) - 1) & 1), abort_flag)) {
                    ok = false;
                    break;
                }
                mbar_arrive_expect_tx(&full[s], tile_bytes);
                tma_load_2d(stages + (size_t)s * L.stage_bytes, &tmap, &full[s], 0,
                            (int32_t)((tile0 + t) * PK_ROWS));
            }
            // every copy issued has landed before the CTA can exit: the last
            // S stages' releases (or, after an abort, their arrivals)
            for (int j = max(0, t - S); j < t; ++j) {
                const int s = j % S;
                if (ok) ok = mbar_wait_or_abort(&empty[s], (uint32_t)((j / S) & 1), abort_flag);
                if (!ok) mbar_wait_bounded(&full[s], (uint32_t)((j / S) & 1));
            }
            if (!ok) give_up();
        }
    } else if (warp == PK_MMA_WARP) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            // descriptors of the K steps differ only in the start address
            // field (16-byte units): chunk kk / 4 of QN x 128 B, 32 B per step;
            // all computed once, so that the loop issues little besides MMAs
            const uint64_t bdesc0 = sw128_desc(smem_u32(qop));
            // mode 1: the lo operand's descriptor start address (16-byte units)
            const uint64_t lo_off = (uint64_t)((W / 2) * QN * 128 / 16);
            uint64_t bd[2 * PK_W_MAX];
#pragma unroll
            for (int kk = 0; kk < 2 * PK_W_MAX; ++kk)
                bd[kk] = bdesc0 + (uint64_t)((kk >> 2) * QN * 8 + (kk & 3) * 2);
            bool ok = true;
            for (int t = 0; t < ntl && ok; ++t) {
                const int b = t & 1;
                const uint32_t use = (uint32_t)(t >> 1);
                if (!mbar_wait_or_abort(&a_full[b], use & 1u, abort_flag) ||
                    !mbar_wait_or_abort(&d_empty[b], (use & 1u) ^ 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dt = tmem_base + (uint32_t)(DCOL0 + b * QN);
                const uint32_t at = tmem_base + (uint32_t)(b * ACOLS);
                if constexpr (F4) {
                    // one K step of 64 elements = 8 TMEM columns of A, 32 B of B
                    const uint32_t sfa = tmem_base + SFCOL, sfb = tmem_base + SFCOL + 8u;
                    mma_f4_tmem_a(dt, at, bd[0], IDESC, sfa, sfb, 0u);
#pragma unroll
                    for (int kk = 1; kk < PK_W_MAX; ++kk)
                        if (kk < ksteps)
                            mma_f4_tmem_a(dt, at + (uint32_t)(8 * kk), bd[kk], IDESC, sfa, sfb, 1u);
                } else {
                    mma_f8_tmem_a(dt, at, bd[0], IDESC, 0u);
                    mma_f8_tmem_a(dt, at, bd[0] + lo_off, IDESC, 1u);
#pragma unroll
                    for (int kk = 1; kk < 2 * PK_W_MAX; ++kk) {
                        if (kk < ksteps) {
                            mma_f8_tmem_a(dt, at + (uint32_t)(8 * kk), bd[kk], IDESC, 1u);
                            mma_f8_tmem_a(dt, at + (uint32_t)(8 * kk), bd[kk] + lo_off, IDESC, 1u);
                        }
                    }
                }
                mma_commit(&d_full[b]);  // one commit per tile: each drains the MMA pipe
            }
            if (!ok) give_up();
            // every MMA issued completes before tensor memory is released
            mma_commit(done);
            if (!mbar_wait_bounded(done, 0)) give_up();
        }
    } else if (warp < PK_UNPACK_WARPS) {
        // ---------------- unpack warps ----------------
        const int h = warp >> 2;               // word pairs h, h + 2, ... of the row
        const int r = (warp & 3) * 32 + lane;  // row in the tile = TMEM lane
        const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
        if (F4 && h == 0) {
            // mode 0: unit scale factors (ue8m0 2^0) for every lane, written
            // before this warp's first A buffer (so before any MMA)
            uint32_t o[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) o[c] = 0x7F7F7F7Fu;
            tmem_st32(tmem_base + lane_off + SFCOL, o);
            tmem_wait_st();
        }
        for (int t = 0; t < ntl; ++t) {
            const int s = t % S, b = t & 1;
            int got = 1;
            if (lane == 0) got = mbar_wait_or_abort(&full[s], (uint32_t)((t / S) & 1), abort_flag);
            got = __shfl_sync(0xffffffffu, got, 0);
            if (!got) {
                if (lane == 0) give_up();
                break;
            }
            const uint64_t* rp =
                reinterpret_cast<const uint64_t*>(stages + (size_t)s * L.stage_bytes) +
                (size_t)r * a.pitch;
            ulonglong2 pw[PK_W_MAX / 4], mw[PK_W_MAX / 4];
#pragma unroll
            for (int i = 0; i < PK_W_MAX / 4; ++i) {
                const int pi = h + 2 * i;
                if (pi < npairs) {
                    pw[i] = reinterpret_cast<const ulonglong2*>(rp)[pi];
                    mw[i] = reinterpret_cast<const ulonglong2*>(rp + W)[pi];
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
            // the MMAs of tile t - 2 (the previous use of A buffer b) are complete;
            // d_full[b] cannot complete again before this warp writes A(t)
            if (lane == 0)
                got = mbar_wait_or_abort(&d_full[b], (uint32_t)(((t >> 1) & 1) ^ 1), abort_flag);
            got = __shfl_sync(0xffffffffu, got, 0);
            if (!got) {
                if (lane == 0) give_up();
                break;
            }
            tc_fence_after();
            const uint32_t abase = tmem_base + lane_off + (uint32_t)(b * ACOLS);
#pragma unroll
            for (int i = 0; i < PK_W_MAX / 4; ++i) {
                const int pi = h + 2 * i;
                if (pi < npairs) {
                    if constexpr (F4) {  // word pair pi: columns 16 pi .. 16 pi + 15
                        uint32_t o[16];
                        unpack_word_f4(pw[i].x, mw[i].x, o);
                        unpack_word_f4(pw[i].y, mw[i].y, o + 8);
                        tmem_st16(abase + (uint32_t)(16 * pi), o);
                    } else {
                        uint32_t o[32];
                        unpack_word(pw[i].x, mw[i].x, o);
                        unpack_word(pw[i].y, mw[i].y, o + 16);
                        tmem_st32(abase + (uint32_t)(32 * pi), o);
                    }
                }
            }
            tmem_wait_st();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&a_full[b]);
        }
    } else if (warp < PK_EPI_WARP0 + PK_EPI_WARPS) {
        // ---------------- epilogue warps ----------------
        // Warp e serves rows of quadrant e % 4 (its TMEM lanes) against
        // queries (e / 4) QH + j, j < QH, with candidate buffers, slice lists
        // and thresholds of its own: no epilogue warp waits for another.
        const int e = warp - PK_EPI_WARP0;
        const int quad = e & 3, qbase = (e >> 2) * QH;
        const int r = quad * 32 + lane;  // row in the tile = TMEM lane
        const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
        const int lslice = slice * PK_LISTS_PER_CTA + quad;  // this warp's list index
        const int nlists = nslices * PK_LISTS_PER_CTA;
        CandT* candw = cand + e * QH * PK_CAP;
        uint64_t* tauw = tau + e * QH;
        float* thrw = thr_s + e * QH;
        int* cntw = cnt + e * QH;
        int* lenw = len + e * QH;
        int* curw = cur + e * QH;
        uint32_t* lminw = lmin + e * QH;
        // candidates of entry j -> the (query, slice) list: sort, merge path,
        // new threshold from the list's k-th key and the union bound
        auto merge = [&](int j, bool fin) {
            const int q = qbase + j, nc = cntw[j];
            CandT* C = candw + j * PK_CAP;
            const int P = next_pow2(nc);
            for (int i = nc + lane; i < P; i += 32) C[i] = ~(CandT)0;
            __syncwarp();
            warp_sort(C, P, lane);
            uint64_t* base = a.lists + ((int64_t)q * nlists + lslice) * 2 * k;
            const int c0 = curw[j], nL = lenw[j];
            const uint64_t* Lst = base + (int64_t)c0 * k;
            uint64_t* out = base + (int64_t)(c0 ^ 1) * k;
            if (k <= PK_STAGE_LIST_K) {
                // the list, read once, is searched in shared memory
                uint64_t* Ls = scratch + e * PK_STAGE_LIST_K;
                for (int i = lane; i < nL; i += 32) Ls[i] = Lst[i];
                __syncwarp();
                Lst = Ls;
            }
            for (int i = lane; i < nL; i += 32) {
                const uint64_t key = Lst[i];
                const int rr = i + lower_bound_cand<MODE>(C, nc, key, row0);
                if (rr < k) out[rr] = key;
            }
            for (int i = lane; i < nc; i += 32) {
                const uint64_t key = pk_key64<MODE>(C[i], row0);
                const int rr = i + lower_bound_u64(Lst, nL, key);
                if (rr < k) out[rr] = key;
            }
            __syncwarp();
            const int nl = nL + nc < k ? nL + nc : k;
            if (lane == 0) {
                uint64_t t_new = nl == k ? out[k - 1] : KEY_NONE;
                const uint32_t T = *reinterpret_cast<volatile uint32_t*>(&ub[q]);
                if (!fin && T != 0xFFFFFFFFu) t_new = min(t_new, pk_bin_key<MODE>(T, a.hshift));
                curw[j] = c0 ^ 1;
                lenw[j] = nl;
                cntw[j] = 0;
                uint64_t tq = min(tauw[j], t_new);
                if (t_new != KEY_NONE) {
                    const unsigned long long old =
                        atomicMin(reinterpret_cast<unsigned long long*>(&a.tau_global[q]),
                                  (unsigned long long)t_new);
                    tq = min(tq, (uint64_t)old);
                }
                tauw[j] = tq;
                if (q < a.nqg) thrw[j] = pk_thr<MODE>(tq, x, a.bias);
            }
            __syncwarp();
        };
        bool ok = true;
        for (int t = 0; t < ntl; ++t) {
            const int b = t & 1;
            int got = 1;
            if (lane == 0) got = mbar_wait_or_abort(&d_full[b], (uint32_t)((t >> 1) & 1), abort_flag);
            got = __shfl_sync(0xffffffffu, got, 0);
            if (!got) {
                if (lane == 0) give_up();
                ok = false;
                break;
            }
            tc_fence_after();
            uint32_t v[QH];
            tmem_ld_wait<QH>(tmem_base + lane_off + (uint32_t)(DCOL0 + b * QN + qbase), v);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&d_empty[b]);
            const int64_t row = (tile0 + t) * PK_ROWS + r;
            // D - threshold per query, then the largest of them (thresholds
            // are finite half-integers, -2^22 or +inf: D - threshold is
            // exact and D = (D - threshold) + threshold)
            const float4* th4 = reinterpret_cast<const float4*>(thrw);
            float gap = -INFINITY;
#pragma unroll
            for (int c = 0; c < QH / 4; ++c) {
                const float4 th = th4[c];
                const float g0 = __uint_as_float(v[4 * c]) - th.x;
                const float g1 = __uint_as_float(v[4 * c + 1]) - th.y;
                const float g2 = __uint_as_float(v[4 * c + 2]) - th.z;
                const float g3 = __uint_as_float(v[4 * c + 3]) - th.w;
                v[4 * c] = __float_as_uint(g0);
                v[4 * c + 1] = __float_as_uint(g1);
                v[4 * c + 2] = __float_as_uint(g2);
                v[4 * c + 3] = __float_as_uint(g3);
                gap = fmaxf(gap, fmaxf(fmaxf(g0, g1), fmaxf(g2, g3)));
            }
            const bool live = gap > 0.f && row < a.ns;
            if (__any_sync(0xffffffffu, live)) {
                uint32_t msk = 0;
#pragma unroll
                for (int j = 0; j < QH; ++j)
                    msk |= (live && __uint_as_float(v[j]) > 0.f ? 1u : 0u) << j;
                const uint32_t any = __reduce_or_sync(0xffffffffu, msk);
                bool need = false;
#pragma unroll
                for (int j = 0; j < QH; ++j) {
                    if (!((any >> j) & 1u)) continue;
                    const int q = qbase + j;
                    // mode 0: Delta = 2x - D lies in [0, 4x] for codes with x
                    // non-zeros; mode 1: the score key bias - D/2 lies in
                    // [0, 2 bias]; clamped so that other codes cannot index
                    // outside the histogram
                    const float dq = __uint_as_float(v[j]) + thrw[j];
                    uint32_t kv, half;
                    if constexpr (MODE == 0) {
                        kv = (uint32_t)min(max(2 * x - __float2int_rn(dq), 0), 4 * x);
                        half = kv >> 1;
                    } else {
                        kv = (uint32_t)min(max(a.bias - (__float2int_rn(dq) >> 1), 0), 2 * a.bias);
                        half = kv >> a.hshift;
                    }
                    bool c = (msk >> j) & 1u;
                    if (c) c = (((uint64_t)kv << 32) | (uint64_t)row) < tauw[j];
                    const uint32_t am = __ballot_sync(0xffffffffu, c);
                    if (!am) continue;
                    const int pos0 = cntw[j];
                    if (c) {
                        const int rank = __popc(am & ((1u << lane) - 1u));
                        const CandT kc = MODE == 0 ? (CandT)half : (CandT)kv;
                        candw[j * PK_CAP + pos0 + rank] =
                            (kc << PK_LOCAL_BITS) | (CandT)(uint32_t)(row - row0);
                        // each row is appended at most once: count it for the union bound
                        atomicAdd(&a.hist[(int64_t)q * a.hist_bins + half], 1u);
                    }
                    const uint32_t wmin = __reduce_min_sync(0xffffffffu, c ? half : 0xFFFFFFFFu);
                    __syncwarp();
                    if (lane == 0) {
                        cntw[j] = pos0 + __popc(am);
                        if (wmin < lminw[j]) {
                            lminw[j] = wmin;
                            atomicMin(&a.minhalf[q], wmin);
                        }
                    }
                    need |= pos0 + __popc(am) >= PK_MERGE_AT;
                    __syncwarp();
                }
                if (need) {
                    for (int j = 0; j < QH; ++j)
                        if (cntw[j] >= PK_MERGE_AT) merge(j, false);
                }
            }
            if ((t & 7) == 7) {
                // other slices' thresholds and the union bound, one query per lane
                if (lane < QH && qbase + lane < a.nqg) {
                    const int q = qbase + lane;
                    uint64_t tq = min(tauw[lane], *reinterpret_cast<volatile uint64_t*>(&a.tau_global[q]));
                    const uint32_t T = *reinterpret_cast<volatile uint32_t*>(&ub[q]);
                    if (T != 0xFFFFFFFFu) tq = min(tq, pk_bin_key<MODE>(T, a.hshift));
                    tauw[lane] = tq;
                    thrw[lane] = pk_thr<MODE>(tq, x, a.bias);
                }
                __syncwarp();
            }
        }
        if (ok) {
            for (int j = 0; j < QH; ++j)
                if (cntw[j] > 0) merge(j, true);
            if (lane < QH) {
                int32_t* m = a.meta + ((int64_t)(qbase + lane) * nlists + lslice) * 2;
                m[0] = lenw[lane];
                m[1] = curw[lane];
            }
        }
        __syncwarp();
        if (lane == 0) atomicAdd(epi_done, 1);
    } else if (warp == PK_HELPER_WARP) {
        // ---------------- union-bound helper ----------------
        // For each query, the smallest T with count(Delta/2 <= T) >= k over
        // the keys all slices have appended (real rows, so no row with a
        // larger Delta/2 can be among the k nearest), scanning the workspace
        // histogram from the smallest appended value up to the previous T.
        while (*reinterpret_cast<volatile int*>(epi_done) < PK_EPI_WARPS &&
               !*reinterpret_cast<volatile int*>(abort_flag)) {
            for (int q = 0; q < a.nqg; ++q) {
                const uint32_t lo = __ldcg(&a.minhalf[q]);
                const uint32_t prev = *reinterpret_cast<volatile uint32_t*>(&ub[q]);
                const uint32_t hi = min(prev, (uint32_t)(a.hist_bins - 1));
                if (lo > hi) continue;
                const uint32_t* H = a.hist + (int64_t)q * a.hist_bins;
                // 8 consecutive bins per lane, 256 per round trip to L2
                uint32_t before = 0, T = 0xFFFFFFFFu;
                for (uint32_t h0 = lo; h0 <= hi && T == 0xFFFFFFFFu; h0 += 256) {
                    const uint32_t hb = h0 + 8u * (uint32_t)lane;
                    uint32_t c8[8], own = 0;
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        c8[u] = hb + u <= hi ? __ldcg(&H[hb + u]) : 0u;
                        own += c8[u];
                    }
                    uint32_t sum = own;  // inclusive scan of the lanes' sums
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t nb = __shfl_up_sync(0xffffffffu, sum, o);
                        if (lane >= o) sum += nb;
                    }
                    const uint32_t hit = __ballot_sync(0xffffffffu, before + sum >= (uint32_t)k);
                    if (hit) {
                        const int l0 = __ffs(hit) - 1;
                        if (lane == l0) {
                            uint32_t cum = before + sum - own;
#pragma unroll
                            for (int u = 0; u < 8; ++u) {
                                cum += c8[u];
                                if (cum >= (uint32_t)k && T == 0xFFFFFFFFu) T = hb + u;
                            }
                        }
                        T = __shfl_sync(0xffffffffu, T, l0);
                    }
                    before += __shfl_sync(0xffffffffu, sum, 31);
                }
                if (lane == 0 && T < prev) *reinterpret_cast<volatile uint32_t*>(&ub[q]) = T;
                __syncwarp();
            }
            __nanosleep(2000);
        }
    }

    // The producer has waited for every copy it issued and the MMA issuer
    // for every MMA (bounded, also after an abort).
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == PK_MMA_WARP)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                     "r"(PK_TMEM_COLS)
                     : "memory");
}

// Per pass: thresholds, histograms and minima of the union bound start empty.
__global__ void pk_init_kernel(uint64_t* tau_global, uint32_t* hist, int hist_words,
                               uint32_t* minhalf) {
    if (threadIdx.x < PK_QN_MAX) {
        tau_global[threadIdx.x] = KEY_NONE;
        minhalf[threadIdx.x] = 0xFFFFFFFFu;
    }
    for (int i = threadIdx.x; i < hist_words; i += blockDim.x) hist[i] = 0u;
}

int pk_stages(int W, int qn, int mode) {
    for (int s = PK_MAX_STAGES; s >= PK_MIN_STAGES; --s)
        if (pk_layout(W, s, qn, mode).total <= (size_t)PK_SMEM_LIMIT) return s;
    return 0;
}

template <int QN, int MODE>
cudaError_t launch_pk(const CUtensorMap& tmap, const PkArgs& a, int nslices, cudaStream_t stream) {
    const size_t smem = pk_layout(a.W, a.stages, QN, MODE).total;
    cudaError_t e = cudaFuncSetAttribute(scan_mma_packed_kernel<QN, MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    TimedLaunch timer(MODE == 0 ? "scan_mma_packed" : "scan_i8q", stream);
    scan_mma_packed_kernel<QN, MODE><<<nslices, PK_THREADS, smem, stream>>>(tmap, a);
    return cudaGetLastError();
}

// Queries per pass of the int8-query mode: two query operands and 64-bit
// candidates leave room for at most 32 in shared memory.
constexpr int PK_I8Q_QN_MAX = 32;

struct PkPlan {
    int nslices;
    int64_t tiles_per_slice, ntiles;
    size_t list_bytes, meta_bytes, hist_bytes, tau_bytes, ws_bytes;
};

PkPlan plan_pk(int64_t ns, int d, int k) {
    PkPlan p{};
    p.ntiles = std::max<int64_t>(1, (ns + PK_ROWS - 1) / PK_ROWS);
    int64_t tps = (p.ntiles + num_sms() - 1) / num_sms();
    tps = std::min(tps, PK_MAX_TILES_PER_SLICE);
    p.tiles_per_slice = tps;
    p.nslices = (int)((p.ntiles + tps - 1) / tps);
    const size_t lists = (size_t)PK_QN_MAX * p.nslices * PK_LISTS_PER_CTA;
    p.list_bytes = pk_align(lists * 2 * k * 8, 256);
    p.meta_bytes = pk_align(lists * 2 * 4, 256);
    p.hist_bytes = pk_align((size_t)PK_QN_MAX * (2 * d + 1) * 4, 256) + 256;  // + minima
    p.tau_bytes = pk_align((size_t)PK_QN_MAX * 8, 256);
    p.ws_bytes = p.list_bytes + p.meta_bytes + p.hist_bytes + p.tau_bytes;
    return p;
}

}  // namespace

bool mma_packed_supported(int64_t ns, int d, int k) {
    const int W = (d + 63) / 64;
    if (W % 2 != 0 || W > PK_W_MAX || k > PK_K_MAX) return false;
    return plan_pk(ns, d, k).nslices * PK_LISTS_PER_CTA <= PK_MAX_SLICES;
}

size_t mma_packed_workspace(int64_t ns, int d, int k) { return plan_pk(ns, d, k).ws_bytes; }

namespace {

// Both modes: MODE 0 takes packed query codes Qp ([nq][2W] uint64), MODE 1
// int8 queries ([nq][d]).
template <int MODE>
int32_t run_pk(const void* Qp, int64_t nq, const uint64_t* S, int64_t ns, int d, int x, int k,
               int64_t* ids, int32_t* dist, void* ws, size_t ws_bytes, int32_t* status,
               cudaStream_t stream) {
    if (!mma_packed_supported(ns, d, k)) return EVP_ERR_UNSUPPORTED;
    const int W = (d + 63) / 64;
    const PkPlan p = plan_pk(ns, d, k);
    if (ws_bytes < p.ws_bytes) return EVP_ERR_NO_MEMORY;

    EncodeTiledFn enc = encode_tiled_fn();
    if (!enc) return EVP_ERR_CUDA;
    CUtensorMap tmap;
    const int pitch = 2 * W + 2;
    cuuint64_t gdim[2] = {(cuuint64_t)(2 * W), (cuuint64_t)ns};
    cuuint64_t gstride[1] = {(cuuint64_t)(16 * W)};
    cuuint32_t box[2] = {(cuuint32_t)pitch, (cuuint32_t)PK_ROWS};
    cuuint32_t estride[2] = {1, 1};
    if (enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<uint64_t*>(S), gdim, gstride,
            box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return EVP_ERR_CUDA;

    uint8_t* w = static_cast<uint8_t*>(ws);
    PkArgs a{};
    a.ns = ns;
    a.W = W;
    a.x = x;
    a.k = k;
    a.d = d;
    a.pitch = pitch;
    a.ntiles = p.ntiles;
    a.tiles_per_slice = p.tiles_per_slice;
    a.lists = reinterpret_cast<uint64_t*>(w);
    a.meta = reinterpret_cast<int32_t*>(w + p.list_bytes);
    a.hist = reinterpret_cast<uint32_t*>(w + p.list_bytes + p.meta_bytes);
    a.minhalf = reinterpret_cast<uint32_t*>(w + p.list_bytes + p.meta_bytes + p.hist_bytes - 256);
    a.tau_global = reinterpret_cast<uint64_t*>(w + p.list_bytes + p.meta_bytes + p.hist_bytes);
    // mode 1: score keys 127 x - score in [0, 254 x], counted in bins of 2^7
    // (at most 2x + 1 bins, the mode-0 histogram's size)
    a.bias = 127 * x;
    a.hshift = 7;
    a.hist_bins = MODE == 0 ? 2 * x + 1 : ((2 * a.bias) >> a.hshift) + 1;
    a.status = status;
    a.stall_fills = MODE == 0 ? take_stall_packed() : -1;

    const int qn_max = MODE == 0 ? PK_QN_MAX : PK_I8Q_QN_MAX;
    for (int64_t q0 = 0; q0 < nq; q0 += qn_max) {
        const int nqg = (int)std::min<int64_t>(qn_max, nq - q0);
        const int qn = nqg <= 16 ? 16 : nqg <= 32 ? 32 : 64;
        if (MODE == 0) a.Q = static_cast<const uint64_t*>(Qp) + q0 * 2 * W;
        else a.Q8 = static_cast<const int8_t*>(Qp) + q0 * d;
        a.nqg = nqg;
        a.stages = pk_stages(W, qn, MODE);
        if (a.stages == 0) return EVP_ERR_UNSUPPORTED;
        {
            TimedLaunch timer("scan_init", stream);
            pk_init_kernel<<<1, 256, 0, stream>>>(a.tau_global, a.hist, PK_QN_MAX * a.hist_bins,
                                                  a.minhalf);
        }
        cudaError_t e;
        if (qn == 16) e = launch_pk<16, MODE>(tmap, a, p.nslices, stream);
        else if (qn == 32) e = launch_pk<32, MODE>(tmap, a, p.nslices, stream);
        else if constexpr (MODE == 0) e = launch_pk<64, MODE>(tmap, a, p.nslices, stream);
        else e = cudaErrorInvalidValue;
        if (e != cudaSuccess) return EVP_ERR_CUDA;
        const int32_t rc = launch_final_merge(
            a.lists, a.meta, a.tau_global, a.hist, a.minhalf, a.hist_bins, nqg,
            p.nslices * PK_LISTS_PER_CTA, k, ids + q0 * k, dist + q0 * k, stream,
            MODE == 0 ? -1 : a.hshift, MODE == 0 ? 0 : a.bias);
        if (rc != EVP_OK) return rc;
    }
    return EVP_OK;
}

}  // namespace

int32_t run_mma_packed_knn(const uint64_t* Q, int64_t nq, const uint64_t* S, int64_t ns, int d,
                           int x, int k, int64_t* ids, int32_t* dist, void* ws, size_t ws_bytes,
                           int32_t* status, cudaStream_t stream) {
    return run_pk<0>(Q, nq, S, ns, d, x, k, ids, dist, ws, ws_bytes, status, stream);
}

int32_t run_i8q_knn(const int8_t* Q8, int64_t nq, const uint64_t* S, int64_t ns, int d, int x,
                    int k, int64_t* ids, int32_t* score, void* ws, size_t ws_bytes,
                    int32_t* status, cudaStream_t stream) {
    return run_pk<1>(Q8, nq, S, ns, d, x, k, ids, score, ws, ws_bytes, status, stream);
}

}  // namespace evp
