// Sparse codes for small x (Sec. 6, "different EVPs": fewer non-zeros) and
// the exhaustive kNN scan over them by masked addition (Sec. 5.1.2).
//
// A sparse code is the list of a vertex's x non-zero dimensions in
// ascending order, one uint16 each: bits 0-14 the dimension, bit 15 set
// where the element is -1.  At x = 64, d = 768 a code takes 128 bytes
// instead of the 192 bytes of the two bitplanes, so a scan that streams the
// database from HBM moves a third less.
//
// evp_pack_sparse (pack_sparse_kernel): bitplane codes -> sparse codes, one
// warp per row; lane w counts the non-zeros of word w, a warp prefix sum
// places them.
//
// ternary_knn_sparse (scan_sparse_kernel): passes of up to 4 queries.  Each
// query element q_i in {-1, 0, +1} is held as the bytes
//   T+[i] = 1 + q_i and T-[i] = 1 - q_i        (both in {0, 1, 2}),
// the 4 queries of a pass packed into one 32-bit word per (sign, dimension),
// in 16 lane-interleaved copies in shared memory (word (sign*1024 + i)*16 +
// c for lanes c and c + 16) so that the 32 lanes' random lookups rarely meet
// in a bank; the table always spans 2 x 1024 dimensions, so an entry's low
// 10 bits and its sign bit index it directly and a malformed entry still
// reads inside it.  For a database row s, the sum over its entries of the word for
// (sign, dimension) is, per byte, A = sum over s's entries of (1 + s_i q_i)
// = x + <q, s>, so Delta = ||q - s||^2 = 2x - 2 <q, s> = 4x - 2A for codes
// with x non-zeros each.  Bytes cannot carry: A <= 2x <= 240 (x <= 120).
// Each warp takes 32 consecutive rows per tile and reads them as one
// contiguous run of 16-byte pieces (lane l takes pieces l, l + 32, ...), so
// every load instruction is fully coalesced; a lane sums the table words of
// its pieces' entries, the partial sums go through shared memory (skewed by
// one word per 32 so that neither side meets in a bank), and lane l adds the
// x / 8 partial sums of row l.  The next tile's pieces are loaded into
// registers while the current tile is scored (the row length is a template
// parameter), so HBM latency overlaps the work of a tile.  Keys (Delta << 32 | row)
// below the CTA's threshold for a query go to a candidate buffer; when a
// buffer may overflow in the next tile, the CTA merges each query's
// candidates into its sorted top-k list (a block bitonic sort of list and
// candidates), shares the list's k-th key through a global per-query
// minimum and takes the smaller of the two as its threshold.  At the end
// each CTA writes its lists; the per-query final merge of the popcount
// path combines them.
#include "evp_internal.cuh"

#include <algorithm>

namespace evp {

namespace {

constexpr int SP_THREADS = 512;     // one row per thread per tile
constexpr int SP_TILE = SP_THREADS;
constexpr int SP_QB = 4;            // queries per pass (bytes of a table word)
constexpr int SP_COPIES = 16;       // lane-interleaved table copies
constexpr int SP_CAP = 1024;        // candidate slots per query: a tile adds <= 512
constexpr int SP_K_MAX = 256;       // largest k of this path
constexpr int SP_SORT = 2048;       // bitonic width: list (<= 256) + candidates (<= 1024)
constexpr int SP_X_MAX = 120;       // bytes of the table sums cannot carry
constexpr int SP_D_MAX = 1024;
constexpr int SP_TAB = 2 * SP_D_MAX;  // table words per copy: (sign, dimension)
constexpr int SP_NV_MAX = SP_X_MAX / 8;  // 16-byte pieces per row
constexpr int SP_WARPS = SP_THREADS / 32;
constexpr int SP_PART = 33 * SP_NV_MAX;  // partial-sum words per warp (skewed)

struct SpArgs {
    const uint64_t* Q;      // this pass's query codes [nqg][2W]
    int nqg;
    const uint16_t* E;      // [ns][x] sparse database codes
    int64_t ns;
    int d, x, k, W;
    int64_t rows_per_slice;
    int q0;                 // first query of the pass (list index)
    int nq_total;
    uint64_t* lists;        // [nq][nslices][2][k]
    int32_t* meta;          // [nq][nslices][2]
    uint64_t* tau_global;   // [nq]
};

__global__ void pack_sparse_kernel(const uint64_t* __restrict__ T, int64_t n, int d, int x,
                                   uint16_t* __restrict__ E, int32_t* __restrict__ status) {
    const int lane = threadIdx.x & 31;
    const int W = (d + 63) / 64;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t row = warp0; row < n; row += nwarps) {
        const uint64_t* t = T + row * 2 * W;
        uint16_t* e = E + row * x;
        int base = 0;
        for (int w0 = 0; w0 < W; w0 += 32) {
            const int w = w0 + lane;
            const uint64_t p = w < W ? t[w] : 0ull, m = w < W ? t[W + w] : 0ull;
            uint64_t nz = p | m;
            const int c = __popcll(nz);
            int off = c;  // inclusive prefix sum over the lanes
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, off, o);
                if (lane >= o) off += v;
            }
            const int total = __shfl_sync(0xffffffffu, off, 31);
            int pos = base + off - c;
            while (nz) {
                const int b = __ffsll((long long)nz) - 1;
                nz &= nz - 1;
                if (pos < x)
                    e[pos] = (uint16_t)((64 * w + b) | (((m >> b) & 1ull) ? 0x8000u : 0u));
                ++pos;
            }
            base += total;
        }
        if (base != x && lane == 0) report(status, EVP_ERR_RANGE);
        for (int i = base + lane; i < x; i += 32) e[i] = 0;  // a short row: defined contents
    }
}

// Ascending bitonic sort of s[0, n) by the whole block (n a power of two,
// at most SP_SORT).
__device__ __forceinline__ void block_sort(uint64_t* s, int n) {
    for (int kk = 2; kk <= n; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n; i += SP_THREADS) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const uint64_t a = s[i], b = s[ixj];
                    if ((a > b) == ((i & kk) == 0)) {
                        s[i] = b;
                        s[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// NV = x / 8: 16-byte pieces per row.
template <int NV>
__global__ void __launch_bounds__(SP_THREADS, 1) scan_sparse_kernel(const SpArgs a) {
    extern __shared__ __align__(16) uint8_t sp_smem[];
    const int d = a.d, x = a.x, k = a.k;
    uint32_t* tab = reinterpret_cast<uint32_t*>(sp_smem);             // [2][1024][SP_COPIES]
    uint64_t* list = reinterpret_cast<uint64_t*>(sp_smem + (size_t)SP_TAB * SP_COPIES * 4);
    uint64_t* cand = list + SP_QB * SP_K_MAX;                          // [SP_QB][SP_CAP]
    uint64_t* sortbuf = cand + SP_QB * SP_CAP;                         // [SP_SORT]
    uint32_t* part = reinterpret_cast<uint32_t*>(sortbuf + SP_SORT) +
                     (threadIdx.x >> 5) * SP_PART;                     // this warp's partials
    __shared__ uint64_t tau[SP_QB];
    __shared__ int cnt[SP_QB], len[SP_QB];
    const int tid = threadIdx.x;
    const int slice = blockIdx.x, nslices = gridDim.x;
    const int64_t row0 = (int64_t)slice * a.rows_per_slice;
    const int64_t row_end = min(row0 + a.rows_per_slice, a.ns);

    // query tables (dimensions >= d hold q = 0)
    for (int i = tid; i < SP_TAB; i += SP_THREADS) {
        const int sgn = i >= SP_D_MAX, dim = i - sgn * SP_D_MAX;
        uint32_t v = 0;
        for (int j = 0; j < SP_QB; ++j) {
            int q = 0;
            if (j < a.nqg && dim < d) {
                const uint64_t* qc = a.Q + (int64_t)j * 2 * a.W;
                q = (int)((qc[dim >> 6] >> (dim & 63)) & 1ull) -
                    (int)((qc[a.W + (dim >> 6)] >> (dim & 63)) & 1ull);
            }
            v |= (uint32_t)(sgn ? 1 - q : 1 + q) << (8 * j);
        }
#pragma unroll
        for (int c = 0; c < SP_COPIES; ++c) tab[i * SP_COPIES + c] = v;
    }
    if (tid < SP_QB) {
        tau[tid] = tid < a.nqg ? KEY_NONE : 0ull;  // padding queries admit nothing
        cnt[tid] = 0;
        len[tid] = 0;
    }
    __syncthreads();
    const uint32_t* mytab = tab + (tid & (SP_COPIES - 1));

    // merge each query's candidates into its list (whole block)
    auto merge_all = [&]() {
        for (int j = 0; j < a.nqg; ++j) {
            const int nc = min(cnt[j], SP_CAP), nl = len[j];
            int n = 2;
            while (n < nl + nc) n <<= 1;
            for (int i = tid; i < n; i += SP_THREADS)
                sortbuf[i] = i < nl ? list[j * SP_K_MAX + i]
                                    : (i < nl + nc ? cand[j * SP_CAP + i - nl] : KEY_NONE);
            __syncthreads();
            block_sort(sortbuf, n);
            const int m = min(nl + nc, k);
            for (int i = tid; i < m; i += SP_THREADS) list[j * SP_K_MAX + i] = sortbuf[i];
            if (tid == 0) {
                len[j] = m;
                cnt[j] = 0;
                uint64_t t = tau[j];
                if (m == k) {
                    const uint64_t kth = sortbuf[k - 1];
                    const unsigned long long old = atomicMin(
                        reinterpret_cast<unsigned long long*>(&a.tau_global[a.q0 + j]),
                        (unsigned long long)kth);
                    t = min(t, min(kth, (uint64_t)old));
                } else {
                    t = min(t, *reinterpret_cast<volatile uint64_t*>(&a.tau_global[a.q0 + j]));
                }
                tau[j] = t;
            }
            __syncthreads();
        }
    };

    // entry -> table word: bits 0-9 the dimension, bit 10 the sign
    auto word_of = [&](uint32_t w) -> uint32_t {
        const uint32_t lo = (w & 0x3FFu) | ((w >> 5) & 0x400u);
        const uint32_t hi = ((w >> 16) & 0x3FFu) | ((w >> 21) & 0x400u);
        return mytab[lo * SP_COPIES] + mytab[hi * SP_COPIES];
    };
    // Warp w scores rows t + 32 w ... t + 32 w + 31 of tile t: pieces
    // (t + 32 w) * NV + 32 u + lane, u < NV, one coalesced run per warp.
    const int lane = tid & 31;
    const uint4* E4 = reinterpret_cast<const uint4*>(a.E);
    const int64_t piece_end = row_end * NV;
    auto load_tile = [&](int64_t t, uint4 (&v)[NV]) {
        const int64_t p0 = (t + (tid - lane)) * NV + lane;
#pragma unroll
        for (int u = 0; u < NV; ++u) {
            const int64_t g = p0 + 32 * u;
            v[u] = g < piece_end ? __ldcs(E4 + g) : make_uint4(0u, 0u, 0u, 0u);
        }
    };
    uint4 cur[NV], nxt[NV];
    load_tile(row0, cur);
    for (int64_t t0 = row0; t0 < row_end; t0 += SP_TILE) {
        if (t0 + SP_TILE < row_end) load_tile(t0 + SP_TILE, nxt);  // in flight meanwhile
        // other CTAs' thresholds: loaded now, taken at the end of the tile
        uint64_t tg = KEY_NONE;
        if (tid < a.nqg) tg = *reinterpret_cast<volatile uint64_t*>(&a.tau_global[a.q0 + tid]);
        // partial sums of this lane's pieces, then row lane's total
#pragma unroll
        for (int u = 0; u < NV; ++u)
            part[33 * u + lane] = word_of(cur[u].x) + word_of(cur[u].y) + word_of(cur[u].z) +
                                  word_of(cur[u].w);
        __syncwarp();
        uint32_t acc = 0;
#pragma unroll
        for (int p = 0; p < NV; ++p) {
            const int g = lane * NV + p;
            acc += part[g + (g >> 5)];
        }
        const int64_t row = t0 + tid;
        if (row < row_end) {
            for (int j = 0; j < a.nqg; ++j) {
                const uint32_t A = (acc >> (8 * j)) & 0xFFu;
                const uint64_t key = ((uint64_t)(uint32_t)(4 * x - 2 * (int)A) << 32) | (uint64_t)row;
                if (key < tau[j]) {
                    const int pos = atomicAdd(&cnt[j], 1);
                    if (pos < SP_CAP) cand[j * SP_CAP + pos] = key;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < NV; ++u) cur[u] = nxt[u];
        __syncthreads();
        // the next tile adds at most SP_TILE candidates per query
        bool full = false;
        for (int j = 0; j < a.nqg; ++j) full |= cnt[j] > SP_CAP - SP_TILE;
        if (full) merge_all();
        else if (tid < a.nqg) tau[tid] = min(tau[tid], tg);
        __syncthreads();
    }
    merge_all();
    for (int j = 0; j < a.nqg; ++j) {
        uint64_t* out = a.lists + ((int64_t)(a.q0 + j) * nslices + slice) * 2 * k;
        for (int i = tid; i < len[j]; i += SP_THREADS) out[i] = list[j * SP_K_MAX + i];
        if (tid == 0) {
            int32_t* mt = a.meta + ((int64_t)(a.q0 + j) * nslices + slice) * 2;
            mt[0] = len[j];
            mt[1] = 0;
        }
    }
}

__global__ void sp_init_kernel(uint64_t* tau_global, int nq) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += gridDim.x * blockDim.x)
        tau_global[i] = KEY_NONE;
}

struct SpPlan {
    int nslices;
    int64_t rows_per_slice;
    size_t list_bytes, meta_bytes, tau_bytes, ws_bytes, smem;
};

SpPlan plan_sparse(int64_t nq, int64_t ns, int d, int k) {
    SpPlan p{};
    const int64_t tiles = std::max<int64_t>(1, (ns + SP_TILE - 1) / SP_TILE);
    p.nslices = (int)std::min<int64_t>(tiles, num_sms());
    const int64_t tps = (tiles + p.nslices - 1) / p.nslices;
    p.rows_per_slice = tps * SP_TILE;
    p.nslices = (int)((tiles + tps - 1) / tps);
    const size_t lists = (size_t)std::max<int64_t>(nq, 1) * p.nslices;
    p.list_bytes = (lists * 2 * k * 8 + 255) / 256 * 256;
    p.meta_bytes = (lists * 2 * 4 + 255) / 256 * 256;
    p.tau_bytes = ((size_t)std::max<int64_t>(nq, 1) * 8 + 255) / 256 * 256;
    p.ws_bytes = p.list_bytes + p.meta_bytes + p.tau_bytes;
    p.smem = (size_t)SP_TAB * SP_COPIES * 4 + (size_t)SP_QB * SP_K_MAX * 8 +
             (size_t)SP_QB * SP_CAP * 8 + (size_t)SP_SORT * 8 +
             (size_t)SP_WARPS * SP_PART * 4;
    return p;
}

}  // namespace

bool sparse_supported(int d, int x, int k) {
    return d >= 1 && d <= SP_D_MAX && x >= 8 && x <= SP_X_MAX && x % 8 == 0 && x <= d &&
           k >= 1 && k <= SP_K_MAX;
}

size_t sparse_workspace(int64_t nq, int64_t ns, int d, int k) {
    return plan_sparse(nq, ns, d, k).ws_bytes;
}

cudaError_t launch_pack_sparse(const uint64_t* T, int64_t n, int d, int x, uint16_t* E,
                               int32_t* status, cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 7) / 8;
    const int64_t cap = (int64_t)num_sms() * 8;
    if (blocks > cap) blocks = cap;
    TimedLaunch timer("pack_sparse", stream);
    pack_sparse_kernel<<<(unsigned)blocks, 256, 0, stream>>>(T, n, d, x, E, status);
    return cudaGetLastError();
}

int32_t run_sparse_knn(const uint64_t* Q, int64_t nq, const uint16_t* E, int64_t ns, int d,
                       int x, int k, int64_t* ids, int32_t* dist, void* ws, size_t ws_bytes,
                       int32_t* status, cudaStream_t stream) {
    if (!sparse_supported(d, x, k)) return EVP_ERR_UNSUPPORTED;
    const SpPlan p = plan_sparse(nq, ns, d, k);
    if (ws_bytes < p.ws_bytes) return EVP_ERR_NO_MEMORY;
    uint8_t* w = static_cast<uint8_t*>(ws);
    SpArgs a{};
    a.E = E;
    a.ns = ns;
    a.d = d;
    a.x = x;
    a.k = k;
    a.W = (d + 63) / 64;
    a.rows_per_slice = p.rows_per_slice;
    a.nq_total = (int)nq;
    a.lists = reinterpret_cast<uint64_t*>(w);
    a.meta = reinterpret_cast<int32_t*>(w + p.list_bytes);
    a.tau_global = reinterpret_cast<uint64_t*>(w + p.list_bytes + p.meta_bytes);
    void (*kern)(const SpArgs) = nullptr;
    switch (x / 8) {
        case 1: kern = scan_sparse_kernel<1>; break;
        case 2: kern = scan_sparse_kernel<2>; break;
        case 3: kern = scan_sparse_kernel<3>; break;
        case 4: kern = scan_sparse_kernel<4>; break;
        case 5: kern = scan_sparse_kernel<5>; break;
        case 6: kern = scan_sparse_kernel<6>; break;
        case 7: kern = scan_sparse_kernel<7>; break;
        case 8: kern = scan_sparse_kernel<8>; break;
        case 9: kern = scan_sparse_kernel<9>; break;
        case 10: kern = scan_sparse_kernel<10>; break;
        case 11: kern = scan_sparse_kernel<11>; break;
        case 12: kern = scan_sparse_kernel<12>; break;
        case 13: kern = scan_sparse_kernel<13>; break;
        case 14: kern = scan_sparse_kernel<14>; break;
        default: kern = scan_sparse_kernel<15>; break;
    }
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem) !=
        cudaSuccess)
        return EVP_ERR_CUDA;
    {
        TimedLaunch timer("scan_init", stream);
        sp_init_kernel<<<1, 256, 0, stream>>>(a.tau_global, (int)nq);
    }
    for (int64_t q0 = 0; q0 < nq; q0 += SP_QB) {
        a.q0 = (int)q0;
        a.nqg = (int)std::min<int64_t>(SP_QB, nq - q0);
        a.Q = Q + q0 * 2 * a.W;
        TimedLaunch timer("scan_sparse", stream);
        kern<<<p.nslices, SP_THREADS, p.smem, stream>>>(a);
        if (cudaGetLastError() != cudaSuccess) return EVP_ERR_CUDA;
    }
    return launch_final_merge(a.lists, a.meta, a.tau_global, nullptr, nullptr, 0, nq, p.nslices,
                              k, ids, dist, stream);
}

}  // namespace evp
