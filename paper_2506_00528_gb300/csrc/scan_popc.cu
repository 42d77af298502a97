// ternary_knn, popcount path: exhaustive scan of packed ternary codes with
// the integer proxy distance Delta and a fused per-query top-k.
//
// Delta(q, s) = ||q - s||^2 over ternary vectors (read of the notation
// table and Sec. 2.6).  With m = v+ | v- (non-zero mask) and sigma = v-
// (sign), per 64-bit word:
//   one_nz  = q.m ^ s.m                 -> elements where exactly one is 0: (v-w)^2 = 1
//   opposed = q.m & s.m & (q.sig ^ s.sig) -> both non-zero, opposite sign:   (v-w)^2 = 4
//   Delta   = sum popc(one_nz) + 4 * sum popc(opposed)
// which equals 2x - 2*b2sp for two codes with x non-zeros each, b2sp being
// the four-term bitplane scalar product of Sec. 5.1.2.
//
// Kernel layout (one CTA per SM, persistent over a contiguous slice of the
// database; 256 threads, one per row, for passes of up to 4 queries (at 10M
// x 768: 2 queries 0.401 ms, against 0.438 with two threads per row each
// taking one query), otherwise 512, two per row each taking half of the
// pass's queries):
//   * database tiles of 256 rows are staged into shared memory by TMA
//     (cp.async.bulk.tensor.2d) through a ring of mbarrier-tracked stages.
//     The box is wider than a row (2(W+p) words, p chosen so the row
//     pitch in 16-byte units is odd); the extra words are filled with 0 by
//     the TMA unit and make the per-thread row reads bank-conflict free;
//   * each thread copies its row into registers, the stage is released at
//     once (its next copy is issued while the rows are scored), and the row
//     is scored from registers;
//   * the pass's queries (up to 16) sit in shared memory as (m, sigma)
//     word pairs and are read by broadcast;
//   * a row whose key (Delta << 32 | row) beats the query's threshold tau
//     is appended to that query's candidate buffer; buffers are merged
//     (bitonic sort + merge-path) into a per-(query, slice) sorted list of
//     the k best, kept in the workspace;
//   * every appended key is also counted in a per-query Delta/2 histogram
//     in the workspace (each row is appended at most once); after a merge,
//     the smallest T with count(Delta/2 <= T) >= k over all slices' keys
//     bounds the answer (those keys are real rows), and so does a full
//     slice list's k-th key.  Both are folded into a global per-query
//     threshold with atomicMin, and every CTA filters with the smaller of
//     its own and the global threshold;
//   * a merge is done by a team of warps per query (all warps of the CTA
//     take part whatever the pass size): bitonic sort, merge path, and the
//     histogram scan for the bound.
// A second kernel merges, per query, the slice lists into the k best: the
// keys at or below the union bound of the complete histogram are gathered
// and sorted directly when there are few of them.
#include "evp_internal.cuh"

#include <algorithm>

namespace evp {

namespace {

constexpr int SCAN_ROWS = 256;                  // rows per tile = threads per CTA
constexpr int CAND_CAP = 512;                   // candidate slots per query (power of 2)
constexpr int MERGE_AT = CAND_CAP - SCAN_ROWS;  // merge before a tile could overflow
constexpr int QB_MAX = 16;
constexpr int MAX_STAGES = 4;
constexpr int SMEM_BUDGET = 225 * 1024;
constexpr int FM_THREADS = 256;                 // final merge: one CTA per query
constexpr int FM_MAX_SLICES = 1024;             // slice lists per query in the final merge
constexpr int FM_GATHER = 2048;                 // keys at or below the threshold hint merged directly
constexpr int FM_OUT_BYTES = (EVP_MAX_K > FM_GATHER ? EVP_MAX_K : FM_GATHER) * 8;  // sort buffer
constexpr int FM_STAGE_BYTES = 160 * 1024;      // lists staged in shared memory up to this size

struct ScanArgs {
    const uint64_t* Q;  // this pass's query codes [nqg][2W]
    int nqg;
    int64_t ns;
    int W;
    int k;
    int pitch;           // uint64 words per staged row
    int stages;
    int64_t tiles_per_slice;
    int64_t ntiles;
    uint64_t* lists;     // [QB_MAX][nslices][2][k]
    int32_t* meta;       // [QB_MAX][nslices][2]: (length, current buffer)
    uint64_t* tau_global;  // [QB_MAX]
    uint32_t* hist;      // [QB_MAX][hist_bins]: Delta/2 of every key any slice appended
    uint32_t* minhalf;   // [QB_MAX]: smallest Delta/2 any slice appended
    int hist_bins;       // 2x + 1
    int32_t* status;
};

__host__ __device__ inline int row_pitch_words(int W) { return 2 * (W + ((W & 1) ? 2 : 1)); }

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct SmemLayout {
    size_t stage_bytes, qv_off, cand_off, tau_off, cnt_off, bar_off, flag_off, total;
};

// Shared-memory carve-up for a pass of `qb` queries (candidate buffers are
// sized by the pass, so small passes leave room for more TMA stages).
__host__ __device__ inline SmemLayout smem_layout(int W, int stages, int qb) {
    SmemLayout L;
    L.stage_bytes = align_up((size_t)SCAN_ROWS * row_pitch_words(W) * 8, 1024);
    L.qv_off = L.stage_bytes * stages;
    L.cand_off = L.qv_off + align_up((size_t)QB_MAX * W * 16, 128);
    L.tau_off = L.cand_off + (size_t)qb * CAND_CAP * 8;
    L.cnt_off = L.tau_off + QB_MAX * 8;
    L.bar_off = L.cnt_off + align_up(4 * QB_MAX * 4, 8);
    L.flag_off = L.bar_off + MAX_STAGES * 8;
    L.total = L.flag_off + 16;
    return L;
}

// Ascending bitonic sort of buf[0, P) (P a power of two) by a team of TT
// threads (t = thread index in the team) that synchronises with `sync`.
template <typename Sync>
__device__ __forceinline__ void team_bitonic_sort(uint64_t* buf, int P, int t, int TT, Sync& sync) {
    for (int kk = 2; kk <= P; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = t; i < P; i += TT) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const uint64_t x0 = buf[i], x1 = buf[ixj];
                    const bool up = (i & kk) == 0;
                    if ((x0 > x1) == up) {
                        buf[i] = x1;
                        buf[ixj] = x0;
                    }
                }
            }
            sync();
        }
    }
}

// The k smallest of two ascending lists L[0, nL) and C[0, nc) (no key in
// both) into out[0, min(nL + nc, k)), by merge path: each key's output rank
// is its own index plus the number of smaller keys in the other list.
__device__ __forceinline__ int team_merge_topk(const uint64_t* L, int nL, const uint64_t* C, int nc,
                                               uint64_t* out, int k, int t, int TT) {
    for (int i = t; i < nL; i += TT) {
        const uint64_t key = L[i];
        const int r = i + lower_bound_u64(C, nc, key);
        if (r < k) out[r] = key;
    }
    for (int j = t; j < nc; j += TT) {
        const uint64_t key = C[j];
        const int r = j + lower_bound_u64(L, nL, key);
        if (r < k) out[r] = key;
    }
    const int total = nL + nc;
    return total < k ? total : k;
}

// TPR threads share a row (each takes QB / TPR of the pass's queries), so a
// CTA runs SCAN_ROWS * TPR threads: more warps to hide the popcount and
// shared-memory latencies than one thread per row would give.
template <int QB, int TPR, int WW, bool EXACT>
__global__ void __launch_bounds__(SCAN_ROWS * TPR, 1)
scan_popc_kernel(const __grid_constant__ CUtensorMap tmap, const ScanArgs a) {
    constexpr int NT = SCAN_ROWS * TPR;
    constexpr int QPT = QB / TPR;
    static_assert(QPT * TPR == QB, "queries split evenly over a row's threads");
    extern __shared__ __align__(1024) uint8_t smem[];
    const SmemLayout L = smem_layout(a.W, a.stages, QB);
    uint64_t* qv = reinterpret_cast<uint64_t*>(smem + L.qv_off);
    uint64_t* cand = reinterpret_cast<uint64_t*>(smem + L.cand_off);
    uint64_t* tau = reinterpret_cast<uint64_t*>(smem + L.tau_off);
    int* cnt = reinterpret_cast<int*>(smem + L.cnt_off);
    int* len = cnt + QB_MAX;
    int* cur = len + QB_MAX;
    uint32_t* lmin = reinterpret_cast<uint32_t*>(cur + QB_MAX);  // smallest Delta/2 this CTA appended
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar_off);
    int* abort_flag = reinterpret_cast<int*>(smem + L.flag_off);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rt = tid % SCAN_ROWS;          // row of the tile this thread scores
    const int qbase = (tid / SCAN_ROWS) * QPT;  // first query of this thread
    const int W = a.W, k = a.k, nslices = gridDim.x, slice = blockIdx.x;
    const int64_t tile0 = (int64_t)slice * a.tiles_per_slice;
    const int64_t tile_end = min(tile0 + a.tiles_per_slice, a.ntiles);
    const int ntl = tile_end > tile0 ? (int)(tile_end - tile0) : 0;
    const uint32_t tile_bytes = (uint32_t)(SCAN_ROWS * a.pitch * 8);

    if (tid == 0) {
        for (int s = 0; s < a.stages; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
        *abort_flag = 0;
    }
    for (int i = tid; i < QB * W; i += NT) {
        const int q = i / W, w = i - q * W;
        uint64_t p = 0, n = 0;
        if (q < a.nqg) {
            p = a.Q[(int64_t)q * 2 * W + w];
            n = a.Q[(int64_t)q * 2 * W + W + w];
        }
        qv[2 * i] = p | n;
        qv[2 * i + 1] = n;
    }
    if (tid < QB) {
        tau[tid] = KEY_NONE;
        cnt[tid] = 0;
        len[tid] = 0;
        cur[tid] = 0;
        lmin[tid] = 0xFFFFFFFFu;
    }
    __syncthreads();
    if (tid == 0) {
        const int pre = min(a.stages, ntl);
        for (int s = 0; s < pre; ++s) {
            mbar_arrive_expect_tx(&bars[s], tile_bytes);
            tma_load_2d(smem + s * L.stage_bytes, &tmap, &bars[s], 0,
                        (int32_t)((tile0 + s) * SCAN_ROWS));
        }
    }

    // Per tile: wait for the stage; merge the earlier tiles' candidates if
    // a buffer could overflow (or, after the last tile, all of them); copy
    // this thread's row into registers and release the stage (its next copy
    // starts at once, so every stage keeps loading while rows are scored);
    // then score the row against the pass's queries from registers.
    int it = 0;
    for (;; ++it) {
        const bool fin = it == ntl;
        const int s = it % a.stages;
        if (!fin && tid == 0 &&
            !mbar_wait_bounded(&bars[s], (uint32_t)((it / a.stages) & 1))) {
            report(a.status, EVP_ERR_TIMEOUT);
            *abort_flag = 1;
        }
        __syncthreads();  // stage s landed; the earlier tiles' candidates are visible
        if (*abort_flag) break;
        uint32_t mask = 0;
#pragma unroll
        for (int q = 0; q < QB; ++q) {
            const int c = cnt[q];
            if (c > MERGE_AT || (fin && c > 0)) mask |= 1u << q;
        }
        if (mask) {
            __syncthreads();  // every thread has read cnt before it changes
            // A team of TEAM warps per query; the pass's queries merge side
            // by side (all warps of the CTA take part, whatever the pass size).
            constexpr int TEAM = NT / 32 >= QB ? NT / 32 / QB : 1;
            constexpr int TT = TEAM * 32;
            const int team = warp / TEAM, t = tid - team * TT;
            auto sync = [&]() {
                if constexpr (TEAM == 1) __syncwarp();
                else named_barrier(1 + team, TT);
            };
            for (int q = team; q < QB; q += NT / TT) {
                if (!((mask >> q) & 1)) continue;
                uint64_t* C = cand + q * CAND_CAP;
                const int nc = cnt[q];
                const int P = next_pow2(nc);
                for (int i = nc + t; i < P; i += TT) C[i] = KEY_NONE;
                sync();
                team_bitonic_sort(C, P, t, TT, sync);
                uint64_t* base = a.lists + ((int64_t)q * nslices + slice) * 2 * k;
                const int c0 = cur[q];
                const int nl = team_merge_topk(base + c0 * k, len[q], C, nc, base + (c0 ^ 1) * k, k,
                                               t, TT);
                sync();  // the new list is complete; C is free
                uint64_t t_new = KEY_NONE;
                if (nl == k) t_new = base[(c0 ^ 1) * k + k - 1];
                if (!fin) {
                    // union bound: the smallest T with count(Delta/2 <= T) >= k
                    // over the keys all slices of the query have appended
                    const uint32_t T = team_kth_bin(a.hist + (int64_t)q * a.hist_bins,
                                                    a.minhalf + q, a.hist_bins, (uint32_t)k,
                                                    reinterpret_cast<uint32_t*>(C), t, TT, sync);
                    if (T != 0xFFFFFFFFu) t_new = min(t_new, (uint64_t)(2u * T + 1u) << 32);
                }
                if (t == 0) {
                    cur[q] = c0 ^ 1;
                    len[q] = nl;
                    cnt[q] = 0;
                    uint64_t tq = min(tau[q], t_new);
                    if (t_new != KEY_NONE) {
                        const unsigned long long old =
                            atomicMin(reinterpret_cast<unsigned long long*>(&a.tau_global[q]),
                                      (unsigned long long)t_new);
                        tq = min(tq, (uint64_t)old);
                    } else {
                        tq = min(tq, *reinterpret_cast<volatile uint64_t*>(&a.tau_global[q]));
                    }
                    tau[q] = tq;
                }
            }
            __syncthreads();
        } else if ((it & 7) == 7 && tid >= NT - QB) {
            // fold in other slices' thresholds now and then, from the last
            // warp (thread 0 issues the copies and must not wait on L2)
            const int q = NT - 1 - tid;
            tau[q] = min(tau[q], *reinterpret_cast<volatile uint64_t*>(&a.tau_global[q]));
        }
        if (fin) break;

        const int64_t row = (tile0 + it) * SCAN_ROWS + rt;
        const bool valid = row < a.ns;
        uint64_t rm[WW], rn[WW];  // the row: non-zero mask m and sign sigma per word
        {
            const uint64_t* rp =
                reinterpret_cast<const uint64_t*>(smem + s * L.stage_bytes) + rt * a.pitch;
            if constexpr (EXACT && WW % 2 == 0) {
                const ulonglong2* rp2 = reinterpret_cast<const ulonglong2*>(rp);
#pragma unroll
                for (int w = 0; w < WW; w += 2) {
                    const ulonglong2 sp = rp2[w / 2], sn = rp2[(WW + w) / 2];
                    rm[w] = sp.x | sn.x;
                    rm[w + 1] = sp.y | sn.y;
                    rn[w] = sn.x;
                    rn[w + 1] = sn.y;
                }
            } else {
#pragma unroll
                for (int w = 0; w < WW; ++w) {
                    const bool in = EXACT || w < W;
                    const uint64_t sp = in ? rp[w] : 0ull, sn = in ? rp[W + w] : 0ull;
                    rm[w] = sp | sn;
                    rn[w] = sn;
                }
            }
        }
        __syncthreads();  // every row is in registers: stage s is free
        if (tid == 0 && it + a.stages < ntl) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bars[s], tile_bytes);
            tma_load_2d(smem + s * L.stage_bytes, &tmap, &bars[s], 0,
                        (int32_t)((tile0 + it + a.stages) * SCAN_ROWS));
        }

        if (valid) {
            const ulonglong2* q2 = reinterpret_cast<const ulonglong2*>(qv) + qbase * W;
            int acc_one[QPT], acc_opp[QPT];
#pragma unroll
            for (int q = 0; q < QPT; ++q) acc_one[q] = acc_opp[q] = 0;
#pragma unroll
            for (int w = 0; w < WW; ++w) {
                if (EXACT || w < W) {
#pragma unroll
                    for (int q = 0; q < QPT; ++q) {
                        const ulonglong2 qq = q2[q * W + w];
                        acc_one[q] += __popcll(qq.x ^ rm[w]);
                        acc_opp[q] += __popcll(qq.x & rm[w] & (qq.y ^ rn[w]));
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < QPT; ++q) {
                const int gq = qbase + q;
                if (gq < a.nqg) {
                    const uint32_t delta = (uint32_t)(acc_one[q] + 4 * acc_opp[q]);
                    const uint64_t key = ((uint64_t)delta << 32) | (uint64_t)row;
                    if (key < tau[gq]) {
                        // warp-aggregated: one slot reservation and one
                        // minimum per warp and query
                        const unsigned am = __activemask();
                        const int leader = __ffs(am) - 1;
                        const int rank = __popc(am & ((1u << lane) - 1u));
                        int pos0 = 0;
                        if (lane == leader) pos0 = atomicAdd(&cnt[gq], __popc(am));
                        pos0 = __shfl_sync(am, pos0, leader);
                        cand[gq * CAND_CAP + pos0 + rank] = key;
                        // each row is appended at most once: count it for the union bound
                        const uint32_t h = delta >> 1;
                        atomicAdd(&a.hist[gq * a.hist_bins + h], 1u);
                        const uint32_t wmin = __reduce_min_sync(am, h);
                        if (lane == leader && wmin < lmin[gq]) {
                            atomicMin(&lmin[gq], wmin);
                            atomicMin(&a.minhalf[gq], wmin);
                        }
                    }
                }
            }
        }
    }

    if (*abort_flag) {
        // drain the loads still in flight before the CTA exits
        if (tid == 0) {
            const int issued = min(ntl, it + a.stages);
            for (int j = it; j < issued; ++j)
                if (!mbar_wait_bounded(&bars[j % a.stages], (uint32_t)((j / a.stages) & 1))) break;
        }
        return;
    }
    if (tid < QB) {
        int32_t* m = a.meta + ((int64_t)tid * nslices + slice) * 2;
        m[0] = len[tid];
        m[1] = cur[tid];
    }
}

// Per pass: thresholds, histograms and minima of the union bound start empty.
__global__ void init_tau_kernel(uint64_t* tau_global, uint32_t* hist, int hist_words,
                                uint32_t* minhalf) {
    if (threadIdx.x < QB_MAX) {
        tau_global[threadIdx.x] = KEY_NONE;
        minhalf[threadIdx.x] = 0xFFFFFFFFu;
    }
    for (int i = threadIdx.x; i < hist_words; i += blockDim.x) hist[i] = 0u;
}

// Per query (one CTA): the k smallest keys of the union of the per-slice
// sorted lists.  With the scan's final threshold as a hint, the keys at or
// below it (at least k of them; usually a few more) are gathered and sorted
// directly.  Otherwise the k-th smallest key T of the union is found bit by
// bit from the top (the smallest T with count(key <= T) >= k), each count
// being a sum of per-list binary searches, with the lists staged in shared
// memory when they fit; then every list contributes its prefix of keys
// <= T (exactly k keys in all, keys being distinct) and those are sorted.
__device__ __forceinline__ int upper_bound_u64(const uint64_t* a, int n, uint64_t key) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] <= key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// The merge of one query q (one CTA): lists [q][nslices][2][k] with meta,
// the scan's threshold tau[q] and histogram hist[q] (either may be absent).
__device__ __forceinline__ void final_merge_query(
    const uint64_t* __restrict__ lists, const int32_t* __restrict__ meta,
    const uint64_t* __restrict__ tau, const uint32_t* __restrict__ hist,
    const uint32_t* __restrict__ minhalf, int hist_bins, int nslices, int k, int kl, int key_bits,
    int stage_lists, int bin_shift, int dist_bias, int64_t* __restrict__ ids,
    int32_t* __restrict__ dist, const int64_t q, uint8_t* smem) {
    // lists hold up to kl keys each (kl <= k: a scan with capped lists)
    __shared__ int red[FM_THREADS / 32];
    __shared__ int total_s;
    uint64_t* out = reinterpret_cast<uint64_t*>(smem);           // sort buffer
    int* lens = reinterpret_cast<int*>(smem + FM_OUT_BYTES);     // nslices
    int* offs = lens + FM_MAX_SLICES;                            // nslices
    uint64_t* staged = reinterpret_cast<uint64_t*>(smem + FM_OUT_BYTES + 2 * FM_MAX_SLICES * 4);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t qbase = q * nslices;

    // Lengths and buffer indices are clamped to the list storage: after a
    // scan that gave up (EVP_ERR_TIMEOUT) some of them were never written,
    // and the merge must still stay inside the workspace.
    for (int s = tid; s < nslices; s += FM_THREADS)
        lens[s] = min(max(meta[(qbase + s) * 2], 0), kl);
    __syncthreads();
    bool staged_now = false;
    auto list_ptr = [&](int s) -> const uint64_t* {
        return staged_now ? staged + (int64_t)s * kl
                          : lists + ((qbase + s) * 2 + (meta[(qbase + s) * 2 + 1] & 1)) * kl;
    };
    auto count_le = [&](uint64_t v) -> int {
        int c = 0;
        for (int s = tid; s < nslices; s += FM_THREADS) c += upper_bound_u64(list_ptr(s), lens[s], v);
        c = __reduce_add_sync(0xffffffffu, c);
        if (lane == 0) red[warp] = c;
        __syncthreads();
        int t = 0;
#pragma unroll
        for (int w = 0; w < FM_THREADS / 32; ++w) t += red[w];
        __syncthreads();
        return t;
    };
    // The scan's final threshold, when given, bounds the k-th smallest key
    // from above (at least k keys of the lists lie at or below it), and so
    // does the smallest T with count(Delta/2 <= T) >= k over the scan's
    // now complete histogram of listed keys; if few keys lie at or below the
    // tighter of the two, they are merged directly.
    uint64_t T = tau ? tau[q] : KEY_NONE;
    if (hist) {
        const uint32_t* H = hist + q * (int64_t)hist_bins;
        const uint32_t lo = minhalf[q];
        __shared__ uint32_t kth_bin;
        if (tid == 0) kth_bin = 0xFFFFFFFFu;
        __syncthreads();
        uint32_t before = 0;
        for (uint32_t h0 = lo; h0 < (uint32_t)hist_bins; h0 += FM_THREADS) {
            const uint32_t h = h0 + (uint32_t)tid;
            const uint32_t c = h < (uint32_t)hist_bins ? H[h] : 0u;
            uint32_t sum = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t nb = __shfl_up_sync(0xffffffffu, sum, o);
                if (lane >= o) sum += nb;
            }
            if (lane == 31) red[warp] = (int)sum;
            __syncthreads();
            uint32_t off = 0, total = 0;
#pragma unroll
            for (int w = 0; w < FM_THREADS / 32; ++w) {
                const uint32_t v = (uint32_t)red[w];
                if (w < warp) off += v;
                total += v;
            }
            sum += off;
            if (c > 0 && before + sum >= (uint32_t)k && before + sum - c < (uint32_t)k) kth_bin = h;
            __syncthreads();
            before += total;
            if (kth_bin != 0xFFFFFFFFu || before >= (uint32_t)k) break;
        }
        // histogram bins are Delta/2 (bin_shift < 0) or (key >> 32) >> bin_shift
        if (kth_bin != 0xFFFFFFFFu)
            T = min(T, bin_shift < 0 ? (uint64_t)(2u * kth_bin + 1u) << 32
                                     : ((uint64_t)(kth_bin + 1u) << bin_shift) << 32);
    }
    int m = T != KEY_NONE ? count_le(T) : FM_GATHER + 1;
    if (m < k || m > FM_GATHER) {
        if (stage_lists) {
            for (int64_t e = tid; e < (int64_t)nslices * kl; e += FM_THREADS) {
                const int s = (int)(e / kl), i = (int)(e - (int64_t)s * kl);
                if (i < lens[s]) staged[e] = lists[((qbase + s) * 2 + (meta[(qbase + s) * 2 + 1] & 1)) * kl + i];
            }
            __syncthreads();
            staged_now = true;
        }
        // smallest T with count(key <= T) >= k, built bit by bit
        T = 0;
        for (int b = key_bits - 1; b >= 0; --b) {
            const uint64_t lowmax = T | ((1ull << b) - 1ull);
            if (count_le(lowmax) < k) T |= 1ull << b;
        }
        m = k;
    }
    // each list's prefix of keys <= T (m keys in all), gathered at
    // exclusive-scan offsets, then sorted
    for (int s = tid; s < nslices; s += FM_THREADS) offs[s] = upper_bound_u64(list_ptr(s), lens[s], T);
    __syncthreads();
    if (tid == 0) {
        int run = 0;
        for (int s = 0; s < nslices; ++s) {
            const int c = offs[s];
            offs[s] = run;
            run += c;
        }
        total_s = run;
    }
    __syncthreads();
    const int cap = max(m, k);
    const int n = min(total_s, min(cap, k));
    int P = 2;
    while (P < cap) P <<= 1;
    for (int i = tid; i < P; i += FM_THREADS) out[i] = KEY_NONE;
    __syncthreads();
    for (int s = tid; s < nslices; s += FM_THREADS) {
        const uint64_t* L = list_ptr(s);
        const int o = offs[s];
        const int c = upper_bound_u64(L, lens[s], T);
        for (int i = 0; i < c && o + i < cap; ++i) out[o + i] = L[i];
    }
    __syncthreads();
    for (int kk = 2; kk <= P; kk <<= 1) {
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
            for (int i = tid; i < P; i += FM_THREADS) {
                const int ixj = i ^ jj;
                if (ixj > i) {
                    const uint64_t a = out[i], b = out[ixj];
                    if ((a > b) == ((i & kk) == 0)) {
                        out[i] = b;
                        out[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int j = tid; j < k; j += FM_THREADS) {
        const uint64_t key = j < n ? out[j] : KEY_NONE;
        ids[q * k + j] = key == KEY_NONE ? -1 : (int64_t)(key & 0xffffffffull);
        dist[q * k + j] = key == KEY_NONE ? -1
                          : dist_bias ? dist_bias - (int32_t)(key >> 32) : (int32_t)(key >> 32);
    }
}

__global__ void __launch_bounds__(FM_THREADS)
final_merge_kernel(const uint64_t* __restrict__ lists, const int32_t* __restrict__ meta,
                   const uint64_t* __restrict__ tau, const uint32_t* __restrict__ hist,
                   const uint32_t* __restrict__ minhalf, int hist_bins, int nslices, int k,
                   int kl, int key_bits, int stage_lists, int bin_shift, int dist_bias,
                   int64_t* __restrict__ ids, int32_t* __restrict__ dist) {
    extern __shared__ __align__(1024) uint8_t smem[];
    final_merge_query(lists, meta, tau, hist, minhalf, hist_bins, nslices, k, kl, key_bits,
                      stage_lists, bin_shift, dist_bias, ids, dist, (int64_t)blockIdx.x, smem);
}

// Several batches in one launch: CTA i merges query i - q0[b] of the batch b
// with q0[b] <= i < q0[b + 1].
__global__ void __launch_bounds__(FM_THREADS)
final_merge_multi_kernel(const FmBatch* __restrict__ tab, int nb, int key_bits) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const int64_t i = blockIdx.x;
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tab[mid].q0 <= i) lo = mid;
        else hi = mid - 1;
    }
    const FmBatch& b = tab[lo];
    final_merge_query(b.lists, b.meta, b.tau, b.hist, b.minhalf, b.hist_bins, b.nslices, b.k,
                      b.kl, key_bits, b.stage, -1, 0, b.ids, b.dist, i - b.q0, smem);
}

int choose_stages(int W, int qb) {
    for (int st = MAX_STAGES; st >= 2; --st)
        if (smem_layout(W, st, qb).total <= (size_t)SMEM_BUDGET) return st;
    return 0;
}

template <int QB, int TPR, int WW, bool EXACT>
cudaError_t launch_scan_w(const CUtensorMap& tmap, const ScanArgs& a, int nslices, size_t smem,
                          cudaStream_t stream) {
    cudaError_t e = cudaFuncSetAttribute(scan_popc_kernel<QB, TPR, WW, EXACT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         SMEM_BUDGET + 2048);
    if (e != cudaSuccess) return e;
    TimedLaunch timer("scan_popc", stream);
    scan_popc_kernel<QB, TPR, WW, EXACT><<<nslices, SCAN_ROWS * TPR, smem, stream>>>(tmap, a);
    return cudaGetLastError();
}

// Rows are held in registers, WW >= W words per plane: the common widths
// (d = 384, 768, 1024) exactly, the others padded to the next of 4, 8, 12, 16.
template <int QB, int TPR>
cudaError_t launch_scan(const CUtensorMap& tmap, const ScanArgs& a, int nslices, size_t smem,
                        cudaStream_t stream) {
    switch (a.W) {
        case 6: return launch_scan_w<QB, TPR, 6, true>(tmap, a, nslices, smem, stream);
        case 12: return launch_scan_w<QB, TPR, 12, true>(tmap, a, nslices, smem, stream);
        case 16: return launch_scan_w<QB, TPR, 16, true>(tmap, a, nslices, smem, stream);
        default: break;
    }
    if (a.W <= 4) return launch_scan_w<QB, TPR, 4, false>(tmap, a, nslices, smem, stream);
    if (a.W <= 8) return launch_scan_w<QB, TPR, 8, false>(tmap, a, nslices, smem, stream);
    if (a.W <= 12) return launch_scan_w<QB, TPR, 12, false>(tmap, a, nslices, smem, stream);
    return launch_scan_w<QB, TPR, 16, false>(tmap, a, nslices, smem, stream);
}

}  // namespace

// Shard results (ids, dist) [nlists][nq][k] -> key lists [nq][nlists][2][k]
// (buffer 0) and meta (valid length, buffer 0): one warp per (query, list).
// A list ends at its first id < 0; ids must lie in [0, 2^31).
__global__ void pack_lists_kernel(const int64_t* __restrict__ ids, const int32_t* __restrict__ dist,
                                  int64_t nq, int nlists, int k, uint64_t* __restrict__ lists,
                                  int32_t* __restrict__ meta, int32_t* __restrict__ status) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nq * nlists) return;
    const int64_t q = w / nlists;
    const int s = (int)(w - q * nlists);
    const int64_t src = ((int64_t)s * nq + q) * k;
    uint64_t* dst = lists + ((q * nlists + s) * 2) * k;
    int len = k;
    for (int i0 = 0; i0 < k; i0 += 32) {
        const int i = i0 + lane;
        const int64_t id = i < k ? ids[src + i] : -1;
        const unsigned bad = __ballot_sync(0xffffffffu, i < k && (id < 0 || id >= (int64_t(1) << 31)));
        if (bad) len = min(len, i0 + __ffs(bad) - 1);
        if (i < k && id >= 0 && id < (int64_t(1) << 31))
            dst[i] = ((uint64_t)(uint32_t)dist[src + i] << 32) | (uint64_t)id;
        if (i < k && id >= (int64_t(1) << 31)) report(status, EVP_ERR_RANGE);
    }
    if (lane == 0) {
        meta[(q * nlists + s) * 2] = len;
        meta[(q * nlists + s) * 2 + 1] = 0;
    }
}

size_t final_merge_smem(int nslices, int k, int* stage) {
    const size_t list_bytes = (size_t)nslices * k * 8;
    *stage = list_bytes <= (size_t)FM_STAGE_BYTES ? 1 : 0;
    return FM_OUT_BYTES + 2 * FM_MAX_SLICES * 4 + (*stage ? list_bytes : 0);
}

int32_t launch_final_merge_multi(const FmBatch* tab, int nb, int64_t total_q, size_t smem,
                                 cudaStream_t stream) {
    if (total_q <= 0) return EVP_OK;
    if (cudaFuncSetAttribute(final_merge_multi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             FM_OUT_BYTES + 2 * FM_MAX_SLICES * 4 + FM_STAGE_BYTES) != cudaSuccess)
        return EVP_ERR_CUDA;
    TimedLaunch timer("final_merge", stream);
    final_merge_multi_kernel<<<(unsigned)total_q, FM_THREADS, smem, stream>>>(tab, nb, 32 + 13);
    return cudaGetLastError() == cudaSuccess ? EVP_OK : EVP_ERR_CUDA;
}

int32_t launch_final_merge(const uint64_t* lists, const int32_t* meta, const uint64_t* tau,
                           const uint32_t* hist, const uint32_t* minhalf, int hist_bins,
                           int64_t nq, int nslices, int k, int64_t* ids, int32_t* dist,
                           cudaStream_t stream, int bin_shift, int dist_bias, int kl) {
    if (nq <= 0) return EVP_OK;
    if (nslices > FM_MAX_SLICES) return EVP_ERR_UNSUPPORTED;
    if (kl <= 0 || kl > k) kl = k;
    const size_t list_bytes = (size_t)nslices * kl * 8;
    const int stage = list_bytes <= (size_t)FM_STAGE_BYTES ? 1 : 0;
    const size_t smem = FM_OUT_BYTES + 2 * FM_MAX_SLICES * 4 + (stage ? list_bytes : 0);
    if (cudaFuncSetAttribute(final_merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             FM_OUT_BYTES + 2 * FM_MAX_SLICES * 4 + FM_STAGE_BYTES) != cudaSuccess)
        return EVP_ERR_CUDA;
    // keys are (Delta << 32 | row) with Delta <= 4 * EVP_MAX_D_SCAN, or
    // (bias - score) << 32 | row with the score key below 2^18
    const int key_bits = 32 + (bin_shift < 0 ? 13 : 18);
    TimedLaunch timer("final_merge", stream);
    final_merge_kernel<<<(unsigned)nq, FM_THREADS, smem, stream>>>(
        lists, meta, tau, hist, minhalf, hist_bins, nslices, k, kl, key_bits, stage, bin_shift,
        dist_bias, ids, dist);
    return cudaGetLastError() == cudaSuccess ? EVP_OK : EVP_ERR_CUDA;
}

size_t merge_topk_workspace(int64_t nq, int nlists, int k) {
    return align_up((size_t)nq * nlists * 2 * k * 8, 256) + align_up((size_t)nq * nlists * 2 * 4, 256);
}

int32_t run_merge_topk(const int64_t* ids, const int32_t* dist, int64_t nq, int nlists, int k,
                       int64_t* out_ids, int32_t* out_dist, void* ws, size_t ws_bytes,
                       int32_t* status, cudaStream_t stream) {
    if (ws_bytes < merge_topk_workspace(nq, nlists, k)) return EVP_ERR_NO_MEMORY;
    uint64_t* lists = static_cast<uint64_t*>(ws);
    int32_t* meta = reinterpret_cast<int32_t*>(static_cast<uint8_t*>(ws) +
                                               align_up((size_t)nq * nlists * 2 * k * 8, 256));
    const int64_t warps = nq * nlists;
    {
        TimedLaunch timer("pack_lists", stream);
        pack_lists_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, stream>>>(
            ids, dist, nq, nlists, k, lists, meta, status);
    }
    if (cudaGetLastError() != cudaSuccess) return EVP_ERR_CUDA;
    return launch_final_merge(lists, meta, nullptr, nullptr, nullptr, 0, nq, nlists, k, out_ids,
                              out_dist, stream);
}

ScanPlan plan_popc_scan(int64_t nq, int64_t ns, int d, int k) {
    ScanPlan p{};
    const int64_t ntiles = std::max<int64_t>(1, (ns + SCAN_ROWS - 1) / SCAN_ROWS);
    const int64_t tps = (ntiles + num_sms() - 1) / num_sms();  // tiles per slice
    p.nslices = (int)((ntiles + tps - 1) / tps);
    p.qb = (int)std::min<int64_t>(QB_MAX, std::max<int64_t>(1, nq));
    p.groups = (int)((nq + QB_MAX - 1) / QB_MAX);
    p.list_bytes = align_up((size_t)QB_MAX * p.nslices * 2 * k * 8, 256);
    p.meta_bytes = align_up((size_t)QB_MAX * p.nslices * 2 * 4, 256);
    // union-bound histograms: Delta/2 in [0, 2x], x <= d
    p.hist_bytes = align_up((size_t)QB_MAX * (2 * d + 1) * 4, 256) + 256;
    p.ws_bytes = p.list_bytes + p.meta_bytes + p.hist_bytes + 256;
    return p;
}

int32_t run_popc_knn(const uint64_t* Q, int64_t nq, const uint64_t* S, int64_t ns, int d,
                     int x, int k, int64_t* ids, int32_t* dist, void* ws, size_t ws_bytes,
                     int32_t* status, cudaStream_t stream) {
    const int W = (d + 63) / 64;
    const ScanPlan p = plan_popc_scan(nq, ns, d, k);
    if (ws_bytes < p.ws_bytes) return EVP_ERR_NO_MEMORY;
    if (choose_stages(W, QB_MAX) == 0) return EVP_ERR_UNSUPPORTED;

    EncodeTiledFn enc = encode_tiled_fn();
    if (!enc) return EVP_ERR_CUDA;
    CUtensorMap tmap;
    const int pitch = row_pitch_words(W);
    cuuint64_t gdim[2] = {(cuuint64_t)(2 * W), (cuuint64_t)ns};
    cuuint64_t gstride[1] = {(cuuint64_t)(16 * W)};
    cuuint32_t box[2] = {(cuuint32_t)pitch, (cuuint32_t)SCAN_ROWS};
    cuuint32_t estride[2] = {1, 1};
    CUresult cr = enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<uint64_t*>(S), gdim,
                      gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return EVP_ERR_CUDA;

    uint8_t* wsb = static_cast<uint8_t*>(ws);
    ScanArgs a{};
    a.ns = ns;
    a.W = W;
    a.k = k;
    a.pitch = pitch;
    a.ntiles = (ns + SCAN_ROWS - 1) / SCAN_ROWS;
    a.tiles_per_slice = (a.ntiles + num_sms() - 1) / num_sms();
    a.lists = reinterpret_cast<uint64_t*>(wsb);
    a.meta = reinterpret_cast<int32_t*>(wsb + p.list_bytes);
    a.tau_global = reinterpret_cast<uint64_t*>(wsb + p.ws_bytes - 256);
    a.hist = reinterpret_cast<uint32_t*>(wsb + p.list_bytes + p.meta_bytes);
    a.minhalf = reinterpret_cast<uint32_t*>(wsb + p.list_bytes + p.meta_bytes + p.hist_bytes - 256);
    a.hist_bins = 2 * x + 1;
    a.status = status;


    for (int g = 0; g < p.groups; ++g) {
        const int64_t q0 = (int64_t)g * QB_MAX;
        const int nqg = (int)std::min<int64_t>(QB_MAX, nq - q0);
        a.Q = Q + q0 * 2 * W;
        a.nqg = nqg;
        const int qb = nqg <= 1 ? 1 : nqg <= 2 ? 2 : nqg <= 4 ? 4 : nqg <= 8 ? 8 : 16;
        a.stages = choose_stages(W, qb);
        const SmemLayout L = smem_layout(W, a.stages, qb);
        {
            TimedLaunch timer("scan_init", stream);
            init_tau_kernel<<<1, 256, 0, stream>>>(a.tau_global, a.hist, QB_MAX * a.hist_bins,
                                                  a.minhalf);
        }
        cudaError_t e;
        if (nqg <= 1) e = launch_scan<1, 1>(tmap, a, p.nslices, L.total, stream);
        else if (nqg <= 2) e = launch_scan<2, 1>(tmap, a, p.nslices, L.total, stream);
        else if (nqg <= 4) e = launch_scan<4, 1>(tmap, a, p.nslices, L.total, stream);
        else if (nqg <= 8) e = launch_scan<8, 2>(tmap, a, p.nslices, L.total, stream);
        else e = launch_scan<16, 2>(tmap, a, p.nslices, L.total, stream);
        if (e != cudaSuccess) return EVP_ERR_CUDA;
        const int32_t rc = launch_final_merge(a.lists, a.meta, a.tau_global, a.hist, a.minhalf,
                                              a.hist_bins, nqg, p.nslices, k,
                                              ids + q0 * k, dist + q0 * k, stream);
        if (rc != EVP_OK) return rc;
    }
    return EVP_OK;
}

}  // namespace evp
