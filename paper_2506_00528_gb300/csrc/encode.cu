// evp_encode kernel: nearest {x,d} EVP vertex of each float32 row
// (Sec. 2.4), packed into the v+/v- bitplanes of Sec. 5.1.2.
//
// One warp per row.  Lane l holds elements j = l + 32 t (t < VPL), so one
// warp load instruction covers 128 contiguous bytes of the row and, for a
// fixed t, the 32 lanes hold exactly the 32-bit half-word t of each plane:
// two warp ballots (selected, negative) give it with no shuffles; lane 0
// stages the ballots in shared memory and lane w assembles words w of v+
// and v-.
//
// Selection of the x largest |u_i|.  Magnitudes order exactly by their
// 31-bit key (float bits with the sign cleared), and for finite values the
// same order is the float order of |u|, so comparisons run on |u| as
// floats.  The threshold tau is the x-th largest key; keys above tau are
// selected and keys equal to tau are taken in ascending element index
// until x are chosen.
//
// Finding tau (exactly) in three steps:
//  1. Bracket.  The x-th largest magnitude varies little from row to row
//     (a few per cent for normalised embeddings), so each warp keeps a
//     running estimate and brackets it, [p1, p2) = estimate x (1 -+ EPS).
//     One pass over the row counts the keys >= p2 and writes the keys inside
//     the bracket to this lane's column in shared memory (lane-interleaved,
//     so the writes never conflict).  tau lies in the bracket iff
//     count(>= p2) < x <= count(>= p2) + count(bracket).
//  2. Refine.  The bracketed keys (a few per lane) are counted into 32
//     equal-width bins of key values; a suffix scan over the bins finds the
//     bin holding the x-th largest, and that bin's keys (a handful) are
//     gathered, one per lane, and ranked against each other.
//  3. Otherwise (a bracket miss, more than 32 keys in the bin, or the first
//     row of a warp) tau is built bit by bit from the top key bit down,
//     counting over all keys at every step.
// Elements past d (the last slot of a row whose d is not a multiple of 32)
// are loaded as NaN, which no comparison selects or counts.
#include "evp_internal.cuh"

namespace evp {

namespace {

constexpr int ENC_THREADS = 256;
constexpr int ENC_WARPS = ENC_THREADS / 32;
constexpr unsigned FULL = 0xffffffffu;
constexpr float ENC_EPS = 0.18f;      // half-width of the bracket, relative to the estimate
constexpr float ENC_EMA = 0.25f;      // weight of the newest threshold in the estimate

// Per-warp shared memory: VPL x 32 column words, 32 histogram bins, a
// 32-slot gather buffer and 2 VPL ballot words.
template <int VPL>
struct EncSmem {
    static constexpr int WORDS = VPL * 32 + 64 + 2 * VPL;
};

// Number of this warp's elements with |u| >= v (v a finite magnitude or +inf;
// a NaN v counts nothing), reduced over the warp.
template <int VPL>
__device__ __forceinline__ int count_ge(const float (&u)[VPL], float v) {
    int c = 0;
#pragma unroll
    for (int t = 0; t < VPL; ++t) c += fabsf(u[t]) >= v ? 1 : 0;
    return __reduce_add_sync(FULL, c);
}

// EXACT: d == 32 VPL (no padding slots).  PREFETCH: the next row is loaded
// into registers while this one is processed.
template <int VPL, bool EXACT, bool PREFETCH>
__global__ void __launch_bounds__(ENC_THREADS)
encode_kernel(const float* __restrict__ U, int64_t n, int d, int x, int W,
              uint64_t* __restrict__ T, int32_t* __restrict__ status) {
    static_assert(VPL >= 1 && VPL <= 64, "VPL range");
    extern __shared__ uint32_t enc_smem[];
    const int lane = threadIdx.x & 31;
    const unsigned lanemask_lt = (1u << lane) - 1u;
    const int64_t warp0 = ((int64_t)blockIdx.x * ENC_THREADS + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * ENC_THREADS) >> 5;
    uint32_t* wsm = enc_smem + (threadIdx.x >> 5) * EncSmem<VPL>::WORDS;
    uint32_t* col = wsm + lane;        // this lane's column: word j at col[32 j]
    uint32_t* hist = wsm + VPL * 32;   // [32] bins of the bracket
    uint32_t* fin = hist + 32;         // [32] keys of the bin holding tau
    uint32_t* bal = fin + 32;          // [2 VPL] ballots: selected, then negative
    const float pad = __int_as_float(0x7fffffff);  // NaN: never counted, never selected

    auto load_row = [&](int64_t row, float (&v)[VPL]) {
        const float* src = U + row * (int64_t)d;
#pragma unroll
        for (int t = 0; t < VPL; ++t) {
            const int j = lane + 32 * t;
            v[t] = (EXACT || j < d) ? __ldcs(src + j) : pad;
        }
    };

    float nxt[VPL];
    int64_t row = warp0;
    if (PREFETCH && row < n) load_row(row, nxt);
    float est = 0.f;  // running estimate of this warp's thresholds (0: none yet)
    for (; row < n; row += nwarps) {
        float u[VPL];
        if constexpr (PREFETCH) {
#pragma unroll
            for (int t = 0; t < VPL; ++t) u[t] = nxt[t];
            if (row + nwarps < n) load_row(row + nwarps, nxt);
        } else {
            load_row(row, u);
        }
        // non-finite input: u * 0 is NaN exactly when u is NaN or infinite
        {
            float z = 0.f;
#pragma unroll
            for (int t = 0; t < VPL; ++t)
                if (EXACT || lane + 32 * t < d) z = fmaf(u[t], 0.f, z);
            if (__any_sync(FULL, z != z) && lane == 0) report(status, EVP_ERR_NONFINITE);
        }

        // 1. bracket [p1, p2) around the estimate
        const float p1f = est * (1.f - ENC_EPS), p2f = est * (1.f + ENC_EPS);
        int above_p2 = 0;
        uint32_t* cp = col;
#pragma unroll
        for (int t = 0; t < VPL; ++t) {
            const float m = fabsf(u[t]);
            const bool ge2 = m >= p2f;
            above_p2 += ge2 ? 1 : 0;
            if (!ge2 && m >= p1f) {
                *cp = __float_as_uint(m);
                cp += 32;
            }
        }
        const int cnt = (int)((cp - col) >> 5);
        const int A = __reduce_add_sync(FULL, above_p2);
        const int L = __reduce_add_sync(FULL, cnt);

        uint32_t tau = 0;
        int need = 0, eqn = 0;
        bool found = false;
        if (A < x && x <= A + L) {
            // 2. refine: 32 bins of 2^s key values from p1
            const uint32_t p1 = __float_as_uint(p1f), p2 = __float_as_uint(p2f);
            const uint32_t wv = (p2 - p1 - 1u) >> 5;
            const int s = wv ? 32 - __clz(wv) : 0;
            hist[lane] = 0u;
            __syncwarp();
            const int maxc = __reduce_max_sync(FULL, cnt);
            for (int j = 0; j < maxc; ++j)
                if (j < cnt) atomicAdd(&hist[(col[32 * j] - p1) >> s], 1u);
            __syncwarp();
            // S = keys in bins >= 31 - lane (lane 0 holds the top bin)
            const uint32_t c = hist[31 - lane];
            uint32_t S = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(FULL, S, o);
                if (lane >= o) S += v;
            }
            const int r = x - A;  // tau is the r-th largest bracketed key
            const int f = __ffs(__ballot_sync(FULL, S >= (uint32_t)r)) - 1;
            const int m = (int)__shfl_sync(FULL, c, f);
            if (m <= 32) {
                const int r2 = r - (int)__shfl_sync(FULL, S - c, f);  // rank within the bin
                const uint32_t B = 31u - (uint32_t)f;
                int base = 0;
                for (int j = 0; j < maxc; ++j) {
                    const uint32_t key = j < cnt ? col[32 * j] : 0u;
                    const bool inb = j < cnt && ((key - p1) >> s) == B;
                    const unsigned bm = __ballot_sync(FULL, inb);
                    if (inb) fin[base + __popc(bm & lanemask_lt)] = key;
                    base += __popc(bm);
                }
                __syncwarp();
                const uint32_t v = lane < m ? fin[lane] : 0u;
                int g = 0, e = 0;
                for (int j = 0; j < m; ++j) {
                    const uint32_t w = __shfl_sync(FULL, v, j);
                    g += w > v ? 1 : 0;
                    e += w == v ? 1 : 0;
                }
                const int f2 =
                    __ffs(__ballot_sync(FULL, lane < m && g < r2 && r2 <= g + e)) - 1;
                tau = __shfl_sync(FULL, v, f2);
                need = r2 - __shfl_sync(FULL, g, f2);
                eqn = __shfl_sync(FULL, e, f2);
                found = true;
            }
            __syncwarp();  // hist and fin are reused by the next row
        }
        if (!found) {
            // 3. exact: tau = max{v : #(key >= v) >= x}, bit by bit
#pragma unroll 1
            for (int b = 30; b >= 0; --b) {
                const uint32_t cand = tau | (1u << b);
                if (count_ge(u, __uint_as_float(cand)) >= x) tau = cand;
            }
            const int gt = count_ge(u, __uint_as_float(tau + 1u));
            need = x - gt;
            eqn = count_ge(u, __uint_as_float(tau)) - gt;
        }
        const float tf = __uint_as_float(tau);
        if (tau > 0u && tau < 0x7f800000u) est = est > 0.f ? est + ENC_EMA * (tf - est) : tf;

        // selection and packing
        const bool all_eq = need >= eqn;  // every key equal to tau is taken
        int base = 0;
#pragma unroll
        for (int t = 0; t < VPL; ++t) {
            const float m = fabsf(u[t]);
            bool sel;
            if (all_eq) {
                sel = m >= tf;
            } else {
                const bool eq = m == tf;
                const unsigned bm = __ballot_sync(FULL, eq);
                const int rank = base + __popc(bm & lanemask_lt);
                base += __popc(bm);
                sel = m > tf || (eq && rank < need);
            }
            const unsigned bs = __ballot_sync(FULL, sel);
            const unsigned bg = __ballot_sync(FULL, u[t] < 0.f);  // -0.0 counts as +1
            if (lane == 0) {
                bal[t] = bs;
                bal[VPL + t] = bg;
            }
        }
        __syncwarp();
        if (lane < W) {
            const uint32_t s0 = bal[2 * lane], g0 = bal[VPL + 2 * lane];
            const uint32_t s1 = 2 * lane + 1 < VPL ? bal[2 * lane + 1] : 0u;
            const uint32_t g1 = 2 * lane + 1 < VPL ? bal[VPL + 2 * lane + 1] : 0u;
            const uint64_t sel = ((uint64_t)s1 << 32) | s0, neg = ((uint64_t)g1 << 32) | g0;
            uint64_t* out = T + row * (int64_t)(2 * W);
            out[lane] = sel & ~neg;
            out[W + lane] = sel & neg;
        }
        __syncwarp();  // bal is rewritten by the next row
    }
}

template <int VPL, bool EXACT>
cudaError_t launch_vpl(const float* U, int64_t n, int d, int x, uint64_t* T, int32_t* status,
                       cudaStream_t stream) {
    // measured: prefetching the next row into registers costs more (register
    // copies, lower occupancy) than it hides at 24-32 rows in flight per SM
    constexpr bool PREFETCH = false;
    auto kern = encode_kernel<VPL, EXACT, PREFETCH>;
    const int W = (d + 63) / 64;
    const size_t smem = (size_t)ENC_WARPS * EncSmem<VPL>::WORDS * 4;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
        return cudaErrorInvalidValue;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, ENC_THREADS, smem) !=
            cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    // persistent: as many warps as are resident, each walking rows with a stride
    int64_t blocks = (n + ENC_WARPS - 1) / ENC_WARPS;
    const int64_t cap = (int64_t)num_sms() * per_sm;
    if (blocks > cap) blocks = cap;
    TimedLaunch timer("encode", stream);
    kern<<<(unsigned)blocks, ENC_THREADS, smem, stream>>>(U, n, d, x, W, T, status);
    return cudaGetLastError();
}

template <int VPL>
cudaError_t launch_v(const float* U, int64_t n, int d, int x, uint64_t* T, int32_t* status,
                     cudaStream_t stream) {
    return d == 32 * VPL ? launch_vpl<VPL, true>(U, n, d, x, T, status, stream)
                         : launch_vpl<VPL, false>(U, n, d, x, T, status, stream);
}

}  // namespace

cudaError_t launch_encode(const float* U, int64_t n, int d, int x, uint64_t* T,
                          int32_t* status, cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    const int vpl = (d + 31) / 32;
    if (vpl <= 1) return launch_v<1>(U, n, d, x, T, status, stream);
    if (vpl <= 2) return launch_v<2>(U, n, d, x, T, status, stream);
    if (vpl <= 4) return launch_v<4>(U, n, d, x, T, status, stream);
    if (vpl <= 8) return launch_v<8>(U, n, d, x, T, status, stream);
    if (vpl <= 12) return launch_v<12>(U, n, d, x, T, status, stream);
    if (vpl <= 16) return launch_v<16>(U, n, d, x, T, status, stream);
    if (vpl <= 24) return launch_v<24>(U, n, d, x, T, status, stream);
    if (vpl <= 32) return launch_v<32>(U, n, d, x, T, status, stream);
    if (vpl <= 48) return launch_v<48>(U, n, d, x, T, status, stream);
    return launch_v<64>(U, n, d, x, T, status, stream);
}

}  // namespace evp
