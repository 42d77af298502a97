// evp_encode kernel: nearest {x,d} EVP vertex of each float32 row
// (Sec. 2.4), packed into the v+/v- bitplanes of Sec. 5.1.2.
//
// One warp per row.  Lane l holds elements j = l + 32 t (t < VPL), so one
// warp load instruction covers 128 contiguous bytes of the row and, for a
// fixed t, the 32 lanes hold exactly the 32-bit half-word t of each plane:
// a warp ballot packs it with no shuffles.
//
// Selection of the x largest |u_i|: the 31-bit magnitude key (float bits
// with the sign cleared) orders magnitudes exactly.  The threshold tau is
// the x-th largest key, found as the largest value with
// count(key >= tau) >= x by a bitwise search from the row's top key bit
// down.  To make each count cheap, every lane first sorts its own keys
// (a merge-exchange comparator network in registers) and stores the sorted
// column in shared memory; a count is then one binary search per lane and
// one warp reduction.  Keys above tau are selected; keys equal to tau are
// taken in ascending element index until x are chosen.
#include "evp_internal.cuh"

#include <utility>

namespace evp {

namespace {

constexpr int ENC_THREADS = 256;
constexpr int ENC_WARPS = ENC_THREADS / 32;
constexpr unsigned FULL = 0xffffffffu;

// Batcher's merge-exchange network for N keys (Knuth, The Art of Computer
// Programming vol. 3, Algorithm 5.2.2M): a fixed list of comparators
// (i, j), i < j, that sorts any input.  The c-th comparator is computed at
// compile time, so the network is straight-line code on registers.
template <int N>
struct MergeExchange {
    // Calls f(i, j) for every comparator in order; stops (returns false)
    // when f returns false.
    template <typename F>
    static constexpr void walk(F&& f) {
        if (N < 2) return;
        int t = 0;
        while ((1 << t) < N) ++t;
        for (int p = 1 << (t - 1); p > 0; p >>= 1) {
            int q = 1 << (t - 1), r = 0, dd = p;
            while (true) {
                for (int i = 0; i < N - dd; ++i)
                    if ((i & p) == r && !f(i, i + dd)) return;
                if (q == p) break;
                dd = q - p;
                q >>= 1;
                r = p;
            }
        }
    }
    static constexpr int count() {
        int c = 0;
        walk([&](int, int) { ++c; return true; });
        return c;
    }
    // end 0: i, end 1: j of comparator number c
    static constexpr int at(int c, int end) {
        int k = 0, out = 0;
        walk([&](int i, int j) {
            if (k++ == c) {
                out = end ? j : i;
                return false;
            }
            return true;
        });
        return out;
    }
    static constexpr int M = count();
};

// Descending sort of s[0, N) in registers by the merge-exchange network.
template <int N, int... C>
__device__ __forceinline__ void sort_desc_net(uint32_t (&s)[N], std::integer_sequence<int, C...>) {
    (
        [&] {
            constexpr int i = MergeExchange<N>::at(C, 0), j = MergeExchange<N>::at(C, 1);
            const uint32_t lo = s[i], hi = s[j];
            s[i] = max(lo, hi);
            s[j] = min(lo, hi);
        }(),
        ...);
}

template <int N>
__device__ __forceinline__ void sort_desc(uint32_t (&s)[N]) {
    sort_desc_net(s, std::make_integer_sequence<int, MergeExchange<N>::M>{});
}

template <int VPL>
__global__ void __launch_bounds__(ENC_THREADS)
encode_kernel(const float* __restrict__ U, int64_t n, int d, int x, int W,
              uint64_t* __restrict__ T, int32_t* __restrict__ status) {
    static_assert(VPL >= 1 && VPL <= 64, "VPL range");
    extern __shared__ uint32_t enc_smem[];  // [ENC_WARPS][VPL][32]: sorted key columns
    const int lane = threadIdx.x & 31;
    const unsigned lanemask_lt = (1u << lane) - 1u;
    const int64_t warp0 = ((int64_t)blockIdx.x * ENC_THREADS + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * ENC_THREADS) >> 5;
    uint32_t* col = enc_smem + (threadIdx.x >> 5) * VPL * 32 + lane;  // this lane's column
    // largest power of two <= VPL: the binary search can then reach any count 0..VPL
    constexpr int TOP = VPL >= 64 ? 64 : VPL >= 32 ? 32 : VPL >= 16 ? 16 : VPL >= 8 ? 8
                      : VPL >= 4 ? 4 : VPL >= 2 ? 2 : 1;

    for (int64_t row = warp0; row < n; row += nwarps) {
        const float* u = U + row * (int64_t)d;
        // this lane's keys in descending order, into its shared-memory column
        {
            uint32_t key[VPL];
            bool bad = false;
#pragma unroll
            for (int t = 0; t < VPL; ++t) {
                const int j = lane + 32 * t;
                key[t] = j < d ? (__float_as_uint(__ldg(u + j)) & 0x7fffffffu) : 0u;
                bad |= key[t] >= 0x7f800000u;
            }
            if (__any_sync(FULL, bad) && lane == 0) report(status, EVP_ERR_NONFINITE);
            sort_desc(key);
            __syncwarp();  // the previous row's searches are done with the column
#pragma unroll
            for (int t = 0; t < VPL; ++t) col[t * 32] = key[t];
            __syncwarp();
        }
        // number of this lane's keys >= v: binary search down the sorted column
        auto count_ge = [&](uint32_t v) -> int {
            int pos = 0;
#pragma unroll
            for (int s = TOP; s >= 1; s >>= 1)
                if (pos + s <= VPL && col[(pos + s - 1) * 32] >= v) pos += s;
            return pos;
        };

        // tau = max{v : #(key >= v) >= x}; bits above the row's largest key
        // cannot be set.  Padding keys are 0 and only count at v = 0, where
        // every real element counts as well.
        const uint32_t kmax = __reduce_max_sync(FULL, col[0]);
        uint32_t tau = 0;
#pragma unroll 1
        for (int b = kmax ? 31 - __clz(kmax) : -1; b >= 0; --b) {
            const uint32_t cand = tau | (1u << b);
            if (__reduce_add_sync(FULL, count_ge(cand)) >= x) tau = cand;
        }
        const int gt = __reduce_add_sync(FULL, count_ge(tau + 1u));
        const int need = x - gt;  // keys equal to tau still to take, lowest index first
        // usually every key equal to tau is taken (no ties beyond the x-th)
        const int eq_real = __reduce_add_sync(FULL, count_ge(tau)) - gt;
        const bool all_eq = tau != 0 && eq_real <= need;

        // selection and packing, from the row read again (L1/L2)
        uint64_t wp = 0, wn = 0;  // this lane's output words (lane < W)
        int base = 0;
#pragma unroll
        for (int t = 0; t < VPL; ++t) {
            const int j = lane + 32 * t;
            const uint32_t b = j < d ? __float_as_uint(__ldg(u + j)) : 0u;
            const uint32_t key = b & 0x7fffffffu;
            bool sel;
            if (all_eq) {
                sel = key >= tau;
            } else {
                const bool eq = key == tau && j < d;
                const unsigned m = __ballot_sync(FULL, eq);
                const int rank = base + __popc(m & lanemask_lt);
                base += __popc(m);
                sel = key > tau || (eq && rank < need);
            }
            const bool ng = (b >> 31) && key != 0;  // u < 0.0f
            const unsigned bp = __ballot_sync(FULL, sel && !ng);
            const unsigned bn = __ballot_sync(FULL, sel && ng);
            if (lane == (t >> 1)) {
                const int sh = (t & 1) * 32;
                wp |= (uint64_t)bp << sh;
                wn |= (uint64_t)bn << sh;
            }
        }
        uint64_t* out = T + row * (int64_t)(2 * W);
        if (lane < W) {
            out[lane] = wp;
            out[W + lane] = wn;
        }
    }
}

template <int VPL>
cudaError_t launch_vpl(const float* U, int64_t n, int d, int x, uint64_t* T, int32_t* status,
                       cudaStream_t stream) {
    const int W = (d + 63) / 64;
    const int64_t warps_needed = n;
    int64_t blocks = (warps_needed + (ENC_THREADS / 32) - 1) / (ENC_THREADS / 32);
    const int64_t cap = (int64_t)num_sms() * 8;  // persistent: 8 CTAs (64 warps) per SM
    if (blocks > cap) blocks = cap;
    const size_t smem = (size_t)ENC_WARPS * VPL * 32 * 4;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(encode_kernel<VPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return cudaErrorInvalidValue;
    TimedLaunch timer("encode", stream);
    encode_kernel<VPL><<<(unsigned)blocks, ENC_THREADS, smem, stream>>>(U, n, d, x, W, T, status);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_encode(const float* U, int64_t n, int d, int x, uint64_t* T,
                          int32_t* status, cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    const int vpl = (d + 31) / 32;
    if (vpl <= 1) return launch_vpl<1>(U, n, d, x, T, status, stream);
    if (vpl <= 2) return launch_vpl<2>(U, n, d, x, T, status, stream);
    if (vpl <= 4) return launch_vpl<4>(U, n, d, x, T, status, stream);
    if (vpl <= 8) return launch_vpl<8>(U, n, d, x, T, status, stream);
    if (vpl <= 12) return launch_vpl<12>(U, n, d, x, T, status, stream);
    if (vpl <= 16) return launch_vpl<16>(U, n, d, x, T, status, stream);
    if (vpl <= 24) return launch_vpl<24>(U, n, d, x, T, status, stream);
    if (vpl <= 32) return launch_vpl<32>(U, n, d, x, T, status, stream);
    if (vpl <= 48) return launch_vpl<48>(U, n, d, x, T, status, stream);
    return launch_vpl<64>(U, n, d, x, T, status, stream);
}

}  // namespace evp
