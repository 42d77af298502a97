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
// count(key >= tau) >= x by a bitwise search from the top key bit down;
// each step is one compare per element and one warp reduction.  Keys above
// tau are selected; keys equal to tau are taken in ascending element index
// until x are chosen.
#include "evp_internal.cuh"

namespace evp {

namespace {

constexpr int ENC_THREADS = 256;
constexpr unsigned FULL = 0xffffffffu;

template <int VPL>
__global__ void __launch_bounds__(ENC_THREADS)
encode_kernel(const float* __restrict__ U, int64_t n, int d, int x, int W,
              uint64_t* __restrict__ T, int32_t* __restrict__ status) {
    static_assert(VPL >= 1 && VPL <= 64, "VPL range");
    const int lane = threadIdx.x & 31;
    const unsigned lanemask_lt = (1u << lane) - 1u;
    const int64_t warp0 = ((int64_t)blockIdx.x * ENC_THREADS + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * ENC_THREADS) >> 5;

    for (int64_t row = warp0; row < n; row += nwarps) {
        const float* u = U + row * (int64_t)d;
        uint32_t key[VPL];
        uint64_t neg = 0;   // bit t: element lane+32t is < 0
        uint64_t real = 0;  // bit t: element lane+32t exists (j < d)
        bool bad = false;
#pragma unroll
        for (int t = 0; t < VPL; ++t) {
            const int j = lane + 32 * t;
            uint32_t b = 0;
            if (j < d) b = __float_as_uint(__ldg(u + j));
            key[t] = b & 0x7fffffffu;
            bad |= key[t] >= 0x7f800000u;
            const bool is_neg = (b >> 31) && key[t] != 0;  // u < 0.0f
            neg |= (uint64_t)is_neg << t;
            real |= (uint64_t)(j < d) << t;
        }
        if (__any_sync(FULL, bad) && lane == 0) report(status, EVP_ERR_NONFINITE);

        // tau = max{v : #(key >= v) >= x}.  Padding keys are 0 and only
        // count at v = 0, where every real element counts as well.
        uint32_t tau = 0;
#pragma unroll 1
        for (int b = 30; b >= 0; --b) {
            const uint32_t cand = tau | (1u << b);
            int c = 0;
#pragma unroll
            for (int t = 0; t < VPL; ++t) c += key[t] >= cand;
            c = __reduce_add_sync(FULL, c);
            if (c >= x) tau = cand;
        }
        int gt = 0;
#pragma unroll
        for (int t = 0; t < VPL; ++t) gt += key[t] > tau;
        gt = __reduce_add_sync(FULL, gt);
        const int need = x - gt;  // keys equal to tau still to take, lowest index first

        uint64_t wp = 0, wn = 0;  // this lane's output words (lane < W)
        int base = 0;
#pragma unroll
        for (int t = 0; t < VPL; ++t) {
            const bool eq = key[t] == tau && ((real >> t) & 1);
            const unsigned m = __ballot_sync(FULL, eq);
            const int rank = base + __popc(m & lanemask_lt);
            base += __popc(m);
            const bool sel = key[t] > tau || (eq && rank < need);
            const bool ng = (neg >> t) & 1;
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
    TimedLaunch timer("encode", stream);
    encode_kernel<VPL><<<(unsigned)blocks, ENC_THREADS, 0, stream>>>(U, n, d, x, W, T, status);
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
