// evp_quantize_i8: the query side of the single-operand translation of
// Sec. 6 -- the database is mapped to EVP vertices, the query keeps its
// values, here as int8 so that every score (Sec. 5.1.2 masked addition)
// is an exact integer.  Symmetric per-query scaling: m = max_i |q_i|,
// scale = 127 / m, q8_i = q_i * scale rounded to the nearest integer, ties
// to even, all in float32 (IEEE division and multiplication, so the result
// does not depend on the GPU); m = 0 gives the zero vector.
//
// One warp per row, grid-stride; lanes hold elements lane + 32 t.
#include "evp_internal.cuh"

namespace evp {

namespace {

constexpr int QZ_THREADS = 256;

__global__ void __launch_bounds__(QZ_THREADS)
quantize_i8_kernel(const float* __restrict__ Q, int64_t n, int d, int8_t* __restrict__ Q8,
                   int32_t* __restrict__ status) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * QZ_THREADS + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * QZ_THREADS) >> 5;
    for (int64_t row = warp0; row < n; row += nwarps) {
        const float* q = Q + row * (int64_t)d;
        int8_t* o = Q8 + row * (int64_t)d;
        // largest magnitude, as its 31-bit key (orders magnitudes exactly);
        // a key >= 0x7f800000 marks NaN or infinity
        uint32_t kmax = 0;
        for (int j = lane; j < d; j += 32) kmax = max(kmax, __float_as_uint(q[j]) & 0x7fffffffu);
        kmax = __reduce_max_sync(0xffffffffu, kmax);
        if (kmax >= 0x7f800000u) {
            if (lane == 0) report(status, EVP_ERR_NONFINITE);
            for (int j = lane; j < d; j += 32) o[j] = 0;
            continue;
        }
        if (kmax == 0u) {
            for (int j = lane; j < d; j += 32) o[j] = 0;
            continue;
        }
        const float scale = __fdiv_rn(127.0f, __uint_as_float(kmax));
        for (int j = lane; j < d; j += 32)
            o[j] = (int8_t)__float2int_rn(__fmul_rn(q[j], scale));
    }
}

}  // namespace

cudaError_t launch_quantize_i8(const float* Q, int64_t n, int d, int8_t* Q8, int32_t* status,
                               cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + QZ_THREADS / 32 - 1) / (QZ_THREADS / 32);
    const int64_t cap = (int64_t)num_sms() * 8;
    if (blocks > cap) blocks = cap;
    TimedLaunch timer("quantize", stream);
    quantize_i8_kernel<<<(unsigned)blocks, QZ_THREADS, 0, stream>>>(Q, n, d, Q8, status);
    return cudaGetLastError();
}

}  // namespace evp
