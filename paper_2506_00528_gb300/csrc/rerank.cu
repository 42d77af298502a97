// rerank kernel: re-order each query's shortlist by the scalar product of
// the original float32 vectors and keep the best k (Sec. 5.3: n > k proxy
// results re-ordered with respect to the original space).
//
// One CTA per query.  The query row is staged in shared memory; each warp
// scores shortlist entries one at a time: the 32 lanes gather the database
// row with coalesced loads (float4 when the row allows it), accumulate a
// running FMA over their strided share of the elements, and combine the 32
// partial sums with a five-level xor butterfly, which leaves the same sum
// on every lane.  The summation order is therefore fixed for a given d.
// Scores become 64-bit keys (~ordered(score) << 32 | id) so that one
// ascending block-wide bitonic sort yields (score descending, id ascending).
#include "evp_internal.cuh"

namespace evp {

namespace {

constexpr int RR_THREADS = 256;
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ uint32_t ordered_ascending(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float from_ordered_ascending(uint32_t o) {
    const uint32_t u = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
    return __uint_as_float(u);
}

template <bool VEC4>
__global__ void __launch_bounds__(RR_THREADS)
rerank_kernel(const float* __restrict__ Q, const float* __restrict__ S, int64_t ns, int d,
              const int64_t* __restrict__ shortlist, int n, int k, int P,
              int64_t* __restrict__ ids, float* __restrict__ scores, int32_t* __restrict__ status) {
    extern __shared__ __align__(16) uint8_t smem[];
    float* qs = reinterpret_cast<float*>(smem);
    uint64_t* keys = reinterpret_cast<uint64_t*>(smem + (((size_t)d * 4 + 15) / 16) * 16);
    const int64_t q = blockIdx.x;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int i = tid; i < d; i += RR_THREADS) qs[i] = Q[q * d + i];
    __syncthreads();

    for (int j = warp; j < P; j += RR_THREADS / 32) {
        uint64_t key = KEY_NONE;
        if (j < n) {
            const int64_t id = shortlist[q * n + j];
            if (id != -1) {
                if (id < 0 || id >= ns) {
                    if (lane == 0) report(status, EVP_ERR_RANGE);
                } else {
                    const float* srow = S + id * (int64_t)d;
                    float acc = 0.f;
                    if (VEC4) {
                        const float4* s4 = reinterpret_cast<const float4*>(srow);
                        const float4* q4 = reinterpret_cast<const float4*>(qs);
                        for (int i = lane; i < (d >> 2); i += 32) {
                            const float4 b = __ldg(s4 + i);
                            const float4 a4 = q4[i];
                            acc = fmaf(a4.x, b.x, acc);
                            acc = fmaf(a4.y, b.y, acc);
                            acc = fmaf(a4.z, b.z, acc);
                            acc = fmaf(a4.w, b.w, acc);
                        }
                    } else {
                        for (int i = lane; i < d; i += 32) acc = fmaf(qs[i], __ldg(srow + i), acc);
                    }
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(FULL, acc, off);
                    if (!isfinite(acc)) {
                        if (lane == 0) report(status, EVP_ERR_NONFINITE);
                    }
                    if (acc == 0.f) acc = 0.f;  // -0.0 ranks as +0.0
                    key = ((uint64_t)(~ordered_ascending(acc)) << 32) | (uint64_t)(uint32_t)id;
                }
            }
        }
        if (lane == 0) keys[j] = key;
    }
    __syncthreads();

    for (int kk = 2; kk <= P; kk <<= 1) {
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
            for (int i = tid; i < P; i += RR_THREADS) {
                const int ixj = i ^ jj;
                if (ixj > i) {
                    const uint64_t a = keys[i], b = keys[ixj];
                    const bool up = (i & kk) == 0;
                    if ((a > b) == up) {
                        keys[i] = b;
                        keys[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }

    for (int j = tid; j < k; j += RR_THREADS) {
        const uint64_t key = keys[j];
        if (key == KEY_NONE) {
            ids[q * k + j] = -1;
            scores[q * k + j] = -INFINITY;
        } else {
            ids[q * k + j] = (int64_t)(key & 0xffffffffull);
            scores[q * k + j] = from_ordered_ascending(~(uint32_t)(key >> 32));
        }
    }
}

}  // namespace

cudaError_t launch_rerank(const float* Q, int64_t nq, const float* S, int64_t ns, int d,
                          const int64_t* shortlist, int n, int k, int64_t* ids, float* scores,
                          int32_t* status, cudaStream_t stream) {
    if (nq <= 0) return cudaSuccess;
    int P = 2;
    while (P < n) P <<= 1;
    const size_t smem = (((size_t)d * 4 + 15) / 16) * 16 + (size_t)P * 8;
    const bool vec4 = (d % 4 == 0) && ((reinterpret_cast<uintptr_t>(S) & 15) == 0);
    const size_t max_smem = (size_t)EVP_MAX_D_RERANK * 4 + (size_t)EVP_MAX_SHORTLIST * 8;
    cudaError_t e;
    TimedLaunch timer("rerank", stream);
    if (vec4) {
        e = cudaFuncSetAttribute(rerank_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)max_smem);
        if (e != cudaSuccess) return e;
        rerank_kernel<true><<<(unsigned)nq, RR_THREADS, smem, stream>>>(
            Q, S, ns, d, shortlist, n, k, P, ids, scores, status);
    } else {
        e = cudaFuncSetAttribute(rerank_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)max_smem);
        if (e != cudaSuccess) return e;
        rerank_kernel<false><<<(unsigned)nq, RR_THREADS, smem, stream>>>(
            Q, S, ns, d, shortlist, n, k, P, ids, scores, status);
    }
    return cudaGetLastError();
}

}  // namespace evp
