// evp_probe_tensor_rate: the dense tensor-core rate of this GPU for the
// instruction shapes the scans issue (measurement support for the roofline
// of the tensor-core scans; the paper has no counterpart).
//
// One CTA per SM (or one CTA pair per two SMs) keeps one thread issuing
// tcgen05.mma back to back on operands resident in shared memory: e4m3
// (kind::f8f6f4, K = 32) or bf16 (kind::f16, K = 16), both with float32
// accumulation in tensor memory.  The operands hold the values the scans
// contract (+1, -1 and 0 in equal shares), so the switching activity -- and
// with it the power draw and the clock the GPU sustains -- resembles the
// scan's.  Every wait is bounded; the launch is timed with CUDA events on
// the caller's stream and the issuing threads count SM clocks.
#include "evp_internal.cuh"

#include <algorithm>
#include <vector>

namespace evp {

namespace {

constexpr int PR_THREADS = 128;
constexpr int PR_A_BYTES = 128 * 128;      // 128 rows x one 128-byte K chunk
constexpr int PR_B_BYTES = 256 * 128;      // up to 256 rows x one K chunk
constexpr int PR_SMEM = 1024 + PR_A_BYTES + PR_B_BYTES + 64;
constexpr int PR_SMEM_LAUNCH = 120 * 1024;  // more than half an SM: one CTA per SM
constexpr uint32_t PR_TMEM_COLS = 256;

__device__ __forceinline__ uint32_t pr_cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void pr_cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// kind: 0 = f8f6f4 (e4m3), 1 = f16 (bf16).  CG: CTAs per instruction.
template <int CG>
__device__ __forceinline__ void pr_mma(int kind, uint32_t d, uint64_t a, uint64_t b,
                                       uint32_t idesc, uint32_t acc) {
    if (kind == 0) {
        if constexpr (CG == 1)
            asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                         "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                         "l"(a), "l"(b), "r"(idesc), "r"(acc)
                         : "memory");
        else
            asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                         "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                         "l"(a), "l"(b), "r"(idesc), "r"(acc)
                         : "memory");
    } else {
        if constexpr (CG == 1)
            asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                         "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                         "l"(a), "l"(b), "r"(idesc), "r"(acc)
                         : "memory");
        else
            asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                         "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                         "l"(a), "l"(b), "r"(idesc), "r"(acc)
                         : "memory");
    }
}

template <int CG>
__global__ void __launch_bounds__(PR_THREADS, 1)
probe_mma_kernel(int kind, int fill, int n, int64_t iters, uint32_t idesc, int64_t* cycles,
                 int32_t* status) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t* smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    uint8_t* A = smem;
    uint8_t* B = smem + PR_A_BYTES;
    uint64_t* done = reinterpret_cast<uint64_t*>(smem + PR_A_BYTES + PR_B_BYTES);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t rank = CG == 2 ? pr_cluster_rank() : 0u;

    // operands: +1 / -1 / 0 in equal shares (a fixed hash of the position),
    // or all zero (fill = 1) or random bytes (fill = 2, e4m3 only)
    const int bytes = PR_A_BYTES + PR_B_BYTES;
    for (int i = tid; i < bytes / 2; i += PR_THREADS) {
        if (fill != 0) {
            const uint32_t h = ((uint32_t)i * 2654435761u + blockIdx.x * 40503u) >> 9;
            uint16_t w = fill == 1 ? 0 : (uint16_t)(h & 0x7777u);  // finite e4m3 bytes
            reinterpret_cast<uint16_t*>(smem)[i] = w;
            continue;
        }
        const uint32_t h = (uint32_t)i * 2654435761u + blockIdx.x * 40503u;
        const uint32_t c0 = (h >> 7) % 3u, c1 = (h >> 17) % 3u;
        uint16_t v;
        if (kind == 0) {
            const uint8_t e[3] = {0x00, 0x38, 0xB8};  // 0, +1, -1 in e4m3
            v = (uint16_t)(e[c0] | (e[c1] << 8));
        } else {
            const uint16_t e[3] = {0x0000, 0x3F80, 0xBF80};  // 0, +1, -1 in bf16
            v = e[c0];
        }
        reinterpret_cast<uint16_t*>(smem)[i] = v;
    }
    if (tid == 0) {
        mbar_init(done, 1);
        fence_mbar_init();
    }
    fence_proxy_async_smem();
    if (warp == 0) {
        if constexpr (CG == 1) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(tmem_slot)),
                         "r"(PR_TMEM_COLS)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        } else {
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(tmem_slot)),
                         "r"(PR_TMEM_COLS)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
        }
    }
    tc_fence_before();
    __syncthreads();
    if constexpr (CG == 2) pr_cluster_sync();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (tid == 0 && rank == 0) {
        const uint64_t a0 = sw128_desc(smem_u32(A)), b0 = sw128_desc(smem_u32(B));
        const long long t0 = clock64();
        for (int64_t i = 0; i < iters; ++i) {
            const uint32_t kk = (uint32_t)(i & 3);  // four 32-byte K steps per 128-byte chunk
            pr_mma<CG>(kind, tmem, a0 + 2 * kk, b0 + 2 * kk, idesc, i > 0 ? 1u : 0u);
        }
        if constexpr (CG == 1)
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(done))
                : "memory");
        else
            asm volatile(
                "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::"
                "cluster.b64 [%0], %1;" ::"r"(smem_u32(done)),
                "h"((uint16_t)3)
                : "memory");
        const bool ok = mbar_wait_bounded(done, 0);
        const long long t1 = clock64();
        if (!ok) report(status, EVP_ERR_TIMEOUT);
        cycles[blockIdx.x / CG] = ok ? (int64_t)(t1 - t0) : -1;
    } else if (tid == 0) {
        if (!mbar_wait_bounded(done, 0)) report(status, EVP_ERR_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if constexpr (CG == 2) pr_cluster_sync();
    tc_fence_after();
    if (warp == 0) {
        if constexpr (CG == 1)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                         "r"(PR_TMEM_COLS)
                         : "memory");
        else
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                         "r"(PR_TMEM_COLS)
                         : "memory");
    }
    (void)n;
}

}  // namespace

}  // namespace evp

extern "C" {

int32_t evp_probe_tensor_rate(int32_t kind, int32_t cta_pair, int32_t n, int64_t iters,
                              double* tflops, double* cycles_per_mma, double* ms, void* stream) {
    using namespace evp;
    const int cg = cta_pair ? 2 : 1;
    const int fill = (kind >> 8) & 3;  // operand values (see evp.h)
    kind &= 0xff;
    if ((kind != 0 && kind != 1) || fill == 3 || (fill == 2 && kind != 0) || n < 16 || n > 256 || n % 16 != 0 || iters < 1 ||
        iters > (int64_t(1) << 26) || !tflops || !cycles_per_mma || !ms)
        return EVP_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int sms = num_sms();
    const int workers = cg == 2 ? sms / 2 : sms;
    const int m = 128 * cg;
    // D = f32; A, B = e4m3 (format 0) or bf16 (format 1); both K-major.
    const uint32_t fmt = kind == 0 ? 0u : 1u;
    const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(n >> 3) << 17) |
                           ((uint32_t)(m >> 4) << 24);
    int64_t* cycles = nullptr;
    int32_t* status = nullptr;
    if (cudaMalloc(&cycles, sizeof(int64_t) * workers) != cudaSuccess) return EVP_ERR_NO_MEMORY;
    if (cudaMalloc(&status, sizeof(int32_t)) != cudaSuccess) {
        cudaFree(cycles);
        return EVP_ERR_NO_MEMORY;
    }
    int32_t rc = EVP_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaMemsetAsync(status, 0, sizeof(int32_t), s);
    cudaError_t err = cudaSuccess;
    if (cg == 1) {
        err = cudaFuncSetAttribute(probe_mma_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   PR_SMEM_LAUNCH);
        if (err == cudaSuccess) {
            cudaEventRecord(e0, s);
            probe_mma_kernel<1><<<workers, PR_THREADS, PR_SMEM_LAUNCH, s>>>(kind, fill, n, iters,
                                                                            idesc, cycles, status);
            err = cudaGetLastError();
            cudaEventRecord(e1, s);
        }
    } else {
        err = cudaFuncSetAttribute(probe_mma_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   PR_SMEM_LAUNCH);
        if (err == cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = 2;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3(2 * (unsigned)workers);
            cfg.blockDim = dim3(PR_THREADS);
            cfg.dynamicSmemBytes = PR_SMEM_LAUNCH;
            cfg.stream = s;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            cudaEventRecord(e0, s);
            err = cudaLaunchKernelEx(&cfg, probe_mma_kernel<2>, kind, fill, n, iters, idesc,
                                     cycles, status);
            cudaEventRecord(e1, s);
        }
    }
    std::vector<int64_t> cyc(workers, -1);
    int32_t st = EVP_OK;
    float t = 0.f;
    if (err == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
        cudaEventElapsedTime(&t, e0, e1) == cudaSuccess &&
        cudaMemcpy(cyc.data(), cycles, sizeof(int64_t) * workers, cudaMemcpyDeviceToHost) ==
            cudaSuccess &&
        cudaMemcpy(&st, status, sizeof(int32_t), cudaMemcpyDeviceToHost) == cudaSuccess) {
        if (st != EVP_OK) {
            rc = st;
        } else {
            double sum = 0.0;
            for (int64_t c : cyc) sum += (double)c;
            const int kdim = kind == 0 ? 32 : 16;
            *ms = t;
            *tflops = 2.0 * m * n * kdim * (double)iters * workers / (t * 1e-3) / 1e12;
            *cycles_per_mma = sum / workers / (double)iters;
        }
    } else {
        cudaGetLastError();
        rc = EVP_ERR_CUDA;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(cycles);
    cudaFree(status);
    return rc;
}

}  // extern "C"
