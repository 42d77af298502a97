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
constexpr int PR_STAGES = 4;               // EXTRA 3: operand buffers cycled through
constexpr int PR_STAGE_BYTES = PR_A_BYTES + PR_B_BYTES;
constexpr int PR_SMEM_LAUNCH = 1024 + PR_STAGES * PR_STAGE_BYTES + 64;  // one CTA per SM
constexpr uint32_t PR_TMEM_COLS = 512;

__device__ __forceinline__ uint32_t pr_cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void pr_cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// KIND: 0 = f8f6f4 (e4m3), 1 = f16 (bf16), 2 = mxf4 (e2m1, K = 64, unit
// ue8m0 scale factors in TMEM columns 384-415 of the accumulator's base).
// CG: CTAs per instruction.
// AMODE 1: A in tensor memory (a = TMEM address), else a shared-memory
// descriptor.  ACC: accumulate into D (0 for the first instruction).
template <int CG, int KIND, int AMODE, int ACC>
__device__ __forceinline__ void pr_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc) {
    if constexpr (AMODE == 1 && CG == 1) {
        static_assert(KIND == 0, "A from TMEM: e4m3");
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
                     "r"((uint32_t)a), "l"(b), "r"(idesc), "n"(ACC)
                     : "memory");
    } else if constexpr (AMODE == 1) {
        static_assert(KIND == 0, "A from TMEM: e4m3");
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
                     "r"((uint32_t)a), "l"(b), "r"(idesc), "n"(ACC)
                     : "memory");
    } else if constexpr (KIND == 2 && CG == 1) {
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X "
                     "[%0], %1, %2, %3, [%5], [%6], p;\n\t}" ::"r"(d),
                     "l"(a), "l"(b), "r"(idesc), "n"(ACC), "r"(d + 384u), "r"(d + 392u)
                     : "memory");
    } else if constexpr (KIND == 2) {
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::2.kind::mxf4.block_scale.scale_vec::2X "
                     "[%0], %1, %2, %3, [%5], [%6], p;\n\t}" ::"r"(d),
                     "l"(a), "l"(b), "r"(idesc), "n"(ACC), "r"(d + 384u), "r"(d + 392u)
                     : "memory");
    } else if constexpr (KIND == 0 && CG == 1) {
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                     "l"(a), "l"(b), "r"(idesc), "n"(ACC)
                     : "memory");
    } else if constexpr (KIND == 0) {
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                     "l"(a), "l"(b), "r"(idesc), "n"(ACC)
                     : "memory");
    } else if constexpr (CG == 1) {
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                     "l"(a), "l"(b), "r"(idesc), "n"(ACC)
                     : "memory");
    } else {
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                     "l"(a), "l"(b), "r"(idesc), "n"(ACC)
                     : "memory");
    }
}

// Store 32 consecutive 32-bit columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void pr_tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
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

// AMODE 0: A in shared memory; 1: A in tensor memory (columns 128-159, the
// accumulator takes columns 0 to n - 1 <= 127).  iters: a multiple of 4.
// EXTRA: what the issuing thread does after every four MMAs besides
// looping (the work a pipelined scan does per stage): 0 nothing, 1 a
// tcgen05.commit to a barrier, 2 a barrier test (already complete) and the
// tcgen05 fence that follows a wait, 3 the next of four distinct operand
// buffers (as a scan streams fresh stages) instead of the same one, 4 a
// switch to the other of two accumulators (columns 0 and 256) every 24
// instructions, restarting it with accumulate = 0 (a scan's tile change), 5
// the other three warps reading columns 256-511 of their TMEM lanes with
// tcgen05.ld throughout (an epilogue draining the other accumulator), 6 the
// switch of 4 without the restart (accumulate = 1 throughout), 7 the restart
// of 4 without the switch (one accumulator, accumulate = 0 every 24); 8 the
// scan's tile structure with run-time loops (per tile of three 4-instruction
// chunks: a barrier test and fence per chunk, a commit per chunk, the
// accumulator switch with accumulate = 0, a commit per tile), 9 the same
// tile with its chunk loop unrolled and compile-time accumulate flags.
template <int CG, int KIND, int AMODE, int EXTRA>
__global__ void __launch_bounds__(PR_THREADS, 1)
probe_mma_kernel(int fill, int64_t iters, uint32_t idesc, int64_t* cycles, int32_t* status) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t* smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    uint8_t* A = smem;
    uint8_t* B = smem + PR_A_BYTES;
    uint64_t* done = reinterpret_cast<uint64_t*>(smem + PR_STAGES * PR_STAGE_BYTES);
    uint64_t* spare = done + 1;  // EXTRA 1: commits; EXTRA 2, 8, 9: tested (complete) barrier
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 4);  // spare + 1, + 2: commits (8, 9)
    int* stop = reinterpret_cast<int*>(tmem_slot + 1);  // EXTRA 5: the issuer is done
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t rank = CG == 2 ? pr_cluster_rank() : 0u;

    // operands: +1 / -1 / 0 in equal shares (a fixed hash of the position),
    // or all zero (fill = 1) or random bytes (fill = 2, e4m3 only)
    const int bytes = PR_STAGES * PR_STAGE_BYTES;
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
        if (KIND == 2) {
            const uint16_t e[3] = {0x0, 0x2, 0xA};  // 0, +1, -1 in e2m1
            const uint32_t c2 = (h >> 23) % 3u, c3 = (h >> 27) % 3u;
            v = (uint16_t)(e[c0] | (e[c1] << 4) | (e[c2] << 8) | (e[c3] << 12));
        } else if (KIND == 0) {
            const uint8_t e[3] = {0x00, 0x38, 0xB8};  // 0, +1, -1 in e4m3
            v = (uint16_t)(e[c0] | (e[c1] << 8));
        } else {
            const uint16_t e[3] = {0x0000, 0x3F80, 0xBF80};  // 0, +1, -1 in bf16
            v = e[c0];
        }
        reinterpret_cast<uint16_t*>(smem)[i] = v;
    }
    if (tid == 0) {
        *stop = 0;
        mbar_init(done, 1);
        mbar_init(spare, 1);
        mbar_init(spare + 1, 1);
        mbar_init(spare + 2, 1);
        fence_mbar_init();
        if (EXTRA == 2 || EXTRA == 8 || EXTRA == 9) mbar_arrive(spare);  // phase 0 complete
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
    if (KIND == 2) {  // unit scale factors (ue8m0 0x7F) in columns 384-415 of every lane
        uint32_t v[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) v[c] = 0x7F7F7F7Fu;
        pr_tmem_st32(tmem + ((uint32_t)(warp * 32) << 16) + 384u, v);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        if constexpr (CG == 2) pr_cluster_sync();
        tc_fence_after();
    }
    if (AMODE == 1) {  // A: this warp's 32 lanes x 32 columns (four K steps of e4m3 bytes)
        uint32_t v[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            const uint32_t h = (uint32_t)(tid * 32 + c) * 2654435761u + blockIdx.x * 40503u;
            uint32_t w = 0;
            for (int b = 0; b < 4; ++b) {
                const uint32_t cb = (h >> (7 + 5 * b)) % 3u;
                const uint32_t e = fill == 1 ? 0u : (cb == 0 ? 0x00u : (cb == 1 ? 0x38u : 0xB8u));
                w |= e << (8 * b);
            }
            v[c] = w;
        }
        pr_tmem_st32(tmem + ((uint32_t)(warp * 32) << 16) + 128u, v);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        if constexpr (CG == 2) pr_cluster_sync();  // both halves of A are written
        tc_fence_after();
    }

    if (tid == 0 && rank == 0) {
        const uint64_t a0 = sw128_desc(smem_u32(A)), b0 = sw128_desc(smem_u32(B));
        const long long t0 = clock64();
        // four 32-byte K steps per 128-byte chunk (A in TMEM: 8 columns each)
        const uint64_t as = AMODE == 1 ? 8 : 2;
        const uint64_t a = AMODE == 1 ? (uint64_t)(tmem + 128u) : a0;
        pr_mma<CG, KIND, AMODE, 0>(tmem, a, b0, idesc);
        pr_mma<CG, KIND, AMODE, 1>(tmem, a + as, b0 + 2, idesc);
        pr_mma<CG, KIND, AMODE, 1>(tmem, a + 2 * as, b0 + 4, idesc);
        pr_mma<CG, KIND, AMODE, 1>(tmem, a + 3 * as, b0 + 6, idesc);
        int extra_ok = 1;
        if constexpr (EXTRA == 8 || EXTRA == 9) {
            // tiles of three chunks of four instructions, accumulators at
            // columns 0 and 256; every barrier involved is already complete
            int ok8 = 1;
            for (int64_t i = 4, tile = 0; i < iters; i += 12, ++tile) {
                const uint32_t dt = tmem + ((uint32_t)(tile & 1) << 8);
                ok8 &= mbar_try_wait(spare, 0) ? 1 : 0;
                tc_fence_after();
                if constexpr (EXTRA == 8) {
#pragma unroll 1
                    for (int kc = 0; kc < 3; ++kc) {
                        ok8 &= mbar_try_wait(spare, 0) ? 1 : 0;
                        tc_fence_after();
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            if (kc > 0 || kk > 0)
                                pr_mma<CG, KIND, AMODE, 1>(dt, a + kk * as, b0 + 2 * kk, idesc);
                            else
                                pr_mma<CG, KIND, AMODE, 0>(dt, a + kk * as, b0 + 2 * kk, idesc);
                        }
                        if constexpr (CG == 1)
                            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(spare + 1)) : "memory");
                        else
                            asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(spare + 1)) : "memory");
                    }
                } else {
#pragma unroll
                    for (int kc = 0; kc < 3; ++kc) {
                        ok8 &= mbar_try_wait(spare, 0) ? 1 : 0;
                        tc_fence_after();
                        if (kc == 0) pr_mma<CG, KIND, AMODE, 0>(dt, a, b0, idesc);
                        else pr_mma<CG, KIND, AMODE, 1>(dt, a, b0, idesc);
                        pr_mma<CG, KIND, AMODE, 1>(dt, a + as, b0 + 2, idesc);
                        pr_mma<CG, KIND, AMODE, 1>(dt, a + 2 * as, b0 + 4, idesc);
                        pr_mma<CG, KIND, AMODE, 1>(dt, a + 3 * as, b0 + 6, idesc);
                        if constexpr (CG == 1)
                            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(spare + 1)) : "memory");
                        else
                            asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(spare + 1)) : "memory");
                    }
                }
                if constexpr (CG == 1)
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(spare + 2)) : "memory");
                else
                    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(spare + 2)) : "memory");
            }
            if (!ok8) report(status, EVP_ERR_INVALID);
        }
        uint64_t so = 0;  // EXTRA 3: start-address offset of the current buffer (16-byte units)
        uint32_t dcur = tmem;  // EXTRA 4: current accumulator
        int nacc = 4;          // EXTRA 4: instructions into it so far
        for (int64_t i = 4; i < ((EXTRA == 8 || EXTRA == 9) ? 0 : iters); i += 4) {
            if constexpr (EXTRA == 4 || EXTRA == 6 || EXTRA == 7) {
                if (nacc == 24) {
                    if (EXTRA != 7) dcur ^= 256u;
                    nacc = 4;
                    if constexpr (EXTRA == 6)
                        pr_mma<CG, KIND, AMODE, 1>(dcur, a, b0, idesc);
                    else
                        pr_mma<CG, KIND, AMODE, 0>(dcur, a, b0, idesc);
                    pr_mma<CG, KIND, AMODE, 1>(dcur, a + as, b0 + 2, idesc);
                    pr_mma<CG, KIND, AMODE, 1>(dcur, a + 2 * as, b0 + 4, idesc);
                    pr_mma<CG, KIND, AMODE, 1>(dcur, a + 3 * as, b0 + 6, idesc);
                    continue;
                }
                nacc += 4;
            }
            if constexpr (EXTRA == 3) so = so == (uint64_t)(3 * (PR_STAGE_BYTES >> 4)) ? 0 : so + (PR_STAGE_BYTES >> 4);
            if constexpr (EXTRA == 1) {
                if constexpr (CG == 1)
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 "
                        "[%0];" ::"r"(smem_u32(spare))
                        : "memory");
                else
                    asm volatile(
                        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 "
                        "[%0];" ::"r"(smem_u32(spare))
                        : "memory");
            } else if constexpr (EXTRA == 2) {
                extra_ok &= mbar_try_wait(spare, 0) ? 1 : 0;
                tc_fence_after();
            }
            pr_mma<CG, KIND, AMODE, 1>(dcur, a + so, b0 + so, idesc);
            pr_mma<CG, KIND, AMODE, 1>(dcur, a + so + as, b0 + so + 2, idesc);
            pr_mma<CG, KIND, AMODE, 1>(dcur, a + so + 2 * as, b0 + so + 4, idesc);
            pr_mma<CG, KIND, AMODE, 1>(dcur, a + so + 3 * as, b0 + so + 6, idesc);
        }
        if (!extra_ok) report(status, EVP_ERR_INVALID);
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
        *reinterpret_cast<volatile int*>(stop) = 1;
        if (!ok) report(status, EVP_ERR_TIMEOUT);
        cycles[blockIdx.x / CG] = ok ? (int64_t)(t1 - t0) : -1;
    } else if (tid == 0) {
        if (!mbar_wait_bounded(done, 0)) report(status, EVP_ERR_TIMEOUT);
    } else if (EXTRA == 5 && warp > 0 && rank == 0) {
        // read this warp's lanes of columns 256-511 until the issuer is done
        // (at most 2^22 rounds)
        uint32_t v[32], acc = 0;
        for (int r = 0; r < (1 << 22); ++r) {
            if (*reinterpret_cast<volatile int*>(stop)) break;
#pragma unroll 1
            for (int c = 0; c < 8; ++c) {
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                    "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                    "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
                    "[%32];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                      "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                      "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]),
                      "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
                      "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
                      "=r"(v[30]), "=r"(v[31])
                    : "r"(tmem + ((uint32_t)(warp * 32) << 16) + 256u + 32u * c));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int u = 0; u < 32; ++u) acc ^= v[u];
            }
        }
        if (acc == 0x9E3779B9u) report(status, EVP_ERR_RANGE);  // keeps the loads
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
}

}  // namespace

}  // namespace evp

extern "C" {

int32_t evp_probe_tensor_rate(int32_t kind, int32_t cta_pair, int32_t n, int64_t iters,
                              double* tflops, double* cycles_per_mma, double* ms, void* stream) {
    using namespace evp;
    const int cg = cta_pair ? 2 : 1;
    const int fill = (kind >> 8) & 3;  // operand values (see evp.h)
    const bool tmem_a = (kind >> 10) & 1, m64 = (kind >> 11) & 1;
    const int extra = (kind >> 12) & 15;  // per-four-MMA extra work (see the kernel)
    kind &= 0xff;
    if ((kind != 0 && kind != 1 && kind != 2) || fill == 3 || (fill == 2 && kind != 0) || n < 16 ||
        n > 256 ||
        n % 16 != 0 || iters < 1 || iters > (int64_t(1) << 26) || !tflops || !cycles_per_mma ||
        !ms)
        return EVP_ERR_INVALID;
    if (m64 && cg != 1) return EVP_ERR_INVALID;
    if (tmem_a && (m64 || kind != 0 || fill == 2 || n > 128)) return EVP_ERR_INVALID;
    if (m64 && n % 8 != 0) return EVP_ERR_INVALID;
    if (extra > 9 || (extra != 0 && (tmem_a || kind != 0))) return EVP_ERR_INVALID;
    if (kind == 2 && (tmem_a || m64 || fill != 0)) return EVP_ERR_INVALID;
    if (extra >= 4 && n > 256) return EVP_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int sms = num_sms();
    const int workers = cg == 2 ? sms / 2 : sms;
    const int m = m64 ? 64 : 128 * cg;
    // D = f32; A, B = e4m3 (format 0) or bf16 (format 1); both K-major.
    // mxf4: A, B = e2m1 (format 1 of the block-scaled kinds), ue8m0 scales.
    const uint32_t fmt = kind == 0 ? 0u : 1u;
    const uint32_t idesc =
        kind == 2 ? (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | (1u << 23) |
                        ((uint32_t)(m >> 4) << 24)
                  : (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(n >> 3) << 17) |
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
    const int64_t iters4 = (iters + 3) / 4 * 4;
    if (cg == 1) {
        void (*kern)(int, int64_t, uint32_t, int64_t*, int32_t*) =
            tmem_a ? probe_mma_kernel<1, 0, 1, 0>
                   : kind == 2 ? probe_mma_kernel<1, 2, 0, 0>
                   : (kind == 1 ? probe_mma_kernel<1, 1, 0, 0>
                                : (extra == 1 ? probe_mma_kernel<1, 0, 0, 1>
                                              : (extra == 2 ? probe_mma_kernel<1, 0, 0, 2>
                                                 : (extra == 3 ? probe_mma_kernel<1, 0, 0, 3>
                                                 : (extra == 4 ? probe_mma_kernel<1, 0, 0, 4>
                                                 : (extra == 5 ? probe_mma_kernel<1, 0, 0, 5>
                                                 : (extra == 6 ? probe_mma_kernel<1, 0, 0, 6>
                                                 : (extra == 7 ? probe_mma_kernel<1, 0, 0, 7>
                                                 : (extra == 8 ? probe_mma_kernel<1, 0, 0, 8>
                                                 : (extra == 9 ? probe_mma_kernel<1, 0, 0, 9>
                                                               : probe_mma_kernel<1, 0, 0, 0>))))))))));
        err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   PR_SMEM_LAUNCH);
        if (err == cudaSuccess) {
            cudaEventRecord(e0, s);
            kern<<<workers, PR_THREADS, PR_SMEM_LAUNCH, s>>>(fill, iters4, idesc, cycles, status);
            err = cudaGetLastError();
            cudaEventRecord(e1, s);
        }
    } else {
        void (*kern)(int, int64_t, uint32_t, int64_t*, int32_t*) =
            tmem_a ? probe_mma_kernel<2, 0, 1, 0>
                   : kind == 2 ? probe_mma_kernel<2, 2, 0, 0>
                   : (kind == 1 ? probe_mma_kernel<2, 1, 0, 0>
                                : (extra == 1 ? probe_mma_kernel<2, 0, 0, 1>
                                              : (extra == 2 ? probe_mma_kernel<2, 0, 0, 2>
                                                 : (extra == 3 ? probe_mma_kernel<2, 0, 0, 3>
                                                 : (extra == 4 ? probe_mma_kernel<2, 0, 0, 4>
                                                 : (extra == 5 ? probe_mma_kernel<2, 0, 0, 5>
                                                 : (extra == 6 ? probe_mma_kernel<2, 0, 0, 6>
                                                 : (extra == 7 ? probe_mma_kernel<2, 0, 0, 7>
                                                 : (extra == 8 ? probe_mma_kernel<2, 0, 0, 8>
                                                 : (extra == 9 ? probe_mma_kernel<2, 0, 0, 9>
                                                               : probe_mma_kernel<2, 0, 0, 0>))))))))));
        err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
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
            err = cudaLaunchKernelEx(&cfg, kern, fill, iters4, idesc, cycles, status);
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
            const int kdim = kind == 0 ? 32 : (kind == 2 ? 64 : 16);
            *ms = t;
            *tflops = 2.0 * m * n * kdim * (double)iters4 * workers / (t * 1e-3) / 1e12;
            *cycles_per_mma = sum / workers / (double)iters4;
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
