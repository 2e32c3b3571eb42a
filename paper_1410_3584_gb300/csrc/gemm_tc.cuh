// BF16 GEMM on the 5th-generation tensor cores (tcgen05, sm_103a) for the dense layers of
// the learned initial guess, plus an FP32 CUDA-core GEMM with the same contract (check mode).
//
//   C[M x N] (FP32) = A[M x K] * B[N x K]^T,  A and B BF16, row-major (K contiguous).
//
// One CTA (4 warps) computes a 128 x BN tile over the K range [z kper, (z + 1) kper) of its
// grid z index (split K: each split writes its partial product to C + z M N; kper = K gives
// the plain product).  Per K chunk of 64 the CTA stages A and B in
// shared memory in the canonical no-swizzle K-major layout (8-row x 16-byte core matrices;
// core matrices adjacent in K are LBO bytes apart, adjacent 8-row groups SBO bytes apart),
// one elected thread issues four 128 x BN x 16 MMAs accumulating in tensor memory and
// commits them to an mbarrier; the CTA waits on the mbarrier (bounded) before reusing the
// buffers.  The epilogue reads the accumulator with tcgen05.ld (warp w owns TMEM lanes
// 32w..32w+31 = rows) and stores FP32.  A wait that runs out sets *err, waits once more
// (bounded) for MMAs in flight, frees the tensor memory and returns.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace nlp {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: no swizzle, K-major
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;        // descriptor version for tcgen05
    return d;                      // base offset 0, layout type 0 (no swizzle)
}

// instruction descriptor, kind::f16: BF16 x BF16 -> F32, A and B K-major, M x N
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase, long long limit) {
    for (long long it = 0; it < limit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred P1;\n mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n selp.b32 %0, 1, 0, P1;\n}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(phase)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// stage rows [r0, r0+R) x K-chunk [k0, k0+64) of a row-major BF16 matrix (ld elements) into
// the core-matrix layout: chunk (row, kg) of 8 elements at ((kg * R/8 + row/8) * 8 + row%8) * 16 B
template <int R>
__device__ __forceinline__ void stage_tile(unsigned char *dst, const __nv_bfloat16 *src, int ld, int r0, int k0) {
    constexpr int CHUNKS = R * 8;   // 16-byte chunks: R rows x 8 groups of 8 K-elements
    for (int c = threadIdx.x; c < CHUNKS; c += blockDim.x) {
        const int row = c >> 3, kg = c & 7;
        const uint4 v = *reinterpret_cast<const uint4 *>(src + (size_t)(r0 + row) * ld + k0 + kg * 8);
        *reinterpret_cast<uint4 *>(dst + ((kg * (R / 8) + (row >> 3)) * 8 + (row & 7)) * 16) = v;
    }
}

constexpr int kGemmSmemBytes = 64 * 1024;

template <int BN>
__global__ void __launch_bounds__(128) k_gemm_bf16_tc(const __nv_bfloat16 *__restrict__ A,
                                                     const __nv_bfloat16 *__restrict__ B, float *__restrict__ C,
                                                     int M, int N, int K, int kper, int *err,
                                                     long long wait_limit) {
    constexpr int BM = 128;
    // A tile at 0, B tile at BM*128 bytes of one dynamic buffer of kGemmSmemBytes: larger than
    // the tiles so that every address an MMA can form from these descriptors stays inside it
    extern __shared__ __align__(1024) unsigned char gemm_smem[];
    unsigned char *sA = gemm_smem, *sB = gemm_smem + BM * 128;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kb = blockIdx.z * kper, ke = min(K, kb + kper);
    C += (size_t)blockIdx.z * M * N;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t mb = smem_u32(&mbar);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"((uint32_t)BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    constexpr uint32_t idesc = umma_idesc_bf16(BM, BN);
    // A: R = 128 -> LBO (next K core matrix) = 16 * 128 B, SBO (next 8 rows) = 128 B
    constexpr uint32_t lboA = (BM / 8) * 128, lboB = (BN / 8) * 128, sbo = 128;
    uint32_t phase = 0;
    bool ok = true;
    for (int k0 = kb; k0 < ke && ok; k0 += 64) {
        stage_tile<BM>(sA, A, K, m0, k0);
        stage_tile<BN>(sB, B, K, n0, k0);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {   // K = 16 per MMA = two core matrices along K
                const uint64_t ad = umma_desc(smem_u32(sA) + ks * 2 * lboA, lboA, sbo);
                const uint64_t bd = umma_desc(smem_u32(sB) + ks * 2 * lboB, lboB, sbo);
                const uint32_t acc = (k0 > kb || ks > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                         : "memory");
        }
        // every thread waits; the CTA continues only if all of them saw the phase complete
        ok = __syncthreads_and(mbar_wait(mb, phase, wait_limit) ? 1 : 0) != 0;
        phase ^= 1u;
    }
    if (!ok) {
        if (threadIdx.x == 0) atomicExch(err, 1);
        mbar_wait(mb, phase ^ 1u, wait_limit);   // let MMAs in flight finish before freeing
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int row = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            uint32_t r[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < M) {
                float *dst = C + (size_t)row * N + n0 + c0;
#pragma unroll
                for (int i = 0; i < 16; ++i) dst[i] = __uint_as_float(r[i]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)BN));
}

// C = sum over the S split-K partials P[z] (M N floats each), added in z order
__global__ void k_splitk_sum(const float *__restrict__ P, int S, int64_t MN, float *__restrict__ C) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < MN; i += (int64_t)gridDim.x * blockDim.x) {
        float t = P[i];
        for (int z = 1; z < S; ++z) t += P[(size_t)z * MN + i];
        C[i] = t;
    }
}

// FP32 CUDA-core GEMM with the same contract (inputs given in FP32), 16 x 16 tiles.
__global__ void k_gemm_f32_simt(const float *__restrict__ A, const float *__restrict__ B, float *__restrict__ C, int M,
                                int N, int K) {
    __shared__ float sA[16][17], sB[16][17];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
    float acc = 0.f;
    for (int k0 = 0; k0 < K; k0 += 16) {
        sA[ty][tx] = (row < M && k0 + tx < K) ? A[(size_t)row * K + k0 + tx] : 0.f;
        sB[ty][tx] = (blockIdx.x * 16 + ty < N && k0 + tx < K) ? B[(size_t)(blockIdx.x * 16 + ty) * K + k0 + tx] : 0.f;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) acc = fmaf(sA[ty][k], sB[tx][k], acc);
        __syncthreads();
    }
    if (row < M && col < N) C[(size_t)row * N + col] = acc;
}

}  // namespace nlp
