// Tensor-core probe for the readout kernel's matrix form: one tcgen05.mma
// shape (kind::f16, M = 128, N = 128, K = 16, FP32 accumulator in tensor
// memory, both operands K-major in shared memory without swizzle, as 8 x 16 B
// core matrices) checked against a host product, then timed.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o probe_umma probe_umma.cu
//   ./probe_umma
// Check: one CTA, D[128][128] = A[128][64] B[128][64]^T with small dyadic
// values (every product and partial sum exact in FP32).
// Rate: 148 CTAs (one per SM, forced by 160 KB of shared memory) issue
// `iters` x 4 MMAs each on resident tiles; flops = 2 M N K per MMA.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <vector>

namespace {

constexpr int kM = 128, kN = 128, kK = 64;
constexpr int kTileBytes = 128 * 16 * 2;  // one K = 16 slice of a 128-row operand
constexpr uint32_t kTmemCols = 512;       // the whole tensor memory (one CTA per SM)
constexpr unsigned long long kWaitNs = 2000000000ull;
constexpr size_t kDynSmem = 160 * 1024;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}
__device__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
    const uint64_t t0 = global_timer_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_timer_ns() - t0 > kWaitNs) return false;
    return true;
}

// Byte offset of element (row, k) in a 128-row x 16 K-major tile: core
// matrices of 8 rows x 16 contiguous bytes, K-adjacent cores 128 B apart,
// row-adjacent cores 256 B apart (4 KB per tile).
__host__ __device__ constexpr uint32_t tile_off(int row, int k) {
    return (row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// Shared-memory matrix descriptor: start address, leading-dimension (K)
// byte offset, stride-dimension (M/N) byte offset, all in 16-byte units;
// bits 46..48 the fixed value 0b001; no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    return static_cast<uint64_t>((addr & 0x3FFFFu) >> 4) | (static_cast<uint64_t>(128 >> 4) << 16) |
           (static_cast<uint64_t>(256 >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: D FP32 (bits 4..5 = 1), A and B FP16
// (bits 7..9, 10..12 = 0), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_f16(int m, int n) {
    return (1u << 4) | (static_cast<uint32_t>(n >> 3) << 17) | (static_cast<uint32_t>(m >> 4) << 24);
}

__global__ void __launch_bounds__(128, 1)
    umma_probe_kernel(const __half* __restrict__ A, const __half* __restrict__ B, float* __restrict__ D, int iters,
                      int* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;
    unsigned char* sB = smem + 4 * kTileBytes;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 8 * kTileBytes);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + 8 * kTileBytes + 64);
    const int tid = threadIdx.x, warp = tid >> 5;

    for (int i = tid; i < kM * kK; i += blockDim.x) {
        const int row = i / kK, k = i % kK;
        *reinterpret_cast<__half*>(sA + (k >> 4) * kTileBytes + tile_off(row, k & 15)) = A[i];
        *reinterpret_cast<__half*>(sB + (k >> 4) * kTileBytes + tile_off(row, k & 15)) = B[i];
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    if (tid == 0) {
        const uint32_t idesc = idesc_f16(kM, kN);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                const uint64_t da = smem_desc(smem_u32(sA + ks * kTileBytes));
                const uint64_t db = smem_desc(smem_u32(sB + ks * kTileBytes));
                const uint32_t acc = (it > 0 || ks > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(acc)
                    : "memory");
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(bar))
                     : "memory");
    }
    const bool ok = __syncthreads_and(mbar_wait_bounded(smem_u32(bar), 0));
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        for (int c = 0; c < kN; c += 16) {
            uint32_t r[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                "%13, %14, %15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(tmem + (static_cast<uint32_t>(32 * warp) << 16) + static_cast<uint32_t>(c)));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (blockIdx.x == 0)
                for (int j = 0; j < 16; ++j) D[(32 * warp + (tid & 31)) * kN + c + j] = __uint_as_float(r[j]);
        }
    } else if (tid == 0) {
        atomicOr(status, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// The readout kernel's issue pattern: per 32-spin block, 4 K slices x 3
// products (A hi B hi, A hi B lo, A lo B hi) from one of two 64 KB stages of
// 16 distinct 4 KB slices, optionally with a commit to an mbarrier and a
// tcgen05 fence after every block. Operand contents are whatever shared
// memory holds (the rate does not depend on them).
__global__ void __launch_bounds__(128, 1) umma_pattern_kernel(int blocks, int commit_each, int* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * 16 * kTileBytes);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + 2 * 16 * kTileBytes + 64);
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // bar[0]: the per-block commits (never waited on); bar[1]: the final commit
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar[0])), "r"(1) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar[1])), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    if (tid == 0) {
        const uint32_t idesc = idesc_f16(kM, kN);
        for (int b = 0; b < blocks; ++b) {
            const uint32_t base = smem_u32(smem + (b & 1) * 16 * kTileBytes);
            if (commit_each) asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int ks = 0; ks < 4; ++ks) {
                const uint64_t ah = smem_desc(base + ks * kTileBytes), al = smem_desc(base + (4 + ks) * kTileBytes);
                const uint64_t bh = smem_desc(base + (8 + ks) * kTileBytes), bl = smem_desc(base + (12 + ks) * kTileBytes);
                const uint64_t ops[3][2] = {{ah, bh}, {ah, bl}, {al, bh}};
                for (int q = 0; q < 3; ++q) {
                    const uint32_t acc = (b > 0 || ks > 0 || q > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n\t.reg .pred p;\n\t"
                        "setp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                        "l"(ops[q][0]), "l"(ops[q][1]), "r"(idesc), "r"(acc)
                        : "memory");
                }
            }
            if (commit_each && b + 1 < blocks)
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&bar[0]))
                             : "memory");
        }
        // completes when every MMA issued above has
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&bar[1]))
                     : "memory");
    }
    const bool ok = __syncthreads_and(mbar_wait_bounded(smem_u32(&bar[1]), 0));
    if (!ok && tid == 0) atomicOr(status, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

}  // namespace

#define CK(x)                                                                          \
    do {                                                                               \
        cudaError_t e_ = (x);                                                          \
        if (e_ != cudaSuccess) {                                                       \
            std::printf("CUDA error %s at %s:%d\n", cudaGetErrorString(e_), __FILE__, __LINE__); \
            return 1;                                                                  \
        }                                                                              \
    } while (0)

int main() {
    std::vector<__half> hA(kM * kK), hB(kN * kK);
    std::vector<float> fA(kM * kK), fB(kN * kK);
    uint32_t s = 12345u;
    auto next = [&]() {
        s = s * 1664525u + 1013904223u;
        return static_cast<int>((s >> 16) % 17) - 8;
    };
    for (int i = 0; i < kM * kK; ++i) {
        fA[i] = next() / 8.0f;
        hA[i] = __float2half(fA[i]);
        fB[i] = next() / 8.0f;
        hB[i] = __float2half(fB[i]);
    }
    __half *dA, *dB;
    float* dD;
    int* dst;
    CK(cudaMalloc(&dA, hA.size() * sizeof(__half)));
    CK(cudaMalloc(&dB, hB.size() * sizeof(__half)));
    CK(cudaMalloc(&dD, kM * kN * sizeof(float)));
    CK(cudaMalloc(&dst, sizeof(int)));
    CK(cudaMemcpy(dA, hA.data(), hA.size() * sizeof(__half), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(dB, hB.data(), hB.size() * sizeof(__half), cudaMemcpyHostToDevice));
    CK(cudaMemset(dD, 0, kM * kN * sizeof(float)));
    CK(cudaMemset(dst, 0, sizeof(int)));
    CK(cudaFuncSetAttribute(umma_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            static_cast<int>(kDynSmem)));

    umma_probe_kernel<<<1, 128, kDynSmem>>>(dA, dB, dD, 1, dst);
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    int st = 0;
    CK(cudaMemcpy(&st, dst, sizeof(int), cudaMemcpyDeviceToHost));
    std::vector<float> hD(kM * kN);
    CK(cudaMemcpy(hD.data(), dD, hD.size() * sizeof(float), cudaMemcpyDeviceToHost));
    double max_err = 0.0, max_ref = 0.0;
    for (int i = 0; i < kM; ++i)
        for (int j = 0; j < kN; ++j) {
            double ref = 0.0;
            for (int k = 0; k < kK; ++k) ref += static_cast<double>(fA[i * kK + k]) * fB[j * kK + k];
            max_err = std::fmax(max_err, std::fabs(ref - hD[i * kN + j]));
            max_ref = std::fmax(max_ref, std::fabs(ref));
        }
    std::printf("check: status %d, max |D - ref| = %.3g (max |ref| %.3g)\n", st, max_err, max_ref);
    if (st != 0 || max_err != 0.0) return 2;

    const int iters = 8192;
    umma_probe_kernel<<<148, 128, kDynSmem>>>(dA, dB, dD, 64, dst);
    CK(cudaDeviceSynchronize());
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0));
    umma_probe_kernel<<<148, 128, kDynSmem>>>(dA, dB, dD, iters, dst);
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    CK(cudaMemcpy(&st, dst, sizeof(int), cudaMemcpyDeviceToHost));
    const double flops = 148.0 * iters * 4 * 2.0 * kM * kN * 16;
    std::printf("rate: status %d, %d MMAs per CTA in %.3f ms: %.1f TFLOP/s\n", st, iters * 4, ms,
                flops / (ms * 1e-3) / 1e12);
    if (st != 0) return 3;

    // the readout kernel's pattern: 1,344 blocks of 12 MMAs per CTA
    CK(cudaFuncSetAttribute(umma_pattern_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            static_cast<int>(2 * 16 * kTileBytes + 256)));
    for (int commit_each = 0; commit_each < 2; ++commit_each) {
        const int blocks = 1344;
        umma_pattern_kernel<<<148, 128, 2 * 16 * kTileBytes + 256>>>(64, commit_each, dst);
        CK(cudaDeviceSynchronize());
        CK(cudaEventRecord(e0));
        umma_pattern_kernel<<<148, 128, 2 * 16 * kTileBytes + 256>>>(blocks, commit_each, dst);
        CK(cudaEventRecord(e1));
        CK(cudaEventSynchronize(e1));
        CK(cudaEventElapsedTime(&ms, e0, e1));
        CK(cudaMemcpy(&st, dst, sizeof(int), cudaMemcpyDeviceToHost));
        const double f = 148.0 * blocks * 12 * 2.0 * kM * kN * 16;
        std::printf("pattern (2 stages x 16 slices, 3 products, commit %s): status %d, %.3f ms: %.1f TFLOP/s\n",
                    commit_each ? "every block" : "at the end", st, ms, f / (ms * 1e-3) / 1e12);
    }
    return st != 0 ? 3 : 0;
}
