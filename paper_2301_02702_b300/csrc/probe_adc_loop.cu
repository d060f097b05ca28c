// Throughput probe of the ADC loop's operation mix, in registers only: per
// sample, 4 spins per thread are summed (the signal) and each is turned by
// its rotator (one complex multiply). Two forms of the same arithmetic: two
// packed f32x2 pairs (as the Bloch kernel runs it) and scalar FP32. Prints
// spin-samples/s at 1, 2 and 4 CTAs of 224 threads per SM. Every thread
// writes one float to its own slot of `out`; nothing else touches memory.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o probe_adc_loop probe_adc_loop.cu
#include <cstdio>
#include <cuda_runtime.h>

typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk(float lo, float hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpk(f32x2 v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__global__ void adc_packed(float* out, int iters, float c0, float s0) {
    f32x2 pr[2], pi[2], qr[2], qi[2], qn[2];
    for (int p = 0; p < 2; ++p) {
        pr[p] = pk(threadIdx.x * 1e-3f + p, 0.5f);
        pi[p] = pk(0.25f, 0.125f * p);
        qr[p] = pk(c0, c0 * 0.999f);
        qi[p] = pk(s0, s0 * 1.001f);
        qn[p] = pk(-s0, -s0 * 1.001f);
    }
    float acc = 0.f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const f32x2 sr2 = add2(pr[0], pr[1]), si2 = add2(pi[0], pi[1]);
            float r0, r1, i0, i1;
            unpk(sr2, r0, r1);
            unpk(si2, i0, i1);
            acc += (r0 + r1) * (i0 + i1);
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                const f32x2 nr = fma2(pr[p], qr[p], mul2(pi[p], qn[p]));
                pi[p] = fma2(pr[p], qi[p], mul2(pi[p], qr[p]));
                pr[p] = nr;
            }
        }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

__global__ void adc_scalar(float* out, int iters, float c0, float s0) {
    float pr[4], pi[4], qr[4], qi[4];
    for (int s = 0; s < 4; ++s) {
        pr[s] = threadIdx.x * 1e-3f + s;
        pi[s] = 0.25f;
        qr[s] = c0 * (1.f - 1e-4f * s);
        qi[s] = s0 * (1.f + 1e-4f * s);
    }
    float acc = 0.f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const float sr = pr[0] + pr[1] + pr[2] + pr[3], si = pi[0] + pi[1] + pi[2] + pi[3];
            acc += sr * si;
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const float nr = fmaf(pr[s], qr[s], -pi[s] * qi[s]);
                pi[s] = fmaf(pr[s], qi[s], pi[s] * qr[s]);
                pr[s] = nr;
            }
        }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

template <typename K>
void run(K k, const char* name, int blocks_per_sm, int threads) {
    int sms;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    const int blocks = sms * blocks_per_sm, iters = 20000;
    float* out;
    cudaMalloc(&out, sizeof(float) * blocks * threads);
    k<<<blocks, threads>>>(out, 10, 0.9999f, 0.01f);
    cudaDeviceSynchronize();
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a);
    k<<<blocks, threads>>>(out, iters, 0.9999f, 0.01f);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms;
    cudaEventElapsedTime(&ms, a, b);
    const double spin_samples = 4.0 * 8 * iters * static_cast<double>(blocks) * threads;
    // 8 algorithmic flops per spin-sample (complex multiply 6, complex add 2)
    printf("%-7s %d x %3d threads/SM: %8.3f ms  %6.3f T spin-samples/s  %5.1f TFLOP/s (8 per spin-sample)\n", name,
           blocks_per_sm, threads, ms, spin_samples / ms / 1e9, 8 * spin_samples / ms / 1e9);
    cudaFree(out);
}

int main() {
    for (int bps : {1, 2, 4}) {
        run(adc_packed, "packed", bps, 224);
        run(adc_scalar, "scalar", bps, 224);
    }
    printf("err: %s\n", cudaGetErrorString(cudaGetLastError()));
    return 0;
}
