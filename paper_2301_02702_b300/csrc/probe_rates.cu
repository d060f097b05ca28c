// Throughput probes behind the roofline of the Bloch kernel: scalar FFMA,
// packed FFMA (fma.rn.f32x2), MUFU ex2 and SHFL rates per SM per clock.
// Every thread writes one float to its own slot of `out` (grid x block
// floats); nothing else touches memory.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o probe_rates probe_rates.cu
#include <cstdio>
#include <cuda_runtime.h>
__global__ void ffma_k(float* out, int iters, float a) {
  float x0=threadIdx.x, x1=x0+1, x2=x0+2, x3=x0+3, x4=x0+4, x5=x0+5, x6=x0+6, x7=x0+7;
  for (int i=0;i<iters;++i){
    #pragma unroll
    for (int u=0;u<8;++u){ x0=fmaf(x0,a,0.5f); x1=fmaf(x1,a,0.5f); x2=fmaf(x2,a,0.5f); x3=fmaf(x3,a,0.5f);
                           x4=fmaf(x4,a,0.5f); x5=fmaf(x5,a,0.5f); x6=fmaf(x6,a,0.5f); x7=fmaf(x7,a,0.5f);}
  }
  out[blockIdx.x*blockDim.x+threadIdx.x]=x0+x1+x2+x3+x4+x5+x6+x7;
}
__device__ __forceinline__ unsigned long long f2(unsigned long long x, unsigned long long a, unsigned long long c){
  unsigned long long r; asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(x), "l"(a), "l"(c)); return r; }
__global__ void ffma2_k(float* out, int iters, float a) {
  unsigned long long av, cv; float2 aa=make_float2(a,a), cc=make_float2(0.5f,0.5f);
  av=*reinterpret_cast<unsigned long long*>(&aa); cv=*reinterpret_cast<unsigned long long*>(&cc);
  unsigned long long x[8];
  for (int k=0;k<8;++k){ float2 t=make_float2(threadIdx.x+k, threadIdx.x+k+0.5f); x[k]=*reinterpret_cast<unsigned long long*>(&t);} 
  for (int i=0;i<iters;++i){
    #pragma unroll
    for (int u=0;u<8;++u){
      #pragma unroll
      for (int k=0;k<8;++k) x[k]=f2(x[k],av,cv);
    }
  }
  float s=0; for(int k=0;k<8;++k){ float2 t=*reinterpret_cast<float2*>(&x[k]); s+=t.x+t.y; }
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
__global__ void mix_k(float* out, int iters, float a) {  // FFMA + FADD + SEL-ish ALU mix 1:1
  float x0=threadIdx.x, x1=x0+1, x2=x0+2, x3=x0+3; int m=threadIdx.x;
  for (int i=0;i<iters;++i){
    #pragma unroll
    for (int u=0;u<16;++u){ x0=fmaf(x0,a,0.5f); x1=fmaf(x1,a,0.5f); m = m ^ (u*7+i); x2 = (m&1)? x2 : x3; x3=fmaf(x3,a,x2);}
  }
  out[blockIdx.x*blockDim.x+threadIdx.x]=x0+x1+x2+x3+m;
}
__global__ void ex2_k(float* out, int iters, float a) {
  float x0=threadIdx.x*1e-3f, x1=x0+1e-3f, x2=x0+2e-3f, x3=x0+3e-3f;
  for (int i=0;i<iters;++i){
    #pragma unroll
    for (int u=0;u<8;++u){ x0=exp2f(-x0); x1=exp2f(-x1); x2=exp2f(-x2); x3=exp2f(-x3);} }
  out[blockIdx.x*blockDim.x+threadIdx.x]=x0+x1+x2+x3;
}
__global__ void shfl_k(float* out, int iters, float a) {
  float x0=threadIdx.x, x1=x0+1, x2=x0+2, x3=x0+3;
  for (int i=0;i<iters;++i){
    #pragma unroll
    for (int u=0;u<8;++u){ x0=__shfl_xor_sync(~0u,x0,1); x1=__shfl_xor_sync(~0u,x1,2); x2=__shfl_xor_sync(~0u,x2,4); x3=__shfl_xor_sync(~0u,x3,8);} }
  out[blockIdx.x*blockDim.x+threadIdx.x]=x0+x1+x2+x3;
}
template<typename K> double run(K k, const char* name, double ops_per_iter_thread, int iters) {
  int sms; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  int blocks = sms*8, threads=256; float* out; cudaMalloc(&out, sizeof(float)*blocks*threads);
  k<<<blocks,threads>>>(out, 10, 1.0001f); cudaDeviceSynchronize();
  cudaEvent_t a,b; cudaEventCreate(&a); cudaEventCreate(&b);
  cudaEventRecord(a); k<<<blocks,threads>>>(out, iters, 1.0001f); cudaEventRecord(b); cudaEventSynchronize(b);
  float ms; cudaEventElapsedTime(&ms,a,b);
  double ops = ops_per_iter_thread * iters * (double)blocks*threads;
  printf("%-8s %8.3f ms  %10.3f Gop/s  %7.2f op/clk/SM @2032MHz\n", name, ms, ops/ms/1e6, ops/(ms*1e-3)/sms/2.032e9);
  cudaFree(out); return ms;
}
int main(){
  run(ffma_k, "ffma", 64, 20000);
  run(ffma2_k, "ffma2x", 128, 20000);   // lane-FMAs
  run(mix_k, "mix", 48, 20000);          // 48 instrs / iter (3 fma + 1 alu pairs...) approx
  run(ex2_k, "ex2", 32, 5000);
  run(shfl_k, "shfl", 32, 5000);
  printf("err: %s\n", cudaGetErrorString(cudaGetLastError()));
}
