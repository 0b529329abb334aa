// microbenchmark: FADD / FADD2 issue throughput vs warps per SM, LDS.128 throughput
#include <cstdio>
#include <cuda_runtime.h>
template <int NACC>
__global__ void fadd_kernel(float* out, int iters, float a) {
  float acc[NACC];
  #pragma unroll
  for (int i = 0; i < NACC; ++i) acc[i] = threadIdx.x * 0.001f + i;
  float b = a * 0.5f;
  for (int it = 0; it < iters; ++it) {
    #pragma unroll
    for (int i = 0; i < NACC; ++i) acc[i] += (i & 1) ? a : b;
  }
  float s = 0; 
  #pragma unroll
  for (int i = 0; i < NACC; ++i) s += acc[i];
  if (s == 12345.f) out[0] = s;
}
template <int NACC>
__global__ void fadd2_kernel(float* out, int iters, float a) {
  unsigned long long acc[NACC/2];
  #pragma unroll
  for (int i = 0; i < NACC/2; ++i) { float2 v = make_float2(threadIdx.x*0.001f+i, i*0.5f); acc[i] = *(unsigned long long*)&v; }
  float2 av = make_float2(a, a*0.5f); unsigned long long ab = *(unsigned long long*)&av;
  for (int it = 0; it < iters; ++it) {
    #pragma unroll
    for (int i = 0; i < NACC/2; ++i) asm volatile("add.rn.f32x2 %0, %0, %1;" : "+l"(acc[i]) : "l"(ab));
  }
  float s = 0;
  #pragma unroll
  for (int i = 0; i < NACC/2; ++i) { float2 v = *(float2*)&acc[i]; s += v.x + v.y; }
  if (s == 12345.f) out[0] = s;
}
__global__ void lds_kernel(float* out, int iters) {
  __shared__ float4 sm[2048];
  for (int i = threadIdx.x; i < 2048; i += blockDim.x) sm[i] = make_float4(i, i+1, i+2, i+3);
  __syncthreads();
  float4 acc = make_float4(0,0,0,0);
  int idx = threadIdx.x;
  for (int it = 0; it < iters; ++it) {
    #pragma unroll
    for (int k = 0; k < 8; ++k) { float4 v = sm[(idx + k*32) & 2047]; acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w; }
    idx += 7;
  }
  if (acc.x == 12345.f) out[0] = acc.x;
}
int main() {
  int dev = 0; cudaDeviceProp p; cudaGetDeviceProperties(&p, dev);
  int sms = p.multiProcessorCount; printf("SMs %d\n", sms);
  float* out; cudaMalloc(&out, 4);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  const int iters = 20000;
  for (int wps = 1; wps <= 8; wps *= 2) {
    int threads = wps * 4 * 32;  // warps per SMSP * 4 SMSP
    for (int v = 0; v < 2; ++v) {
      for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0);
        if (v == 0) fadd_kernel<36><<<sms, threads>>>(out, iters, 1.0f);
        else fadd2_kernel<36><<<sms, threads>>>(out, iters, 1.0f);
        cudaEventRecord(e1); cudaEventSynchronize(e1);
        float ms; cudaEventElapsedTime(&ms, e0, e1);
        double adds = (double)sms * threads * iters * 36;
        if (rep) printf("%s warps/SMSP=%d  %.2f Tadd/s  (%.3f ms)\n", v ? "FADD2" : "FADD ", wps, adds / ms / 1e9, ms);
      }
    }
  }
  for (int wps = 1; wps <= 8; wps *= 2) {
    int threads = wps * 128;
    for (int rep = 0; rep < 2; ++rep) {
      cudaEventRecord(e0);
      lds_kernel<<<sms, threads>>>(out, iters);
      cudaEventRecord(e1); cudaEventSynchronize(e1);
      float ms; cudaEventElapsedTime(&ms, e0, e1);
      double bytes = (double)sms * threads * iters * 8 * 16;
      if (rep) printf("LDS.128 warps/SMSP=%d  %.1f B/clk/SM at 2.07GHz (%.3f ms)\n", wps, bytes / (ms*1e-3) / sms / 2.07e9, ms);
    }
  }
  cudaError_t err = cudaGetLastError(); printf("err %s\n", cudaGetErrorString(err));
  return 0;
}
