// TMEM <-> register throughput microbenchmark (tcgen05.st / tcgen05.ld 32x32b)
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

#define R32(p) "=r"(p[0]),"=r"(p[1]),"=r"(p[2]),"=r"(p[3]),"=r"(p[4]),"=r"(p[5]),"=r"(p[6]),"=r"(p[7]),"=r"(p[8]),"=r"(p[9]),"=r"(p[10]),"=r"(p[11]),"=r"(p[12]),"=r"(p[13]),"=r"(p[14]),"=r"(p[15]),"=r"(p[16]),"=r"(p[17]),"=r"(p[18]),"=r"(p[19]),"=r"(p[20]),"=r"(p[21]),"=r"(p[22]),"=r"(p[23]),"=r"(p[24]),"=r"(p[25]),"=r"(p[26]),"=r"(p[27]),"=r"(p[28]),"=r"(p[29]),"=r"(p[30]),"=r"(p[31])
#define W32(p) "r"(p[0]),"r"(p[1]),"r"(p[2]),"r"(p[3]),"r"(p[4]),"r"(p[5]),"r"(p[6]),"r"(p[7]),"r"(p[8]),"r"(p[9]),"r"(p[10]),"r"(p[11]),"r"(p[12]),"r"(p[13]),"r"(p[14]),"r"(p[15]),"r"(p[16]),"r"(p[17]),"r"(p[18]),"r"(p[19]),"r"(p[20]),"r"(p[21]),"r"(p[22]),"r"(p[23]),"r"(p[24]),"r"(p[25]),"r"(p[26]),"r"(p[27]),"r"(p[28]),"r"(p[29]),"r"(p[30]),"r"(p[31])
#define REGS "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}"
#define REGS1 "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32}"

__device__ __forceinline__ void tm_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 " REGS ", [%32];" : R32(r) : "r"(taddr));
}
__device__ __forceinline__ void tm_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], " REGS1 ";" :: "r"(taddr), W32(r) : "memory");
}
__device__ __forceinline__ void tm_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__global__ void __launch_bounds__(256, 1) tmem_bench(float* out, int iters, int mode, int nwarps_active) {
  __shared__ uint32_t taddr_s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    uint32_t dst = (uint32_t)__cvta_generic_to_shared(&taddr_s);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" :: "r"(dst) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t base = taddr_s;
  const uint32_t lb = (uint32_t)(32 * (warp & 3)) << 16;
  const uint32_t c0 = (uint32_t)(warp >> 2) * 256;
  uint32_t r[32];
  #pragma unroll
  for (int i = 0; i < 32; ++i) r[i] = __float_as_uint((float)(lane + i));
  float acc = 0.f;
  if (warp < nwarps_active) {
    tm_st32(base + lb + c0, r);
    tm_st32(base + lb + c0 + 32, r);
    tm_st32(base + lb + c0 + 64, r);
    tm_wait_st();
    for (int it = 0; it < iters; ++it) {
      const uint32_t col = c0 + ((it * 7) & 63);       // dynamic (warp-uniform) column offset
      if (mode == 0) {            // ld only, consume one value
        uint32_t v[32]; tm_ld32(base + lb + col, v); tm_wait_ld();
        acc += __uint_as_float(v[it & 31 ? 0 : 1]);
      } else if (mode == 1) {     // ld + 32 FADD
        uint32_t v[32]; tm_ld32(base + lb + col, v); tm_wait_ld();
        #pragma unroll
        for (int i = 0; i < 32; ++i) acc += __uint_as_float(v[i]);
      } else if (mode == 2) {     // two lds in flight, then wait
        uint32_t v[32], u[32]; tm_ld32(base + lb + col, v); tm_ld32(base + lb + col + 33, u); tm_wait_ld();
        acc += __uint_as_float(v[5]) + __uint_as_float(u[7]);
      } else {                    // st only
        r[it & 31] += 1u; tm_st32(base + lb + c0 + 128 + ((it * 5) & 63), r); tm_wait_st();
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" :: "r"(base) : "memory");
  if (acc == 1234.5f) out[0] = acc;
}

int main() {
  cudaDeviceProp p; cudaGetDeviceProperties(&p, 0);
  const int sms = p.multiProcessorCount;
  float* out; cudaMalloc(&out, 4);
  cudaFuncSetAttribute(tmem_bench, cudaFuncAttributeMaxDynamicSharedMemorySize, 120 * 1024);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  const char* names[] = {"ld x32 only", "ld x32 + 32 FADD", "2x ld x32 in flight", "st x32 only"};
  for (int mode = 0; mode < 4; ++mode)
    for (int nw = 4; nw <= 8; nw += 4) {
      const int iters = 20000;
      for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0);
        tmem_bench<<<sms, 256, 120 * 1024>>>(out, iters, mode, nw);
        cudaEventRecord(e1); cudaEventSynchronize(e1);
        float ms; cudaEventElapsedTime(&ms, e0, e1);
        double per = (mode == 2) ? 2 : 1;
        double bytes = (double)sms * nw * iters * per * 32 * 32 * 4;
        cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) { printf("error %s\n", cudaGetErrorString(err)); return 1; }
        if (rep) printf("%-22s warps=%d  %.3f ms  %.1f B/clk/SM at 2.07 GHz\n", names[mode], nw, ms, bytes / (ms * 1e-3) / sms / 2.07e9);
      }
    }
  return 0;
}
