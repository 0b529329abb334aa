// Allocation-free statistics entry point (no counterpart in the paper).
//
// Some callers cannot call cudaMalloc: a real-time beam pipeline whose device
// memory is budgeted once at start-up and must not allocate afterwards
// (cudaMalloc/cudaFree can synchronise the device and stall the streams that
// carry live data), or code running where another runtime owns the device
// allocator.  dd_stats_f32_noalloc gives them the mean and standard deviation
// of a float32 device buffer (the quantities the search thresholds use) while
// allocating nothing: its per-block partial results live in the file-scope
// device array below, which every GPU that loads the library holds until the
// process exits.
#include "dd_device.cuh"
#include "dd_internal.h"

#include <mutex>

namespace dd {

constexpr int kNaThreads = 256;
constexpr int kNaPer = 16;                                 // elements per thread
constexpr int64_t kNaBlockElems = (int64_t)kNaThreads * kNaPer;
constexpr int kNaMaxBlocks = 65536;                        // 1.5 MB of partials
constexpr int64_t kNaMaxElems = kNaBlockElems * kNaMaxBlocks;   // 2^28 elements (1 GiB of float32)

// Shared by every call on a device; each call overwrites the first
// ceil(n / 4096) records before reading them, so nothing needs clearing.
static __device__ __align__(256) StatF g_noalloc_partials[kNaMaxBlocks];

__global__ void __launch_bounds__(kNaThreads) noalloc_partials_kernel(const float *__restrict__ x, int64_t n,
                                                                      StatF *__restrict__ part)
{
    const int64_t base = (int64_t)blockIdx.x * kNaBlockElems;
    float v[kNaPer];
    int cnt = 0;
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kNaPer; ++k) {
        const int64_t i = base + (int64_t)k * kNaThreads + threadIdx.x;
        v[k] = i < n ? x[i] : 0.f;
        if (i < n) { ++cnt; s += v[k]; }
    }
    const float m = cnt ? s / (float)cnt : 0.f;
    float q = 0.f;
#pragma unroll
    for (int k = 0; k < kNaPer; ++k) {
        const int64_t i = base + (int64_t)k * kNaThreads + threadIdx.x;
        if (i < n) { const float d = v[k] - m; q += d * d; }
    }
    block_stat_f32(cnt, s, q, part + blockIdx.x);
}

// One block: mean = sum n_b*mean_b / N, M2 = sum [M2_b + n_b (mean_b - mean)^2].
__global__ void __launch_bounds__(1024) noalloc_finalize_kernel(const StatF *__restrict__ part, int np,
                                                                double *__restrict__ mu_sigma)
{
    __shared__ double sa[1024], sb[1024];
    double n = 0, s = 0;
    for (int i = threadIdx.x; i < np; i += 1024) { n += part[i].n; s += part[i].n * part[i].mean; }
    sa[threadIdx.x] = n; sb[threadIdx.x] = s;
    __syncthreads();
    for (int h = 512; h > 0; h >>= 1) {
        if (threadIdx.x < h) { sa[threadIdx.x] += sa[threadIdx.x + h]; sb[threadIdx.x] += sb[threadIdx.x + h]; }
        __syncthreads();
    }
    const double N = sa[0];
    const double M = sb[0] / N;
    __syncthreads();
    double q = 0;
    for (int i = threadIdx.x; i < np; i += 1024) {
        const double e = part[i].mean - M;
        q += part[i].m2 + part[i].n * e * e;
    }
    sa[threadIdx.x] = q;
    __syncthreads();
    for (int h = 512; h > 0; h >>= 1) {
        if (threadIdx.x < h) sa[threadIdx.x] += sa[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) { mu_sigma[0] = M; mu_sigma[1] = sqrt(sa[0] / N); }
}

// Device address of g_noalloc_partials, looked up once per device with that
// device current (host code cannot use the symbol itself as an address).
static std::mutex g_na_mu;
static StatF *g_na_ptr[64] = {};

static int noalloc_scratch(StatF **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return set_error(DD_ERR_ARG, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> g(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
        g_na_ptr[dev] = static_cast<StatF *>(p);
    }
    *out = g_na_ptr[dev];
    return DD_OK;
}

}  // namespace dd

using namespace dd;

extern "C" int dd_stats_f32_noalloc(const float *x_dev, int64_t n, double *mu_sigma_dev, void *stream)
{
    if (!x_dev || !mu_sigma_dev) return set_error(DD_ERR_ARG, "NULL buffer");
    if (n < 1) return set_error(DD_ERR_ARG, "n must be >= 1");
    if (n > kNaMaxElems)
        return set_error(DD_ERR_ARG, "n = %lld exceeds the allocation-free maximum of %lld elements",
                         (long long)n, (long long)kNaMaxElems);
    StatF *part = nullptr;
    int rc = noalloc_scratch(&part);
    if (rc) return rc;
    const int nb = (int)((n + kNaBlockElems - 1) / kNaBlockElems);
    cudaStream_t s = (cudaStream_t)stream;
    noalloc_partials_kernel<<<nb, kNaThreads, 0, s>>>(x_dev, n, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch noalloc_partials_kernel");
    noalloc_finalize_kernel<<<1, 1024, 0, s>>>(part, nb, mu_sigma_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch noalloc_finalize_kernel");
    return DD_OK;
}
