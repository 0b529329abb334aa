// Device helpers shared by the de-dispersion kernels: input conversion and
// per-block partial statistics (Section 3: mean and standard deviation over
// the whole processed buffer).
//
// Floating-point partials are formed without FP64 divisions in the hot path
// (GB300 executes FP64 at a small fraction of the FP32 rate): a thread keeps
// (count, sum, M2 about its own mean) in FP32, a warp combines them with the
// exact two-level identity M2 = sum_i [M2_i + n_i (mean_i - mean)^2], and one
// thread per block does the same over the warps in FP64 with one division.
#pragma once

#include "dd_internal.h"

namespace dd {

template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<uint8_t>(uint8_t v) { return (float)v; }
template <> __device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }

// n values of this thread with sum s and M2 q (about s/n).  All threads of the
// block must call it; thread 0 writes the block's (count, mean, M2).
__device__ __forceinline__ void block_stat_f32(int n, float s, float q, StatF *dst)
{
    __shared__ int shn[32];
    __shared__ float shm[32], shq[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    int nw = n;
    float sw = s;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        nw += __shfl_xor_sync(0xffffffffu, nw, off);
        sw += __shfl_xor_sync(0xffffffffu, sw, off);
    }
    const float mw = nw ? sw / (float)nw : 0.f;
    const float mt = n ? s / (float)n : 0.f;
    const float d = mt - mw;
    float qw = q + (float)n * d * d;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) qw += __shfl_xor_sync(0xffffffffu, qw, off);
    if (lane == 0) { shn[warp] = nw; shm[warp] = mw; shq[warp] = qw; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double N = 0, S = 0;
        for (int w = 0; w < nwarps; ++w) { N += shn[w]; S += (double)shn[w] * shm[w]; }
        const double M = N > 0 ? S / N : 0.0;
        double Q = 0;
        for (int w = 0; w < nwarps; ++w) {
            const double e = (double)shm[w] - M;
            Q += (double)shq[w] + (double)shn[w] * e * e;
        }
        dst->n = N; dst->mean = M; dst->m2 = Q;
    }
}

__device__ __forceinline__ void block_stat_i(long long n, long long s, unsigned long long q, StatI *dst)
{
    __shared__ long long shn[32], shs[32];
    __shared__ unsigned long long shq[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        n += __shfl_xor_sync(0xffffffffu, n, off);
        s += __shfl_xor_sync(0xffffffffu, s, off);
        q += __shfl_xor_sync(0xffffffffu, q, off);
    }
    if (lane == 0) { shn[warp] = n; shs[warp] = s; shq[warp] = q; }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long N = 0, S = 0;
        unsigned long long Q = 0;
        for (int w = 0; w < nwarps; ++w) { N += shn[w]; S += shs[w]; Q += shq[w]; }
        dst->n = N; dst->sum = S; dst->sumsq = Q;
    }
}

}  // namespace dd
