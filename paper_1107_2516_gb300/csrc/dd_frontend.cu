// Front end of the real-time pipeline (Section 5, Tables 5-6): the
// channeliser (an nfft-point FFT of each block of a subband's complex
// voltages), the intensity |X|^2 summed over polarisations, and the corner
// turn to channel-major order, fused into one pass over the voltages.
//
// Thread = one block b of one subband s: it loads nfft complex samples per
// polarisation with 16-byte loads (consecutive threads read consecutive
// blocks: coalesced), transforms them in registers (radix-2, decimation in
// time), and writes the nfft intensities to rows s*nfft + j of the output at
// column b.  Consecutive threads write consecutive columns of each row, so
// the corner turn needs no shared-memory transpose.  Every voltage is read
// once (8 bytes per sample and polarisation) and every intensity written once
// (4 bytes per nfft samples): the kernel is HBM-bound.
#include "dd_internal.h"

#include <algorithm>

namespace dd {

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// In-place radix-2 DIT FFT of F points (F a power of two), forward sign.
template <int F>
__device__ __forceinline__ void fft_inplace(float2 (&x)[F])
{
    // bit-reversal permutation
#pragma unroll
    for (int i = 0; i < F; ++i) {
        int r = 0;
#pragma unroll
        for (int b = 1, v = i; b < F; b <<= 1, v >>= 1) r = (r << 1) | (v & 1);
        if (r > i) { const float2 t = x[i]; x[i] = x[r]; x[r] = t; }
    }
#pragma unroll
    for (int len = 2; len <= F; len <<= 1) {
#pragma unroll
        for (int m = 0; m < len / 2; ++m) {
            float sn, cs;
            sincospif(-2.0f * (float)m / (float)len, &sn, &cs);     // W_len^m
            const float2 w = make_float2(cs, sn);
#pragma unroll
            for (int i = 0; i < F; i += len) {
                const float2 u = x[i + m], v = cmul(w, x[i + m + len / 2]);
                x[i + m] = make_float2(u.x + v.x, u.y + v.y);
                x[i + m + len / 2] = make_float2(u.x - v.x, u.y - v.y);
            }
        }
    }
}

template <int F, int NPOL>
__global__ void __launch_bounds__(256) channelise_kernel(const float2 *__restrict__ volt, int nsub,
                                                         int64_t nsamp, int64_t nblk,
                                                         float *__restrict__ out, int64_t out_pitch)
{
    const int s = blockIdx.y;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nblk;
         b += (int64_t)gridDim.x * blockDim.x) {
        float pw[F];
#pragma unroll
        for (int k = 0; k < F; ++k) pw[k] = 0.f;
#pragma unroll
        for (int p = 0; p < NPOL; ++p) {
            const float4 *src = reinterpret_cast<const float4 *>(volt + ((size_t)p * nsub + s) * nsamp + b * F);
            float2 x[F];
#pragma unroll
            for (int q = 0; q < F / 2; ++q) {
                const float4 v = __ldg(src + q);
                x[2 * q] = make_float2(v.x, v.y);
                x[2 * q + 1] = make_float2(v.z, v.w);
            }
            fft_inplace<F>(x);
#pragma unroll
            for (int k = 0; k < F; ++k) pw[k] += x[k].x * x[k].x + x[k].y * x[k].y;
        }
        // channel j of the subband: bin (F/2 - 1 - j) mod F (descending frequency)
#pragma unroll
        for (int j = 0; j < F; ++j)
            out[((size_t)s * F + j) * out_pitch + b] = pw[(F / 2 - 1 - j + F) % F];
    }
}

template <int F>
static cudaError_t channelise_launch(const float2 *v, int npol, int nsub, int64_t nsamp, float *out,
                                     int64_t out_pitch, cudaStream_t s)
{
    const int64_t nblk = nsamp / F;
    const dim3 grid((unsigned)std::min<int64_t>((nblk + 255) / 256, 65535), (unsigned)nsub);
    if (npol == 1)
        channelise_kernel<F, 1><<<grid, 256, 0, s>>>(v, nsub, nsamp, nblk, out, out_pitch);
    else
        channelise_kernel<F, 2><<<grid, 256, 0, s>>>(v, nsub, nsamp, nblk, out, out_pitch);
    return cudaGetLastError();
}

}  // namespace dd

using namespace dd;

extern "C" int dd_channelise(const void *volt_dev, int32_t npol, int32_t nsub, int64_t nsamp, int32_t nfft,
                             float *out_dev, int64_t out_pitch, void *stream)
{
    if (!volt_dev || !out_dev) return set_error(DD_ERR_ARG, "NULL buffer");
    if (npol < 1 || npol > 2) return set_error(DD_ERR_ARG, "npol must be 1 or 2");
    if (nsub < 1 || nsub > 65535) return set_error(DD_ERR_ARG, "nsub must be in 1..65535");
    if (nfft != 2 && nfft != 4 && nfft != 8 && nfft != 16 && nfft != 32)
        return set_error(DD_ERR_ARG, "nfft must be 2, 4, 8, 16 or 32");
    if (nsamp < nfft || nsamp % 2) return set_error(DD_ERR_ARG, "nsamp must be even and >= nfft");
    if ((uintptr_t)volt_dev & 15u) return set_error(DD_ERR_ARG, "voltages must be 16-byte aligned");
    if (out_pitch < nsamp / nfft) return set_error(DD_ERR_ARG, "out_pitch < nsamp / nfft");
    const float2 *v = static_cast<const float2 *>(volt_dev);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    switch (nfft) {
    case 2: e = channelise_launch<2>(v, npol, nsub, nsamp, out_dev, out_pitch, s); break;
    case 4: e = channelise_launch<4>(v, npol, nsub, nsamp, out_dev, out_pitch, s); break;
    case 8: e = channelise_launch<8>(v, npol, nsub, nsamp, out_dev, out_pitch, s); break;
    case 16: e = channelise_launch<16>(v, npol, nsub, nsamp, out_dev, out_pitch, s); break;
    default: e = channelise_launch<32>(v, npol, nsub, nsamp, out_dev, out_pitch, s); break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "launch channelise_kernel");
    return DD_OK;
}
