// Generic de-dispersion kernel (kernel 1), statistics and the boxcar
// threshold search.
//
// Section 3.1 (brute force): out[dm][t] = sum_c in[c][t + d(c,dm)].
// Section 3 (output stage): mean and standard deviation over the whole
// processed buffer, an n-sigma threshold, every point above it reported.
#include "dd_internal.h"
#include "dd_device.cuh"

#include <algorithm>
#include <cmath>
#include <type_traits>

namespace dd {

// ---------------------------------------------------------------------------
// Kernel 1: generic shared-memory de-dispersion.
//
// Block = kGenDms DM trials x kGenTile samples.  For each stage of `chunk`
// channels the block copies, per channel, the input span covering all its
// DM trials ([t0 + base, t0 + base + kGenTile + span)) into shared memory,
// converting to float; each thread then adds, for each of its samples and
// DM trials, the element at its delay offset.  One shared load per add.
// With chunk == 0 (span too large for shared memory) it reads global memory
// directly.
// ---------------------------------------------------------------------------
template <typename Tin, bool kInt>
__global__ void __launch_bounds__(kGenThreads)
generic_kernel(const Tin *__restrict__ in, int64_t pitch, int64_t nsamp_in, int nchans,
               const int32_t *__restrict__ goffs,   // [dmblk][nchans][kGenDms]
               const int32_t *__restrict__ gbase,   // [dmblk][nchans]
               const int32_t *__restrict__ gspan,   // [dmblk][nchans]
               int ndm, int64_t nout, void *__restrict__ out_, void *__restrict__ partials,
               int chunk, int stride)
{
    extern __shared__ float smem[];
    const int tid = threadIdx.x;
    const int64_t t0 = (int64_t)blockIdx.x * kGenTile;
    const int blk = blockIdx.y;
    const int dm0 = blk * kGenDms;
    const int ndb = min(kGenDms, ndm - dm0);
    const int32_t *boffs = goffs + (size_t)blk * nchans * kGenDms;
    const int32_t *bbase = gbase + (size_t)blk * nchans;
    const int32_t *bspan = gspan + (size_t)blk * nchans;

    float acc[kGenDms][kGenTimes];
#pragma unroll
    for (int j = 0; j < kGenDms; ++j)
#pragma unroll
        for (int k = 0; k < kGenTimes; ++k) acc[j][k] = 0.f;

    if (chunk > 0) {
        float *rows = smem;
        int *offs = reinterpret_cast<int *>(smem + (size_t)chunk * stride);
        for (int c0 = 0; c0 < nchans; c0 += chunk) {
            const int cn = min(chunk, nchans - c0);
            __syncthreads();
            for (int i = tid; i < cn * kGenDms; i += kGenThreads)
                offs[i] = boffs[(size_t)c0 * kGenDms + i];
            for (int c = 0; c < cn; ++c) {
                const int64_t s0 = t0 + bbase[c0 + c];
                const int len = kGenTile + bspan[c0 + c];
                const Tin *src = in + (size_t)(c0 + c) * pitch;
                float *dst = rows + (size_t)c * stride;
                for (int i = tid; i < len; i += kGenThreads) {
                    const int64_t s = s0 + i;
                    dst[i] = (s < nsamp_in) ? to_f(src[s]) : 0.f;
                }
            }
            __syncthreads();
            for (int c = 0; c < cn; ++c) {
                const float *r = rows + (size_t)c * stride + tid;
                const int *o = offs + c * kGenDms;
#pragma unroll
                for (int j = 0; j < kGenDms; ++j) {
                    const int oj = o[j];
#pragma unroll
                    for (int k = 0; k < kGenTimes; ++k) acc[j][k] += r[oj + k * kGenThreads];
                }
            }
        }
    } else {
        for (int c = 0; c < nchans; ++c) {
            const Tin *src = in + (size_t)c * pitch + bbase[c];
            const int32_t *o = boffs + (size_t)c * kGenDms;
#pragma unroll
            for (int j = 0; j < kGenDms; ++j) {
                const int oj = o[j];
#pragma unroll
                for (int k = 0; k < kGenTimes; ++k) {
                    const int64_t s = t0 + tid + k * kGenThreads + oj;
                    if (s + bbase[c] < nsamp_in) acc[j][k] += to_f(src[s]);
                }
            }
        }
    }

    // Epilogue: store, then per-block partial statistics.
    const int64_t pidx = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    if constexpr (kInt) {
        int32_t *out = reinterpret_cast<int32_t *>(out_);
        long long n = 0, s = 0;
        unsigned long long q = 0;
#pragma unroll
        for (int j = 0; j < kGenDms; ++j)
#pragma unroll
            for (int k = 0; k < kGenTimes; ++k) {
                const int64_t t = t0 + tid + k * kGenThreads;
                if (j < ndb && t < nout) {
                    const int v = __float2int_rn(acc[j][k]);
                    out[(size_t)(dm0 + j) * nout + t] = v;
                    n += 1; s += v; q += (unsigned long long)((long long)v * v);
                }
            }
        block_stat_i(n, s, q, reinterpret_cast<StatI *>(partials) + pidx);
    } else {
        float *out = reinterpret_cast<float *>(out_);
        int n = 0;
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < kGenDms; ++j)
#pragma unroll
            for (int k = 0; k < kGenTimes; ++k) {
                const int64_t t = t0 + tid + k * kGenThreads;
                if (j < ndb && t < nout) {
                    out[(size_t)(dm0 + j) * nout + t] = acc[j][k];
                    n += 1; s += acc[j][k];
                }
            }
        const float m = n ? s / (float)n : 0.f;
        float q = 0.f;
#pragma unroll
        for (int j = 0; j < kGenDms; ++j)
#pragma unroll
            for (int k = 0; k < kGenTimes; ++k) {
                const int64_t t = t0 + tid + k * kGenThreads;
                if (j < ndb && t < nout) { const float d = acc[j][k] - m; q += d * d; }
            }
        block_stat_f32(n, s, q, reinterpret_cast<StatF *>(partials) + pidx);
    }
}

// ---------------------------------------------------------------------------
// Statistics straight from an `out` buffer (used when dd_search is given a
// buffer other than the one the last dd_execute produced).
// ---------------------------------------------------------------------------
constexpr int kStatThreads = 256;
constexpr int kStatPer = 16;   // elements per thread

template <bool kInt>
__global__ void __launch_bounds__(kStatThreads)
stats_kernel(const void *__restrict__ out_, int64_t total, void *__restrict__ partials)
{
    const int64_t base = (int64_t)blockIdx.x * kStatThreads * kStatPer;
    if constexpr (kInt) {
        const int32_t *x = reinterpret_cast<const int32_t *>(out_);
        long long n = 0, s = 0;
        unsigned long long q = 0;
        for (int k = 0; k < kStatPer; ++k) {
            const int64_t i = base + (int64_t)k * kStatThreads + threadIdx.x;
            if (i < total) { const long long v = x[i]; n++; s += v; q += (unsigned long long)(v * v); }
        }
        block_stat_i(n, s, q, reinterpret_cast<StatI *>(partials) + blockIdx.x);
    } else {
        const float *x = reinterpret_cast<const float *>(out_);
        float v[kStatPer];
        int n = 0;
        float s = 0.f;
        for (int k = 0; k < kStatPer; ++k) {
            const int64_t i = base + (int64_t)k * kStatThreads + threadIdx.x;
            v[k] = i < total ? x[i] : 0.f;
            if (i < total) { n++; s += v[k]; }
        }
        const float m = n ? s / (float)n : 0.f;
        float q = 0.f;
        for (int k = 0; k < kStatPer; ++k) {
            const int64_t i = base + (int64_t)k * kStatThreads + threadIdx.x;
            if (i < total) { const float d = v[k] - m; q += d * d; }
        }
        block_stat_f32(n, s, q, reinterpret_cast<StatF *>(partials) + blockIdx.x);
    }
}

// ---------------------------------------------------------------------------
// Finalise: merge the per-block partials into mu and sigma (population, over
// the whole buffer) and form the per-width thresholds
//   T_w = w*mu + k*sigma*sqrt(w)
// in double (Section 3's n-sigma test applied to boxcar sums).  Each
// threshold is stored as the largest float <= T_w and as floor(T_w), so the
// kernels' FP32 / integer comparisons decide B_w > T_w exactly as a double
// comparison of the same B_w would.  One block of 1024 threads.
// ---------------------------------------------------------------------------
constexpr int kFinThreads = 1024;

template <bool kInt>
__global__ void __launch_bounds__(kFinThreads)
finalize_kernel(const void *__restrict__ partials, int64_t np, const int32_t *__restrict__ widths,
                int nw, double k, SearchParams *__restrict__ prm)
{
    __shared__ double mu_s, sg_s;
    if constexpr (kInt) {
        __shared__ long long sn[kFinThreads], ss[kFinThreads];
        __shared__ unsigned long long sq_lo[kFinThreads], sq_hi[kFinThreads];
        const StatI *p = reinterpret_cast<const StatI *>(partials);
        long long n = 0, s = 0;
        unsigned __int128 q = 0;
        for (int64_t i = threadIdx.x; i < np; i += kFinThreads) {
            n += p[i].n; s += p[i].sum; q += (unsigned __int128)p[i].sumsq;
        }
        sn[threadIdx.x] = n; ss[threadIdx.x] = s;
        sq_lo[threadIdx.x] = (unsigned long long)q;
        sq_hi[threadIdx.x] = (unsigned long long)(q >> 64);
        __syncthreads();
        for (int h = kFinThreads / 2; h > 0; h >>= 1) {
            if (threadIdx.x < h) {
                const int o = threadIdx.x + h;
                sn[threadIdx.x] += sn[o];
                ss[threadIdx.x] += ss[o];
                unsigned __int128 a = ((unsigned __int128)sq_hi[threadIdx.x] << 64) | sq_lo[threadIdx.x];
                unsigned __int128 b = ((unsigned __int128)sq_hi[o] << 64) | sq_lo[o];
                a += b;
                sq_lo[threadIdx.x] = (unsigned long long)a;
                sq_hi[threadIdx.x] = (unsigned long long)(a >> 64);
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const long long N = sn[0], S = ss[0];
            const unsigned __int128 Q = ((unsigned __int128)sq_hi[0] << 64) | sq_lo[0];
            // N*Q - S^2 >= 0 exactly (Cauchy-Schwarz), then one rounding each.
            const __int128 num = (__int128)((unsigned __int128)N * Q) - (__int128)S * (__int128)S;
            const double dn = (double)N;
            mu_s = (double)S / dn;
            sg_s = sqrt((double)num / (dn * dn));
        }
    } else {
        // Two passes over the partials, no division per partial:
        //   mean = sum n_b*mean_b / N,  M2 = sum [M2_b + n_b*(mean_b - mean)^2].
        __shared__ double sa[kFinThreads], sb[kFinThreads];
        const StatF *p = reinterpret_cast<const StatF *>(partials);
        double n = 0, s = 0;
        for (int64_t i = threadIdx.x; i < np; i += kFinThreads) { n += p[i].n; s += p[i].n * p[i].mean; }
        sa[threadIdx.x] = n; sb[threadIdx.x] = s;
        __syncthreads();
        for (int h = kFinThreads / 2; h > 0; h >>= 1) {
            if (threadIdx.x < h) { sa[threadIdx.x] += sa[threadIdx.x + h]; sb[threadIdx.x] += sb[threadIdx.x + h]; }
            __syncthreads();
        }
        const double N = sa[0];
        const double M = N > 0 ? sb[0] / N : 0.0;
        __syncthreads();
        double q = 0;
        for (int64_t i = threadIdx.x; i < np; i += kFinThreads) {
            const double e = p[i].mean - M;
            q += p[i].m2 + p[i].n * e * e;
        }
        sa[threadIdx.x] = q;
        __syncthreads();
        for (int h = kFinThreads / 2; h > 0; h >>= 1) {
            if (threadIdx.x < h) sa[threadIdx.x] += sa[threadIdx.x + h];
            __syncthreads();
        }
        if (threadIdx.x == 0) { mu_s = M; sg_s = sqrt(sa[0] / N); }
    }
    __syncthreads();
    if (threadIdx.x == 0) { prm->mu = mu_s; prm->sigma = sg_s; prm->nw = nw; }
    if (threadIdx.x < nw) {
        const double w = (double)widths[threadIdx.x];
        const double T = w * mu_s + k * sg_s * sqrt(w);
        prm->thr_f[threadIdx.x] = __double2float_rd(T);
        double f = floor(T);
        f = fmin(fmax(f, -4.0e18), 4.0e18);
        prm->thr_i[threadIdx.x] = (long long)f;
    }
}

// ---------------------------------------------------------------------------
// Per-DM-row statistics (search option): one block per row reads the row once.
// Float rows: each thread sums x - K and (x - K)^2 in FP32 with K its first
// value (a shift near the mean keeps the second moment free of cancellation),
// the block merges (n, mean, M2) in FP64.  Integer rows: exact int64 sums,
// 128-bit merge.  Then mu_row, sigma_row (population) and the row's
// thresholds T_w = w*mu_row + k*sigma_row*sqrt(w) in the exact float/integer
// forms of finalize_kernel.
// ---------------------------------------------------------------------------
constexpr int kRowThreads = 512;

template <bool kInt>
__global__ void __launch_bounds__(kRowThreads)
row_stats_kernel(const void *__restrict__ out_, int64_t nout, const int32_t *__restrict__ widths, int nw,
                 double k, RowParams *__restrict__ rp)
{
    __shared__ double sa[kRowThreads], sb[kRowThreads], sc[kRowThreads];
    __shared__ double mu_s, sg_s;
    const int row = blockIdx.x;
    const int tid = threadIdx.x;
    if constexpr (kInt) {
        const int32_t *x = reinterpret_cast<const int32_t *>(out_) + (size_t)row * nout;
        long long n = 0, s = 0, q = 0;
        for (int64_t t = tid; t < nout; t += kRowThreads) {
            const long long v = x[t];
            n++; s += v; q += v * v;
        }
        __shared__ long long sn[kRowThreads], ss[kRowThreads];
        __shared__ unsigned long long ql[kRowThreads], qh[kRowThreads];
        sn[tid] = n; ss[tid] = s; ql[tid] = (unsigned long long)q; qh[tid] = 0;
        __syncthreads();
        for (int h = kRowThreads / 2; h > 0; h >>= 1) {
            if (tid < h) {
                sn[tid] += sn[tid + h];
                ss[tid] += ss[tid + h];
                unsigned __int128 a = ((unsigned __int128)qh[tid] << 64) | ql[tid];
                const unsigned __int128 b = ((unsigned __int128)qh[tid + h] << 64) | ql[tid + h];
                a += b;
                ql[tid] = (unsigned long long)a;
                qh[tid] = (unsigned long long)(a >> 64);
            }
            __syncthreads();
        }
        if (tid == 0) {
            const long long N = sn[0], S = ss[0];
            const unsigned __int128 Q = ((unsigned __int128)qh[0] << 64) | ql[0];
            const __int128 num = (__int128)((unsigned __int128)N * Q) - (__int128)S * (__int128)S;
            const double dn = (double)N;
            mu_s = (double)S / dn;
            sg_s = sqrt((double)num / (dn * dn));
        }
    } else {
        const float *x = reinterpret_cast<const float *>(out_) + (size_t)row * nout;
        const float K = tid < nout ? x[tid] : 0.f;
        float s = 0.f, q = 0.f;
        int n = 0;
        for (int64_t t = tid; t < nout; t += kRowThreads) {
            const float d = x[t] - K;
            s += d; q += d * d; n++;
        }
        // thread (n, mean, M2) in double: mean = K + s/n, M2 = q - s^2/n
        const double dn = (double)n;
        const double m = n ? (double)K + (double)s / dn : 0.0;
        const double m2 = n ? fmax((double)q - (double)s * (double)s / dn, 0.0) : 0.0;
        sa[tid] = dn; sb[tid] = dn * m;
        __syncthreads();
        for (int h = kRowThreads / 2; h > 0; h >>= 1) {
            if (tid < h) { sa[tid] += sa[tid + h]; sb[tid] += sb[tid + h]; }
            __syncthreads();
        }
        const double N = sa[0], M = N > 0 ? sb[0] / N : 0.0;
        __syncthreads();
        const double e = m - M;
        sc[tid] = m2 + dn * e * e;
        __syncthreads();
        for (int h = kRowThreads / 2; h > 0; h >>= 1) {
            if (tid < h) sc[tid] += sc[tid + h];
            __syncthreads();
        }
        if (tid == 0) { mu_s = M; sg_s = sqrt(sc[0] / N); }
    }
    __syncthreads();
    if (tid == 0) { rp[row].mu = mu_s; rp[row].sigma = sg_s; }
    if (tid < nw) {
        const double w = (double)widths[tid];
        const double T = w * mu_s + k * sg_s * sqrt(w);
        rp[row].thr_f[tid] = __double2float_rd(T);
        double f = floor(T);
        f = fmin(fmax(f, -4.0e18), 4.0e18);
        rp[row].thr_i[tid] = (long long)f;
    }
}

// ---------------------------------------------------------------------------
// Boxcar threshold search.  Block = one DM row x kSearchTile samples; thread
// owns kSearchPer consecutive samples.  For the widths in ascending order it
// extends B_w at its first sample from the previous width's sum, then slides
// it along its samples (B_w(t+1) = B_w(t) + x[t+w] - x[t]), testing
// B_w > T_w at each (t, w).  Only FP32 (or integer) arithmetic runs here;
// hits are appended with one atomic each and their S/N is formed afterwards
// by cand_snr_kernel.  The shared tile is padded one word per 16 so the
// per-thread windows fall in distinct banks.
// ---------------------------------------------------------------------------
constexpr int kSearchThreads = 256;
constexpr int kSearchPer = 16;
constexpr int kSearchTile = kSearchThreads * kSearchPer;

__host__ __device__ __forceinline__ int spad(int i) { return i + (i >> 4); }

template <bool kInt>
__global__ void __launch_bounds__(kSearchThreads)
search_kernel(const void *__restrict__ out_, int64_t nout,
              const int32_t *__restrict__ wsorted, int nw, int wmax,
              const SearchParams *__restrict__ prm, const RowParams *__restrict__ rp,
              dd_candidate *__restrict__ cands, int64_t cap, unsigned long long *__restrict__ count)
{
    using T = typename std::conditional<kInt, int32_t, float>::type;
    using Acc = typename std::conditional<kInt, long long, float>::type;
    extern __shared__ __align__(16) unsigned char sraw[];
    __shared__ int sw[kMaxWidths], sidx[kMaxWidths];
    __shared__ float thf[kMaxWidths];
    __shared__ long long thi[kMaxWidths];
    T *x = reinterpret_cast<T *>(sraw);
    const int row = blockIdx.y;
    const int64_t t0 = (int64_t)blockIdx.x * kSearchTile;
    const int len = kSearchTile + wmax - 1;
    if (threadIdx.x < nw) {
        sw[threadIdx.x] = wsorted[threadIdx.x];
        sidx[threadIdx.x] = wsorted[nw + threadIdx.x];
        thf[threadIdx.x] = rp ? rp[blockIdx.y].thr_f[sidx[threadIdx.x]] : prm->thr_f[sidx[threadIdx.x]];
        thi[threadIdx.x] = rp ? rp[blockIdx.y].thr_i[sidx[threadIdx.x]] : prm->thr_i[sidx[threadIdx.x]];
    }
    const T *src = reinterpret_cast<const T *>(out_) + (size_t)row * nout;
    for (int i = threadIdx.x; i < len; i += kSearchThreads) {
        const int64_t t = t0 + i;
        x[spad(i)] = t < nout ? src[t] : (T)0;
    }
    __syncthreads();
    const int base = threadIdx.x * kSearchPer;
    const int64_t tb = t0 + base;
    if (tb >= nout) return;
    Acc b0 = 0;          // running B_w at the thread's first sample
    int wprev = 0;
    for (int p = 0; p < nw; ++p) {
        const int w = sw[p];
        for (int j = wprev; j < w; ++j) b0 += (Acc)x[spad(base + j)];
        wprev = w;
        Acc b = b0;
        for (int i = 0; i < kSearchPer; ++i) {
            const int64_t t = tb + i;
            if (t + w > nout) break;
            if (i > 0) b += (Acc)x[spad(base + i - 1 + w)] - (Acc)x[spad(base + i - 1)];
            bool hit;
            if constexpr (kInt) hit = b > thi[p];
            else hit = b > thf[p];
            if (hit) {
                const unsigned long long pos = atomicAdd(count, 1ull);
                if ((int64_t)pos < cap) {
                    dd_candidate c;
                    c.dm_idx = row; c.width_idx = sidx[p]; c.t = t;
                    c.snr = 0.f; c.reserved = 0.f; c.value = (double)b;
                    cands[pos] = c;
                }
            }
        }
    }
}

// The same search for the common width set {1, 2, 4, ..., 2^(K-1)}.  The
// tile is staged with kSearchPer independent loads per thread; each thread
// then copies its kSearchPer samples plus the 2^(K-1) - 1 that follow into
// registers and forms the boxcars as a doubling tree, B_2w(i) = B_w(i) +
// B_w(i + w): one add per sample and width, no shared-memory traffic in the
// loop (the sliding form needs two shared words per sample and width).
// Integer data stay in int32 (at most 65536 channels x 255 x 64 < 2^31).
template <bool kInt, int K>
__global__ void __launch_bounds__(kSearchThreads)
search_pow2_kernel(const void *__restrict__ out_, int64_t nout, const int32_t *__restrict__ wsorted,
                   const SearchParams *__restrict__ prm, const RowParams *__restrict__ rp,
                   dd_candidate *__restrict__ cands, int64_t cap, unsigned long long *__restrict__ count)
{
    using T = typename std::conditional<kInt, int32_t, float>::type;
    constexpr int W = 1 << (K - 1);                 // widest boxcar
    constexpr int kWin = kSearchPer + W - 1;
    extern __shared__ __align__(16) unsigned char sraw[];
    __shared__ int sidx[K];
    __shared__ float thf[K];
    __shared__ long long thi[K];
    T *x = reinterpret_cast<T *>(sraw);
    const int row = blockIdx.y;
    const int64_t t0 = (int64_t)blockIdx.x * kSearchTile;
    if (threadIdx.x < K) {
        const int o = wsorted[K + threadIdx.x];     // original index of sorted width 2^threadIdx.x
        sidx[threadIdx.x] = o;
        thf[threadIdx.x] = rp ? rp[blockIdx.y].thr_f[o] : prm->thr_f[o];
        thi[threadIdx.x] = rp ? rp[blockIdx.y].thr_i[o] : prm->thr_i[o];
    }
    const T *src = reinterpret_cast<const T *>(out_) + (size_t)row * nout + t0;
    const int64_t avail = nout - t0;                // > 0
    T r[kSearchPer];
#pragma unroll
    for (int q = 0; q < kSearchPer; ++q) {
        const int i = q * kSearchThreads + threadIdx.x;
        r[q] = i < avail ? src[i] : (T)0;
    }
#pragma unroll
    for (int q = 0; q < kSearchPer; ++q) x[spad(q * kSearchThreads + threadIdx.x)] = r[q];
    if ((int)threadIdx.x < W - 1) {
        const int i = kSearchTile + threadIdx.x;
        x[spad(i)] = i < avail ? src[i] : (T)0;
    }
    __syncthreads();
    const int base = threadIdx.x * kSearchPer;
    if (base >= avail) return;
    const int64_t rem = avail - base;               // samples from this thread's first one on
    T b[kWin];
#pragma unroll
    for (int k = 0; k < kWin; ++k) b[k] = x[spad(base + k)];
    // hits as bits p*16 + i (width 2^p, sample i): the unrolled loop stays
    // compact; the rare appends run once below
    unsigned long long hits[2] = {0ull, 0ull};
#pragma unroll
    for (int p = 0; p < K; ++p) {
        const int w = 1 << p;
        if (p > 0) {
            // b[k] = B_{w/2}(k) -> B_w(k); ascending k reads b[k + w/2] before it changes
#pragma unroll
            for (int k = 0; k + w <= kWin; ++k) b[k] = b[k] + b[k + w / 2];
        }
        unsigned m = 0;
#pragma unroll
        for (int i = 0; i < kSearchPer; ++i) {
            bool hit;
            if constexpr (kInt) hit = (long long)b[i] > thi[p];
            else hit = b[i] > thf[p];
            m |= (unsigned)hit << i;
        }
        const int64_t lim = rem - w + 1;            // tests with t + w <= nout
        if (lim < kSearchPer) m &= lim > 0 ? (1u << lim) - 1u : 0u;
        hits[p >> 2] |= (unsigned long long)m << (16 * (p & 3));
    }
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
        unsigned long long bits = hits[h];
        while (bits) {
            const int bit = __ffsll((long long)bits) - 1;
            bits &= bits - 1;
            const int p = 4 * h + (bit >> 4), i = bit & 15, w = 1 << p;
            // B_w(i) again, by the same pairwise tree (bit-identical value)
            T v[1 << (K - 1)];
            for (int q = 0; q < w; ++q) v[q] = x[spad(base + i + q)];
            for (int d = 1; d < w; d *= 2)
                for (int q = 0; q + d < w; q += 2 * d) v[q] = v[q] + v[q + d];
            const unsigned long long pos = atomicAdd(count, 1ull);
            if ((int64_t)pos < cap) {
                dd_candidate c;
                c.dm_idx = row; c.width_idx = sidx[p]; c.t = t0 + base + i;
                c.snr = 0.f; c.reserved = 0.f; c.value = (double)v[0];
                cands[pos] = c;
            }
        }
    }
}

template <bool kInt, int K>
static void launch_search_pow2(dim3 grid, cudaStream_t s, const void *out, const dd_plan *p)
{
    const size_t smem = (size_t)(spad(kSearchTile + (1 << (K - 1)) - 1) + 1) * 4;
    search_pow2_kernel<kInt, K><<<grid, kSearchThreads, smem, s>>>(out, p->nsamp_out, p->d_wsorted, p->d_params,
                                                                    p->row_stats ? p->d_rowprm : nullptr,
                                                                    p->d_cands, p->cand_cap, p->d_count);
}

// K if the plan's widths are exactly {1, 2, ..., 2^(K-1)} with K <= 7, else 0.
static int pow2_widths(const dd_plan *p)
{
    std::vector<int> w(p->widths.begin(), p->widths.end());
    std::sort(w.begin(), w.end());
    if (w.size() > 7) return 0;
    for (size_t i = 0; i < w.size(); ++i)
        if (w[i] != (1 << i)) return 0;
    return (int)w.size();
}

template <bool kInt>
static void launch_search_pow2_k(int K, dim3 grid, cudaStream_t s, const void *out, const dd_plan *p)
{
    switch (K) {
    case 1: launch_search_pow2<kInt, 1>(grid, s, out, p); break;
    case 2: launch_search_pow2<kInt, 2>(grid, s, out, p); break;
    case 3: launch_search_pow2<kInt, 3>(grid, s, out, p); break;
    case 4: launch_search_pow2<kInt, 4>(grid, s, out, p); break;
    case 5: launch_search_pow2<kInt, 5>(grid, s, out, p); break;
    case 6: launch_search_pow2<kInt, 6>(grid, s, out, p); break;
    default: launch_search_pow2<kInt, 7>(grid, s, out, p); break;
    }
}

// Boxcars that cross a chunk boundary (streaming search variant): per DM row,
// x = [the previous chunk's last L outputs | this chunk's first L outputs],
// L = wmax - 1; every window of width w starting at i in [L - w + 1, L) (it
// starts in the previous chunk and ends in this one) is tested against this
// chunk's thresholds.  Hits get t = i - L < 0: the window starts |t| samples
// before this chunk's first output.  S/N is formed on the host.
template <bool kInt>
__global__ void __launch_bounds__(128)
boundary_search_kernel(const void *__restrict__ tail_, const void *__restrict__ out_, int64_t nout, int L,
                       const int32_t *__restrict__ widths, int nw, const SearchParams *__restrict__ prm,
                       const RowParams *__restrict__ rp, dd_candidate *__restrict__ cands, int64_t cap,
                       unsigned long long *__restrict__ count)
{
    using T = typename std::conditional<kInt, int32_t, float>::type;
    using Acc = typename std::conditional<kInt, long long, float>::type;
    extern __shared__ __align__(16) unsigned char sraw[];
    T *x = reinterpret_cast<T *>(sraw);
    const int row = blockIdx.x;
    const T *tail = reinterpret_cast<const T *>(tail_) + (size_t)row * L;
    const T *head = reinterpret_cast<const T *>(out_) + (size_t)row * nout;
    for (int i = threadIdx.x; i < L; i += blockDim.x) { x[i] = tail[i]; x[L + i] = head[i]; }
    __syncthreads();
    for (int q = threadIdx.x; q < nw * L; q += blockDim.x) {
        const int p = q / L, i = q - p * L, w = widths[p];
        if (i < L - w + 1) continue;                 // window ends before this chunk
        Acc b = 0;
        for (int j = 0; j < w; ++j) b += (Acc)x[i + j];
        bool hit;
        if constexpr (kInt) hit = (long long)b > (rp ? rp[row].thr_i[p] : prm->thr_i[p]);
        else hit = b > (rp ? rp[row].thr_f[p] : prm->thr_f[p]);
        if (hit) {
            const unsigned long long pos = atomicAdd(count, 1ull);
            if ((int64_t)pos < cap) {
                dd_candidate c;
                c.dm_idx = row; c.width_idx = p; c.t = (int64_t)i - L;
                c.snr = 0.f; c.reserved = 0.f; c.value = (double)b;
                cands[pos] = c;
            }
        }
    }
}

int boundary_search_launch(dd_plan *p, const void *tail, const void *out, int L, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(p->d_count, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "memset count");
    const int32_t *w_orig = p->d_wsorted + 2 * p->nwidths;
    const RowParams *rp = p->row_stats ? p->d_rowprm : nullptr;
    const size_t smem = (size_t)2 * L * 4;
    if (p->dtype == DD_U8)
        boundary_search_kernel<true><<<(unsigned)p->ndm, 128, smem, s>>>(tail, out, p->nsamp_out, L, w_orig, p->nwidths,
                                                                        p->d_params, rp, p->d_cands, p->cand_cap,
                                                                        p->d_count);
    else
        boundary_search_kernel<false><<<(unsigned)p->ndm, 128, smem, s>>>(tail, out, p->nsamp_out, L, w_orig,
                                                                         p->nwidths, p->d_params, rp, p->d_cands,
                                                                         p->cand_cap, p->d_count);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch boundary_search_kernel");
    return DD_OK;
}

// S/N of the compacted hits: (B_w - w*mu) / (sigma*sqrt(w)), in double.
__global__ void cand_snr_kernel(dd_candidate *__restrict__ cands, const unsigned long long *__restrict__ count,
                                int64_t cap, const int32_t *__restrict__ widths, const SearchParams *__restrict__ prm,
                                const RowParams *__restrict__ rp)
{
    const int64_t n = min((int64_t)*count, cap);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double w = (double)widths[cands[i].width_idx];
        const double mu = rp ? rp[cands[i].dm_idx].mu : prm->mu;
        const double sg = rp ? rp[cands[i].dm_idx].sigma : prm->sigma;
        cands[i].snr = (float)((cands[i].value - w * mu) / (sg * sqrt(w)));
    }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
static size_t stat_size(const dd_plan *p)
{
    return p->dtype == DD_U8 ? sizeof(StatI) : sizeof(StatF);
}

// The dynamic shared-memory limit is a per-kernel (not per-plan) attribute:
// set it once to everything the device allows so that plans of different
// geometry never lower it under one another.
cudaError_t allow_max_dynamic_smem(const void *fn, size_t optin)
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, fn);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(optin - a.sharedSizeBytes));
}

int ensure_partials_public(dd_plan *p, int64_t n)
{
    if (n <= p->n_partials_cap) return DD_OK;
    if (p->d_partials) cudaFree(p->d_partials);
    p->d_partials = nullptr;
    p->n_partials_cap = 0;
    cudaError_t e = cudaMalloc(&p->d_partials, (size_t)n * stat_size(p));
    if (e != cudaSuccess) return set_error(DD_ERR_NOMEM, "cudaMalloc(partials, %lld): %s",
                                           (long long)n, cudaGetErrorString(e));
    p->n_partials_cap = n;
    return DD_OK;
}

int generic_configure(dd_plan *p)
{
    const int nblk = (p->ndm + kGenDms - 1) / kGenDms;
    const int C = p->nchans;
    std::vector<int32_t> offs((size_t)nblk * C * kGenDms), base((size_t)nblk * C), span((size_t)nblk * C);
    int maxspan = 0;
    for (int b = 0; b < nblk; ++b) {
        const int dm0 = b * kGenDms, ndb = std::min(kGenDms, p->ndm - dm0);
        for (int c = 0; c < C; ++c) {
            int lo = INT32_MAX, hi = INT32_MIN;
            for (int j = 0; j < ndb; ++j) {
                const int d = p->delays[(size_t)(dm0 + j) * C + c];
                lo = std::min(lo, d); hi = std::max(hi, d);
            }
            base[(size_t)b * C + c] = lo;
            span[(size_t)b * C + c] = hi - lo;
            maxspan = std::max(maxspan, hi - lo);
            for (int j = 0; j < kGenDms; ++j) {
                const int jj = std::min(j, ndb - 1);
                offs[((size_t)b * C + c) * kGenDms + j] = p->delays[(size_t)(dm0 + jj) * C + c] - lo;
            }
        }
    }
    // Shared-memory geometry: rows of kGenTile + maxspan floats (rounded to 4).
    const int stride = ((kGenTile + maxspan + 3) / 4) * 4;
    const size_t budget = std::min<size_t>(p->smem_optin, 100 * 1024);
    const size_t per_chan = (size_t)stride * sizeof(float) + kGenDms * sizeof(int);
    int chunk = (int)std::min<size_t>(16, budget / per_chan);
    if (chunk < 1) chunk = 0;
    p->gen_stride = stride;
    p->gen_chunk = chunk;
    p->gen_smem = chunk ? (size_t)chunk * per_chan : 0;

    // Device copies, packed as [offs | base | span] in one allocation.
    void *dptr = nullptr;
    const size_t bytes = (offs.size() + base.size() + span.size()) * sizeof(int32_t);
    cudaError_t e = cudaMalloc(&dptr, bytes);
    if (e != cudaSuccess) return set_error(DD_ERR_NOMEM, "cudaMalloc(generic tables): %s", cudaGetErrorString(e));
    int32_t *d = static_cast<int32_t *>(dptr);
    e = cudaMemcpy(d, offs.data(), offs.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d + offs.size(), base.data(), base.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d + offs.size() + base.size(), span.data(), span.size() * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(dptr); return cuda_fail(e, "upload generic tables"); }
    p->d_gen = d;
    if (chunk) {
        auto set = [&](const void *fn) {
            return allow_max_dynamic_smem(fn, p->smem_optin);
        };
        cudaError_t a = cudaSuccess;
        a = set((const void *)generic_kernel<float, false>);
        if (a == cudaSuccess) a = set((const void *)generic_kernel<__half, false>);
        if (a == cudaSuccess) a = set((const void *)generic_kernel<uint8_t, true>);
        if (a != cudaSuccess) return cuda_fail(a, "cudaFuncSetAttribute(generic)");
    }
    return DD_OK;
}

int generic_execute(dd_plan *p, const void *in, int64_t pitch, void *out, cudaStream_t s)
{
    const int nblk = (p->ndm + kGenDms - 1) / kGenDms;
    const int64_t ntile = (p->nsamp_out + kGenTile - 1) / kGenTile;
    if (ntile > INT32_MAX || nblk > 65535) return set_error(DD_ERR_ARG, "problem too large for kernel 1 grid");
    const int64_t np = ntile * nblk;
    int rc = ensure_partials_public(p, np);
    if (rc) return rc;
    const size_t noffs = (size_t)nblk * p->nchans * kGenDms;
    const int32_t *goffs = p->d_gen;
    const int32_t *gbase = goffs + noffs;
    const int32_t *gspan = gbase + (size_t)nblk * p->nchans;
    dim3 grid((unsigned)ntile, (unsigned)nblk);
    switch (p->dtype) {
    case DD_F32:
        generic_kernel<float, false><<<grid, kGenThreads, p->gen_smem, s>>>(
            (const float *)in, pitch, p->nsamp_in, p->nchans, goffs, gbase, gspan, p->ndm,
            p->nsamp_out, out, p->d_partials, p->gen_chunk, p->gen_stride);
        break;
    case DD_F16:
        generic_kernel<__half, false><<<grid, kGenThreads, p->gen_smem, s>>>(
            (const __half *)in, pitch, p->nsamp_in, p->nchans, goffs, gbase, gspan, p->ndm,
            p->nsamp_out, out, p->d_partials, p->gen_chunk, p->gen_stride);
        break;
    case DD_U8:
        generic_kernel<uint8_t, true><<<grid, kGenThreads, p->gen_smem, s>>>(
            (const uint8_t *)in, pitch, p->nsamp_in, p->nchans, goffs, gbase, gspan, p->ndm,
            p->nsamp_out, out, p->d_partials, p->gen_chunk, p->gen_stride);
        break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch generic_kernel");
    p->n_partials = np;
    p->stats_out = out;
    return DD_OK;
}

int stats_from_out(dd_plan *p, const void *out, cudaStream_t s)
{
    const int64_t total = (int64_t)p->ndm * p->nsamp_out;
    const int64_t per = (int64_t)kStatThreads * kStatPer;
    const int64_t nb = (total + per - 1) / per;
    if (nb > INT32_MAX) return set_error(DD_ERR_ARG, "buffer too large for the stats kernel");
    int rc = ensure_partials_public(p, nb);
    if (rc) return rc;
    if (p->dtype == DD_U8)
        stats_kernel<true><<<(unsigned)nb, kStatThreads, 0, s>>>(out, total, p->d_partials);
    else
        stats_kernel<false><<<(unsigned)nb, kStatThreads, 0, s>>>(out, total, p->d_partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch stats_kernel");
    p->n_partials = nb;
    p->stats_out = out;
    return DD_OK;
}

int search_launch(dd_plan *p, const void *out, cudaStream_t s)
{
    const bool isint = p->dtype == DD_U8;
    // widths are stored original-order in [0,nw) of d_wsorted's tail region
    const int32_t *w_orig = p->d_wsorted + 2 * p->nwidths;
    if (isint)
        finalize_kernel<true><<<1, kFinThreads, 0, s>>>(p->d_partials, p->n_partials, w_orig,
                                                        p->nwidths, p->sigma_k, p->d_params);
    else
        finalize_kernel<false><<<1, kFinThreads, 0, s>>>(p->d_partials, p->n_partials, w_orig,
                                                         p->nwidths, p->sigma_k, p->d_params);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch finalize_kernel");
    const RowParams *rp = nullptr;
    if (p->row_stats && p->d_rowprm) {
        if (isint)
            row_stats_kernel<true><<<(unsigned)p->ndm, kRowThreads, 0, s>>>(out, p->nsamp_out, w_orig, p->nwidths,
                                                                           p->sigma_k, p->d_rowprm);
        else
            row_stats_kernel<false><<<(unsigned)p->ndm, kRowThreads, 0, s>>>(out, p->nsamp_out, w_orig, p->nwidths,
                                                                            p->sigma_k, p->d_rowprm);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "launch row_stats_kernel");
        rp = p->d_rowprm;
    }
    e = cudaMemsetAsync(p->d_count, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "memset count");
    int wmax = 0;
    for (int w : p->widths) wmax = std::max(wmax, w);
    const int64_t ntile = (p->nsamp_out + kSearchTile - 1) / kSearchTile;
    dim3 grid((unsigned)ntile, (unsigned)p->ndm);
    const size_t smem = (size_t)(spad(kSearchTile + wmax - 1) + 1) * 4;
    const int K = pow2_widths(p);
    if (K) {
        if (isint) launch_search_pow2_k<true>(K, grid, s, out, p);
        else launch_search_pow2_k<false>(K, grid, s, out, p);
    } else if (isint)
        search_kernel<true><<<grid, kSearchThreads, smem, s>>>(out, p->nsamp_out, p->d_wsorted, p->nwidths,
                                                               wmax, p->d_params, rp, p->d_cands, p->cand_cap,
                                                               p->d_count);
    else
        search_kernel<false><<<grid, kSearchThreads, smem, s>>>(out, p->nsamp_out, p->d_wsorted, p->nwidths,
                                                                wmax, p->d_params, rp, p->d_cands, p->cand_cap,
                                                                p->d_count);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch search_kernel");
    cand_snr_kernel<<<64, 256, 0, s>>>(p->d_cands, p->d_count, p->cand_cap, w_orig, p->d_params, rp);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch cand_snr_kernel");
    return DD_OK;
}

}  // namespace dd
