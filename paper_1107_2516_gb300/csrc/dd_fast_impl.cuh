// Kernel 2: register-blocked brute-force de-dispersion (Section 3.1),
//   out[dm][t] = sum_c in[c][t + d(c,dm)],
// templated on the thread tile (TR samples x 4 DM trials) and the number of
// warps per block (NW).  Each configuration is instantiated in its own
// translation unit (dd_fast_t*.cu); the host side (dd_fast.cu) builds the
// per-plan tables and picks a configuration (autotuner).
//
// Block = NW warps = 4*NW DM trials x 32*TR samples.  Warp w owns DM trials
// 4w..4w+3 of the block; lane l owns samples TR*l .. TR*l+TR-1 of the tile.
//
// For each channel the block stages, with one TMA bulk copy per channel, the
// input span covering all DM trials of the block into shared memory.  A
// warp's four delays at channel c are d_j = b + j*A + e_j with e_j in [0, j]
// for uniformly spaced DM trials (A = floor of the per-step delay increment),
// so a thread loads ONE window of TR + 3A + 6 samples and adds it, at four
// warp-uniform offsets, into its four DM rows: one shared load feeds up to
// ~2.5 adds instead of one.  The uniform offset is resolved by a warp-uniform
// switch over statically unrolled add sequences (registers cannot be indexed
// dynamically); the step A selects one of kAMax+1 specialised channel bodies.
// Channel/warp pairs that do not fit the pattern use a per-DM window.
//
// The epilogue transposes the register tile through shared memory for
// coalesced stores and emits per-block partial statistics (Section 3).
#pragma once

#include "dd_device.cuh"
#include "dd_internal.h"

namespace dd {

constexpr int kDR = 4;          // DM trials per thread
constexpr int kAMax = 12;       // largest specialised step
constexpr int kGeneric = 255;   // descriptor step value of the fallback path
constexpr int kStages = 3;      // shared-memory stages

struct FastLaunch {
    const void *in;
    int64_t pitch, nsamp_in_al;
    int nchans, ndm;
    int64_t nout;
    const uint32_t *desc;
    const int32_t *base, *goff;
    int rs, ch, bar_off, nblk;
    int64_t ntile;
    int dgroup;
    void *out, *partials;
    int *err;
    size_t smem;
    int dtype;                   // dd_dtype of `in` (batched launches)
};

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t gtimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait: gives up after limit_ns (default ~2 s), records
// DD_ERR_TIMEOUT, returns false.
constexpr uint64_t kWaitLimitNs = 2000000000ull;
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err,
                                          uint64_t limit_ns = kWaitLimitNs)
{
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    while (!mbar_test(bar, parity)) {
        if (gtimer() - t0 > limit_ns) {
            atomicExch(err, DD_ERR_TIMEOUT);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// L2 policy that keeps lines in the cache ahead of normal ones (input rows
// that other blocks of the same time tile stage again soon)
__device__ __forceinline__ uint64_t l2_evict_last()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// bulk_g2s with an L2 cache policy for the source lines
__device__ __forceinline__ void bulk_g2s_hint(void *dst, const void *src, uint32_t bytes, uint64_t *bar, uint64_t pol)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
                 : "memory");
}

// ------------------------------------------------------------- window loads
template <typename Tin> struct Win;

template <> struct Win<float> {
    // N elements (multiple of 4) from a 16-B aligned shared address
    template <int N> static __device__ __forceinline__ void load(float (&w)[N], const float *p)
    {
#pragma unroll
        for (int k = 0; k < N / 4; ++k) {
            const float4 v = reinterpret_cast<const float4 *>(p)[k];
            w[4 * k] = v.x; w[4 * k + 1] = v.y; w[4 * k + 2] = v.z; w[4 * k + 3] = v.w;
        }
    }
};

template <> struct Win<__half> {
    template <int N> static __device__ __forceinline__ void load(float (&w)[N], const __half *p)
    {
#pragma unroll
        for (int k = 0; k < N / 4; ++k) {
            const uint2 v = reinterpret_cast<const uint2 *>(p)[k];
            const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&v.x));
            const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&v.y));
            w[4 * k] = a.x; w[4 * k + 1] = a.y; w[4 * k + 2] = b.x; w[4 * k + 3] = b.y;
        }
    }
};

template <> struct Win<uint8_t> {
    template <int N> static __device__ __forceinline__ void load(float (&w)[N], const uint8_t *p)
    {
#pragma unroll
        for (int k = 0; k < N / 4; ++k) {
            const uint32_t v = reinterpret_cast<const uint32_t *>(p)[k];
            w[4 * k] = (float)(v & 0xffu);
            w[4 * k + 1] = (float)((v >> 8) & 0xffu);
            w[4 * k + 2] = (float)((v >> 16) & 0xffu);
            w[4 * k + 3] = (float)(v >> 24);
        }
    }
};

// ------------------------------------------------------------- add sequences
template <int TR, int OFF, int N>
__device__ __forceinline__ void add_row(float (&a)[TR], const float (&w)[N])
{
    static_assert(OFF + TR <= N, "window too short");
#pragma unroll
    for (int i = 0; i < TR; ++i) a[i] += w[OFF + i];
}

// DM j of the warp: offset j*A + q, q in [0, j+3] (warp-uniform).  Four
// switch cases plus a short if-chain: a flat switch over all j+4 cases makes
// the register allocator keep extra live values and spill.
template <int TR, int J, int A, int N>
__device__ __forceinline__ void add_dm(float (&a)[TR], const float (&w)[N], int q)
{
    constexpr int B = J * A;
    switch (q) {
    case 0: add_row<TR, B + 0>(a, w); break;
    case 1: add_row<TR, B + 1>(a, w); break;
    case 2: add_row<TR, B + 2>(a, w); break;
    case 3: add_row<TR, B + 3>(a, w); break;
    default:
        if constexpr (J >= 1) { if (q == 4) { add_row<TR, B + 4>(a, w); break; } }
        if constexpr (J >= 2) { if (q == 5) { add_row<TR, B + 5>(a, w); break; } }
        if constexpr (J >= 3) { if (q == 6) { add_row<TR, B + 6>(a, w); break; } }
        break;
    }
}

// Window length (elements, multiple of 4) of the step-A body.
__host__ __device__ constexpr int win_len(int TR, int A) { return ((kDR - 1) * A + (kDR - 1) + 3 + TR + 3) / 4 * 4; }

template <typename Tin, int TR, int A>
__device__ __forceinline__ void chan_pattern(float (&acc)[kDR][TR], const Tin *row, uint32_t desc)
{
    constexpr int N = win_len(TR, A);
    float w[N];
    Win<Tin>::template load<N>(w, row);
    add_dm<TR, 0, A>(acc[0], w, (int)(desc & 7u));
    add_dm<TR, 1, A>(acc[1], w, (int)((desc >> 3) & 7u));
    add_dm<TR, 2, A>(acc[2], w, (int)((desc >> 6) & 7u));
    add_dm<TR, 3, A>(acc[3], w, (int)((desc >> 9) & 7u));
}

// Fallback for channel/warp pairs off the pattern: one aligned window per DM.
template <typename Tin, int TR>
__device__ __forceinline__ void chan_generic(float (&acc)[kDR][TR], const Tin *row_base, int lane,
                                             const int32_t *__restrict__ goff)
{
#pragma unroll
    for (int j = 0; j < kDR; ++j) {
        const int o = __ldg(goff + j) + TR * lane;
        const Tin *p = row_base + (o & ~3);
        float w[TR + 4];
        Win<Tin>::template load<TR + 4>(w, p);
        switch (o & 3) {
        case 0: add_row<TR, 0>(acc[j], w); break;
        case 1: add_row<TR, 1>(acc[j], w); break;
        case 2: add_row<TR, 2>(acc[j], w); break;
        default: add_row<TR, 3>(acc[j], w); break;
        }
    }
}

template <typename Tin, int TR>
__device__ __forceinline__ void chan_dispatch(float (&acc)[kDR][TR], const Tin *row_base, int lane,
                                              uint32_t desc, const int32_t *__restrict__ goff)
{
    const Tin *row = row_base + (int)(desc >> 20) * 4 + TR * lane;
    switch ((int)((desc >> 12) & 0xffu)) {
    case 0: chan_pattern<Tin, TR, 0>(acc, row, desc); break;
    case 1: chan_pattern<Tin, TR, 1>(acc, row, desc); break;
    case 2: chan_pattern<Tin, TR, 2>(acc, row, desc); break;
    case 3: chan_pattern<Tin, TR, 3>(acc, row, desc); break;
    case 4: chan_pattern<Tin, TR, 4>(acc, row, desc); break;
    case 5: chan_pattern<Tin, TR, 5>(acc, row, desc); break;
    case 6: chan_pattern<Tin, TR, 6>(acc, row, desc); break;
    case 7: chan_pattern<Tin, TR, 7>(acc, row, desc); break;
    case 8: chan_pattern<Tin, TR, 8>(acc, row, desc); break;
    case 9: chan_pattern<Tin, TR, 9>(acc, row, desc); break;
    case 10: chan_pattern<Tin, TR, 10>(acc, row, desc); break;
    case 11: chan_pattern<Tin, TR, 11>(acc, row, desc); break;
    case 12: chan_pattern<Tin, TR, 12>(acc, row, desc); break;
    default: chan_generic<Tin, TR>(acc, row_base, lane, goff); break;
    }
}

// ------------------------------------------------------------------- kernel
// One work item: DM block `blk` (4*NW trials) x the time tile starting at t0
// of the plan described by `a`.  `gstage` is the block's running stage count:
// the mbarrier ring persists across the items a persistent block processes,
// so stage s of this item uses buffer (gstage+s) % kStages and the parity of
// (gstage+s) / kStages.  Returns false if a bounded wait gave up.
template <typename Tin, bool kInt, int TR, int NW>
__device__ __forceinline__ bool process_tile(const FastLaunch &a, int blk, int64_t t0, int64_t lin,
                                             unsigned char *smem, uint64_t *bar, uint32_t &gstage)
{
    static_assert(TR % 8 == 4, "TR must be 4 x odd: conflict-free 16-byte window loads");
    constexpr int kTile = 32 * TR, kDmBlk = kDR * NW;
    const Tin *__restrict__ in = static_cast<const Tin *>(a.in);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nchans = a.nchans, rs = a.rs, ch = a.ch;
    const int dm0 = blk * kDmBlk;

    // layout: [kStages][ch][rs] Tin rows | [kStages][ch][NW] desc | ... | mbar
    // (the epilogue reuses the start of shared memory for the output transpose)
    const size_t stage_elems = (size_t)ch * rs;
    Tin *rows = reinterpret_cast<Tin *>(smem);
    uint32_t *sdesc = reinterpret_cast<uint32_t *>(smem + kStages * stage_elems * sizeof(Tin));

    const uint32_t *bdesc = a.desc + (size_t)blk * nchans * NW;
    const int32_t *bbase = a.base + (size_t)blk * nchans;
    const int32_t *bgoff = a.goff + (size_t)blk * nchans * NW * kDR;
    const int nst = (nchans + ch - 1) / ch;
    const uint32_t g0 = gstage;

    // bytes of one row copy: clamped at the (aligned) end of the input row
    auto row_bytes = [&](int c, int64_t &g) -> uint32_t {
        g = t0 + bbase[c];
        int64_t n = a.nsamp_in_al - g;
        n = n < 0 ? 0 : (n > rs ? rs : n);
        return (uint32_t)(n * (int64_t)sizeof(Tin));
    };
    auto issue = [&](int s) {
        const int buf = (int)((g0 + s) % kStages);
        const int c0 = s * ch;
        const int cn = min(ch, nchans - c0);
        uint32_t bytes = (uint32_t)(cn * NW * sizeof(uint32_t));
        for (int cc = 0; cc < cn; ++cc) { int64_t g; bytes += row_bytes(c0 + cc, g); }
        mbar_arrive_tx(&bar[buf], bytes);
        bulk_g2s(sdesc + (size_t)buf * ch * NW, bdesc + (size_t)c0 * NW,
                 (uint32_t)(cn * NW * sizeof(uint32_t)), &bar[buf]);
        for (int cc = 0; cc < cn; ++cc) {
            int64_t g;
            const uint32_t nb = row_bytes(c0 + cc, g);
            if (nb)
                bulk_g2s(rows + (size_t)buf * stage_elems + (size_t)cc * rs,
                         in + (size_t)(c0 + cc) * a.pitch + g, nb, &bar[buf]);
        }
    };

    float acc[kDR][TR];
#pragma unroll
    for (int j = 0; j < kDR; ++j)
#pragma unroll
        for (int i = 0; i < TR; ++i) acc[j][i] = 0.f;

    if (tid == 0)
        for (int s = 0; s < kStages - 1 && s < nst; ++s) issue(s);

    bool ok = true;
    for (int s = 0; s < nst; ++s) {
        // buffer of stage s+kStages-1 was last read in stage s-1, which every
        // thread finished before the __syncthreads that ended it
        if (tid == 0 && s + kStages - 1 < nst) issue(s + kStages - 1);
        const uint32_t g = g0 + s;
        const int buf = (int)(g % kStages);
        if (!mbar_wait(&bar[buf], (g / kStages) & 1u, a.err)) { ok = false; break; }
        const int c0 = s * ch;
        const int cn = min(ch, nchans - c0);
        const Tin *srow = rows + (size_t)buf * stage_elems;
        const uint32_t *sd = sdesc + (size_t)buf * ch * NW;
        for (int cc = 0; cc < cn; ++cc)
            chan_dispatch<Tin, TR>(acc, srow + (size_t)cc * rs, lane, sd[cc * NW + warp],
                                   bgoff + ((size_t)(c0 + cc) * NW + warp) * kDR);
        __syncthreads();
    }
    gstage = g0 + nst;
    if (!ok) return false;

    // ---------------------------------------------------------------- epilogue
    const int64_t nout = a.nout;
    const int64_t tb = t0 + (int64_t)TR * lane;
    const int valid_t = (int)max((int64_t)0, min((int64_t)TR, nout - tb));
    float *stile = reinterpret_cast<float *>(smem) + (size_t)warp * kDR * kTile;
#pragma unroll
    for (int j = 0; j < kDR; ++j)
#pragma unroll
        for (int k = 0; k < TR / 4; ++k)
            *reinterpret_cast<float4 *>(stile + j * kTile + TR * lane + 4 * k) =
                make_float4(acc[j][4 * k], acc[j][4 * k + 1], acc[j][4 * k + 2], acc[j][4 * k + 3]);
    const int lim = (int)min((int64_t)kTile, nout - t0);

    if constexpr (kInt) {
        long long n = 0, s = 0;
        unsigned long long q = 0;
#pragma unroll
        for (int j = 0; j < kDR; ++j) {
            const bool dv = dm0 + warp * kDR + j < a.ndm;
#pragma unroll
            for (int i = 0; i < TR; ++i)
                if (dv && i < valid_t) {
                    const long long v = __float2int_rn(acc[j][i]);
                    n++; s += v; q += (unsigned long long)(v * v);
                }
        }
        __syncwarp();
        int32_t *out = reinterpret_cast<int32_t *>(a.out);
        for (int j = 0; j < kDR; ++j) {
            const int dm = dm0 + warp * kDR + j;
            if (dm >= a.ndm) break;
            int32_t *orow = out + (size_t)dm * nout + t0;
            for (int m = lane; m < lim; m += 32) orow[m] = __float2int_rn(stile[j * kTile + m]);
        }
        block_stat_i(n, s, q, reinterpret_cast<StatI *>(a.partials) + lin);
    } else {
        int n = 0;
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < kDR; ++j) {
            const bool dv = dm0 + warp * kDR + j < a.ndm;
#pragma unroll
            for (int i = 0; i < TR; ++i)
                if (dv && i < valid_t) { n++; s += acc[j][i]; }
        }
        const float m = n ? s / (float)n : 0.f;
        float q = 0.f;
#pragma unroll
        for (int j = 0; j < kDR; ++j) {
            const bool dv = dm0 + warp * kDR + j < a.ndm;
#pragma unroll
            for (int i = 0; i < TR; ++i)
                if (dv && i < valid_t) { const float d = acc[j][i] - m; q += d * d; }
        }
        __syncwarp();
        float *out = reinterpret_cast<float *>(a.out);
        for (int j = 0; j < kDR; ++j) {
            const int dm = dm0 + warp * kDR + j;
            if (dm >= a.ndm) break;
            float *orow = out + (size_t)dm * nout + t0;
            for (int m = lane; m < lim; m += 32) orow[m] = stile[j * kTile + m];
        }
        block_stat_f32(n, s, q, reinterpret_cast<StatF *>(a.partials) + lin);
    }
    return true;
}

// Raster: DM blocks in groups of a.dgroup; within a group the time tiles
// advance slowest, so concurrently resident blocks read nearby input spans
// (better L2 reuse than sweeping all DM blocks of a tile at once).
template <int TR>
__device__ __forceinline__ void raster(const FastLaunch &a, int64_t lin, int &blk, int64_t &t0)
{
    const int64_t per_group = (int64_t)a.dgroup * a.ntile;
    const int64_t grp = lin / per_group;
    const int64_t rr = lin - grp * per_group;
    const int gsize = min(a.dgroup, a.nblk - (int)grp * a.dgroup);
    blk = (int)grp * a.dgroup + (int)(rr % gsize);
    t0 = (rr / gsize) * (int64_t)(32 * TR);
}

// One plan: one block per work item, grid = nblk * ntile.
template <typename Tin, bool kInt, int TR, int NW>
__global__ void __launch_bounds__(NW * 32, 1) fast_kernel(FastLaunch a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + a.bar_off);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
        mbar_fence_init();
    }
    __syncthreads();
    int blk;
    int64_t t0;
    raster<TR>(a, blockIdx.x, blk, t0);
    uint32_t gstage = 0;
    process_tile<Tin, kInt, TR, NW>(a, blk, t0, blockIdx.x, smem, bar, gstage);
}

// Batched plans (uneven beams, mixed input types): a persistent grid pulls
// work items (beam, linear tile index) from a device queue ordered heaviest
// first, so beams of different channel counts and lengths share one launch.
struct BatchLaunch {
    const FastLaunch *beams;     // [nbeams], each with its own tables and buffers
    const uint2 *items;          // [nitems] (beam, linear tile index within the beam)
    int nitems;
    int bar_off;
    unsigned int *counter;       // work-queue head, zeroed before the launch
    int *err;
};

template <int TR, int NW>
__global__ void __launch_bounds__(NW * 32, 1) batch_kernel(BatchLaunch b)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_item;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + b.bar_off);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
        mbar_fence_init();
    }
    __syncthreads();
    uint32_t gstage = 0;
    while (true) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(b.counter, 1u);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= b.nitems) break;
        const uint2 w = b.items[it];
        const FastLaunch &a = b.beams[w.x];
        int blk;
        int64_t t0;
        raster<TR>(a, w.y, blk, t0);
        bool ok;
        switch (a.dtype) {
        case DD_F32: ok = process_tile<float, false, TR, NW>(a, blk, t0, w.y, smem, bar, gstage); break;
        case DD_F16: ok = process_tile<__half, false, TR, NW>(a, blk, t0, w.y, smem, bar, gstage); break;
        default: ok = process_tile<uint8_t, true, TR, NW>(a, blk, t0, w.y, smem, bar, gstage); break;
        }
        if (!ok) break;
        // the epilogue's generic-proxy shared accesses must be ordered before
        // the next item's TMA writes into the same bytes
        __syncthreads();
        if (threadIdx.x == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
}

// Launch one configuration for one input type.  Grid: nblk * ntile blocks.
template <int TR, int NW>
cudaError_t fast_launch_cfg(dd_dtype t, const FastLaunch &a, cudaStream_t s)
{
    const unsigned grid = (unsigned)(a.ntile * a.nblk);
    switch (t) {
    case DD_F32: fast_kernel<float, false, TR, NW><<<grid, NW * 32, a.smem, s>>>(a); break;
    case DD_F16: fast_kernel<__half, false, TR, NW><<<grid, NW * 32, a.smem, s>>>(a); break;
    case DD_U8: fast_kernel<uint8_t, true, TR, NW><<<grid, NW * 32, a.smem, s>>>(a); break;
    }
    return cudaGetLastError();
}

template <int TR, int NW>
cudaError_t fast_prepare_cfg(size_t optin)
{
    cudaError_t e = allow_max_dynamic_smem((const void *)fast_kernel<float, false, TR, NW>, optin);
    if (e == cudaSuccess) e = allow_max_dynamic_smem((const void *)fast_kernel<__half, false, TR, NW>, optin);
    if (e == cudaSuccess) e = allow_max_dynamic_smem((const void *)fast_kernel<uint8_t, true, TR, NW>, optin);
    if (e == cudaSuccess) e = allow_max_dynamic_smem((const void *)batch_kernel<TR, NW>, optin);
    return e;
}

template <int TR, int NW>
cudaError_t batch_launch_cfg(const BatchLaunch &b, int grid, size_t smem, cudaStream_t s)
{
    batch_kernel<TR, NW><<<grid, NW * 32, smem, s>>>(b);
    return cudaGetLastError();
}

// Configurations compiled into the library: {samples per thread, warps}.
struct FastShape { int tr, nw; };
constexpr int kNumFastCfg = 3;
constexpr FastShape kFastCfg[kNumFastCfg] = {{36, 8}, {20, 12}, {28, 8}};

cudaError_t fast_launch_t36w8(dd_dtype t, const FastLaunch &a, cudaStream_t s);
cudaError_t fast_launch_t20w12(dd_dtype t, const FastLaunch &a, cudaStream_t s);
cudaError_t fast_launch_t28w8(dd_dtype t, const FastLaunch &a, cudaStream_t s);
cudaError_t fast_prepare_t36w8(size_t optin);
cudaError_t fast_prepare_t20w12(size_t optin);
cudaError_t fast_prepare_t28w8(size_t optin);
cudaError_t batch_launch_t36w8(const BatchLaunch &b, int grid, size_t smem, cudaStream_t s);
cudaError_t batch_launch_t20w12(const BatchLaunch &b, int grid, size_t smem, cudaStream_t s);
cudaError_t batch_launch_t28w8(const BatchLaunch &b, int grid, size_t smem, cudaStream_t s);

}  // namespace dd
