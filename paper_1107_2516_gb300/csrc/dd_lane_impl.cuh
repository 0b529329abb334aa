// Kernel 3: lane-interleaved brute-force de-dispersion (Section 3.1),
//   out[dm][t] = sum_c in[c][t + d(c,dm)].
//
// Block = NW warps sharing one time tile of 32*TI samples; lane l owns
// samples t0 + l + 32*i (i < TI) and each warp owns DR DM trials, so a thread
// accumulates DR x TI outputs.  Per channel the block stages (one TMA bulk
// copy) the input span of all its DM trials; for each DM trial a warp adds
// row[o + l + 32 i] with o the trial's warp-uniform offset: 32 consecutive
// words per load, conflict-free at any alignment, no branches.  Every add
// costs one shared-memory word, so the kernel is bounded by shared-memory
// bandwidth (32 words/clk/SM = 1/4 of the FP32 add rate); it trades kernel
// 2's register reuse for straight-line code and high occupancy.
#pragma once

#include "dd_fast_impl.cuh"

namespace dd {

struct LaneLaunch {
    const void *in;
    int64_t pitch, nsamp_in_al;
    int nchans, ndm;
    int64_t nout;
    const int32_t *offs;   // [nblk][nchans][NW*DR] element offsets within the staged row
    const int32_t *base;   // [nblk][nchans] row start relative to the tile start (aligned)
    int rs, ch, bar_off, nblk;
    int64_t ntile;
    int dgroup;
    void *out, *partials;
    int *err;
    size_t smem;
    int dtype;             // dd_dtype of `in` (batched launches)
    int64_t t_base;        // lane_kernel: first output sample of the launch's tile range
    int kind;              // mixed batch: 0 = this kernel 3 launch, 1 = the beam's kernel 5 launch
};

template <typename Tin> __device__ __forceinline__ float lane_ld(const Tin *p);
template <> __device__ __forceinline__ float lane_ld<float>(const float *p) { return *p; }
template <> __device__ __forceinline__ float lane_ld<__half>(const __half *p) { return __half2float(*p); }
template <> __device__ __forceinline__ float lane_ld<uint8_t>(const uint8_t *p) { return (float)*p; }

// DM block / time tile of linear block index `lin` (DM blocks in groups, time
// tiles slowest within a group, as kernel 2).
template <int TI>
__device__ __forceinline__ void lane_raster(const LaneLaunch &a, int64_t lin, int &blk, int64_t &t0)
{
    const int64_t per_group = (int64_t)a.dgroup * a.ntile;
    const int64_t grp = lin / per_group;
    const int64_t rr = lin - grp * per_group;
    const int gsize = min(a.dgroup, a.nblk - (int)grp * a.dgroup);
    blk = (int)grp * a.dgroup + (int)(rr % gsize);
    t0 = (rr / gsize) * (32 * TI);
}

// One work item: DM block `blk` x the time tile at t0 of the plan in `a`;
// partials record `lin`.  `gstage` is the block's running stage count (the
// mbarrier ring persists across the items of a persistent block: stage s
// of this item uses buffer (gstage+s) % kStages, parity (gstage+s) / kStages).
// Returns false if a bounded wait gave up.
// The tile addresses the block's dynamic shared memory through the extern
// symbol (not a pointer argument), so that its loads and stores stay
// shared-space instructions in the out-of-line copies the persistent kernels
// call.
template <typename Tin, bool kInt, int TI, int DR, int NW>
__device__ __forceinline__ bool lane_tile(const LaneLaunch &a, int blk, int64_t t0, int64_t lin,
                                          uint64_t *bar, uint32_t &gstage)
{
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int kDmBlk = DR * NW;
    const Tin *__restrict__ in = static_cast<const Tin *>(a.in);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nchans = a.nchans, rs = a.rs, ch = a.ch;
    const int dm0 = blk * kDmBlk;

    // layout: [kStages][ch][rs] Tin rows | [kStages][ch][kDmBlk] int32 offsets | mbar at bar_off
    const size_t stage_elems = (size_t)ch * rs;
    Tin *rows = reinterpret_cast<Tin *>(smem);
    int32_t *soffs = reinterpret_cast<int32_t *>(smem + kStages * stage_elems * sizeof(Tin));
    const int32_t *boffs = a.offs + (size_t)blk * nchans * kDmBlk;
    const int32_t *bbase = a.base + (size_t)blk * nchans;
    const int nst = (nchans + ch - 1) / ch;
    const uint32_t g0 = gstage;

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
        uint32_t bytes = (uint32_t)(cn * kDmBlk * sizeof(int32_t));
        for (int cc = 0; cc < cn; ++cc) { int64_t g; bytes += row_bytes(c0 + cc, g); }
        mbar_arrive_tx(&bar[buf], bytes);
        bulk_g2s(soffs + (size_t)buf * ch * kDmBlk, boffs + (size_t)c0 * kDmBlk,
                 (uint32_t)(cn * kDmBlk * sizeof(int32_t)), &bar[buf]);
        for (int cc = 0; cc < cn; ++cc) {
            int64_t g;
            const uint32_t nb = row_bytes(c0 + cc, g);
            if (nb)
                bulk_g2s(rows + (size_t)buf * stage_elems + (size_t)cc * rs,
                         in + (size_t)(c0 + cc) * a.pitch + g, nb, &bar[buf]);
        }
    };

    float acc[DR][TI];
#pragma unroll
    for (int j = 0; j < DR; ++j)
#pragma unroll
        for (int i = 0; i < TI; ++i) acc[j][i] = 0.f;

    if (tid == 0)
        for (int s = 0; s < kStages - 1 && s < nst; ++s) issue(s);

    bool ok = true;
    for (int s = 0; s < nst; ++s) {
        if (tid == 0 && s + kStages - 1 < nst) issue(s + kStages - 1);
        const uint32_t g = g0 + s;
        const int buf = (int)(g % kStages);
        if (!mbar_wait(&bar[buf], (g / kStages) & 1u, a.err)) { ok = false; break; }
        const int cn = min(ch, nchans - s * ch);
        const Tin *srow = rows + (size_t)buf * stage_elems + lane;
        const int32_t *so = soffs + (size_t)buf * ch * kDmBlk + warp * DR;
        for (int cc = 0; cc < cn; ++cc) {
            const Tin *r = srow + (size_t)cc * rs;
            // the warp's DR offsets: uniform 16-byte loads, one shared-memory
            // wavefront per 4 offsets (the data path is the kernel's bound)
            int o[DR];
            static_assert(DR % 4 == 0, "offsets are loaded 4 at a time");
#pragma unroll
            for (int j = 0; j < DR; j += 4) {
                const int4 v = *reinterpret_cast<const int4 *>(so + cc * kDmBlk + j);
                o[j] = v.x; o[j + 1] = v.y; o[j + 2] = v.z; o[j + 3] = v.w;
            }
#pragma unroll
            for (int j = 0; j < DR; ++j) {
                const Tin *p = r + o[j];
#pragma unroll
                for (int i = 0; i < TI; ++i) acc[j][i] += lane_ld<Tin>(p + 32 * i);
            }
        }
        __syncthreads();
    }
    gstage = g0 + nst;
    if (!ok) return false;

    // epilogue: lanes hold consecutive samples, so stores are coalesced directly
    const int64_t nout = a.nout;
    if constexpr (kInt) {
        long long n = 0, s = 0;
        unsigned long long q = 0;
        int32_t *out = reinterpret_cast<int32_t *>(a.out);
#pragma unroll
        for (int j = 0; j < DR; ++j) {
            const int dm = dm0 + warp * DR + j;
#pragma unroll
            for (int i = 0; i < TI; ++i) {
                const int64_t t = t0 + lane + 32 * i;
                if (dm < a.ndm && t < nout) {
                    const long long v = __float2int_rn(acc[j][i]);
                    out[(size_t)dm * nout + t] = (int32_t)v;
                    n++; s += v; q += (unsigned long long)(v * v);
                }
            }
        }
        block_stat_i(n, s, q, reinterpret_cast<StatI *>(a.partials) + lin);
    } else {
        int n = 0;
        float s = 0.f;
        float *out = reinterpret_cast<float *>(a.out);
#pragma unroll
        for (int j = 0; j < DR; ++j) {
            const int dm = dm0 + warp * DR + j;
#pragma unroll
            for (int i = 0; i < TI; ++i) {
                const int64_t t = t0 + lane + 32 * i;
                if (dm < a.ndm && t < nout) {
                    out[(size_t)dm * nout + t] = acc[j][i];
                    n++; s += acc[j][i];
                }
            }
        }
        const float m = n ? s / (float)n : 0.f;
        float q = 0.f;
#pragma unroll
        for (int j = 0; j < DR; ++j) {
            const int dm = dm0 + warp * DR + j;
#pragma unroll
            for (int i = 0; i < TI; ++i) {
                const int64_t t = t0 + lane + 32 * i;
                if (dm < a.ndm && t < nout) { const float d = acc[j][i] - m; q += d * d; }
            }
        }
        block_stat_f32(n, s, q, reinterpret_cast<StatF *>(a.partials) + lin);
    }
    return true;
}

// One plan: one block per work item, grid = nblk * ntile.
template <typename Tin, bool kInt, int TI, int DR, int NW, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB) lane_kernel(LaneLaunch a)
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
    lane_raster<TI>(a, blockIdx.x, blk, t0);
    t0 += a.t_base;
    uint32_t gstage = 0;
    lane_tile<Tin, kInt, TI, DR, NW>(a, blk, t0, blockIdx.x, bar, gstage);
}

// lane_tile as an out-of-line function: the persistent kernel calls one per
// input type, each compiled with the full register budget.
template <typename Tin, bool kInt, int TI, int DR, int NW>
__device__ __noinline__ bool lane_tile_call(const LaneLaunch &a, int blk, int64_t t0, int64_t lin,
                                            uint64_t *bar, uint32_t &gstage)
{
    return lane_tile<Tin, kInt, TI, DR, NW>(a, blk, t0, lin, bar, gstage);
}

// Batched plans with kernel 3: a persistent grid (MINB blocks per SM) pulls
// work items (beam, linear tile index) from a device queue, heaviest beams
// first; each beam brings its own tables, buffers and input type.
struct ShareLaunch;

struct LaneBatchLaunch {
    const LaneLaunch *beams;
    const uint2 *items;
    int nitems;
    int bar_off;
    unsigned int *counter;
    const ShareLaunch *sbeams;   // mixed batch: each kind-1 beam's kernel 5 launch
};

template <int TI, int DR, int NW, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB) lane_batch_kernel(LaneBatchLaunch b)
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
        const LaneLaunch &a = b.beams[w.x];
        int blk;
        int64_t t0;
        lane_raster<TI>(a, w.y, blk, t0);
        bool ok;
        switch (a.dtype) {
        case DD_F32: ok = lane_tile_call<float, false, TI, DR, NW>(a, blk, t0, w.y, bar, gstage); break;
        case DD_F16: ok = lane_tile_call<__half, false, TI, DR, NW>(a, blk, t0, w.y, bar, gstage); break;
        default: ok = lane_tile_call<uint8_t, true, TI, DR, NW>(a, blk, t0, w.y, bar, gstage); break;
        }
        if (!ok) break;
        __syncthreads();
        if (threadIdx.x == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
}

template <int TI, int DR, int NW, int MINB>
cudaError_t lane_launch_cfg(dd_dtype t, const LaneLaunch &a, cudaStream_t s)
{
    const unsigned grid = (unsigned)(a.ntile * a.nblk);
    switch (t) {
    case DD_F32: lane_kernel<float, false, TI, DR, NW, MINB><<<grid, NW * 32, a.smem, s>>>(a); break;
    case DD_F16: lane_kernel<__half, false, TI, DR, NW, MINB><<<grid, NW * 32, a.smem, s>>>(a); break;
    case DD_U8: lane_kernel<uint8_t, true, TI, DR, NW, MINB><<<grid, NW * 32, a.smem, s>>>(a); break;
    }
    return cudaGetLastError();
}

template <int TI, int DR, int NW, int MINB>
cudaError_t lane_prepare_cfg(size_t optin)
{
    cudaError_t e = allow_max_dynamic_smem((const void *)lane_kernel<float, false, TI, DR, NW, MINB>, optin);
    if (e == cudaSuccess)
        e = allow_max_dynamic_smem((const void *)lane_kernel<__half, false, TI, DR, NW, MINB>, optin);
    if (e == cudaSuccess)
        e = allow_max_dynamic_smem((const void *)lane_kernel<uint8_t, true, TI, DR, NW, MINB>, optin);
    if (e == cudaSuccess)
        e = allow_max_dynamic_smem((const void *)lane_batch_kernel<TI, DR, NW, MINB>, optin);
    return e;
}

// Persistent launch: grid = MINB blocks per SM (the occupancy the shared
// memory budget of the configuration allows).
template <int TI, int DR, int NW, int MINB>
cudaError_t lane_batch_launch_cfg(const LaneBatchLaunch &b, int sms, size_t smem, cudaStream_t s)
{
    lane_batch_kernel<TI, DR, NW, MINB><<<sms * MINB, NW * 32, smem, s>>>(b);
    return cudaGetLastError();
}

// Configurations compiled into the library: {samples per lane, DM trials per
// warp, warps per block, resident blocks per SM the register budget targets}.
struct LaneShape { int ti, dr, nw, minb; };
constexpr int kNumLaneCfg = 4;
constexpr LaneShape kLaneCfg[kNumLaneCfg] = {{16, 4, 8, 2}, {16, 8, 8, 1}, {16, 8, 4, 3}, {8, 16, 4, 3}};

cudaError_t lane_launch_c0(dd_dtype t, const LaneLaunch &a, cudaStream_t s);
cudaError_t lane_launch_c1(dd_dtype t, const LaneLaunch &a, cudaStream_t s);
cudaError_t lane_launch_c2(dd_dtype t, const LaneLaunch &a, cudaStream_t s);
cudaError_t lane_launch_c3(dd_dtype t, const LaneLaunch &a, cudaStream_t s);
cudaError_t lane_prepare_c0(size_t optin);
cudaError_t lane_prepare_c1(size_t optin);
cudaError_t lane_prepare_c2(size_t optin);
cudaError_t lane_prepare_c3(size_t optin);
cudaError_t lane_batch_launch_c0(const LaneBatchLaunch &b, int sms, size_t smem, cudaStream_t s);
cudaError_t lane_batch_launch_c1(const LaneBatchLaunch &b, int sms, size_t smem, cudaStream_t s);
cudaError_t lane_batch_launch_c2(const LaneBatchLaunch &b, int sms, size_t smem, cudaStream_t s);
cudaError_t lane_batch_launch_c3(const LaneBatchLaunch &b, int sms, size_t smem, cudaStream_t s);

}  // namespace dd
