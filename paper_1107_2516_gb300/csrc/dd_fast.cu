// Kernel 2: register-blocked brute-force de-dispersion (Section 3.1),
//   out[dm][t] = sum_c in[c][t + d(c,dm)].
//
// Block = 8 warps = 32 DM trials x 1152 samples.  Warp w owns DM trials
// 4w..4w+3 of the block; lane l owns samples 36l..36l+35 of the tile, so a
// thread accumulates a 4 x 36 register tile.
//
// For each channel the block stages, with one TMA bulk copy per channel, the
// input span covering all 32 DM trials into shared memory.  A warp's four
// delays at channel c are d_j = b + j*A + e_j with e_j in [0, j] for uniformly
// spaced DM trials (A = floor of the per-step delay increment), so a thread
// loads ONE window of 36 + 3A + 6 samples and adds it, at four warp-uniform
// offsets, into its four DM rows: one shared load feeds up to ~2.5 adds
// instead of one.  The uniform offset is resolved by a warp-uniform switch
// over a few statically unrolled add sequences (registers cannot be indexed
// dynamically); the step A selects one of A_MAX+1 specialised channel bodies.
// Channel/warp pairs that do not fit the pattern fall back to a per-DM window.
//
// The epilogue transposes the register tile through shared memory for
// coalesced stores and emits per-block partial statistics (Section 3).
#include "dd_internal.h"
#include "dd_device.cuh"

#include <algorithm>
#include <climits>
#include <cstring>

namespace dd {

constexpr int kTR = 36;                    // samples per thread (4 * odd: conflict-free 16-B loads)
constexpr int kDR = 4;                     // DM trials per thread
constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kTile = 32 * kTR;            // 1152 samples per block
constexpr int kDmBlk = kWarps * kDR;       // 32 DM trials per block
constexpr int kAMax = 12;                  // largest specialised step
constexpr int kGeneric = 255;
constexpr int kStages = 3;

struct FastPlan {
    int nblk = 0;                // DM blocks
    int rs = 0;                  // shared row stride in elements (multiple of 16)
    int ch = 0;                  // channels per stage
    size_t smem = 0;
    uint32_t *d_desc = nullptr;  // [nblk][nchans][kWarps]
    int32_t *d_base = nullptr;   // [nblk][nchans] smem-row start (aligned, relative to t0)
    int32_t *d_goff = nullptr;   // [nblk][nchans][kWarps][kDR] generic offsets (elements)
    int *d_err = nullptr;
    int al = 4;                  // row alignment in elements (16 bytes)
    int bar_off = 0;             // byte offset of the stage mbarriers in shared memory
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

// Bounded wait: gives up after ~2 s, records DD_ERR_TIMEOUT, returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err)
{
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    while (!mbar_test(bar, parity)) {
        if (gtimer() - t0 > 2000000000ull) {
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

// ------------------------------------------------------------- window loads
template <typename Tin> struct Win;

template <> struct Win<float> {
    // n elements (multiple of 4) from 16-B aligned shared address
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
template <int OFF, int N>
__device__ __forceinline__ void add36(float (&a)[kTR], const float (&w)[N])
{
    static_assert(OFF + kTR <= N, "window too short");
#pragma unroll
    for (int i = 0; i < kTR; ++i) a[i] += w[OFF + i];
}

// DM j of the warp: offset j*A + q, q in [0, j+3] (warp-uniform).
template <int J, int A, int N>
__device__ __forceinline__ void add_dm(float (&a)[kTR], const float (&w)[N], int q)
{
    constexpr int B = J * A;
    switch (q) {
    case 0: add36<B + 0>(a, w); break;
    case 1: add36<B + 1>(a, w); break;
    case 2: add36<B + 2>(a, w); break;
    case 3: add36<B + 3>(a, w); break;
    default:
        if constexpr (J >= 1) { if (q == 4) { add36<B + 4>(a, w); break; } }
        if constexpr (J >= 2) { if (q == 5) { add36<B + 5>(a, w); break; } }
        if constexpr (J >= 3) { if (q == 6) { add36<B + 6>(a, w); break; } }
        break;
    }
}

template <int A> struct WLen { static constexpr int v = ((kDR - 1) * A + (kDR - 1) + 3 + kTR + 3) / 4 * 4; };

template <typename Tin, int A>
__device__ __forceinline__ void chan_pattern(float (&acc)[kDR][kTR], const Tin *row, uint32_t desc)
{
    constexpr int N = WLen<A>::v;
    float w[N];
    Win<Tin>::template load<N>(w, row);
    add_dm<0, A>(acc[0], w, (int)(desc & 7u));
    add_dm<1, A>(acc[1], w, (int)((desc >> 3) & 7u));
    add_dm<2, A>(acc[2], w, (int)((desc >> 6) & 7u));
    add_dm<3, A>(acc[3], w, (int)((desc >> 9) & 7u));
}

// Fallback for channel/warp pairs off the pattern: one aligned window per DM.
template <typename Tin>
__device__ __forceinline__ void chan_generic(float (&acc)[kDR][kTR], const Tin *row_base, int lane,
                                             const int32_t *__restrict__ goff)
{
#pragma unroll
    for (int j = 0; j < kDR; ++j) {
        const int o = __ldg(goff + j) + kTR * lane;
        const Tin *p = row_base + (o & ~3);
        float w[kTR + 4];
        Win<Tin>::template load<kTR + 4>(w, p);
        switch (o & 3) {
        case 0: add36<0>(acc[j], w); break;
        case 1: add36<1>(acc[j], w); break;
        case 2: add36<2>(acc[j], w); break;
        default: add36<3>(acc[j], w); break;
        }
    }
}

template <typename Tin>
__device__ __forceinline__ void chan_dispatch(float (&acc)[kDR][kTR], const Tin *row_base, int lane,
                                              uint32_t desc, const int32_t *__restrict__ goff)
{
    const int A = (int)((desc >> 12) & 0xffu);
    const Tin *row = row_base + (int)(desc >> 20) * 4 + kTR * lane;
    switch (A) {
    case 0: chan_pattern<Tin, 0>(acc, row, desc); break;
    case 1: chan_pattern<Tin, 1>(acc, row, desc); break;
    case 2: chan_pattern<Tin, 2>(acc, row, desc); break;
    case 3: chan_pattern<Tin, 3>(acc, row, desc); break;
    case 4: chan_pattern<Tin, 4>(acc, row, desc); break;
    case 5: chan_pattern<Tin, 5>(acc, row, desc); break;
    case 6: chan_pattern<Tin, 6>(acc, row, desc); break;
    case 7: chan_pattern<Tin, 7>(acc, row, desc); break;
    case 8: chan_pattern<Tin, 8>(acc, row, desc); break;
    case 9: chan_pattern<Tin, 9>(acc, row, desc); break;
    case 10: chan_pattern<Tin, 10>(acc, row, desc); break;
    case 11: chan_pattern<Tin, 11>(acc, row, desc); break;
    case 12: chan_pattern<Tin, 12>(acc, row, desc); break;
    default: chan_generic<Tin>(acc, row_base, lane, goff); break;
    }
}

// ------------------------------------------------------------------- kernel
template <typename Tin, bool kInt>
__global__ void __launch_bounds__(kThreads, 1)
fast_kernel(const Tin *__restrict__ in, int64_t pitch, int64_t nsamp_in_al, int nchans, int ndm,
            int64_t nout, const uint32_t *__restrict__ desc, const int32_t *__restrict__ base,
            const int32_t *__restrict__ goff, int rs, int ch, int bar_off, void *__restrict__ out_,
            void *__restrict__ partials, int *__restrict__ err)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int blk = blockIdx.x;
    const int64_t t0 = (int64_t)blockIdx.y * kTile;
    const int dm0 = blk * kDmBlk;

    // layout: [kStages][ch][rs] Tin rows | [kStages][ch][kWarps] desc | ... | mbar at bar_off
    // (the epilogue reuses [0, bar_off) for the output transpose)
    const size_t stage_elems = (size_t)ch * rs;
    Tin *rows = reinterpret_cast<Tin *>(smem);
    uint32_t *sdesc = reinterpret_cast<uint32_t *>(smem + kStages * stage_elems * sizeof(Tin));
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + bar_off);

    const uint32_t *bdesc = desc + (size_t)blk * nchans * kWarps;
    const int32_t *bbase = base + (size_t)blk * nchans;
    const int32_t *bgoff = goff + (size_t)blk * nchans * kWarps * kDR;
    const int nst = (nchans + ch - 1) / ch;

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
        mbar_fence_init();
    }
    __syncthreads();

    auto issue = [&](int s) {
        const int buf = s % kStages;
        const int c0 = s * ch;
        const int cn = min(ch, nchans - c0);
        // bytes of one row copy: clamped at the (aligned) end of the input row
        auto row_bytes = [&](int c, int64_t &g) -> uint32_t {
            g = t0 + bbase[c];
            int64_t n = nsamp_in_al - g;
            n = n < 0 ? 0 : (n > rs ? rs : n);
            return (uint32_t)(n * (int64_t)sizeof(Tin));
        };
        uint32_t bytes = (uint32_t)(cn * kWarps * sizeof(uint32_t));
        for (int cc = 0; cc < cn; ++cc) { int64_t g; bytes += row_bytes(c0 + cc, g); }
        mbar_arrive_tx(&bar[buf], bytes);
        bulk_g2s(sdesc + (size_t)buf * ch * kWarps, bdesc + (size_t)c0 * kWarps,
                 (uint32_t)(cn * kWarps * sizeof(uint32_t)), &bar[buf]);
        for (int cc = 0; cc < cn; ++cc) {
            int64_t g;
            const uint32_t nb = row_bytes(c0 + cc, g);
            if (nb)
                bulk_g2s(rows + (size_t)buf * stage_elems + (size_t)cc * rs,
                         in + (size_t)(c0 + cc) * pitch + g, nb, &bar[buf]);
        }
    };

    float acc[kDR][kTR];
#pragma unroll
    for (int j = 0; j < kDR; ++j)
#pragma unroll
        for (int i = 0; i < kTR; ++i) acc[j][i] = 0.f;

    if (tid == 0)
        for (int s = 0; s < kStages - 1 && s < nst; ++s) issue(s);

    bool ok = true;
    for (int s = 0; s < nst; ++s) {
        if (tid == 0 && s + kStages - 1 < nst) issue(s + kStages - 1);
        const int buf = s % kStages;
        if (!mbar_wait(&bar[buf], (uint32_t)((s / kStages) & 1), err)) { ok = false; break; }
        const int c0 = s * ch;
        const int cn = min(ch, nchans - c0);
        const Tin *srow = rows + (size_t)buf * stage_elems;
        const uint32_t *sd = sdesc + (size_t)buf * ch * kWarps;
        for (int cc = 0; cc < cn; ++cc) {
            const uint32_t dsc = sd[cc * kWarps + warp];
            chan_dispatch<Tin>(acc, srow + (size_t)cc * rs, lane, dsc,
                               bgoff + ((size_t)(c0 + cc) * kWarps + warp) * kDR);
        }
        __syncthreads();
    }
    if (!ok) return;

    // ---------------------------------------------------------------- epilogue
    const int64_t pidx = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    const int64_t tb = t0 + (int64_t)kTR * lane;
    const int valid_t = (int)max((int64_t)0, min((int64_t)kTR, nout - tb));
    float *stile = reinterpret_cast<float *>(smem) + (size_t)warp * kDR * kTile;
#pragma unroll
    for (int j = 0; j < kDR; ++j)
#pragma unroll
        for (int k = 0; k < kTR / 4; ++k)
            *reinterpret_cast<float4 *>(stile + j * kTile + kTR * lane + 4 * k) =
                make_float4(acc[j][4 * k], acc[j][4 * k + 1], acc[j][4 * k + 2], acc[j][4 * k + 3]);

    if constexpr (kInt) {
        long long n = 0, s = 0;
        unsigned long long q = 0;
#pragma unroll
        for (int j = 0; j < kDR; ++j) {
            const bool dv = dm0 + warp * kDR + j < ndm;
#pragma unroll
            for (int i = 0; i < kTR; ++i)
                if (dv && i < valid_t) {
                    const long long v = __float2int_rn(acc[j][i]);
                    n++; s += v; q += (unsigned long long)(v * v);
                }
        }
        __syncwarp();
        int32_t *out = reinterpret_cast<int32_t *>(out_);
        for (int j = 0; j < kDR; ++j) {
            const int dm = dm0 + warp * kDR + j;
            if (dm >= ndm) break;
            int32_t *orow = out + (size_t)dm * nout + t0;
            const int lim = (int)min((int64_t)kTile, nout - t0);
            for (int m = lane; m < lim; m += 32) orow[m] = __float2int_rn(stile[j * kTile + m]);
        }
        block_stat_i(n, s, q, reinterpret_cast<StatI *>(partials) + pidx);
    } else {
        int n = 0;
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < kDR; ++j) {
            const bool dv = dm0 + warp * kDR + j < ndm;
#pragma unroll
            for (int i = 0; i < kTR; ++i)
                if (dv && i < valid_t) { n++; s += acc[j][i]; }
        }
        const float m = n ? s / (float)n : 0.f;
        float q = 0.f;
#pragma unroll
        for (int j = 0; j < kDR; ++j) {
            const bool dv = dm0 + warp * kDR + j < ndm;
#pragma unroll
            for (int i = 0; i < kTR; ++i)
                if (dv && i < valid_t) { const float d = acc[j][i] - m; q += d * d; }
        }
        __syncwarp();
        float *out = reinterpret_cast<float *>(out_);
        for (int j = 0; j < kDR; ++j) {
            const int dm = dm0 + warp * kDR + j;
            if (dm >= ndm) break;
            float *orow = out + (size_t)dm * nout + t0;
            const int lim = (int)min((int64_t)kTile, nout - t0);
            for (int m = lane; m < lim; m += 32) orow[m] = stile[j * kTile + m];
        }
        block_stat_f32(n, s, q, reinterpret_cast<StatF *>(partials) + pidx);
    }
}

// ------------------------------------------------------------------ host side
static int elem_align(dd_dtype t) { return (int)(16 / in_elem_bytes(t)); }

int fast_configure(dd_plan *p)
{
    p->fast = nullptr;
    const int C = p->nchans, D = p->ndm;
    const int nblk = (D + kDmBlk - 1) / kDmBlk;
    const int AL = elem_align(p->dtype);
    std::vector<uint32_t> desc((size_t)nblk * C * kWarps);
    std::vector<int32_t> base((size_t)nblk * C);
    std::vector<int32_t> goff((size_t)nblk * C * kWarps * kDR);
    auto dl = [&](int dm, int c) { return p->delays[(size_t)std::min(dm, D - 1) * C + c]; };
    long long need = 0;   // largest element index any lane touches, + 1
    for (int b = 0; b < nblk; ++b) {
        for (int c = 0; c < C; ++c) {
            int lo = INT_MAX;
            for (int j = 0; j < kDmBlk; ++j) lo = std::min(lo, dl(b * kDmBlk + j, c));
            const int row0 = lo - (lo % AL);       // aligned row start (t0 is a multiple of AL)
            base[(size_t)b * C + c] = row0;
            for (int w = 0; w < kWarps; ++w) {
                int d[kDR], bw = INT_MAX;
                for (int j = 0; j < kDR; ++j) { d[j] = dl(b * kDmBlk + w * kDR + j, c); bw = std::min(bw, d[j]); }
                const int off = bw - row0;           // window offset of the warp's base in the row
                int A = kGeneric;
                const int o1 = d[1] - d[0];
                if (d[0] == bw) {
                    for (int cand = std::max(0, o1 - 1); cand <= o1 && A == kGeneric; ++cand) {
                        bool fits = cand <= kAMax;
                        for (int j = 1; j < kDR && fits; ++j) {
                            const int e = d[j] - d[0] - j * cand;
                            fits = e >= 0 && e <= j;
                        }
                        if (fits) A = cand;
                    }
                }
                const int wsoff = off & ~3, rem = off & 3;
                if (A != kGeneric && wsoff / 4 < (1 << 12)) {
                    uint32_t dd = 0;
                    for (int j = 0; j < kDR; ++j) {
                        const uint32_t q = (uint32_t)(rem + (d[j] - d[0] - j * A));
                        dd |= q << (3 * j);
                    }
                    dd |= (uint32_t)A << 12;
                    dd |= (uint32_t)(wsoff / 4) << 20;
                    desc[((size_t)b * C + c) * kWarps + w] = dd;
                    const int wl = ((kDR - 1) * A + (kDR - 1) + 3 + kTR + 3) / 4 * 4;
                    need = std::max<long long>(need, (long long)wsoff + kTR * 31 + wl);
                } else {
                    desc[((size_t)b * C + c) * kWarps + w] = (uint32_t)kGeneric << 12;
                    for (int j = 0; j < kDR; ++j) {
                        const int o = d[j] - row0;
                        goff[(((size_t)b * C + c) * kWarps + w) * kDR + j] = o;
                        need = std::max<long long>(need, (long long)(o & ~3) + kTR * 31 + kTR + 4);
                    }
                }
            }
        }
    }
    const int rs = (int)((need + 15) / 16 * 16);
    const size_t eb = in_elem_bytes(p->dtype);
    const size_t budget = std::min<size_t>(p->smem_optin, 227 * 1024) - 1024;
    const size_t per_ch = (size_t)rs * eb + kWarps * sizeof(uint32_t);
    int ch = (int)std::min<size_t>(16, budget / (kStages * per_ch));
    const size_t epi = (size_t)kWarps * kDR * kTile * sizeof(float);
    if (ch < 1 || epi > budget) return DD_OK;   // kernel 2 unavailable: rows too long
    const size_t bar_off = (std::max(epi, (size_t)kStages * ch * per_ch) + 15) / 16 * 16;
    const size_t smem = bar_off + kStages * sizeof(uint64_t);
    if (smem > budget + 1024) return DD_OK;

    FastPlan *f = new FastPlan();
    f->nblk = nblk; f->rs = rs; f->ch = ch; f->smem = smem; f->al = AL; f->bar_off = (int)bar_off;
    cudaError_t e = cudaMalloc(&f->d_desc, desc.size() * 4);
    if (e == cudaSuccess) e = cudaMalloc(&f->d_base, base.size() * 4);
    if (e == cudaSuccess) e = cudaMalloc(&f->d_goff, goff.size() * 4);
    if (e == cudaSuccess) e = cudaMalloc(&f->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(f->d_desc, desc.data(), desc.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(f->d_base, base.data(), base.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(f->d_goff, goff.data(), goff.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(f->d_err, 0, sizeof(int));
    const void *fn = p->dtype == DD_F32 ? (const void *)fast_kernel<float, false>
                   : p->dtype == DD_F16 ? (const void *)fast_kernel<__half, false>
                                        : (const void *)fast_kernel<uint8_t, true>;
    if (e == cudaSuccess) e = allow_max_dynamic_smem(fn, p->smem_optin);
    p->fast = f;
    if (e != cudaSuccess) {
        fast_release(p);
        return cuda_fail(e, "kernel 2 setup");
    }
    return DD_OK;
}

int fast_error(dd_plan *p, cudaStream_t s)
{
    FastPlan *f = static_cast<FastPlan *>(p->fast);
    if (!f) return DD_OK;
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, f->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "read kernel-2 status");
    if (h) {
        cudaMemsetAsync(f->d_err, 0, sizeof(int), s);
        return set_error(h, "kernel 2 gave up waiting for its input copies (status %d)", h);
    }
    return DD_OK;
}

int fast_execute(dd_plan *p, const void *in, int64_t pitch, void *out, cudaStream_t s)
{
    FastPlan *f = static_cast<FastPlan *>(p->fast);
    if (!f) return set_error(DD_ERR_ARG, "kernel 2 unavailable for this plan");
    const int AL = f->al;
    if (((uintptr_t)in & 15u) || (pitch % AL)) {
        // TMA bulk copies need 16-byte aligned rows: run the generic kernel.
        return generic_execute(p, in, pitch, out, s);
    }
    const int64_t ntile = (p->nsamp_out + kTile - 1) / kTile;
    if (ntile > 65535) return generic_execute(p, in, pitch, out, s);
    const int64_t np = ntile * f->nblk;
    int rc = ensure_partials_public(p, np);
    if (rc) return rc;
    const int64_t nin_al = (p->nsamp_in + AL - 1) / AL * AL;
    dim3 grid((unsigned)f->nblk, (unsigned)ntile);
    switch (p->dtype) {
    case DD_F32:
        fast_kernel<float, false><<<grid, kThreads, f->smem, s>>>(
            (const float *)in, pitch, nin_al, p->nchans, p->ndm, p->nsamp_out, f->d_desc, f->d_base, f->d_goff,
            f->rs, f->ch, f->bar_off, out, p->d_partials, f->d_err);
        break;
    case DD_F16:
        fast_kernel<__half, false><<<grid, kThreads, f->smem, s>>>(
            (const __half *)in, pitch, nin_al, p->nchans, p->ndm, p->nsamp_out, f->d_desc, f->d_base, f->d_goff,
            f->rs, f->ch, f->bar_off, out, p->d_partials, f->d_err);
        break;
    case DD_U8:
        fast_kernel<uint8_t, true><<<grid, kThreads, f->smem, s>>>(
            (const uint8_t *)in, pitch, nin_al, p->nchans, p->ndm, p->nsamp_out, f->d_desc, f->d_base, f->d_goff,
            f->rs, f->ch, f->bar_off, out, p->d_partials, f->d_err);
        break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch fast_kernel");
    p->n_partials = np;
    p->stats_out = out;
    return DD_OK;
}

void fast_release(dd_plan *p)
{
    FastPlan *f = static_cast<FastPlan *>(p->fast);
    if (!f) return;
    if (f->d_desc) cudaFree(f->d_desc);
    if (f->d_base) cudaFree(f->d_base);
    if (f->d_goff) cudaFree(f->d_goff);
    if (f->d_err) cudaFree(f->d_err);
    delete f;
    p->fast = nullptr;
}

}  // namespace dd
