// Kernel 5: the Section 3.1 sum with exactly shared subband partial sums,
//   out[dm][t] = sum_c in[c][t + d(c,dm)]
//              = sum_s P_s,pat(dm)[t + d(ref(s),dm)],
//   P_s,pat[u] = sum_{c in s} in[c][u + r_pat(c)],  r_pat(c) = d(c,dm) - d(ref(s),dm),
// over subbands s of CS consecutive channels, ref(s) the subband's channel
// with the smallest delay.  DM trials of a block whose relative delays
// r(c) within a subband coincide (a "pattern") share one partial sum: the
// result is exactly the brute-force sum (same integer delays; FP32 rounding
// order differs), computed with (#patterns x CS + #trials) shared-memory
// words per subband and output tile instead of #trials x CS.
//
// Block = NW warps on a tile of 32*TI samples (lanes interleaved as kernel 3)
// and DR*NW DM trials.  Per subband (one TMA stage: its CS input rows and
// its table record):
//   stage 1: the block forms every pattern's partial sum over the samples
//            its trials need (P, double-buffered in shared memory);
//   stage 2: each warp adds, for its trials, P_pat[t + offset] (one
//            conflict-free shared word per add, as kernel 3).
// One __syncthreads per subband: stage 1 of subband s+1 writes the other P
// buffer while stage 2 of s reads this one; each warp takes its trials'
// offsets into registers during stage 1 (the stage's record may be reused by
// the next TMA copy before stage 2 ends).  The input ring has two stages
// (kShStages): one subband's work covers the next one's copy, and the shared
// memory saved keeps three blocks per SM.
#pragma once

#include "dd_lane_impl.cuh"

namespace dd {

constexpr int kShStages = 2;     // input ring of kernel 5

// Table record of one (DM block, subband), int32 (16-byte multiple):
//   [0 .. DB) q_j (index into P of trial j's t = t0 term) | [DB] npat |
//   [DB+1 .. DB+1+CS) rowoff_c (staged-row index of u = 0 for channel c) |
//   per pattern p < NPMAX: {poff, lo, W, r_0 .. r_{CS-1}}.
template <int CS, int NPMAX, int DB>
struct ShareRec {
    static_assert(DB % 4 == 0, "trial offsets are loaded 4 at a time");
    static constexpr int kTrial = 0;
    static constexpr int kNpat = DB;
    static constexpr int kRowoff = DB + 1;
    static constexpr int kPat = DB + 1 + CS;            // first pattern field
    static constexpr int kPatLen = 3 + CS;
    static constexpr int kLen = (kPat + NPMAX * kPatLen + 3) / 4 * 4;
};

struct ShareLaunch {
    const void *in;
    int64_t pitch, nsamp_in_al;
    int nchans, ndm, nsub;
    int64_t nout;
    const int32_t *rec;    // [nblk][nsub][kLen]
    const int32_t *base;   // [nblk][nchans] staged row start relative to the tile start (aligned)
    int rs, pmax, bar_off, nblk;
    int64_t ntile;
    int dgroup;
    void *out, *partials;
    int *err;
    size_t smem;
};

template <typename Tin, bool kInt, int TI, int DR, int NW, int CS, int NPMAX, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB) share_kernel(ShareLaunch a)
{
    constexpr int kDmBlk = DR * NW, kT = NW * 32;
    using R = ShareRec<CS, NPMAX, kDmBlk>;
    extern __shared__ __align__(128) unsigned char smem[];
    const Tin *__restrict__ in = static_cast<const Tin *>(a.in);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rs = a.rs, nsub = a.nsub;

    int blk;
    int64_t t0;
    {
        LaneLaunch r{};
        r.dgroup = a.dgroup; r.ntile = a.ntile; r.nblk = a.nblk;
        lane_raster<TI>(r, blockIdx.x, blk, t0);
    }
    const int dm0 = blk * kDmBlk;

    // layout: [kShStages][CS][rs] Tin rows | [kShStages][kLen] int32 records |
    //         [2][pmax] float P | mbarriers
    const size_t stage_elems = (size_t)CS * rs;
    Tin *rows = reinterpret_cast<Tin *>(smem);
    int32_t *srec = reinterpret_cast<int32_t *>(smem + kShStages * stage_elems * sizeof(Tin));
    float *P = reinterpret_cast<float *>(srec + kShStages * R::kLen);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + a.bar_off);
    const int32_t *brec = a.rec + (size_t)blk * nsub * R::kLen;
    const int32_t *bbase = a.base + (size_t)blk * a.nchans;

    if (tid == 0) {
        for (int s = 0; s < kShStages; ++s) mbar_init(&bar[s], 1);
        mbar_fence_init();
    }
    __syncthreads();

    auto row_bytes = [&](int c, int64_t &g) -> uint32_t {
        g = t0 + bbase[c];
        int64_t n = a.nsamp_in_al - g;
        n = n < 0 ? 0 : (n > rs ? rs : n);
        return (uint32_t)(n * (int64_t)sizeof(Tin));
    };
    auto issue = [&](int s) {
        const int buf = s % kShStages;
        uint32_t bytes = (uint32_t)(R::kLen * sizeof(int32_t));
        for (int cc = 0; cc < CS; ++cc) { int64_t g; bytes += row_bytes(s * CS + cc, g); }
        mbar_arrive_tx(&bar[buf], bytes);
        bulk_g2s(srec + (size_t)buf * R::kLen, brec + (size_t)s * R::kLen, (uint32_t)(R::kLen * sizeof(int32_t)),
                 &bar[buf]);
        for (int cc = 0; cc < CS; ++cc) {
            int64_t g;
            const uint32_t nb = row_bytes(s * CS + cc, g);
            if (nb)
                bulk_g2s(rows + (size_t)buf * stage_elems + (size_t)cc * rs,
                         in + (size_t)(s * CS + cc) * a.pitch + g, nb, &bar[buf]);
        }
    };

    float acc[DR][TI];
#pragma unroll
    for (int j = 0; j < DR; ++j)
#pragma unroll
        for (int i = 0; i < TI; ++i) acc[j][i] = 0.f;

    if (tid == 0)
        for (int s = 0; s < kShStages - 1 && s < nsub; ++s) issue(s);

    bool ok = true;
    int q[DR];
    for (int s = 0; s < nsub; ++s) {
        if (tid == 0 && s + kShStages - 1 < nsub) issue(s + kShStages - 1);
        const int buf = s % kShStages;
        if (ok) ok = mbar_wait(&bar[buf], (uint32_t)((s / kShStages) & 1), a.err);
        const int32_t *rec = srec + (size_t)buf * R::kLen;
        const Tin *srow = rows + (size_t)buf * stage_elems;
        float *Pb = P + (size_t)(s & 1) * a.pmax;
        // stage 1: every pattern's partial sum over the samples its trials need
        const int npat = rec[R::kNpat];
        int rowoff[CS];
#pragma unroll
        for (int c = 0; c < CS; ++c) rowoff[c] = rec[R::kRowoff + c];
        for (int p = 0; p < npat; ++p) {
            const int32_t *pr = rec + R::kPat + p * R::kPatLen;
            const int poff = pr[0], lo = pr[1], W = pr[2];
            const Tin *src[CS];
#pragma unroll
            for (int c = 0; c < CS; ++c) src[c] = srow + (size_t)c * rs + rowoff[c] + lo + pr[3 + c];
#pragma unroll 4
            for (int u = tid; u < W; u += kT) {
                float v = lane_ld<Tin>(src[0] + u);
#pragma unroll
                for (int c = 1; c < CS; ++c) v += lane_ld<Tin>(src[c] + u);
                Pb[poff + u] = v;
            }
        }
        // this warp's trials: index of their t = t0 term in P
#pragma unroll
        for (int j = 0; j < DR; j += 4) {
            const int4 v = *reinterpret_cast<const int4 *>(rec + R::kTrial + warp * DR + j);
            q[j] = v.x; q[j + 1] = v.y; q[j + 2] = v.z; q[j + 3] = v.w;
        }
        __syncthreads();
        // stage 2: one shared word per add
#pragma unroll
        for (int j = 0; j < DR; ++j) {
            const float *pp = Pb + q[j] + lane;
#pragma unroll
            for (int i = 0; i < TI; ++i) acc[j][i] += pp[32 * i];
        }
    }
    ok = __syncthreads_and(ok);
    if (!ok) return;

    const int64_t nout = a.nout;
    if constexpr (kInt) {
        long long n = 0, s = 0;
        unsigned long long qq = 0;
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
                    n++; s += v; qq += (unsigned long long)(v * v);
                }
            }
        }
        block_stat_i(n, s, qq, reinterpret_cast<StatI *>(a.partials) + blockIdx.x);
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
        float qq = 0.f;
#pragma unroll
        for (int j = 0; j < DR; ++j) {
            const int dm = dm0 + warp * DR + j;
#pragma unroll
            for (int i = 0; i < TI; ++i) {
                const int64_t t = t0 + lane + 32 * i;
                if (dm < a.ndm && t < nout) { const float d = acc[j][i] - m; qq += d * d; }
            }
        }
        block_stat_f32(n, s, qq, reinterpret_cast<StatF *>(a.partials) + blockIdx.x);
    }
}

// Compiled shapes: subbands of 4 channels, at most 8 patterns per (block,
// subband), 8 trials per warp, 4 warps (32 trials); {samples per lane,
// resident blocks per SM the register budget targets}.
constexpr int kShDR = 8, kShNW = 4, kShCS = 4, kShNP = 8;
using ShareRecC = ShareRec<kShCS, kShNP, kShDR * kShNW>;
struct ShareShape { int ti, minb; };
constexpr int kNumShareCfg = 2;
constexpr ShareShape kShareCfg[kNumShareCfg] = {{16, 3}, {8, 5}};

cudaError_t share_launch(int k, dd_dtype t, const ShareLaunch &a, cudaStream_t s);
cudaError_t share_prepare(int k, size_t optin);

}  // namespace dd
