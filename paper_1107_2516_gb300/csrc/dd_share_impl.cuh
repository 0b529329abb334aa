// Kernel 5: the Section 3.1 sum with exactly shared subband partial sums,
//   out[dm][t] = sum_c in[c][t + d(c,dm)]
//              = sum_s P_s,pat(dm)[t + d(ref(s),dm)],
//   P_s,pat[u] = sum_{c in s} in[c][u + r_pat(c)],  r_pat(c) = d(c,dm) - d(ref(s),dm),
// over subbands s of CS consecutive channels, ref(s) the subband's channel
// with the smallest delay.  DM trials of a block whose relative delays
// r(c) within a subband coincide (a "pattern") share one partial sum: the
// result is exactly the brute-force sum (same integer delays; FP32 rounding
// order differs), computed with about #patterns x (CS + 1) + #trials
// shared-memory words per subband and output sample instead of #trials x CS.
//
// Block = NW warps on a tile of 32*TI samples (lanes interleaved as kernel 3)
// and DR*NW DM trials.  Per subband (one TMA stage: its CS input rows and
// its table record):
//   stage 1: the block forms every pattern's partial sum over the samples
//            its trials need (P, double-buffered in shared memory).  The
//            patterns' sums are laid end to end in one index space e < E,
//            cut into rows of 32 (each row inside one pattern), and each warp
//            sums the contiguous run of rows the table assigns it, four rows
//            per step: the pattern's fields are uniform in the warp and
//            reloaded only where a pattern ends, and every warp gets the same
//            number of rows;
//   stage 2: each warp adds, for its trials, P_pat[t + offset] (one
//            conflict-free shared word per add, as kernel 3).
// One __syncthreads per subband: stage 1 of subband s+1 writes the other P
// buffer while stage 2 of s reads this one; each warp takes its trials'
// offsets into registers during stage 1 (the stage's record may be reused by
// the next TMA copy before stage 2 ends).  The input ring has NS stages:
// NS - 1 subbands' copies are in flight while one is summed.  The tile body
// (share_tile) serves the one-plan kernel and the persistent batch kernel.
#pragma once

#include "dd_lane_impl.cuh"

namespace dd {

// Table record of one (DM block, subband), int32 (16-byte multiple):
//   [0 .. DB) q_j (index into P of trial j's t = t0 term) | [DB] E (the
//   subband's P length) | 3 unused |
//   per pattern p < NPMAX, kPatLen words: {end_p, b_0 .. b_{CS-1}, start_p,
//   rows_p, unused} |
//   stage-1 split: [kWarp + w] (w <= kMaxWarps) first row of warp w (the
//   row count R at w = the block's warp count), [kWarp + kMaxWarps + 1 + w]
//   the pattern holding that row.
// start_p / end_p = the index range of pattern p's sums in P; b_c such that
// the term of channel c in P[e] (e in pattern p) is staged element b_c + e of
// the stage's rows (b_c = c * rs + the row offset of the pattern's first
// sample minus start_p); rows_p = the rows of 32 sums before pattern p (the
// patterns' sums are cut into rows of 32, each row inside one pattern).
template <int CS, int NPMAX, int DB>
struct ShareRec {
    static_assert(DB % 4 == 0, "trial offsets are loaded 4 at a time");
    static_assert(CS + 3 <= 8, "pattern record: end, CS row offsets, start, rows before");
    static constexpr int kTrial = 0;
    static constexpr int kE = DB;
    static constexpr int kPat = DB + 4;                 // first pattern field (16-byte aligned)
    static constexpr int kPatLen = 8;
    static constexpr int kPatStart = 1 + CS, kPatRows = 2 + CS;
    static constexpr int kMaxWarps = 8;
    static constexpr int kWarp = kPat + NPMAX * kPatLen;
    static constexpr int kLen = kWarp + (2 * kMaxWarps + 1 + 3) / 4 * 4;
};

struct ShareLaunch {
    const void *in;
    int64_t pitch, nsamp_in_al;
    int nchans, ndm, nsub;
    int64_t nout;
    const int32_t *rec;    // [nblk][nsub][kLen]
    const int32_t *base;   // [nblk][nchans] staged row start relative to the tile start (aligned)
    const int32_t *rlen;   // [nblk][nchans] elements of that row the block's trials read (<= rs, aligned)
    int rs, pmax, bar_off, nblk;
    int64_t ntile;         // tiles of this launch, starting at output sample t_base
    int64_t t_base;
    int dgroup;
    void *out, *partials;
    int *err;
    size_t smem;
    int skew;              // 1: DM block b takes the time tiles in a rotated order (share_raster)
};

// DM block / time tile of linear block index `lin`, as lane_raster, and with
// a.skew set (a launch over every time tile of the plan) each DM block's
// tiles rotated back by its own delay offset: block b takes tile (s - k_b)
// mod ntile where lane_raster gives tile s, k_b = the block's row start in
// the middle channel in whole tiles.  Blocks that run at the same time then
// stage nearly the same input columns instead of windows up to the whole
// delay span apart, so the staged input stays in L2 between them.  A
// permutation of each block's tiles: every (block, tile) is still taken once.
template <int TI>
__device__ __forceinline__ void share_raster(const ShareLaunch &a, int64_t lin, int &blk, int64_t &t0)
{
    LaneLaunch r{};
    r.dgroup = a.dgroup; r.ntile = a.ntile; r.nblk = a.nblk;
    lane_raster<TI>(r, lin, blk, t0);
    if (a.skew) {
        constexpr int64_t kTile = 32 * TI;
        const int64_t k = ((int64_t)a.base[(size_t)blk * a.nchans + a.nchans / 2] / kTile) % a.ntile;
        t0 = ((t0 / kTile + a.ntile - k) % a.ntile) * kTile;
    }
}

// Stage 1 of one subband: P[e] for e < E (the patterns' sums end to end).
// Each pattern's sums form rows of 32 consecutive e (the last one partial);
// warp w takes the contiguous rows the record assigns it (the host splits
// the R rows in order, warp 0 a smaller share), so a row's pattern (its fields) is
// uniform in the warp and changes only at pattern ends, and lane l sums
// element row_start + l of each of its rows: whole rows RPS at a time with
// the pattern's offsets set up once (every load of a step issued before its
// stores), then the pattern's leftover rows in predicated steps of LRS rows.
template <typename Tin, typename R, int CS, int NW, int RPS = 4, int LRS = RPS>
__device__ __forceinline__ void share_stage1(const int32_t *rec, const Tin *srow, float *Pb, int warp, int lane)
{
    static_assert(NW <= R::kMaxWarps, "stage-1 split recorded for at most kMaxWarps warps");
    int r = rec[R::kWarp + warp];
    const int r1 = rec[R::kWarp + warp + 1];
    int p = rec[R::kWarp + R::kMaxWarps + 1 + warp];
    while (r < r1) {
        const int32_t *pr = rec + R::kPat + p * R::kPatLen;
        int b[R::kPatLen];
#pragma unroll
        for (int v = 0; v < R::kPatLen; v += 4) {
            const int4 x = *reinterpret_cast<const int4 *>(pr + v);
            b[v] = x.x; b[v + 1] = x.y; b[v + 2] = x.z; b[v + 3] = x.w;
        }
        const int pend = b[0], pst = b[R::kPatStart], pexcl = b[R::kPatRows];
        const int rend = min(r1, pexcl + ((pend - pst + 31) >> 5));
        const int rfull = min(rend, pexcl + ((pend - pst) >> 5));    // rows wholly inside the pattern
        // row r's element for this lane: e = e0 + 32 r
        const int e0 = pst - (pexcl << 5) + lane;
        int src[CS];                                                   // staged element of channel c at e0
#pragma unroll
        for (int c = 0; c < CS; ++c) src[c] = b[1 + c] + e0;
        for (; r + RPS <= rfull; r += RPS) {
            // all RPS x CS loads before the RPS stores: the staged rows and P
            // are both shared memory, so the compiler may not move a store
            // above a later load
            float x[RPS][CS];
#pragma unroll
            for (int u = 0; u < RPS; ++u)
#pragma unroll
                for (int c = 0; c < CS; ++c) x[u][c] = lane_ld<Tin>(srow + (src[c] + ((r + u) << 5)));
#pragma unroll
            for (int u = 0; u < RPS; ++u) {
                float v = x[u][0];
#pragma unroll
                for (int c = 1; c < CS; ++c) v += x[u][c];
                Pb[e0 + ((r + u) << 5)] = v;
            }
        }
        for (; r < rend; r += LRS) {
            // the pattern's leftover rows (fewer than RPS whole rows and the
            // partial last one), LRS per step; only the rows and lanes inside
            // the pattern load and store
            float x[LRS][CS];
            bool in[LRS];
#pragma unroll
            for (int u = 0; u < LRS; ++u) {
                const int o = (r + u) << 5;
                in[u] = r + u < rend && e0 + o < pend;
#pragma unroll
                for (int c = 0; c < CS; ++c) x[u][c] = in[u] ? lane_ld<Tin>(srow + (src[c] + o)) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < LRS; ++u) {
                float v = x[u][0];
#pragma unroll
                for (int c = 1; c < CS; ++c) v += x[u][c];
                if (in[u]) Pb[e0 + ((r + u) << 5)] = v;
            }
        }
        r = rend;
        ++p;
    }
}

// One thread's share of the block's partial statistics.
template <bool kInt> struct ShareStat;
template <> struct ShareStat<true> { long long n = 0, s = 0; unsigned long long q = 0; };
template <> struct ShareStat<false> { int n = 0; float s = 0.f, q = 0.f; };

// Store one warp's DR trials x 32*TI samples and accumulate their statistics.
template <bool kInt, int TI, int DR>
__device__ __forceinline__ void share_store(const ShareLaunch &a, const float (&acc)[DR][TI], int dmw, int64_t t0,
                                            int lane, ShareStat<kInt> &st)
{
    const int64_t nout = a.nout;
    if constexpr (kInt) {
        int32_t *out = reinterpret_cast<int32_t *>(a.out);
#pragma unroll
        for (int j = 0; j < DR; ++j) {
            const int dm = dmw + j;
#pragma unroll
            for (int i = 0; i < TI; ++i) {
                const int64_t t = t0 + lane + 32 * i;
                if (dm < a.ndm && t < nout) {
                    const long long v = __float2int_rn(acc[j][i]);
                    __stcs(&out[(size_t)dm * nout + t], (int32_t)v);
                    st.n++; st.s += v; st.q += (unsigned long long)(v * v);
                }
            }
        }
    } else {
        float *out = reinterpret_cast<float *>(a.out);
#pragma unroll
        for (int j = 0; j < DR; ++j) {
            const int dm = dmw + j;
#pragma unroll
            for (int i = 0; i < TI; ++i) {
                const int64_t t = t0 + lane + 32 * i;
                if (dm < a.ndm && t < nout) {
                    __stcs(&out[(size_t)dm * nout + t], acc[j][i]);   // streamed: read back only by the search
                    st.n++; st.s += acc[j][i];
                }
            }
        }
        const float m = st.n ? st.s / (float)st.n : 0.f;
#pragma unroll
        for (int j = 0; j < DR; ++j) {
            const int dm = dmw + j;
#pragma unroll
            for (int i = 0; i < TI; ++i) {
                const int64_t t = t0 + lane + 32 * i;
                if (dm < a.ndm && t < nout) { const float d = acc[j][i] - m; st.q += d * d; }
            }
        }
    }
}

// The block's partial statistics into record `lin` (every thread of the
// block calls this).
template <bool kInt>
__device__ __forceinline__ void share_stat_flush(const ShareLaunch &a, const ShareStat<kInt> &st, int64_t lin)
{
    if constexpr (kInt)
        block_stat_i(st.n, st.s, st.q, reinterpret_cast<StatI *>(a.partials) + lin);
    else
        block_stat_f32(st.n, st.s, st.q, reinterpret_cast<StatF *>(a.partials) + lin);
}

// One work item: DM block `blk` x the time tile at t0; partial statistics
// record `lin`.  bar[NS] is the block's input ring; `gstage` its running stage
// count (a persistent block keeps the ring across items: subband s of this
// item uses buffer (gstage + s) % NS, parity ((gstage + s) / NS) & 1).
// Returns false if a bounded wait gave up.
template <typename Tin, bool kInt, int TI, int DR, int NW, int CS, int NPMAX, int NS>
__device__ __forceinline__ bool share_tile(const ShareLaunch &a, int blk, int64_t t0, int64_t lin,
                                           uint64_t *bar, uint32_t &gstage)
{
    extern __shared__ __align__(128) unsigned char smem[];   // as lane_tile: shared-space accesses
    constexpr int kDmBlk = DR * NW, kT = NW * 32;
    using R = ShareRec<CS, NPMAX, kDmBlk>;
    const Tin *__restrict__ in = static_cast<const Tin *>(a.in);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rs = a.rs, nsub = a.nsub;
    const int dm0 = blk * kDmBlk;

    // layout: [NS][CS][rs] Tin rows | [NS][kLen] int32 records | [2][pmax] float P
    const size_t stage_elems = (size_t)CS * rs;
    Tin *rows = reinterpret_cast<Tin *>(smem);
    int32_t *srec = reinterpret_cast<int32_t *>(smem + NS * stage_elems * sizeof(Tin));
    float *P = reinterpret_cast<float *>(srec + NS * R::kLen);
    const int32_t *brec = a.rec + (size_t)blk * nsub * R::kLen;
    const int32_t *bbase = a.base + (size_t)blk * a.nchans;
    const uint32_t g0 = gstage;
    gstage += (uint32_t)nsub;

    // thread 0 issues subband s's copies with its rows' start offsets loaded
    // one subband earlier (the global loads' latency stays off the barrier path)
    // each channel's row: the rl elements its DM trials read from column
    // t0 + b on (fewer than rs near the top of the band), cut at the input's end
    auto row_bytes = [&](int b, int rl, int64_t &g) -> uint32_t {
        g = t0 + b;
        int64_t n = a.nsamp_in_al - g;
        n = n < 0 ? 0 : (n > rl ? rl : n);
        return (uint32_t)(n * (int64_t)sizeof(Tin));
    };
    auto issue = [&](int s, const int (&rb)[CS], const int (&rl)[CS]) {
        const int buf = (int)((g0 + s) % NS);
        uint32_t bytes = (uint32_t)(R::kLen * sizeof(int32_t));
#pragma unroll
        for (int cc = 0; cc < CS; ++cc) { int64_t g; bytes += row_bytes(rb[cc], rl[cc], g); }
        mbar_arrive_tx(&bar[buf], bytes);
        bulk_g2s(srec + (size_t)buf * R::kLen, brec + (size_t)s * R::kLen, (uint32_t)(R::kLen * sizeof(int32_t)),
                 &bar[buf]);
        const uint64_t pol = l2_evict_last();          // other DM blocks of this tile stage these rows soon
#pragma unroll
        for (int cc = 0; cc < CS; ++cc) {
            int64_t g;
            const uint32_t nb = row_bytes(rb[cc], rl[cc], g);
            if (nb)
                bulk_g2s_hint(rows + (size_t)buf * stage_elems + (size_t)cc * rs,
                              in + (size_t)(s * CS + cc) * a.pitch + g, nb, &bar[buf], pol);
        }
    };
    const int32_t *blen = a.rlen + (size_t)blk * a.nchans;
    int rb[CS], rl[CS];
    auto load_rb = [&](int s) {
#pragma unroll
        for (int cc = 0; cc < CS; ++cc) { rb[cc] = bbase[s * CS + cc]; rl[cc] = blen[s * CS + cc]; }
    };

    float acc[DR][TI];
#pragma unroll
    for (int j = 0; j < DR; ++j)
#pragma unroll
        for (int i = 0; i < TI; ++i) acc[j][i] = 0.f;

    if (tid == 0) {
        for (int s = 0; s < NS - 1 && s < nsub; ++s) { load_rb(s); issue(s, rb, rl); }
        if (NS - 1 < nsub) load_rb(NS - 1);
    }

    bool ok = true;
    int q[DR];
    for (int s = 0; s < nsub; ++s) {
        if (tid == 0 && s + NS - 1 < nsub) {
            issue(s + NS - 1, rb, rl);
            if (s + NS < nsub) load_rb(s + NS);
        }
        const int buf = (int)((g0 + s) % NS);
        if (ok) ok = mbar_wait(&bar[buf], (uint32_t)(((g0 + s) / NS) & 1), a.err);
        const int32_t *rec = srec + (size_t)buf * R::kLen;
        const Tin *srow = rows + (size_t)buf * stage_elems;
        float *Pb = P + (size_t)(s & 1) * a.pmax;
        // stage 1: every pattern's partial sum over the samples its trials need
        share_stage1<Tin, R, CS, NW>(rec, srow, Pb, warp, lane);
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
    if (!ok) return false;
    ShareStat<kInt> st;
    share_store<kInt, TI, DR>(a, acc, dm0 + warp * DR, t0, lane, st);
    share_stat_flush<kInt>(a, st, lin);
    return true;
}

// One plan: one block per work item, grid = nblk * ntile.
template <typename Tin, bool kInt, int TI, int DR, int NW, int CS, int NPMAX, int NS, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB) share_kernel(ShareLaunch a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + a.bar_off);
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(&bar[s], 1);
        mbar_fence_init();
    }
    __syncthreads();
    int blk;
    int64_t t0;
    share_raster<TI>(a, blockIdx.x, blk, t0);
    t0 += a.t_base;
    uint32_t gstage = 0;
    share_tile<Tin, kInt, TI, DR, NW, CS, NPMAX, NS>(a, blk, t0, blockIdx.x, bar, gstage);
}

// share_tile as an out-of-line function for the persistent batch kernel.
template <typename Tin, bool kInt, int TI, int DR, int NW, int CS, int NPMAX, int NS>
__device__ __noinline__ bool share_tile_call(const ShareLaunch &a, int blk, int64_t t0, int64_t lin,
                                             uint64_t *bar, uint32_t &gstage)
{
    return share_tile<Tin, kInt, TI, DR, NW, CS, NPMAX, NS>(a, blk, t0, lin, bar, gstage);
}

// Persistent batch of beams, each on kernel 5 (kind 1: its ShareLaunch) or on
// kernel 3 (kind 0: its LaneLaunch) with the same block geometry (DR*NW
// trials x 32*TI samples), so both enumerate the same work items.  Two input
// rings: kernel 3's kStages mbarriers at b.bar_off, kernel 5's NS right after;
// each with its own running stage count.
template <int TI, int DR, int NW, int CS, int NPMAX, int NS, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB) mixed_batch_kernel(LaneBatchLaunch b)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_item;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + b.bar_off), *sbar = bar + kStages;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
        for (int s = 0; s < NS; ++s) mbar_init(&sbar[s], 1);
        mbar_fence_init();
    }
    __syncthreads();
    uint32_t gl = 0, gs = 0;
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
        if (a.kind == 1) {
            const ShareLaunch &sa = b.sbeams[w.x];
            switch (a.dtype) {
            case DD_F32: ok = share_tile_call<float, false, TI, DR, NW, CS, NPMAX, NS>(sa, blk, t0, w.y, sbar, gs); break;
            case DD_F16: ok = share_tile_call<__half, false, TI, DR, NW, CS, NPMAX, NS>(sa, blk, t0, w.y, sbar, gs); break;
            default: ok = share_tile_call<uint8_t, true, TI, DR, NW, CS, NPMAX, NS>(sa, blk, t0, w.y, sbar, gs); break;
            }
        } else {
            switch (a.dtype) {
            case DD_F32: ok = lane_tile_call<float, false, TI, DR, NW>(a, blk, t0, w.y, bar, gl); break;
            case DD_F16: ok = lane_tile_call<__half, false, TI, DR, NW>(a, blk, t0, w.y, bar, gl); break;
            default: ok = lane_tile_call<uint8_t, true, TI, DR, NW>(a, blk, t0, w.y, bar, gl); break;
            }
        }
        if (!ok) break;
        __syncthreads();
        if (threadIdx.x == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
}

// Arrive on an mbarrier (no transaction bytes); release semantics at CTA scope.
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Partial statistics of warps [gw0, gw0 + ngw) of the block (the accumulator
// warps of the warp-specialised kernel; the others have left): the same
// combination as block_stat_f32 / block_stat_i over those warps only, joined
// by named barrier 1.  Every thread of those warps calls it; the group's
// first thread writes record `lin`.
template <bool kInt>
__device__ __forceinline__ void group_stat_flush(const ShareLaunch &a, const ShareStat<kInt> &st, int64_t lin,
                                                 int gw0, int ngw)
{
    __shared__ double gn[32], gm[32], gq[32];
    __shared__ long long gs[32], gc[32];
    __shared__ unsigned long long gu[32];
    const int lane = threadIdx.x & 31, w = (threadIdx.x >> 5) - gw0;
    if constexpr (kInt) {
        long long n = st.n, s = st.s;
        unsigned long long q = st.q;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            n += __shfl_xor_sync(0xffffffffu, n, off);
            s += __shfl_xor_sync(0xffffffffu, s, off);
            q += __shfl_xor_sync(0xffffffffu, q, off);
        }
        if (lane == 0) { gc[w] = n; gs[w] = s; gu[w] = q; }
    } else {
        int nw = st.n;
        float sw = st.s;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            nw += __shfl_xor_sync(0xffffffffu, nw, off);
            sw += __shfl_xor_sync(0xffffffffu, sw, off);
        }
        const float mw = nw ? sw / (float)nw : 0.f;
        const float mt = st.n ? st.s / (float)st.n : 0.f;
        const float d = mt - mw;
        float qw = st.q + (float)st.n * d * d;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) qw += __shfl_xor_sync(0xffffffffu, qw, off);
        if (lane == 0) { gn[w] = nw; gm[w] = mw; gq[w] = qw; }
    }
    asm volatile("bar.sync 1, %0;" ::"r"(ngw * 32) : "memory");
    if (w == 0 && lane == 0) {
        if constexpr (kInt) {
            long long N = 0, S = 0;
            unsigned long long Q = 0;
            for (int v = 0; v < ngw; ++v) { N += gc[v]; S += gs[v]; Q += gu[v]; }
            StatI *dst = reinterpret_cast<StatI *>(a.partials) + lin;
            dst->n = N; dst->sum = S; dst->sumsq = Q;
        } else {
            double N = 0, S = 0;
            for (int v = 0; v < ngw; ++v) { N += gn[v]; S += gn[v] * (double)gm[v]; }
            const double M = N > 0 ? S / N : 0.0;
            double Q = 0;
            for (int v = 0; v < ngw; ++v) {
                const double e = (double)gm[v] - M;
                Q += (double)gq[v] + gn[v] * e * e;
            }
            StatF *dst = reinterpret_cast<StatF *>(a.partials) + lin;
            dst->n = N; dst->mean = M; dst->m2 = Q;
        }
    }
}

// Registers of the warp-specialised block: a launch of T threads gets at
// most 65536 / T per thread (a multiple of 8).  When that is below what the
// stage-2 warps need (their DR x TI accumulators: kWsAccRegs), the stage-1
// warps give registers back with setmaxnreg.dec and the stage-2 warps take
// them with setmaxnreg.inc; the two shares together stay within the block's
// launch allocation (checked on the host against the compiled register count
// before the shape is used: an increase the block cannot cover would wait
// forever).
constexpr int kWsAccRegs = 168;
template <int NW, int PW>
struct WsRegs {
    static constexpr int kThreads = (NW + PW) * 32;
    static constexpr int kLaunch = (65536 / kThreads) / 8 * 8 > 255 ? 248 : (65536 / kThreads) / 8 * 8;
    static constexpr bool kSplit = kLaunch < kWsAccRegs;
    // stage-1 warps' share: what the launch leaves after the stage-2 warps' 168,
    // 8 registers short of the most that would fit (slack for the compiled count)
    static constexpr int kProd = kSplit ? ((NW + PW) * kLaunch - NW * kWsAccRegs) / PW / 8 * 8 - 8 : kLaunch;
    static_assert(!kSplit || (kProd >= 24 && kProd % 8 == 0), "stage-1 warps need at least 24 registers");
    static_assert(!kSplit || (PW % 4 == 0 && NW % 4 == 0), "setmaxnreg acts on whole warpgroups");
    // the compiled register count per thread the split needs
    static constexpr int kNeed = kSplit ? (PW * kProd + NW * kWsAccRegs + NW + PW - 1) / (NW + PW) : 0;
};

// Kernel 5, warp-specialised: the same two stages on separate warps.  Warps
// [0, PW) form subband s's partial sums (stage 1) into P slot s % PB and copy
// the block's trial offsets next to them; warps [PW, PW + NW) add slot s into
// their trials' accumulators (stage 2).  Hand-offs are mbarriers, not a block
// barrier per subband:
//   full[i]   input stage i has landed (TMA transaction bytes),
//   empty[i]  every stage-1 warp is done with input stage i,
//   pfull[b]  every stage-1 warp has written slot b,
//   pempty[b] every stage-2 warp has read slot b,
// so stage 1 runs up to PB - 1 subbands ahead of stage 2 and the two keep the
// shared-memory pipe busy together.  Lane 0 of warp 0 issues the input copies
// NS - 1 subbands ahead: at the top of subband s, those of subband s + NS - 1
// into the stage subband s - 1 used, once every stage-1 warp is done with it.
// One block per SM: NW * DR trials x 32 * TI samples of accumulators take
// most of the register file, the stage-1 warps the rest.
// Every wait is bounded; a warp whose wait gives up stops, the others then
// give up on theirs, and the issuing thread waits (bounded) for its copies
// still in flight before it returns.
template <typename Tin, bool kInt, int TI, int DR, int NW, int PW, int CS, int NPMAX, int NS, int PB>
__global__ void __launch_bounds__((NW + PW) * 32, 1) share_ws_kernel(ShareLaunch a)
{
    using Regs = WsRegs<NW, PW>;
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int kDmBlk = DR * NW;
    using R = ShareRec<CS, NPMAX, kDmBlk>;
    static_assert(NS >= 2 && PB >= 2, "input ring and slot ring need two entries");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rs = a.rs, nsub = a.nsub;

    // layout: [NS][CS][rs] Tin rows | [NS][kLen] int32 records |
    //         [PB] slots {int32 q[kDmBlk], float P[pmax]} | mbarriers at bar_off
    const size_t stage_elems = (size_t)CS * rs;
    Tin *rows = reinterpret_cast<Tin *>(smem);
    int32_t *srec = reinterpret_cast<int32_t *>(smem + NS * stage_elems * sizeof(Tin));
    int32_t *slots = srec + NS * R::kLen;
    const size_t slot_len = (size_t)kDmBlk + a.pmax;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + a.bar_off);
    uint64_t *empty = full + NS, *pfull = full + 2 * NS, *pempty = full + 2 * NS + PB;
    if (tid == 0) {
        for (int i = 0; i < NS; ++i) { mbar_init(&full[i], 1); mbar_init(&empty[i], PW); }
        for (int b = 0; b < PB; ++b) { mbar_init(&pfull[b], PW); mbar_init(&pempty[b], NW); }
        mbar_fence_init();
    }
    __syncthreads();
    int blk;
    int64_t t0;
    share_raster<TI>(a, blockIdx.x, blk, t0);
    t0 += a.t_base;

    if (warp < PW) {
        // ---- stage 1 (and the input copies)
        if constexpr (Regs::kSplit) asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(Regs::kProd));
        const Tin *__restrict__ in = static_cast<const Tin *>(a.in);
        const int32_t *brec = a.rec + (size_t)blk * nsub * R::kLen;
        const int32_t *bbase = a.base + (size_t)blk * a.nchans;
        const int32_t *blen = a.rlen + (size_t)blk * a.nchans;
        auto row_bytes = [&](int b, int rl, int64_t &g) -> uint32_t {
            g = t0 + b;
            int64_t n = a.nsamp_in_al - g;
            n = n < 0 ? 0 : (n > rl ? rl : n);
            return (uint32_t)(n * (int64_t)sizeof(Tin));
        };
        int rb[CS], rl[CS];
        auto load_rb = [&](int s) {
#pragma unroll
            for (int cc = 0; cc < CS; ++cc) { rb[cc] = bbase[s * CS + cc]; rl[cc] = blen[s * CS + cc]; }
        };
        auto issue = [&](int s) {
            const int buf = s % NS;
            uint32_t bytes = (uint32_t)(R::kLen * sizeof(int32_t));
#pragma unroll
            for (int cc = 0; cc < CS; ++cc) { int64_t g; bytes += row_bytes(rb[cc], rl[cc], g); }
            mbar_arrive_tx(&full[buf], bytes);
            bulk_g2s(srec + (size_t)buf * R::kLen, brec + (size_t)s * R::kLen, (uint32_t)(R::kLen * sizeof(int32_t)),
                     &full[buf]);
            const uint64_t pol = l2_evict_last();
#pragma unroll
            for (int cc = 0; cc < CS; ++cc) {
                int64_t g;
                const uint32_t nb = row_bytes(rb[cc], rl[cc], g);
                if (nb)
                    bulk_g2s_hint(rows + (size_t)buf * stage_elems + (size_t)cc * rs,
                                  in + (size_t)(s * CS + cc) * a.pitch + g, nb, &full[buf], pol);
            }
        };
        int issued = 0;   // copies issued (thread 0)
        if (tid == 0) {
            for (; issued < NS - 1 && issued < nsub; ++issued) { load_rb(issued); issue(issued); }
            if (issued < nsub) load_rb(issued);
        }
        bool ok = true;
        int s = 0;
        for (; s < nsub; ++s) {
            if (warp == 0) {
                // refill the stage subband s - 1 used once every stage-1 warp is done with it
                bool go = true;
                if (lane == 0 && issued < nsub) {
                    if (s >= 1) go = mbar_wait(&empty[(s - 1) % NS], (uint32_t)(((s - 1) / NS) & 1), a.err);
                    if (go) {
                        issue(issued);
                        ++issued;
                        if (issued < nsub) load_rb(issued);
                    }
                }
                ok = __shfl_sync(0xffffffffu, go ? 1 : 0, 0) != 0;
            }
            const int pb = s % PB, ib = s % NS;
            if (ok && s >= PB) ok = mbar_wait(&pempty[pb], (uint32_t)(((s / PB) - 1) & 1), a.err);
            if (ok) ok = mbar_wait(&full[ib], (uint32_t)((s / NS) & 1), a.err);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            const int32_t *rec = srec + (size_t)ib * R::kLen;
            int32_t *slot = slots + (size_t)pb * slot_len;
            // whole rows 8 per step (no accumulators here), leftovers 4 per step
            share_stage1<Tin, R, CS, PW, 8, 4>(rec, rows + (size_t)ib * stage_elems,
                                               reinterpret_cast<float *>(slot + kDmBlk), warp, lane);
            if (warp == PW - 1)
                for (int j = lane; j < kDmBlk; j += 32) slot[j] = rec[R::kTrial + j];
            __syncwarp();
            if (lane == 0) { mbar_arrive(&pfull[pb]); mbar_arrive(&empty[ib]); }
        }
        // after a wait gave up: let the copies still in flight land before leaving
        if (tid == 0)
            for (int u = s; u < issued; ++u) mbar_wait(&full[u % NS], (uint32_t)((u / NS) & 1), a.err);
        return;
    }

    // ---- stage 2: one shared word per add
    if constexpr (Regs::kSplit) asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kWsAccRegs));
    const int cw = warp - PW;
    float acc[DR][TI];
#pragma unroll
    for (int j = 0; j < DR; ++j)
#pragma unroll
        for (int i = 0; i < TI; ++i) acc[j][i] = 0.f;
    bool ok = true;
    for (int s = 0; s < nsub; ++s) {
        const int pb = s % PB;
        ok = __all_sync(0xffffffffu, mbar_wait(&pfull[pb], (uint32_t)((s / PB) & 1), a.err));
        if (!ok) break;
        const int32_t *slot = slots + (size_t)pb * slot_len;
        const float *Pb = reinterpret_cast<const float *>(slot + kDmBlk);
        int q[DR];
#pragma unroll
        for (int j = 0; j < DR; j += 4) {
            const int4 v = *reinterpret_cast<const int4 *>(slot + cw * DR + j);
            q[j] = v.x; q[j + 1] = v.y; q[j + 2] = v.z; q[j + 3] = v.w;
        }
#pragma unroll
        for (int j = 0; j < DR; ++j) {
            const float *pp = Pb + q[j] + lane;
#pragma unroll
            for (int i = 0; i < TI; ++i) acc[j][i] += pp[32 * i];
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&pempty[pb]);
    }
    ShareStat<kInt> st;
    if (ok) share_store<kInt, TI, DR>(a, acc, blk * kDmBlk + cw * DR, t0, lane, st);
    group_stat_flush<kInt>(a, st, blockIdx.x, PW, NW);
}

// Compiled shapes: subbands of 4 channels, at most 16 patterns per (block,
// subband); {samples per lane, DM trials per warp, warps (stage-2 warps in
// the warp-specialised form), resident blocks per SM the register budget
// targets, input stages, stage-1 warps (0: the one-barrier-per-subband
// kernel, whose warps do both stages), partial-sum slots, stage-1 rows of
// warp 0 in percent of another warp's (its first thread issues the input
// copies, which hold it for ~1000 cycles per subband: a smaller share keeps
// it from being the last one at each subband's barrier or hand-off)}.
constexpr int kShCS = 4, kShNP = 16;
struct ShareShape { int ti, dr, nw, minb, ns, pw, pb, w0; };
constexpr int kNumShareCfg = 4;
constexpr ShareShape kShareCfg[kNumShareCfg] = {
    {16, 8, 4, 3, 2, 0, 2, 70}, {8, 8, 4, 5, 2, 0, 2, 70}, {16, 8, 6, 2, 2, 0, 2, 70}, {16, 8, 8, 1, 3, 8, 3, 50}};
template <int DB>
using ShareRecDB = ShareRec<kShCS, kShNP, DB>;

cudaError_t share_launch(int k, dd_dtype t, const ShareLaunch &a, cudaStream_t s);
cudaError_t share_prepare(int k, size_t optin);
// false if shape k's kernels were compiled with fewer registers than its
// register split needs (the shape is then not used)
bool share_regs_ok(int k);
// Mixed persistent batch of kernel 5 shape 0 and kernel 3 shape 2 (the same
// block geometry): grid = sms * that shape's resident blocks per SM.
cudaError_t mixed_batch_launch(const LaneBatchLaunch &b, int sms, size_t smem, cudaStream_t s);
cudaError_t mixed_batch_prepare(size_t optin);
int mixed_batch_occupancy(size_t smem);   // resident blocks per SM with `smem` dynamic bytes
constexpr int kMixedLane = 2, kMixedShare = 0;

}  // namespace dd
