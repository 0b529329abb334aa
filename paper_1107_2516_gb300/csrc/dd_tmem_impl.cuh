// Kernel 4: brute-force de-dispersion (Section 3.1) through tensor memory,
//   out[dm][t] = sum_c in[c][t + d(c,dm)].
//
// Kernel 3 loads one shared-memory word per add and is capped by the
// shared-memory data path (32 words/clk/SM, a quarter of the FP32 add rate).
// Reuse needs a dynamically indexable per-thread window, which registers are
// not; TMEM is: a tcgen05.ld reads any (warp-uniform) column offset of the
// 32 TMEM lanes a warp owns.
//
// Block = NW warps on one time tile of 32*N samples; lane l owns the N
// consecutive outputs t0 + N*l .. +N-1, warp w the DM trials w*DBW .. +DBW
// of the block's NW*DBW.  Per channel c each warp
//   fill:  copies its window in[c][t0 + row0 + wbase + N*l + k], k < 8*kc8,
//          shared -> registers -> TMEM (its lanes, its column range; row0 =
//          the block's smallest delay, wbase = the warp's smallest delay above
//          it; N = 4 mod 8 makes the lanes' vector loads conflict-free);
//   read:  for each trial j, a tcgen05.ld of N columns at the offset
//          d(c,dm_j) - row0 - wbase gives in[c][t + d(c,dm_j)] for the lane's
//          N outputs, added into registers.
// One staged word serves DBW adds: shared-memory words per add drop to
// (span + N) / (N * DBW), span = the warp's delay spread at channel c.  The
// window is double-buffered in TMEM (channel parity) and the loads are
// software-pipelined (the next batch of trials is in flight while the
// previous one is added).  The TMA stage ring of input rows is the one of
// kernels 2 and 3.
//
// Measured on GB300 this kernel is slower than kernel 3: the TMEM fill
// (tcgen05.st) and the load round trip leave it latency-bound at the two
// warps per scheduler that its accumulators allow.
#pragma once

#include "dd_fast_impl.cuh"

namespace dd {

struct TmemLaunch {
    const void *in;
    int64_t pitch, nsamp_in_al;
    int nchans, ndm;
    int64_t nout;
    const int32_t *tab;    // [nblk][nchans][dbp]: per warp {wbase, kc8, DBW column offsets}
    const int32_t *base;   // [nblk][nchans] row0 relative to the tile start (aligned)
    int rs, ch, bar_off, nblk, dbp, wmax;
    int64_t ntile;
    int dgroup;
    void *out, *partials;
    int *err;
    size_t smem;
};

// ------------------------------------------------------------- TMEM helpers
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// 8 columns of this thread's TMEM lane from 8 floats
__device__ __forceinline__ void tc_st8(uint32_t taddr, const float (&w)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
                 ::"r"(taddr), "f"(w[0]), "f"(w[1]), "f"(w[2]), "f"(w[3]),
                   "f"(w[4]), "f"(w[5]), "f"(w[6]), "f"(w[7])
                 : "memory");
}

__device__ __forceinline__ void tc_ld4(uint32_t taddr, float *v)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
                 : "r"(taddr));
}

__device__ __forceinline__ void tc_ld8(uint32_t taddr, float *v)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]),
                   "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
                 : "r"(taddr));
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, float *v)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]),
                   "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]),
                   "=f"(v[8]), "=f"(v[9]), "=f"(v[10]), "=f"(v[11]),
                   "=f"(v[12]), "=f"(v[13]), "=f"(v[14]), "=f"(v[15])
                 : "r"(taddr));
}

// N consecutive columns (N a multiple of 4) as x16 / x8 / x4 pieces
template <int N>
__device__ __forceinline__ void tc_ldn(uint32_t taddr, float (&v)[N])
{
    static_assert(N % 4 == 0, "TMEM read width");
#pragma unroll
    for (int k = 0; k + 16 <= N; k += 16) tc_ld16(taddr + k, v + k);
    constexpr int r = N % 16;
    if constexpr (r >= 8) tc_ld8(taddr + (N - r), v + (N - r));
    if constexpr (r % 8 == 4) tc_ld4(taddr + (N - 4), v + (N - 4));
}

// ------------------------------------------------------------------ kernel
// Completion wait for one batch of TMEM loads; the batch's registers are
// in-out operands so no use of them can be scheduled before the wait.
template <int M>
__device__ __forceinline__ void tc_wait_ld_regs(float (&v)[M])
{
    static_assert(M % 4 == 0 && M <= 64, "wait operand count");
#pragma unroll
    for (int k = 0; k < M; k += 4) {
        if (k == 0)
            asm volatile("tcgen05.wait::ld.sync.aligned;" : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3]) :: "memory");
        else
            asm volatile("" : "+f"(v[k]), "+f"(v[k + 1]), "+f"(v[k + 2]), "+f"(v[k + 3]) :: "memory");
    }
}

template <typename Tin, bool kInt, int N, int DBW, int NW, int TPW>
__global__ void __launch_bounds__(32 * NW, 1) tmem_kernel(TmemLaunch a)
{
    static_assert(N % 8 == 4, "N = 4 mod 8 keeps the lanes' window loads conflict-free");
    static_assert(DBW % TPW == 0 && (DBW / TPW) % 2 == 0, "an even number of load batches per channel");
    static_assert(NW == 4 || NW == 8 || NW == 16, "warps per block");
    constexpr int kTile = 32 * N, kDmBlk = DBW * NW;
    constexpr int kColsWarp = 512 / (NW / 4);     // TMEM columns of one warp (its lane quarter is shared)
    constexpr int kBuf = kColsWarp / 2;            // double buffer
    constexpr int kRec = DBW + 2;                  // per warp: wbase, kc8, DBW offsets
    constexpr int kNB = DBW / TPW;                 // load batches per channel
    extern __shared__ __align__(128) unsigned char smem[];
    const Tin *__restrict__ in = static_cast<const Tin *>(a.in);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nchans = a.nchans, rs = a.rs, ch = a.ch, dbp = a.dbp;

    // raster: DM blocks in groups, time tiles slowest within a group
    const int64_t lin = blockIdx.x;
    const int64_t per_group = (int64_t)a.dgroup * a.ntile;
    const int64_t grp = lin / per_group;
    const int64_t rr = lin - grp * per_group;
    const int gsize = min(a.dgroup, a.nblk - (int)grp * a.dgroup);
    const int blk = (int)grp * a.dgroup + (int)(rr % gsize);
    const int64_t t0 = (rr / gsize) * kTile;
    const int dm0 = blk * kDmBlk + warp * DBW;

    // layout: [kStages][ch][rs] Tin rows | [kStages][ch][dbp] int32 | mbarriers | TMEM address
    const size_t stage_elems = (size_t)ch * rs;
    Tin *rows = reinterpret_cast<Tin *>(smem);
    int32_t *stab = reinterpret_cast<int32_t *>(smem + kStages * stage_elems * sizeof(Tin));
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + a.bar_off);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + a.bar_off + kStages * sizeof(uint64_t));
    const int32_t *btab = a.tab + (size_t)blk * nchans * dbp;
    const int32_t *bbase = a.base + (size_t)blk * nchans;
    const int nst = (nchans + ch - 1) / ch;

    if (warp == 0) {
        // one block per SM (shared memory + registers): all 512 columns
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;"
                     ::"r"(smem_addr(tslot)) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
        mbar_fence_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t twarp = *tslot + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * kColsWarp);

    auto row_bytes = [&](int c, int64_t &g) -> uint32_t {
        g = t0 + bbase[c];
        int64_t n = a.nsamp_in_al - g;
        n = n < 0 ? 0 : (n > rs ? rs : n);
        return (uint32_t)(n * (int64_t)sizeof(Tin));
    };
    auto issue = [&](int s) {
        const int buf = s % kStages;
        const int c0 = s * ch;
        const int cn = min(ch, nchans - c0);
        uint32_t bytes = (uint32_t)(cn * dbp * sizeof(int32_t));
        for (int cc = 0; cc < cn; ++cc) { int64_t g; bytes += row_bytes(c0 + cc, g); }
        mbar_arrive_tx(&bar[buf], bytes);
        bulk_g2s(stab + (size_t)buf * ch * dbp, btab + (size_t)c0 * dbp,
                 (uint32_t)(cn * dbp * sizeof(int32_t)), &bar[buf]);
        for (int cc = 0; cc < cn; ++cc) {
            int64_t g;
            const uint32_t nb = row_bytes(c0 + cc, g);
            if (nb)
                bulk_g2s(rows + (size_t)buf * stage_elems + (size_t)cc * rs,
                         in + (size_t)(c0 + cc) * a.pitch + g, nb, &bar[buf]);
        }
    };
    if (tid == 0)
        for (int s = 0; s < kStages && s < nst; ++s) issue(s);

    float acc[DBW][N];
#pragma unroll
    for (int j = 0; j < DBW; ++j)
#pragma unroll
        for (int i = 0; i < N; ++i) acc[j][i] = 0.f;

    const int lrow = lane * N;          // this lane's window start relative to the warp base
    int ocur[DBW], onext[DBW];
    bool ok = true;

    // Copy channel n's window (this warp's trials) into TMEM buffer n&1 and
    // fetch its column offsets; releases the stage after its last channel.
    auto fill = [&](int n) {
        const int S = n / ch, cc = n - S * ch, buf = S % kStages;
        if (cc == 0 && ok) ok = mbar_wait(&bar[buf], (uint32_t)((S / kStages) & 1), a.err);
        const int32_t *tb = stab + ((size_t)buf * ch + cc) * dbp + warp * kRec;
        const int wbase = tb[0], kc8 = tb[1];
#pragma unroll
        for (int j = 0; j < DBW; ++j) onext[j] = tb[2 + j];
        const Tin *row = rows + (size_t)buf * stage_elems + (size_t)cc * rs + wbase + lrow;
        const uint32_t tcol = twarp + (uint32_t)((n & 1) * kBuf);
        for (int k = 0; k < kc8; ++k) {
            float w[8];
            Win<Tin>::template load<8>(w, row + 8 * k);
            tc_st8(tcol + 8 * k, w);
        }
    };
    auto release = [&](int n) {
        if (n % ch == ch - 1 || n == nchans - 1) {
            __syncthreads();
            const int S = n / ch + kStages;
            if (tid == 0 && S < nst) issue(S);
        }
    };
    auto ld_batch = [&](int c, int b, float (&v)[TPW][N]) {
        const uint32_t tcol = twarp + (uint32_t)((c & 1) * kBuf);
#pragma unroll
        for (int jj = 0; jj < TPW; ++jj) tc_ldn<N>(tcol + ocur[b * TPW + jj], v[jj]);
    };
    auto add_batch = [&](int b, float (&v)[TPW][N]) {
#pragma unroll
        for (int jj = 0; jj < TPW; ++jj)
#pragma unroll
            for (int i = 0; i < N; ++i) acc[b * TPW + jj][i] += v[jj][i];
    };

    // prologue: channel 0 in TMEM, its first batch in flight
    fill(0);
    tc_wait_st();
    release(0);
#pragma unroll
    for (int j = 0; j < DBW; ++j) ocur[j] = onext[j];
    float va[TPW][N], vb[TPW][N];
    ld_batch(0, 0, va);

    // pipeline: the next load batch is in flight while the previous one is added
    for (int c = 0; c < nchans; ++c) {
        const bool more = c + 1 < nchans;
#pragma unroll
        for (int b = 0; b < kNB; b += 2) {
            tc_wait_ld_regs<TPW * N>(reinterpret_cast<float (&)[TPW * N]>(va));
            ld_batch(c, b + 1, vb);
            if (b == 0 && more) fill(c + 1);
            add_batch(b, va);
            tc_wait_ld_regs<TPW * N>(reinterpret_cast<float (&)[TPW * N]>(vb));
            if (b + 2 < kNB) {
                ld_batch(c, b + 2, va);
            } else if (more) {
                tc_wait_st();
#pragma unroll
                for (int j = 0; j < DBW; ++j) ocur[j] = onext[j];
                ld_batch(c + 1, 0, va);
            }
            add_batch(b + 1, vb);
        }
        if (more) release(c + 1);
    }

    tc_fence_before();
    ok = __syncthreads_and(ok);
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(*tslot) : "memory");
    if (!ok) return;

    // epilogue: lane l holds outputs t0 + N*l .. +N-1 of the warp's DBW trials
    const int64_t nout = a.nout;
    const int64_t tl = t0 + lrow;
    if constexpr (kInt) {
        long long cnt = 0, s = 0;
        unsigned long long qq = 0;
        int32_t *out = reinterpret_cast<int32_t *>(a.out);
#pragma unroll
        for (int j = 0; j < DBW; ++j) {
            const int dm = dm0 + j;
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const int64_t t = tl + i;
                if (dm < a.ndm && t < nout) {
                    const long long v = __float2int_rn(acc[j][i]);
                    out[(size_t)dm * nout + t] = (int32_t)v;
                    cnt++; s += v; qq += (unsigned long long)(v * v);
                }
            }
        }
        block_stat_i(cnt, s, qq, reinterpret_cast<StatI *>(a.partials) + lin);
    } else {
        int cnt = 0;
        float s = 0.f;
        float *out = reinterpret_cast<float *>(a.out);
#pragma unroll
        for (int j = 0; j < DBW; ++j) {
            const int dm = dm0 + j;
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const int64_t t = tl + i;
                if (dm < a.ndm && t < nout) {
                    out[(size_t)dm * nout + t] = acc[j][i];
                    cnt++; s += acc[j][i];
                }
            }
        }
        const float mean = cnt ? s / (float)cnt : 0.f;
        float qq = 0.f;
#pragma unroll
        for (int j = 0; j < DBW; ++j) {
            const int dm = dm0 + j;
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const int64_t t = tl + i;
                if (dm < a.ndm && t < nout) { const float d = acc[j][i] - mean; qq += d * d; }
            }
        }
        block_stat_f32(cnt, s, qq, reinterpret_cast<StatF *>(a.partials) + lin);
    }
}

template <int N, int DBW, int NW, int TPW>
cudaError_t tmem_launch_cfg(dd_dtype t, const TmemLaunch &a, cudaStream_t s)
{
    const unsigned grid = (unsigned)(a.ntile * a.nblk);
    switch (t) {
    case DD_F32: tmem_kernel<float, false, N, DBW, NW, TPW><<<grid, 32 * NW, a.smem, s>>>(a); break;
    case DD_F16: tmem_kernel<__half, false, N, DBW, NW, TPW><<<grid, 32 * NW, a.smem, s>>>(a); break;
    case DD_U8: tmem_kernel<uint8_t, true, N, DBW, NW, TPW><<<grid, 32 * NW, a.smem, s>>>(a); break;
    }
    return cudaGetLastError();
}

template <int N, int DBW, int NW, int TPW>
cudaError_t tmem_prepare_cfg(size_t optin)
{
    cudaError_t e = allow_max_dynamic_smem((const void *)tmem_kernel<float, false, N, DBW, NW, TPW>, optin);
    if (e == cudaSuccess)
        e = allow_max_dynamic_smem((const void *)tmem_kernel<__half, false, N, DBW, NW, TPW>, optin);
    if (e == cudaSuccess)
        e = allow_max_dynamic_smem((const void *)tmem_kernel<uint8_t, true, N, DBW, NW, TPW>, optin);
    return e;
}

// Configurations compiled into the library: {outputs per lane, DM trials per
// warp, warps per block, trials per TMEM load batch}.
struct TmemShape { int n, dbw, nw, tpw; };
constexpr int kNumTmemCfg = 2;
constexpr TmemShape kTmemCfg[kNumTmemCfg] = {{20, 4, 8, 2}, {12, 8, 8, 4}};

cudaError_t tmem_launch_c0(dd_dtype t, const TmemLaunch &a, cudaStream_t s);
cudaError_t tmem_launch_c1(dd_dtype t, const TmemLaunch &a, cudaStream_t s);
cudaError_t tmem_prepare_c0(size_t optin);
cudaError_t tmem_prepare_c1(size_t optin);

}  // namespace dd
