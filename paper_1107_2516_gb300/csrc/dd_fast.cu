// Kernel 2 host side: per-plan tables for each compiled tile configuration,
// launch, and the autotuner that picks (configuration, raster group) by
// timing them on the caller's data.
#include "dd_fast_impl.cuh"
#include "dd_lane_impl.cuh"
#include "dd_tmem_impl.cuh"
#include "dd_share_impl.cuh"

#include <algorithm>
#include <climits>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <array>

namespace dd {

struct FastCfgData {
    bool ok = false;
    int tr = 0, nw = 0;
    int nblk = 0;                // DM blocks of 4*nw trials
    int rs = 0;                  // shared row stride in elements (multiple of 16)
    int ch = 0;                  // channels per stage
    int bar_off = 0;             // byte offset of the stage mbarriers
    size_t smem = 0;
    uint32_t *d_desc = nullptr;  // [nblk][nchans][nw] packed window descriptors
    int32_t *d_base = nullptr;   // [nblk][nchans] row start relative to the tile start (aligned)
    int32_t *d_goff = nullptr;   // [nblk][nchans][nw][4] fallback offsets (elements)
    double last_ms = -1.0;       // autotuner timing
};

struct LaneCfgData {
    bool ok = false;
    int ti = 0, dr = 0, nw = 0;
    int nblk = 0, rs = 0, ch = 0, bar_off = 0;
    int64_t reach = 0;           // input columns a tile at t0 reads lie below t0 + reach
    size_t smem = 0;
    int32_t *d_offs = nullptr;   // [nblk][nchans][nw*dr] offsets within the staged row
    int32_t *d_base = nullptr;   // [nblk][nchans] row start relative to the tile start
};

struct TmemCfgData {
    bool ok = false;
    int n = 0, dbw = 0, nw = 0;
    int nblk = 0, rs = 0, ch = 0, bar_off = 0, dbp = 0, wmax = 0;
    size_t smem = 0;
    int32_t *d_tab = nullptr;    // [nblk][nchans][dbp] per-warp window records
    int32_t *d_base = nullptr;   // [nblk][nchans] row start relative to the tile start
};

struct ShareCfgData {
    bool ok = false;
    int nblk = 0, nsub = 0, rs = 0, pmax = 0, bar_off = 0;
    int64_t reach = 0;           // input columns a tile at t0 reads lie below t0 + reach
    size_t smem = 0;
    int32_t *d_rec = nullptr;    // [nblk][nsub][kLen] subband records
    int32_t *d_base = nullptr;   // [2][nblk][nchans] staged row starts, then staged row lengths
};

// Tile configurations: indices [0, kNumFastCfg) are kernel 2 shapes,
// [kNumFastCfg, kLaneEnd) kernel 3 shapes, [kLaneEnd, kShareBeg) kernel 4,
// [kShareBeg, kNumAllCfg) kernel 5.
constexpr int kLaneEnd = kNumFastCfg + kNumLaneCfg;
constexpr int kShareBeg = kLaneEnd + kNumTmemCfg;
constexpr int kNumAllCfg = kShareBeg + kNumShareCfg;

constexpr int kHostChunks = 8;   // input column chunks of the pipelined host path

struct FastPlan {
    FastCfgData cfg[kNumFastCfg];
    LaneCfgData lane[kNumLaneCfg];
    TmemCfgData tm[kNumTmemCfg];
    ShareCfgData sh[kNumShareCfg];
    int active = -1;
    int dgroup = 8;
    int al = 4;                  // row alignment in elements (16 bytes)
    int *d_err = nullptr;
    // dd_process_host's pipelined input copy (created on first use)
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t copy_ev[kHostChunks + 1] = {};
};

static int elem_align(dd_dtype t) { return (int)(16 / in_elem_bytes(t)); }

static cudaError_t launch_cfg(int k, dd_dtype t, const FastLaunch &a, cudaStream_t s)
{
    switch (k) {
    case 0: return fast_launch_t36w8(t, a, s);
    case 1: return fast_launch_t20w12(t, a, s);
    default: return fast_launch_t28w8(t, a, s);
    }
}

static cudaError_t prepare_cfg(int k, size_t optin)
{
    switch (k) {
    case 0: return fast_prepare_t36w8(optin);
    case 1: return fast_prepare_t20w12(optin);
    default: return fast_prepare_t28w8(optin);
    }
}

static cudaError_t launch_lane(int k, dd_dtype t, const LaneLaunch &a, cudaStream_t s)
{
    switch (k) {
    case 0: return lane_launch_c0(t, a, s);
    case 1: return lane_launch_c1(t, a, s);
    case 2: return lane_launch_c2(t, a, s);
    default: return lane_launch_c3(t, a, s);
    }
}

static cudaError_t prepare_lane(int k, size_t optin)
{
    switch (k) {
    case 0: return lane_prepare_c0(optin);
    case 1: return lane_prepare_c1(optin);
    case 2: return lane_prepare_c2(optin);
    default: return lane_prepare_c3(optin);
    }
}

static void free_lane(LaneCfgData &c)
{
    if (c.d_offs) cudaFree(c.d_offs);
    if (c.d_base) cudaFree(c.d_base);
    c.d_offs = nullptr; c.d_base = nullptr;
    c.ok = false;
}

// Kernel 3 tables: per (DM block, channel) the aligned row start and every
// DM trial's offset in the row.  c.ok stays false if rows do not fit.
static int build_lane(const dd_plan *p, int ti, int dr, int nw, int minb, LaneCfgData &c)
{
    c = LaneCfgData();
    c.ti = ti; c.dr = dr; c.nw = nw;
    const int C = p->nchans, D = p->ndm, DB = dr * nw;
    const int nblk = (D + DB - 1) / DB;
    const int AL = elem_align(p->dtype);
    std::vector<int32_t> offs((size_t)nblk * C * DB), base((size_t)nblk * C);
    long long need = 0;
    for (int b = 0; b < nblk; ++b)
        for (int ch = 0; ch < C; ++ch) {
            int lo = INT_MAX, hi = 0;
            for (int j = 0; j < DB; ++j) {
                const int d = p->delays[(size_t)std::min(b * DB + j, D - 1) * C + ch];
                lo = std::min(lo, d); hi = std::max(hi, d);
            }
            const int row0 = lo - (lo % AL);
            base[(size_t)b * C + ch] = row0;
            for (int j = 0; j < DB; ++j)
                offs[((size_t)b * C + ch) * DB + j] = p->delays[(size_t)std::min(b * DB + j, D - 1) * C + ch] - row0;
            need = std::max<long long>(need, (long long)(hi - row0) + 32LL * ti);
        }
    const int rs = (int)((need + 15) / 16 * 16);
    const size_t eb = in_elem_bytes(p->dtype);
    // shared memory of one block: the SM's 228 KB split between `minb` resident blocks
    const size_t budget = std::min<size_t>(p->smem_optin, (228 * 1024) / (size_t)minb - 1024) - 1024;
    const size_t per_ch = (size_t)rs * eb + DB * sizeof(int32_t);
    const int ch = (int)std::min<size_t>(16, budget / (kStages * per_ch));
    if (ch < 1) return DD_OK;
    c.bar_off = (int)(((size_t)kStages * ch * per_ch + 15) / 16 * 16);
    c.smem = (size_t)c.bar_off + kStages * sizeof(uint64_t);
    c.reach = (int64_t)*std::max_element(base.begin(), base.end()) + rs;
    c.nblk = nblk; c.rs = rs; c.ch = ch;
    cudaError_t e = cudaMalloc(&c.d_offs, offs.size() * 4);
    if (e == cudaSuccess) e = cudaMalloc(&c.d_base, base.size() * 4);
    if (e == cudaSuccess) e = cudaMemcpy(c.d_offs, offs.data(), offs.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c.d_base, base.data(), base.size() * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { free_lane(c); return cuda_fail(e, "kernel 3 tables"); }
    c.ok = true;
    return DD_OK;
}

static cudaError_t launch_tmem(int k, dd_dtype t, const TmemLaunch &a, cudaStream_t s)
{
    return k == 0 ? tmem_launch_c0(t, a, s) : tmem_launch_c1(t, a, s);
}

static cudaError_t prepare_tmem(int k, size_t optin)
{
    return k == 0 ? tmem_prepare_c0(optin) : tmem_prepare_c1(optin);
}

static void free_tmem(TmemCfgData &c)
{
    if (c.d_tab) cudaFree(c.d_tab);
    if (c.d_base) cudaFree(c.d_base);
    c.d_tab = nullptr; c.d_base = nullptr;
    c.ok = false;
}

// Kernel 4 tables.  Per (DM block, channel): the block's aligned row start
// (base), and per warp {wbase, kc8, DBW column offsets}: the warp's window
// starts wbase elements into the staged row (a multiple of 4), spans 8*kc8
// columns, and trial j reads columns offs[j] .. offs[j]+N-1 of it.  c.ok
// stays false if a window exceeds the warp's TMEM buffer or the rows do not
// fit in shared memory.
static int build_tmem(const dd_plan *p, int n, int dbw, int nw, TmemCfgData &c)
{
    c = TmemCfgData();
    c.n = n; c.dbw = dbw; c.nw = nw;
    const int C = p->nchans, D = p->ndm, DB = dbw * nw;
    const int nblk = (D + DB - 1) / DB;
    const int AL = elem_align(p->dtype);
    const int rec = dbw + 2;
    const int dbp = (nw * rec + 3) / 4 * 4;
    const int kbuf = 512 / (nw / 4) / 2;           // TMEM columns of one window buffer
    std::vector<int32_t> tab((size_t)nblk * C * dbp, 0), base((size_t)nblk * C);
    auto dl = [&](int dm, int ch) { return p->delays[(size_t)std::min(dm, D - 1) * C + ch]; };
    long long need = 0;
    int wmax = 0;
    for (int b = 0; b < nblk; ++b)
        for (int ch = 0; ch < C; ++ch) {
            int lo = INT_MAX;
            for (int j = 0; j < DB; ++j) lo = std::min(lo, dl(b * DB + j, ch));
            const int row0 = lo - (lo % AL);
            base[(size_t)b * C + ch] = row0;
            for (int w = 0; w < nw; ++w) {
                int wlo = INT_MAX, whi = 0;
                for (int j = 0; j < dbw; ++j) {
                    const int d = dl(b * DB + w * dbw + j, ch) - row0;
                    wlo = std::min(wlo, d); whi = std::max(whi, d);
                }
                const int wbase = wlo - (wlo % 4);
                const int kc8 = (whi - wbase + n + 7) / 8;
                int32_t *t = &tab[((size_t)b * C + ch) * dbp + (size_t)w * rec];
                t[0] = wbase; t[1] = kc8;
                for (int j = 0; j < dbw; ++j) t[2 + j] = dl(b * DB + w * dbw + j, ch) - row0 - wbase;
                wmax = std::max(wmax, 8 * kc8);
                need = std::max<long long>(need, (long long)wbase + 31LL * n + 8LL * kc8);
            }
        }
    if (wmax > kbuf) return DD_OK;
    const int rs = (int)((need + 15) / 16 * 16);
    const size_t eb = in_elem_bytes(p->dtype);
    const size_t budget = std::min<size_t>(p->smem_optin, 227 * 1024) - 1024 - 64;
    const size_t per_ch = (size_t)rs * eb + (size_t)dbp * sizeof(int32_t);
    const int ch = (int)std::min<size_t>(16, budget / (kStages * per_ch));
    if (ch < 1) return DD_OK;
    c.bar_off = (int)(((size_t)kStages * ch * per_ch + 15) / 16 * 16);
    c.smem = (size_t)c.bar_off + kStages * sizeof(uint64_t) + 16;
    // more than half of the SM's shared memory: one block (and one 512-column
    // TMEM allocation) per SM
    c.smem = std::max<size_t>(c.smem, std::min<size_t>(p->smem_optin, 120 * 1024));
    c.nblk = nblk; c.rs = rs; c.ch = ch; c.dbp = dbp; c.wmax = wmax;
    cudaError_t e = cudaMalloc(&c.d_tab, tab.size() * 4);
    if (e == cudaSuccess) e = cudaMalloc(&c.d_base, base.size() * 4);
    if (e == cudaSuccess) e = cudaMemcpy(c.d_tab, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c.d_base, base.data(), base.size() * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { free_tmem(c); return cuda_fail(e, "kernel 4 tables"); }
    c.ok = true;
    return DD_OK;
}

static void free_share(ShareCfgData &c)
{
    if (c.d_rec) cudaFree(c.d_rec);
    if (c.d_base) cudaFree(c.d_base);
    c.d_rec = nullptr; c.d_base = nullptr;
    c.ok = false;
}

// Kernel 5 tables.  Per (DM block, subband of kShCS channels): the trials'
// relative delays r(c) = d(c,dm) - d(ref,dm) (ref = the subband's highest
// frequency) grouped into patterns; per pattern the range of P samples its
// trials need and where they sit in the packed P buffer; per trial the index
// of its t = t0 term.  c.ok stays false when the channel count is not a
// multiple of kShCS, a (block, subband) has more than kShNP patterns, or the
// buffers do not fit three blocks per SM.
// Kernel 5's tables of shape k for a delay table [D][C] (host only): per
// (DM block, subband) record (layout of ShareRec) and per (DM block, channel)
// staged row start; T.ok stays false if a (block, subband) has more than
// kShNP delay patterns.
struct ShareTables {
    std::vector<int32_t> rec, base;   // base: [2][nblk][nchans] row starts, then row lengths
    int nblk = 0, nsub = 0, rs = 0, pmax = 0, klen = 0;
    bool ok = false;
};

template <int DB>
static void share_tables_db(const int32_t *delays, int D, int C, double foff, dd_dtype dtype, int k,
                            ShareTables &T)
{
    T = ShareTables();
    constexpr int CS = kShCS, NP = kShNP;
    // the stage-1 split goes to the warps that run stage 1 (the stage-1 warps
    // of the warp-specialised shape, else all of the block's warps)
    const int TILE = 32 * kShareCfg[k].ti, nw = kShareCfg[k].pw > 0 ? kShareCfg[k].pw : kShareCfg[k].nw;
    using R = ShareRecDB<DB>;
    if (nw > R::kMaxWarps) return;
    if (C % CS) return;
    const int S = C / CS, nblk = (D + DB - 1) / DB;
    const int AL = elem_align(dtype);
    std::vector<int32_t> rec((size_t)nblk * S * R::kLen, 0), base((size_t)2 * nblk * C);
    std::vector<int> npat((size_t)nblk * S);
    auto dl = [&](int dm, int ch) { return delays[(size_t)std::min(dm, D - 1) * C + ch]; };
    long long need = 0;
    int pmax = 0;
    for (int b = 0; b < nblk; ++b)
        for (int s = 0; s < S; ++s) {
            const int ref = foff < 0.0 ? s * CS : s * CS + CS - 1;
            int dref[DB], pid[DB];
            std::vector<std::array<int, CS>> pats;
            int dmin = INT_MAX;
            for (int j = 0; j < DB; ++j) {
                dref[j] = dl(b * DB + j, ref);
                dmin = std::min(dmin, dref[j]);
                std::array<int, CS> r;
                for (int cc = 0; cc < CS; ++cc) r[cc] = dl(b * DB + j, s * CS + cc) - dref[j];
                int q = 0;
                while (q < (int)pats.size() && pats[q] != r) ++q;
                if (q == (int)pats.size()) pats.push_back(r);
                pid[j] = q;
            }
            if ((int)pats.size() > NP) return;
            int32_t *t = &rec[((size_t)b * S + s) * R::kLen];
            int rowoff[CS];
            for (int cc = 0; cc < CS; ++cc) {
                int lo = INT_MAX, hi = 0;
                for (int j = 0; j < DB; ++j) {
                    const int d = dl(b * DB + j, s * CS + cc);
                    lo = std::min(lo, d); hi = std::max(hi, d);
                }
                const int b0 = lo - (lo % AL);
                base[(size_t)b * C + s * CS + cc] = b0;
                // elements of the row this block's trials read, a whole number of
                // 16-byte units (<= rs, which rounds the largest up to 16 elements)
                const long long nr = (long long)(hi - b0) + TILE;
                base[(size_t)nblk * C + (size_t)b * C + s * CS + cc] = (int32_t)((nr + AL - 1) / AL * AL);
                rowoff[cc] = dmin - b0;
                need = std::max<long long>(need, nr);
            }
            // patterns end to end in P; b_c without the row stride (added once rs is known)
            int poff = 0, rows = 0;
            std::vector<int> plo(pats.size()), pof(pats.size()), prow(pats.size() + 1);
            for (int q = 0; q < (int)pats.size(); ++q) {
                int lo = INT_MAX, hi = INT_MIN;
                for (int j = 0; j < DB; ++j)
                    if (pid[j] == q) { lo = std::min(lo, dref[j] - dmin); hi = std::max(hi, dref[j] - dmin); }
                const int W = hi - lo + TILE;
                int32_t *pr = t + R::kPat + q * R::kPatLen;
                pr[0] = poff + W;
                for (int cc = 0; cc < CS; ++cc) pr[1 + cc] = rowoff[cc] + lo + pats[q][cc] - poff;
                pr[R::kPatStart] = poff;
                pr[R::kPatRows] = rows;
                plo[q] = lo;
                pof[q] = poff;
                prow[q] = rows;
                poff += W;
                rows += (W + 31) / 32;
            }
            prow[pats.size()] = rows;
            // stage-1 split: warp w's first row and the pattern holding it.
            // Warp 0 (whose first thread issues the input copies and waits
            // while the copy engine takes them) gets kShareCfg[k].w0 percent
            // of another warp's share of the rows, the others equal shares.
            {
                const long long w0 = kShareCfg[k].w0, tot = w0 + 100LL * (nw - 1);
                t[R::kWarp] = 0;
                for (int w = 1; w <= nw; ++w)
                    t[R::kWarp + w] = (int)(((long long)rows * (w0 + 100LL * (w - 1)) + tot / 2) / tot);
            }
            for (int w = 0; w < nw; ++w) {
                const int r0 = t[R::kWarp + w];
                int q = 0;
                while (q + 1 < (int)pats.size() && prow[q + 1] <= r0) ++q;
                t[R::kWarp + R::kMaxWarps + 1 + w] = q;
            }
            t[R::kE] = poff;
            pmax = std::max(pmax, poff);
            npat[(size_t)b * S + s] = (int)pats.size();
            for (int j = 0; j < DB; ++j) t[R::kTrial + j] = pof[pid[j]] + (dref[j] - dmin - plo[pid[j]]);
        }
    const int rs = (int)((need + 15) / 16 * 16);
    for (size_t r = 0; r < npat.size(); ++r)
        for (int q = 0; q < npat[r]; ++q)
            for (int cc = 0; cc < CS; ++cc) rec[r * R::kLen + R::kPat + q * R::kPatLen + 1 + cc] += cc * rs;
    T.rec.swap(rec);
    T.base.swap(base);
    T.nblk = nblk; T.nsub = S; T.rs = rs; T.pmax = pmax; T.klen = R::kLen;
    T.ok = true;
}

static void share_tables(const int32_t *delays, int D, int C, double foff, dd_dtype dtype, int k, ShareTables &T)
{
    switch (kShareCfg[k].dr * kShareCfg[k].nw) {
    case 32: share_tables_db<32>(delays, D, C, foff, dtype, k, T); break;
    case 48: share_tables_db<48>(delays, D, C, foff, dtype, k, T); break;
    case 64: share_tables_db<64>(delays, D, C, foff, dtype, k, T); break;
    default: T = ShareTables(); break;
    }
}

static int build_share(const dd_plan *p, int k, ShareCfgData &c)
{
    c = ShareCfgData();
    if (!share_regs_ok(k)) return DD_OK;
    ShareTables T;
    share_tables(p->delays.data(), p->ndm, p->nchans, p->foff, p->dtype, k, T);
    if (!T.ok) return DD_OK;
    const size_t eb = in_elem_bytes(p->dtype);
    // shared memory: input stages | records | partial-sum buffers | mbarriers;
    // the shape's target blocks per SM if it fits, else fewer (>= 2).  The
    // warp-specialised shape (one block per SM): pb slots of the block's trial
    // offsets and a P buffer, and full/empty mbarriers per input stage and slot.
    const ShareShape &sh = kShareCfg[k];
    const int nis = sh.ns, minb = sh.minb;
    const int pm4 = (T.pmax + 3) / 4 * 4;
    const size_t rows_b = (size_t)nis * kShCS * T.rs * eb, rec_b = (size_t)nis * T.klen * 4;
    const size_t p_b = sh.pw > 0 ? (size_t)sh.pb * (sh.dr * sh.nw + pm4) * 4 : (size_t)2 * pm4 * 4;
    const size_t bar_off = (rows_b + rec_b + p_b + 15) / 16 * 16;
    const size_t nbar = sh.pw > 0 ? 2 * (size_t)(nis + sh.pb) : (size_t)nis;
    const size_t need_b = bar_off + nbar * sizeof(uint64_t);
    bool fits = false;
    for (int nb = minb; nb >= std::min(minb, 2) && !fits; --nb)
        fits = need_b <= std::min<size_t>(p->smem_optin, (228 * 1024) / nb - 1024) - 1024;
    if (!fits) return DD_OK;
    c.reach = (int64_t)*std::max_element(T.base.begin(), T.base.begin() + (size_t)T.nblk * p->nchans) + T.rs;
    c.nblk = T.nblk; c.nsub = T.nsub; c.rs = T.rs; c.pmax = pm4; c.bar_off = (int)bar_off;
    c.smem = need_b;
    cudaError_t e = cudaMalloc(&c.d_rec, T.rec.size() * 4);
    if (e == cudaSuccess) e = cudaMalloc(&c.d_base, T.base.size() * 4);
    if (e == cudaSuccess) e = cudaMemcpy(c.d_rec, T.rec.data(), T.rec.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c.d_base, T.base.data(), T.base.size() * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { free_share(c); return cuda_fail(e, "kernel 5 tables"); }
    c.ok = true;
    return DD_OK;
}

static void free_cfg(FastCfgData &c)
{
    if (c.d_desc) cudaFree(c.d_desc);
    if (c.d_base) cudaFree(c.d_base);
    if (c.d_goff) cudaFree(c.d_goff);
    c.d_desc = nullptr; c.d_base = nullptr; c.d_goff = nullptr;
    c.ok = false;
}

// Build the descriptor tables of one configuration.  Returns DD_OK with
// c.ok == false when the configuration cannot run the plan (rows too long
// for shared memory).
static int build_cfg(const dd_plan *p, int tr, int nw, FastCfgData &c)
{
    c = FastCfgData();
    c.tr = tr; c.nw = nw;
    const int C = p->nchans, D = p->ndm, DB = kDR * nw;
    const int nblk = (D + DB - 1) / DB;
    const int AL = elem_align(p->dtype);
    std::vector<uint32_t> desc((size_t)nblk * C * nw);
    std::vector<int32_t> base((size_t)nblk * C);
    std::vector<int32_t> goff((size_t)nblk * C * nw * kDR);
    auto dl = [&](int dm, int ch) { return p->delays[(size_t)std::min(dm, D - 1) * C + ch]; };
    long long need = 0;   // largest element index any lane touches, + 1
    for (int b = 0; b < nblk; ++b) {
        for (int ch = 0; ch < C; ++ch) {
            int lo = INT_MAX;
            for (int j = 0; j < DB; ++j) lo = std::min(lo, dl(b * DB + j, ch));
            const int row0 = lo - (lo % AL);       // aligned row start (tile starts are multiples of AL)
            base[(size_t)b * C + ch] = row0;
            for (int w = 0; w < nw; ++w) {
                int d[kDR], bw = INT_MAX;
                for (int j = 0; j < kDR; ++j) { d[j] = dl(b * DB + w * kDR + j, ch); bw = std::min(bw, d[j]); }
                const int off = bw - row0;         // warp base within the row
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
                const size_t di = ((size_t)b * C + ch) * nw + w;
                if (A != kGeneric && wsoff / 4 < (1 << 12)) {
                    uint32_t dd = 0;
                    for (int j = 0; j < kDR; ++j)
                        dd |= (uint32_t)(rem + (d[j] - d[0] - j * A)) << (3 * j);
                    dd |= (uint32_t)A << 12;
                    dd |= (uint32_t)(wsoff / 4) << 20;
                    desc[di] = dd;
                    need = std::max<long long>(need, (long long)wsoff + tr * 31 + win_len(tr, A));
                } else {
                    desc[di] = (uint32_t)kGeneric << 12;
                    for (int j = 0; j < kDR; ++j) {
                        const int o = d[j] - row0;
                        goff[di * kDR + j] = o;
                        need = std::max<long long>(need, (long long)(o & ~3) + tr * 31 + tr + 4);
                    }
                }
            }
        }
    }
    const int rs = (int)((need + 15) / 16 * 16);
    const size_t eb = in_elem_bytes(p->dtype);
    const size_t budget = std::min<size_t>(p->smem_optin, 227 * 1024) - 1024;
    const size_t per_ch = (size_t)rs * eb + nw * sizeof(uint32_t);
    const int ch = (int)std::min<size_t>(16, budget / (kStages * per_ch));
    const size_t epi = (size_t)nw * kDR * 32 * tr * sizeof(float);
    if (ch < 1 || epi > budget) return DD_OK;
    const size_t bar_off = (std::max(epi, (size_t)kStages * ch * per_ch) + 15) / 16 * 16;
    const size_t smem = bar_off + kStages * sizeof(uint64_t);
    if (smem > budget + 1024) return DD_OK;
    c.nblk = nblk; c.rs = rs; c.ch = ch; c.bar_off = (int)bar_off; c.smem = smem;
    // the fallback offsets are only read for descriptors marked generic
    bool any_generic = false;
    for (uint32_t dd : desc) any_generic |= ((dd >> 12) & 0xffu) == (uint32_t)kGeneric;
    if (!any_generic) goff.assign(kDR, 0);
    cudaError_t e = cudaMalloc(&c.d_desc, desc.size() * 4);
    if (e == cudaSuccess) e = cudaMalloc(&c.d_base, base.size() * 4);
    if (e == cudaSuccess) e = cudaMalloc(&c.d_goff, goff.size() * 4);
    if (e == cudaSuccess) e = cudaMemcpy(c.d_desc, desc.data(), desc.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c.d_base, base.data(), base.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c.d_goff, goff.data(), goff.size() * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_cfg(c);
        return cuda_fail(e, "kernel 2 tables");
    }
    c.ok = true;
    return DD_OK;
}

// Process-wide cache of autotuner choices, keyed by the plan's shape.
using TuneKey = std::tuple<int, int, int, int64_t, double, double, double, double, double>;
static std::mutex g_tune_mu;
static std::map<TuneKey, std::pair<int, int>> g_tune_cache;

static TuneKey tune_key(const dd_plan *p)
{
    const double d0 = p->dm_list.front(), d1 = p->dm_list.back();
    return TuneKey(p->nchans, p->ndm, (int)p->dtype, p->nsamp_in, p->fch1, p->foff, p->tsamp, d0, d1);
}

static bool cfg_ok(const FastPlan *f, int k)
{
    if (k < 0 || k >= kNumAllCfg) return false;
    if (k < kNumFastCfg) return f->cfg[k].ok;
    if (k < kLaneEnd) return f->lane[k - kNumFastCfg].ok;
    return k < kShareBeg ? f->tm[k - kLaneEnd].ok : f->sh[k - kShareBeg].ok;
}

int fast_configure(dd_plan *p)
{
    p->fast = nullptr;
    FastPlan *f = new FastPlan();
    f->al = elem_align(p->dtype);
    int rc = DD_OK;
    for (int k = 0; k < kNumFastCfg && rc == DD_OK; ++k)
        rc = build_cfg(p, kFastCfg[k].tr, kFastCfg[k].nw, f->cfg[k]);
    for (int k = 0; k < kNumLaneCfg && rc == DD_OK; ++k)
        rc = build_lane(p, kLaneCfg[k].ti, kLaneCfg[k].dr, kLaneCfg[k].nw, kLaneCfg[k].minb, f->lane[k]);
    for (int k = 0; k < kNumTmemCfg && rc == DD_OK; ++k)
        rc = build_tmem(p, kTmemCfg[k].n, kTmemCfg[k].dbw, kTmemCfg[k].nw, f->tm[k]);
    for (int k = 0; k < kNumShareCfg && rc == DD_OK; ++k) rc = build_share(p, k, f->sh[k]);
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < kNumFastCfg && rc == DD_OK && e == cudaSuccess; ++k)
        if (f->cfg[k].ok) e = prepare_cfg(k, p->smem_optin);
    for (int k = 0; k < kNumLaneCfg && rc == DD_OK && e == cudaSuccess; ++k)
        if (f->lane[k].ok) e = prepare_lane(k, p->smem_optin);
    for (int k = 0; k < kNumTmemCfg && rc == DD_OK && e == cudaSuccess; ++k)
        if (f->tm[k].ok) e = prepare_tmem(k, p->smem_optin);
    for (int k = 0; k < kNumShareCfg && rc == DD_OK && e == cudaSuccess; ++k)
        if (f->sh[k].ok) e = share_prepare(k, p->smem_optin);
    if (rc == DD_OK && e == cudaSuccess) e = cudaMalloc(&f->d_err, sizeof(int));
    if (rc == DD_OK && e == cudaSuccess) e = cudaMemset(f->d_err, 0, sizeof(int));
    p->fast = f;
    if (rc == DD_OK && e != cudaSuccess) rc = cuda_fail(e, "kernel 2 setup");
    if (rc != DD_OK) { fast_release(p); return rc; }
    // default: the first available configuration in the order of measured
    // speed (kernel 5 shapes where their tables fit, then kernel 3, then
    // kernel 2); the autotuner may change it
    static const int pref[] = {kShareBeg + 3, kShareBeg + 2, kShareBeg + 0, kShareBeg + 1, kNumFastCfg + 2,
                               kNumFastCfg + 0, kNumFastCfg + 3, kNumFastCfg + 1, 1, 0, 2};
    for (int k : pref)
        if (cfg_ok(f, k)) { f->active = k; break; }
    if (f->active < 0) { fast_release(p); return DD_OK; }   // tiled kernels unavailable
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tune_cache.find(tune_key(p));
    if (it != g_tune_cache.end() && cfg_ok(f, it->second.first)) {
        f->active = it->second.first;
        f->dgroup = it->second.second;
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

// Partial-statistics record size of the plan's input type.
static size_t stat_bytes(const dd_plan *p) { return p->dtype == DD_U8 ? sizeof(StatI) : sizeof(StatF); }

// Kernel 3 on output tiles [tile_lo, tile_hi) (tile_hi < 0: all tiles); the
// partial statistics of tile j land where a whole-plan launch puts them.
static int lane_run(dd_plan *p, int k, int dgroup, const void *in, int64_t pitch, void *out, cudaStream_t s,
                    int64_t tile_lo = 0, int64_t tile_hi = -1)
{
    FastPlan *f = static_cast<FastPlan *>(p->fast);
    LaneCfgData &c = f->lane[k];
    const int tile = 32 * c.ti;
    const int64_t ntile = (p->nsamp_out + tile - 1) / tile;
    if (ntile * c.nblk > INT32_MAX) return generic_execute(p, in, pitch, out, s);
    if (tile_hi < 0) tile_hi = ntile;
    const int64_t np = ntile * c.nblk;
    int rc = ensure_partials_public(p, np);
    if (rc) return rc;
    if (tile_hi <= tile_lo) return DD_OK;
    LaneLaunch a{};
    a.in = in; a.pitch = pitch;
    a.nsamp_in_al = (p->nsamp_in + f->al - 1) / f->al * f->al;
    a.nchans = p->nchans; a.ndm = p->ndm; a.nout = p->nsamp_out;
    a.offs = c.d_offs; a.base = c.d_base;
    a.rs = c.rs; a.ch = c.ch; a.bar_off = c.bar_off; a.nblk = c.nblk;
    a.ntile = tile_hi - tile_lo; a.t_base = tile_lo * tile;
    a.dgroup = std::max(1, std::min(dgroup, c.nblk));
    a.out = out; a.err = f->d_err; a.smem = c.smem;
    a.partials = static_cast<char *>(p->d_partials) + (size_t)(tile_lo * c.nblk) * stat_bytes(p);
    cudaError_t e = launch_lane(k, p->dtype, a, s);
    if (e != cudaSuccess) return cuda_fail(e, "launch lane_kernel");
    p->n_partials = np;
    p->stats_out = out;
    return DD_OK;
}

static int tmem_run(dd_plan *p, int k, int dgroup, const void *in, int64_t pitch, void *out, cudaStream_t s)
{
    FastPlan *f = static_cast<FastPlan *>(p->fast);
    TmemCfgData &c = f->tm[k];
    const int tile = 32 * c.n;
    const int64_t ntile = (p->nsamp_out + tile - 1) / tile;
    if (ntile * c.nblk > INT32_MAX) return generic_execute(p, in, pitch, out, s);
    const int64_t np = ntile * c.nblk;
    int rc = ensure_partials_public(p, np);
    if (rc) return rc;
    TmemLaunch a;
    a.in = in; a.pitch = pitch;
    a.nsamp_in_al = (p->nsamp_in + f->al - 1) / f->al * f->al;
    a.nchans = p->nchans; a.ndm = p->ndm; a.nout = p->nsamp_out;
    a.tab = c.d_tab; a.base = c.d_base;
    a.rs = c.rs; a.ch = c.ch; a.bar_off = c.bar_off; a.nblk = c.nblk; a.dbp = c.dbp; a.wmax = c.wmax;
    a.ntile = ntile; a.dgroup = std::max(1, std::min(dgroup, c.nblk));
    a.out = out; a.partials = p->d_partials; a.err = f->d_err; a.smem = c.smem;
    cudaError_t e = launch_tmem(k, p->dtype, a, s);
    if (e != cudaSuccess) return cuda_fail(e, "launch tmem_kernel");
    p->n_partials = np;
    p->stats_out = out;
    return DD_OK;
}

// Kernel 5 on output tiles [tile_lo, tile_hi), as lane_run.
static int share_run(dd_plan *p, int k, int dgroup, const void *in, int64_t pitch, void *out, cudaStream_t s,
                     int64_t tile_lo = 0, int64_t tile_hi = -1)
{
    FastPlan *f = static_cast<FastPlan *>(p->fast);
    ShareCfgData &c = f->sh[k];
    const int tile = 32 * kShareCfg[k].ti;
    const int64_t ntile = (p->nsamp_out + tile - 1) / tile;
    if (ntile * c.nblk > INT32_MAX) return generic_execute(p, in, pitch, out, s);
    if (tile_hi < 0) tile_hi = ntile;
    const int64_t np = ntile * c.nblk;
    int rc = ensure_partials_public(p, np);
    if (rc) return rc;
    if (tile_hi <= tile_lo) return DD_OK;
    ShareLaunch a{};
    a.in = in; a.pitch = pitch;
    a.nsamp_in_al = (p->nsamp_in + f->al - 1) / f->al * f->al;
    a.nchans = p->nchans; a.ndm = p->ndm; a.nsub = c.nsub; a.nout = p->nsamp_out;
    a.rec = c.d_rec; a.base = c.d_base; a.rlen = c.d_base + (size_t)c.nblk * p->nchans;
    a.rs = c.rs; a.pmax = c.pmax; a.bar_off = c.bar_off; a.nblk = c.nblk;
    a.ntile = tile_hi - tile_lo; a.t_base = tile_lo * tile;
    a.dgroup = std::max(1, std::min(dgroup, c.nblk));
    a.out = out; a.err = f->d_err; a.smem = c.smem;
    a.skew = tile_lo == 0 && tile_hi == ntile ? 1 : 0;   // whole-plan launches only (a tile range must stay in range)
    a.partials = static_cast<char *>(p->d_partials) + (size_t)(tile_lo * c.nblk) * stat_bytes(p);
    cudaError_t e = share_launch(k, p->dtype, a, s);
    if (e != cudaSuccess) return cuda_fail(e, "launch share_kernel");
    p->n_partials = np;
    p->stats_out = out;
    return DD_OK;
}

static int fast_run(dd_plan *p, int k, int dgroup, const void *in, int64_t pitch, void *out, cudaStream_t s)
{
    if (k >= kShareBeg) return share_run(p, k - kShareBeg, dgroup, in, pitch, out, s);
    if (k >= kLaneEnd) return tmem_run(p, k - kLaneEnd, dgroup, in, pitch, out, s);
    if (k >= kNumFastCfg) return lane_run(p, k - kNumFastCfg, dgroup, in, pitch, out, s);
    FastPlan *f = static_cast<FastPlan *>(p->fast);
    FastCfgData &c = f->cfg[k];
    const int tile = 32 * c.tr;
    const int64_t ntile = (p->nsamp_out + tile - 1) / tile;
    if (ntile * c.nblk > INT32_MAX) return generic_execute(p, in, pitch, out, s);
    const int64_t np = ntile * c.nblk;
    int rc = ensure_partials_public(p, np);
    if (rc) return rc;
    FastLaunch a;
    a.in = in; a.pitch = pitch;
    a.nsamp_in_al = (p->nsamp_in + f->al - 1) / f->al * f->al;
    a.nchans = p->nchans; a.ndm = p->ndm; a.nout = p->nsamp_out;
    a.desc = c.d_desc; a.base = c.d_base; a.goff = c.d_goff;
    a.rs = c.rs; a.ch = c.ch; a.bar_off = c.bar_off; a.nblk = c.nblk;
    a.ntile = ntile; a.dgroup = std::max(1, std::min(dgroup, c.nblk));
    a.out = out; a.partials = p->d_partials; a.err = f->d_err; a.smem = c.smem;
    cudaError_t e = launch_cfg(k, p->dtype, a, s);
    if (e != cudaSuccess) return cuda_fail(e, "launch fast_kernel");
    p->n_partials = np;
    p->stats_out = out;
    return DD_OK;
}

int fast_execute(dd_plan *p, const void *in, int64_t pitch, void *out, cudaStream_t s)
{
    FastPlan *f = static_cast<FastPlan *>(p->fast);
    if (!f) return set_error(DD_ERR_ARG, "kernel 2 unavailable for this plan");
    // TMA bulk copies need 16-byte aligned rows; otherwise run the generic kernel.
    if (((uintptr_t)in & 15u) || (pitch % f->al)) return generic_execute(p, in, pitch, out, s);
    return fast_run(p, f->active, f->dgroup, in, pitch, out, s);
}

// Schedule of the pipelined host path for nsamp_out outputs in tiles of
// `tile` samples whose inputs lie below t0 + reach: up to kHostChunks chunks,
// chunk c copies input columns up to col_end[c] (multiples of 64, the last
// one the whole pitch) and then launches tiles up to tile_end[c].  Returns
// the number of chunks.
static int host_chunks(int64_t nsamp_out, int64_t pitch, int tile, int64_t reach, int64_t *col_end,
                       int64_t *tile_end)
{
    const int64_t ntile = (nsamp_out + tile - 1) / tile;
    const int nch = (int)std::min<int64_t>(kHostChunks, ntile);
    int64_t col = 0;
    for (int c = 0; c < nch; ++c) {
        tile_end[c] = ntile * (c + 1) / nch;
        const int64_t need = c == nch - 1 ? pitch : std::min<int64_t>(pitch, (tile_end[c] * tile + reach + 63) / 64 * 64);
        col = std::max(col, need);
        col_end[c] = col;
    }
    return nch;
}

// dd_process_host with kernels 3 and 5: the input goes to the device in
// kHostChunks column chunks on the plan's copy stream, and after chunk k the
// output tiles whose input it completes run on `s` while the next chunk is
// in flight.  Tile j (outputs from t0 = j * tile) reads input columns below
// t0 + reach, so tiles [T_k, T_k+1) need columns below T_k+1 * tile + reach.
// Returns kNotPipelined (nothing done) for the other kernels.
int fast_execute_host(dd_plan *p, const void *in_host, int64_t pitch, void *in_dev, void *out, cudaStream_t s)
{
    FastPlan *f = static_cast<FastPlan *>(p->fast);
    if (!f || ((uintptr_t)in_dev & 15u) || (pitch % f->al)) return kNotPipelined;
    const int k = f->active;
    int tile, nblk;
    int64_t reach;
    if (k >= kShareBeg) {
        tile = 32 * kShareCfg[k - kShareBeg].ti;
        reach = f->sh[k - kShareBeg].reach;
        nblk = f->sh[k - kShareBeg].nblk;
    } else if (k >= kNumFastCfg && k < kLaneEnd) {
        tile = 32 * f->lane[k - kNumFastCfg].ti;
        reach = f->lane[k - kNumFastCfg].reach;
        nblk = f->lane[k - kNumFastCfg].nblk;
    } else {
        return kNotPipelined;
    }
    // plans whose grid would fall back to the generic kernel (which reads the
    // whole input) take the unsplit path
    if ((p->nsamp_out + tile - 1) / tile * nblk > INT32_MAX) return kNotPipelined;
    cudaError_t e = cudaSuccess;
    if (!f->copy_stream) {
        e = cudaStreamCreateWithFlags(&f->copy_stream, cudaStreamNonBlocking);
        for (int i = 0; i <= kHostChunks && e == cudaSuccess; ++i)
            e = cudaEventCreateWithFlags(&f->copy_ev[i], cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "copy stream");
    }
    const size_t eb = in_elem_bytes(p->dtype);
    // the copies wait for earlier work on `s` (it may still read the staging buffer)
    e = cudaEventRecord(f->copy_ev[kHostChunks], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(f->copy_stream, f->copy_ev[kHostChunks], 0);
    if (e != cudaSuccess) return cuda_fail(e, "order input copy");
    int64_t col_end[kHostChunks], tile_end[kHostChunks];
    const int nch = host_chunks(p->nsamp_out, pitch, tile, reach, col_end, tile_end);
    int64_t col = 0, tlo = 0;
    for (int c = 0; c < nch; ++c) {
        const int64_t thi = tile_end[c], end = col_end[c];
        if (end > col) {
            e = cudaMemcpy2DAsync(static_cast<char *>(in_dev) + col * eb, (size_t)pitch * eb,
                                  static_cast<const char *>(in_host) + col * eb, (size_t)pitch * eb,
                                  (size_t)(end - col) * eb, (size_t)p->nchans, cudaMemcpyHostToDevice,
                                  f->copy_stream);
            if (e == cudaSuccess) e = cudaEventRecord(f->copy_ev[c], f->copy_stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, f->copy_ev[c], 0);
            if (e != cudaSuccess) return cuda_fail(e, "H2D input chunk");
            col = end;
        }
        const int rc = k >= kShareBeg ? share_run(p, k - kShareBeg, f->dgroup, in_dev, pitch, out, s, tlo, thi)
                                      : lane_run(p, k - kNumFastCfg, f->dgroup, in_dev, pitch, out, s, tlo, thi);
        if (rc) return rc;
        tlo = thi;
    }
    return DD_OK;
}

int fast_autotune(dd_plan *p, const void *in, int64_t pitch, void *out, cudaStream_t s)
{
    FastPlan *f = static_cast<FastPlan *>(p->fast);
    if (!f) return DD_OK;
    if (((uintptr_t)in & 15u) || (pitch % f->al)) return DD_OK;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return set_error(DD_ERR_CUDA, "cudaEventCreate");
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return set_error(DD_ERR_CUDA, "cudaEventCreate"); }
    float best = 1e30f;
    int bk = f->active, bg = f->dgroup, rc = DD_OK;
    // largest raster group first: on a tie (within 0.5%) it keeps the least DRAM
    // traffic (64: every DM block of the usual plans in one group, each time
    // tile's blocks together)
    const int groups[] = {64, 16, 8, 4};
    // kernels 5, 3 and 2, each in its order of measured speed, so that a tie
    // keeps the earlier one (kernel 5's warp-specialised 64-trial shape first, then the 48-trial one: fewest input
    // re-reads); kernel 4 (slower on every plan measured) runs only on request
    static const int order[] = {kShareBeg + 3, kShareBeg + 2, kShareBeg + 0, kShareBeg + 1, kNumFastCfg + 2,
                                kNumFastCfg + 0, kNumFastCfg + 3, kNumFastCfg + 1, 1, 0, 2};
    static_assert(sizeof(order) / sizeof(order[0]) == kNumAllCfg - kNumTmemCfg, "every timed configuration once");
    for (int k : order) {
        if (rc != DD_OK) break;
        if (!cfg_ok(f, k)) continue;
        rc = fast_run(p, k, 8, in, pitch, out, s);             // warm-up (caches, clocks)
        for (int gi = 0; gi < 4 && rc == DD_OK; ++gi) {
            cudaEventRecord(e0, s);
            rc = fast_run(p, k, groups[gi], in, pitch, out, s);
            cudaEventRecord(e1, s);
            if (rc) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) { rc = set_error(DD_ERR_CUDA, "autotune sync"); break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (k < kNumFastCfg) f->cfg[k].last_ms = ms;
            if (ms < best * 0.995f) { best = ms; bk = k; bg = groups[gi]; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    rc = fast_error(p, s);
    if (rc) return rc;
    f->active = bk;
    f->dgroup = bg;
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune_cache[tune_key(p)] = {bk, bg};
    return DD_OK;
}

int fast_set_tile(dd_plan *p, int cfg, int dgroup)
{
    FastPlan *f = static_cast<FastPlan *>(p->fast);
    if (!f) return set_error(DD_ERR_ARG, "kernel 2 unavailable for this plan");
    if (!cfg_ok(f, cfg))
        return set_error(DD_ERR_ARG, "tile configuration %d not available for this plan", cfg);
    if (dgroup < 1) return set_error(DD_ERR_ARG, "raster group must be >= 1");
    f->active = cfg;
    f->dgroup = dgroup;
    return DD_OK;
}

int fast_get_tile(const dd_plan *p, int *cfg, int *dgroup, int *tr, int *nw)
{
    const FastPlan *f = static_cast<const FastPlan *>(p->fast);
    if (!f) return set_error(DD_ERR_ARG, "kernel 2 unavailable for this plan");
    if (cfg) *cfg = f->active;
    if (dgroup) *dgroup = f->dgroup;
    if (f->active < kNumFastCfg) {
        if (tr) *tr = f->cfg[f->active].tr;
        if (nw) *nw = f->cfg[f->active].nw;
    } else if (f->active < kLaneEnd) {
        if (tr) *tr = f->lane[f->active - kNumFastCfg].ti;
        if (nw) *nw = f->lane[f->active - kNumFastCfg].nw;
    } else if (f->active < kShareBeg) {
        if (tr) *tr = f->tm[f->active - kLaneEnd].n;
        if (nw) *nw = f->tm[f->active - kLaneEnd].nw;
    } else {
        if (tr) *tr = kShareCfg[f->active - kShareBeg].ti;
        if (nw) *nw = kShareCfg[f->active - kShareBeg].nw;
    }
    return DD_OK;
}

int fast_kernel_id(const dd_plan *p)
{
    const FastPlan *f = static_cast<const FastPlan *>(p->fast);
    if (!f || f->active < kNumFastCfg) return 2;
    if (f->active < kLaneEnd) return 3;
    return f->active < kShareBeg ? 4 : 5;
}

void fast_release(dd_plan *p)
{
    FastPlan *f = static_cast<FastPlan *>(p->fast);
    if (!f) return;
    for (int k = 0; k < kNumFastCfg; ++k) free_cfg(f->cfg[k]);
    for (int k = 0; k < kNumLaneCfg; ++k) free_lane(f->lane[k]);
    for (int k = 0; k < kNumTmemCfg; ++k) free_tmem(f->tm[k]);
    for (int k = 0; k < kNumShareCfg; ++k) free_share(f->sh[k]);
    if (f->d_err) cudaFree(f->d_err);
    if (f->copy_stream) {
        cudaStreamSynchronize(f->copy_stream);
        for (int i = 0; i <= kHostChunks; ++i)
            if (f->copy_ev[i]) cudaEventDestroy(f->copy_ev[i]);
        cudaStreamDestroy(f->copy_stream);
    }
    delete f;
    p->fast = nullptr;
}

}  // namespace dd

// ===================================================================== batch
// Several plans (beams) in one persistent launch of batch_kernel.

struct dd_batch {
    std::vector<dd_plan *> plans;
    int device = 0;
    int cfg = -1;                          // shared tile configuration (-1: no persistent launch)
    std::vector<int> k2;                   // beams in the persistent launch
    std::vector<int> sep;                  // beams run by their own dd_execute launch
    uint2 *d_items = nullptr;
    int nitems = 0;
    dd::FastLaunch *d_beams = nullptr, *h_beams = nullptr;   // h_beams pinned (graph-capturable copy)
    dd::LaneLaunch *d_lbeams = nullptr, *h_lbeams = nullptr; // the same for kernel 3 configurations
    dd::ShareLaunch *d_sbeams = nullptr, *h_sbeams = nullptr; // kernel 5 beams of the mixed configuration
    std::vector<int> kind;                 // mixed configuration: 1 = the beam runs kernel 5
    std::vector<int> k5;                   // mixed configuration, own launches: the kernel 5 shape each beam runs
    bool per_beam = false;                 // launch mode: each beam's own kernel launch instead of one persistent grid
    unsigned int *d_counter = nullptr;
    int *d_err = nullptr;
    int bar_off = 0;
    size_t smem = 0;
    int grid = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace dd {

static FastPlan *fp(const dd_plan *p) { return static_cast<FastPlan *>(p->fast); }

// The batch's mixed configuration: kernel 5 shape kMixedShare for the beams
// whose tables exist and fit the shape's blocks per SM, kernel 3 shape
// kMixedLane (the same block geometry) for the others.
constexpr int kMixedCfg = kShareBeg + kMixedShare;

static bool mixed_share_ok(const dd_plan *p, const FastPlan *f)
{
    const ShareCfgData &c = f->sh[kMixedShare];
    const int nb = kShareCfg[kMixedShare].minb;
    return c.ok && c.smem <= std::min<size_t>(p->smem_optin, (228 * 1024) / nb - 1024) - 1024;
}

// Geometry of configuration k (kernel 2 or kernel 3, or the mixed one: its
// kernel 3 shape's) of a plan's tables.
struct BatchGeom { bool ok; int tile, nblk, bar_off; };
static BatchGeom batch_geom(const FastPlan *f, int k)
{
    if (k == kMixedCfg) k = kNumFastCfg + kMixedLane;
    if (!f || k < 0 || k >= kLaneEnd) return {false, 0, 0, 0};
    if (k < kNumFastCfg) {
        const FastCfgData &c = f->cfg[k];
        return {c.ok, 32 * c.tr, c.nblk, c.bar_off};
    }
    const LaneCfgData &c = f->lane[k - kNumFastCfg];
    return {c.ok, 32 * c.ti, c.nblk, c.bar_off};
}

static cudaError_t batch_launch_lane(int k, const LaneBatchLaunch &b, int sms, size_t smem, cudaStream_t s)
{
    switch (k) {
    case 0: return lane_batch_launch_c0(b, sms, smem, s);
    case 1: return lane_batch_launch_c1(b, sms, smem, s);
    case 2: return lane_batch_launch_c2(b, sms, smem, s);
    default: return lane_batch_launch_c3(b, sms, smem, s);
    }
}

// Work items for configuration k: every (beam, linear tile) of the beams that
// can use it, heaviest beams (most channels per item) first.
static int batch_build(dd_batch *B, int k)
{
    B->k2.clear();
    B->sep.clear();
    for (int i = 0; i < (int)B->plans.size(); ++i) {
        const FastPlan *f = fp(B->plans[i]);
        if (batch_geom(f, k).ok) B->k2.push_back(i); else B->sep.push_back(i);
    }
    std::vector<int> order = B->k2;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return B->plans[a]->nchans > B->plans[b]->nchans;
    });
    std::vector<uint2> items;
    int bar_off = 0;
    B->kind.assign(B->plans.size(), 0);
    for (int i : order) {
        const dd_plan *p = B->plans[i];
        const BatchGeom c = batch_geom(fp(p), k);
        const int64_t ntile = (p->nsamp_out + c.tile - 1) / c.tile;
        const int64_t n = ntile * c.nblk;
        if ((int64_t)items.size() + n > INT32_MAX) return set_error(DD_ERR_ARG, "batch too large");
        for (int64_t l = 0; l < n; ++l) items.push_back(make_uint2((unsigned)i, (unsigned)l));
        bar_off = std::max(bar_off, c.bar_off);
        if (k == kMixedCfg && mixed_share_ok(p, fp(p))) {
            B->kind[i] = 1;
            bar_off = std::max(bar_off, fp(p)->sh[kMixedShare].bar_off);
        }
    }
    B->k5.assign(B->plans.size(), -1);
    if (k == kMixedCfg && B->per_beam) {
        // own launches: every beam with kernel 5 tables runs its first
        // available kernel 5 shape in the order of measured speed (the shape
        // it would start on alone), the others kernel 3's mixed shape
        static const int k5pref[] = {kShareBeg + 3, kShareBeg + 2, kShareBeg + 0, kShareBeg + 1};
        for (int i : order) {
            B->kind[i] = 0;
            for (int c : k5pref)
                if (cfg_ok(fp(B->plans[i]), c)) { B->kind[i] = 1; B->k5[i] = c; break; }
        }
    } else if (k == kMixedCfg) {
        // keep the shape's resident blocks per SM: the kernel 5 beams with the
        // largest shared-memory layouts go back to kernel 3 until they fit
        constexpr int nbar = kStages + kShareCfg[kMixedShare].ns;
        int lane_off = 0;
        for (int i : order) lane_off = std::max(lane_off, batch_geom(fp(B->plans[i]), k).bar_off);
        for (;;) {
            int worst = -1, off = lane_off;
            for (int i : order)
                if (B->kind[i]) {
                    const int o = fp(B->plans[i])->sh[kMixedShare].bar_off;
                    off = std::max(off, o);
                    if (worst < 0 || o > fp(B->plans[worst])->sh[kMixedShare].bar_off) worst = i;
                }
            bar_off = off;
            if (worst < 0 || off == lane_off ||
                mixed_batch_occupancy((size_t)off + nbar * sizeof(uint64_t)) >= kShareCfg[kMixedShare].minb)
                break;
            B->kind[worst] = 0;
        }
    }
    if (B->d_items) cudaFree(B->d_items);
    B->d_items = nullptr;
    B->nitems = (int)items.size();
    B->cfg = B->k2.empty() ? -1 : k;
    B->bar_off = bar_off;
    B->smem = (size_t)bar_off + (kStages + (k == kMixedCfg ? kShareCfg[kMixedShare].ns : 0)) * sizeof(uint64_t);
    if (!items.empty()) {
        cudaError_t e = cudaMalloc(&B->d_items, items.size() * sizeof(uint2));
        if (e == cudaSuccess)
            e = cudaMemcpy(B->d_items, items.data(), items.size() * sizeof(uint2), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "batch work items");
    }
    return DD_OK;
}

// Everything the launches need, allocated before any capture.
static int batch_prepare(dd_batch *B)
{
    for (int i : B->k2) {
        dd_plan *p = B->plans[i];
        const BatchGeom c = batch_geom(fp(p), B->cfg);
        const int64_t ntile = (p->nsamp_out + c.tile - 1) / c.tile;
        int rc = ensure_partials_public(p, ntile * c.nblk);
        if (rc) return rc;
        if (B->k5.size() == B->plans.size() && B->k5[i] >= kShareBeg) {
            // the beam's own kernel 5 launch (a capture must not allocate)
            const int j = B->k5[i] - kShareBeg;
            const int64_t t5 = (p->nsamp_out + 32 * kShareCfg[j].ti - 1) / (32 * kShareCfg[j].ti);
            rc = ensure_partials_public(p, t5 * fp(p)->sh[j].nblk);
            if (rc) return rc;
        }
    }
    return DD_OK;
}

static int batch_enqueue(dd_batch *B, const void *const *ins, const int64_t *pitches, void *const *outs,
                         cudaStream_t s)
{
    for (size_t i = 0; i < B->plans.size(); ++i) {
        if (!ins[i] || !outs[i]) return set_error(DD_ERR_ARG, "NULL buffer for beam %d", (int)i);
        if (pitches[i] < B->plans[i]->nsamp_in) return set_error(DD_ERR_ARG, "pitch < nsamp_in for beam %d", (int)i);
    }
    int rc = batch_prepare(B);
    if (rc) return rc;
    std::vector<int> own(B->sep);
    if (B->per_beam && B->cfg >= 0) {
        // each beam's single-plan kernel on its batch configuration, in turn
        for (int i : B->k2) {
            dd_plan *p = B->plans[i];
            FastPlan *f = fp(p);
            if (((uintptr_t)ins[i] & 15u) || (pitches[i] % f->al))
                return set_error(DD_ERR_ARG, "beam %d: input rows must be 16-byte aligned in a batch", i);
            const int k = B->cfg != kMixedCfg ? B->cfg : B->kind[i] ? B->k5[i] : kNumFastCfg + kMixedLane;
            rc = fast_run(p, k, f->dgroup, ins[i], pitches[i], outs[i], s);
            if (rc) return rc;
        }
    } else if (B->cfg >= kNumFastCfg) {
        const bool mixed = B->cfg == kMixedCfg;
        const int kl = mixed ? kMixedLane : B->cfg - kNumFastCfg;
        for (int i : B->k2) {
            dd_plan *p = B->plans[i];
            FastPlan *f = fp(p);
            if (((uintptr_t)ins[i] & 15u) || (pitches[i] % f->al))
                return set_error(DD_ERR_ARG, "beam %d: input rows must be 16-byte aligned in a batch", i);
            const LaneCfgData &c = f->lane[kl];
            LaneLaunch &a = B->h_lbeams[i];
            a.in = ins[i]; a.pitch = pitches[i];
            a.nsamp_in_al = (p->nsamp_in + f->al - 1) / f->al * f->al;
            a.nchans = p->nchans; a.ndm = p->ndm; a.nout = p->nsamp_out;
            a.offs = c.d_offs; a.base = c.d_base;
            a.rs = c.rs; a.ch = c.ch; a.bar_off = B->bar_off; a.nblk = c.nblk;
            a.ntile = (p->nsamp_out + 32 * c.ti - 1) / (32 * c.ti);
            a.dgroup = std::max(1, std::min(f->dgroup, c.nblk));
            a.out = outs[i]; a.partials = p->d_partials; a.err = f->d_err; a.smem = B->smem;
            a.dtype = (int)p->dtype;
            a.t_base = 0;
            a.kind = mixed ? B->kind[i] : 0;
            if (a.kind) {
                const ShareCfgData &sc = f->sh[kMixedShare];
                ShareLaunch &sa = B->h_sbeams[i];
                sa = ShareLaunch{};
                sa.in = ins[i]; sa.pitch = pitches[i];
                sa.nsamp_in_al = a.nsamp_in_al;
                sa.nchans = p->nchans; sa.ndm = p->ndm; sa.nsub = sc.nsub; sa.nout = p->nsamp_out;
                sa.rec = sc.d_rec; sa.base = sc.d_base; sa.rlen = sc.d_base + (size_t)sc.nblk * p->nchans;
                sa.rs = sc.rs; sa.pmax = sc.pmax; sa.bar_off = B->bar_off; sa.nblk = sc.nblk;
                sa.ntile = a.ntile; sa.t_base = 0; sa.dgroup = a.dgroup;
                sa.out = outs[i]; sa.partials = p->d_partials; sa.err = f->d_err; sa.smem = B->smem;
            }
        }
        cudaError_t e = cudaMemcpyAsync(B->d_lbeams, B->h_lbeams, B->plans.size() * sizeof(LaneLaunch),
                                        cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && mixed)
            e = cudaMemcpyAsync(B->d_sbeams, B->h_sbeams, B->plans.size() * sizeof(ShareLaunch),
                                cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(B->d_counter, 0, sizeof(unsigned int), s);
        if (e != cudaSuccess) return cuda_fail(e, "batch setup");
        LaneBatchLaunch bl;
        bl.beams = B->d_lbeams; bl.items = B->d_items; bl.nitems = B->nitems;
        bl.bar_off = B->bar_off; bl.counter = B->d_counter; bl.sbeams = B->d_sbeams;
        e = mixed ? mixed_batch_launch(bl, B->grid, B->smem, s) : batch_launch_lane(kl, bl, B->grid, B->smem, s);
        if (e != cudaSuccess) return cuda_fail(e, mixed ? "launch mixed_batch_kernel" : "launch lane_batch_kernel");
        for (int i : B->k2) {
            dd_plan *p = B->plans[i];
            p->n_partials = B->h_lbeams[i].ntile * B->h_lbeams[i].nblk;
            p->stats_out = outs[i];
        }
    } else if (B->cfg >= 0) {
        for (int i : B->k2) {
            dd_plan *p = B->plans[i];
            FastPlan *f = fp(p);
            if (((uintptr_t)ins[i] & 15u) || (pitches[i] % f->al))
                return set_error(DD_ERR_ARG, "beam %d: input rows must be 16-byte aligned in a batch", i);
            const FastCfgData &c = f->cfg[B->cfg];
            FastLaunch &a = B->h_beams[i];
            a.in = ins[i]; a.pitch = pitches[i];
            a.nsamp_in_al = (p->nsamp_in + f->al - 1) / f->al * f->al;
            a.nchans = p->nchans; a.ndm = p->ndm; a.nout = p->nsamp_out;
            a.desc = c.d_desc; a.base = c.d_base; a.goff = c.d_goff;
            a.rs = c.rs; a.ch = c.ch; a.bar_off = B->bar_off; a.nblk = c.nblk;
            a.ntile = (p->nsamp_out + 32 * c.tr - 1) / (32 * c.tr);
            a.dgroup = std::max(1, std::min(f->dgroup, c.nblk));
            a.out = outs[i]; a.partials = p->d_partials; a.err = f->d_err; a.smem = B->smem;
            a.dtype = (int)p->dtype;
        }
        cudaError_t e = cudaMemcpyAsync(B->d_beams, B->h_beams, B->plans.size() * sizeof(FastLaunch),
                                        cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(B->d_counter, 0, sizeof(unsigned int), s);
        if (e != cudaSuccess) return cuda_fail(e, "batch setup");
        BatchLaunch bl;
        bl.beams = B->d_beams; bl.items = B->d_items; bl.nitems = B->nitems;
        bl.bar_off = B->bar_off; bl.counter = B->d_counter; bl.err = B->d_err;
        switch (B->cfg) {
        case 0: e = batch_launch_t36w8(bl, B->grid, B->smem, s); break;
        case 1: e = batch_launch_t20w12(bl, B->grid, B->smem, s); break;
        default: e = batch_launch_t28w8(bl, B->grid, B->smem, s); break;
        }
        if (e != cudaSuccess) return cuda_fail(e, "launch batch_kernel");
        for (int i : B->k2) {
            dd_plan *p = B->plans[i];
            p->n_partials = B->h_beams[i].ntile * B->h_beams[i].nblk;
            p->stats_out = outs[i];
        }
    }
    for (int i : own) {
        rc = generic_execute(B->plans[i], ins[i], pitches[i], outs[i], s);
        if (rc) return rc;
    }
    for (size_t i = 0; i < B->plans.size(); ++i) {
        rc = search_launch(B->plans[i], outs[i], s);
        if (rc) return rc;
    }
    return DD_OK;
}

}  // namespace dd

using namespace dd;

extern "C" {

int dd_host_chunk_schedule(int64_t nsamp_out, int64_t pitch, int32_t tile, int64_t reach, int64_t *col_end,
                           int64_t *tile_end, int32_t *n)
{
    if (!col_end || !tile_end || !n || nsamp_out < 1 || tile < 1 || reach < 0 || pitch < 1)
        return set_error(DD_ERR_ARG, "bad schedule arguments");
    *n = host_chunks(nsamp_out, pitch, tile, reach, col_end, tile_end);
    return DD_OK;
}

int dd_share_tables(const int32_t *delays, int32_t ndm, int32_t nchans, double foff, int32_t dtype,
                    int32_t config, int32_t *info, int32_t *rec_out, int64_t rec_cap, int32_t *base_out,
                    int64_t base_cap)
{
    if (!delays || !info || ndm < 1 || nchans < 1) return set_error(DD_ERR_ARG, "bad table arguments");
    if (dtype != DD_F32 && dtype != DD_U8 && dtype != DD_F16) return set_error(DD_ERR_ARG, "bad dtype %d", dtype);
    if (config < kShareBeg || config >= kShareBeg + kNumShareCfg)
        return set_error(DD_ERR_ARG, "configuration %d is not a kernel 5 shape", config);
    ShareTables T;
    share_tables(delays, ndm, nchans, foff, (dd_dtype)dtype, config - kShareBeg, T);
    info[0] = T.ok ? 1 : 0;
    info[1] = T.nblk; info[2] = T.nsub; info[3] = T.rs; info[4] = T.pmax; info[5] = T.klen;
    if (!T.ok) return DD_OK;
    if (rec_out) {
        if (rec_cap < (int64_t)T.rec.size()) return set_error(DD_ERR_ARG, "record buffer too small");
        memcpy(rec_out, T.rec.data(), T.rec.size() * 4);
    }
    if (base_out) {
        if (base_cap < (int64_t)T.base.size()) return set_error(DD_ERR_ARG, "row-start buffer too small");
        memcpy(base_out, T.base.data(), T.base.size() * 4);
    }
    return DD_OK;
}

int dd_batch_create(dd_plan *const *plans, int32_t nplans, dd_batch **out)
{
    if (!out) return set_error(DD_ERR_ARG, "batch_out is NULL");
    *out = nullptr;
    if (!plans || nplans < 1) return set_error(DD_ERR_ARG, "need >= 1 plan");
    int dev = 0;
    cudaGetDevice(&dev);
    for (int i = 0; i < nplans; ++i) {
        if (!plans[i]) return set_error(DD_ERR_ARG, "plan %d is NULL", i);
        if (plans[i]->device != dev) return set_error(DD_ERR_ARG, "plan %d lives on another device", i);
    }
    dd_batch *B = new dd_batch();
    B->plans.assign(plans, plans + nplans);
    B->device = dev;
    B->grid = std::max(1, plans[0]->sm_count);
    // first configuration, in the order of measured speed (kernel 3 shapes,
    // then kernel 2), that every tiled-kernel beam can use
    static const int pref[] = {kMixedCfg, kNumFastCfg + 2, kNumFastCfg + 0, kNumFastCfg + 3, kNumFastCfg + 1, 1, 0, 2};
    int k = -1;
    for (int c : pref) {
        if (k >= 0) break;
        bool all = false, some = false;
        for (int i = 0; i < nplans; ++i) {
            const FastPlan *f = fp(plans[i]);
            if (!f) continue;
            some = true;
            all = batch_geom(f, c).ok;
            if (!all) break;
        }
        if (some && all) k = c;
    }
    cudaError_t e = cudaMalloc(&B->d_beams, nplans * sizeof(FastLaunch));
    if (e == cudaSuccess) e = cudaMallocHost(&B->h_beams, nplans * sizeof(FastLaunch));
    if (e == cudaSuccess) e = cudaMalloc(&B->d_lbeams, nplans * sizeof(LaneLaunch));
    if (e == cudaSuccess) e = cudaMallocHost(&B->h_lbeams, nplans * sizeof(LaneLaunch));
    if (e == cudaSuccess) e = cudaMalloc(&B->d_sbeams, nplans * sizeof(ShareLaunch));
    if (e == cudaSuccess) e = cudaMallocHost(&B->h_sbeams, nplans * sizeof(ShareLaunch));
    if (e == cudaSuccess) e = mixed_batch_prepare(plans[0]->smem_optin);
    if (e == cudaSuccess) e = cudaMalloc(&B->d_counter, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc(&B->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(B->d_err, 0, sizeof(int));
    int rc = e == cudaSuccess ? DD_OK : cuda_fail(e, "batch allocation");
    if (rc == DD_OK) {
        memset(B->h_beams, 0, nplans * sizeof(FastLaunch));
        memset(B->h_lbeams, 0, nplans * sizeof(LaneLaunch));
        memset(B->h_sbeams, 0, nplans * sizeof(ShareLaunch));
        rc = batch_build(B, k);
    }
    if (rc != DD_OK) { dd_batch_destroy(B); return rc; }
    *out = B;
    return DD_OK;
}

int dd_batch_destroy(dd_batch *B)
{
    if (!B) return DD_OK;
    cudaDeviceSynchronize();
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    if (B->d_items) cudaFree(B->d_items);
    if (B->d_beams) cudaFree(B->d_beams);
    if (B->h_beams) cudaFreeHost(B->h_beams);
    if (B->d_lbeams) cudaFree(B->d_lbeams);
    if (B->h_lbeams) cudaFreeHost(B->h_lbeams);
    if (B->d_sbeams) cudaFree(B->d_sbeams);
    if (B->h_sbeams) cudaFreeHost(B->h_sbeams);
    if (B->d_counter) cudaFree(B->d_counter);
    if (B->d_err) cudaFree(B->d_err);
    delete B;
    return DD_OK;
}

int dd_batch_execute(dd_batch *B, const void *const *ins, const int64_t *pitches, void *const *outs, void *stream)
{
    if (!B || !ins || !pitches || !outs) return set_error(DD_ERR_ARG, "NULL argument");
    return batch_enqueue(B, ins, pitches, outs, (cudaStream_t)stream);
}

int dd_batch_capture(dd_batch *B, const void *const *ins, const int64_t *pitches, void *const *outs, void *stream)
{
    if (!B || !ins || !pitches || !outs) return set_error(DD_ERR_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    if (!s) return set_error(DD_ERR_ARG, "graph capture needs a non-default stream");
    int rc = batch_prepare(B);
    if (rc) return rc;
    if (B->exec) { cudaGraphExecDestroy(B->exec); B->exec = nullptr; }
    if (B->graph) { cudaGraphDestroy(B->graph); B->graph = nullptr; }
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    rc = batch_enqueue(B, ins, pitches, outs, s);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    B->graph = g;
    e = cudaGraphInstantiate(&B->exec, g, 0);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    return DD_OK;
}

int dd_batch_launch(dd_batch *B, void *stream)
{
    if (!B || !B->exec) return set_error(DD_ERR_ARG, "no captured graph");
    cudaError_t e = cudaGraphLaunch(B->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    return DD_OK;
}

int dd_batch_results(dd_batch *B, int32_t beam, dd_candidate *cand_host, int64_t capacity, int64_t *n_found,
                     void *stream)
{
    if (!B || beam < 0 || beam >= (int)B->plans.size()) return set_error(DD_ERR_ARG, "bad beam index");
    if (!n_found || capacity < 0 || (capacity > 0 && !cand_host)) return set_error(DD_ERR_ARG, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, B->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "batch status");
    if (h) return set_error(h, "batch kernel gave up waiting for its input copies");
    dd_plan *p = B->plans[beam];
    return search_readback(p, cand_host, capacity, n_found, s, p->cand_cap);
}

int dd_batch_autotune(dd_batch *B, const void *const *ins, const int64_t *pitches, void *const *outs, void *stream)
{
    if (!B) return set_error(DD_ERR_ARG, "batch is NULL");
    if (B->cfg < 0) return DD_OK;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return set_error(DD_ERR_CUDA, "cudaEventCreate");
    float best = 1e30f;
    int bk = B->cfg, rc = DD_OK;
    std::vector<int> cfgs;
    for (int k = 0; k < kLaneEnd; ++k) cfgs.push_back(k);
    cfgs.push_back(kMixedCfg);
    bool bpb = B->per_beam;
    for (int k : cfgs) {
        bool all = true;
        for (int i = 0; i < (int)B->plans.size(); ++i) {
            const FastPlan *f = fp(B->plans[i]);
            if (f && !batch_geom(f, k).ok) all = false;
        }
        if (!all) continue;
        // the persistent grid, and (kernel 3 and the mixed configuration) each beam's own launch
        for (int pb = 0; pb < (k >= kNumFastCfg ? 2 : 1) && rc == DD_OK; ++pb) {
            B->per_beam = pb == 1;
            rc = batch_build(B, k);
            if (!rc) rc = batch_enqueue(B, ins, pitches, outs, s);           // warm-up
            if (!rc) { cudaEventRecord(e0, s); rc = batch_enqueue(B, ins, pitches, outs, s); cudaEventRecord(e1, s); }
            if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = set_error(DD_ERR_CUDA, "autotune sync");
            float ms = 0.f;
            if (!rc) cudaEventElapsedTime(&ms, e0, e1);
            if (!rc && ms < best) { best = ms; bk = k; bpb = pb == 1; }
        }
        if (rc != DD_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    B->per_beam = bpb;
    if (rc) return rc;
    if (B->exec) { cudaGraphExecDestroy(B->exec); B->exec = nullptr; }
    if (B->graph) { cudaGraphDestroy(B->graph); B->graph = nullptr; }
    return batch_build(B, bk);
}

int dd_batch_set_config(dd_batch *B, int32_t config)
{
    if (!B) return set_error(DD_ERR_ARG, "batch is NULL");
    if ((config < 0 || config >= kLaneEnd) && config != kMixedCfg)
        return set_error(DD_ERR_ARG, "batch configuration %d out of range", config);
    cudaDeviceSynchronize();
    if (B->exec) { cudaGraphExecDestroy(B->exec); B->exec = nullptr; }
    if (B->graph) { cudaGraphDestroy(B->graph); B->graph = nullptr; }
    return batch_build(B, config);
}

int dd_batch_set_launch_mode(dd_batch *B, int32_t per_beam)
{
    if (!B) return set_error(DD_ERR_ARG, "batch is NULL");
    if (per_beam != 0 && per_beam != 1) return set_error(DD_ERR_ARG, "launch mode must be 0 or 1");
    cudaDeviceSynchronize();
    if (B->exec) { cudaGraphExecDestroy(B->exec); B->exec = nullptr; }
    if (B->graph) { cudaGraphDestroy(B->graph); B->graph = nullptr; }
    B->per_beam = per_beam == 1;
    return batch_build(B, B->cfg);
}

int dd_batch_launch_mode(const dd_batch *B, int32_t *per_beam)
{
    if (!B || !per_beam) return set_error(DD_ERR_ARG, "NULL argument");
    *per_beam = B->per_beam ? 1 : 0;
    return DD_OK;
}

int dd_batch_beam_config(const dd_batch *B, int32_t beam, int32_t *config)
{
    if (!B || !config) return set_error(DD_ERR_ARG, "NULL argument");
    if (beam < 0 || beam >= (int32_t)B->plans.size()) return set_error(DD_ERR_ARG, "beam %d out of range", beam);
    *config = -1;
    if (B->cfg < 0 || std::find(B->k2.begin(), B->k2.end(), beam) == B->k2.end()) return DD_OK;
    if (B->cfg == kMixedCfg)
        *config = !B->kind[beam] ? kNumFastCfg + kMixedLane : B->per_beam ? B->k5[beam] : kMixedCfg;
    else *config = B->cfg;
    return DD_OK;
}

int dd_batch_info(const dd_batch *B, int32_t *config, int64_t *nitems, int32_t *n_separate)
{
    if (!B) return set_error(DD_ERR_ARG, "batch is NULL");
    if (config) *config = B->cfg;
    if (nitems) *nitems = B->nitems;
    if (n_separate) *n_separate = (int32_t)B->sep.size();
    return DD_OK;
}

}  // extern "C"
