// Kernel 2 host side: per-plan tables for each compiled tile configuration,
// launch, and the autotuner that picks (configuration, raster group) by
// timing them on the caller's data.
#include "dd_fast_impl.cuh"

#include <algorithm>
#include <climits>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

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

struct FastPlan {
    FastCfgData cfg[kNumFastCfg];
    int active = -1;
    int dgroup = 8;
    int al = 4;                  // row alignment in elements (16 bytes)
    int *d_err = nullptr;
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

int fast_configure(dd_plan *p)
{
    p->fast = nullptr;
    FastPlan *f = new FastPlan();
    f->al = elem_align(p->dtype);
    int rc = DD_OK;
    for (int k = 0; k < kNumFastCfg && rc == DD_OK; ++k)
        rc = build_cfg(p, kFastCfg[k].tr, kFastCfg[k].nw, f->cfg[k]);
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < kNumFastCfg && rc == DD_OK && e == cudaSuccess; ++k)
        if (f->cfg[k].ok) e = prepare_cfg(k, p->smem_optin);
    if (rc == DD_OK && e == cudaSuccess) e = cudaMalloc(&f->d_err, sizeof(int));
    if (rc == DD_OK && e == cudaSuccess) e = cudaMemset(f->d_err, 0, sizeof(int));
    p->fast = f;
    if (rc == DD_OK && e != cudaSuccess) rc = cuda_fail(e, "kernel 2 setup");
    if (rc != DD_OK) { fast_release(p); return rc; }
    for (int k = 0; k < kNumFastCfg; ++k)
        if (f->cfg[k].ok) { f->active = k; break; }
    if (f->active < 0) { fast_release(p); return DD_OK; }   // kernel 2 unavailable
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tune_cache.find(tune_key(p));
    if (it != g_tune_cache.end() && f->cfg[it->second.first].ok) {
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

static int fast_run(dd_plan *p, int k, int dgroup, const void *in, int64_t pitch, void *out, cudaStream_t s)
{
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
    const int groups[] = {4, 8, 16};
    for (int k = 0; k < kNumFastCfg && rc == DD_OK; ++k) {
        if (!f->cfg[k].ok) continue;
        rc = fast_run(p, k, 8, in, pitch, out, s);             // warm-up (caches, clocks)
        for (int gi = 0; gi < 3 && rc == DD_OK; ++gi) {
            cudaEventRecord(e0, s);
            rc = fast_run(p, k, groups[gi], in, pitch, out, s);
            cudaEventRecord(e1, s);
            if (rc) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) { rc = set_error(DD_ERR_CUDA, "autotune sync"); break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            f->cfg[k].last_ms = ms;
            if (ms < best) { best = ms; bk = k; bg = groups[gi]; }
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
    if (cfg < 0 || cfg >= kNumFastCfg || !f->cfg[cfg].ok)
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
    if (tr) *tr = f->cfg[f->active].tr;
    if (nw) *nw = f->cfg[f->active].nw;
    return DD_OK;
}

void fast_release(dd_plan *p)
{
    FastPlan *f = static_cast<FastPlan *>(p->fast);
    if (!f) return;
    for (int k = 0; k < kNumFastCfg; ++k) free_cfg(f->cfg[k]);
    if (f->d_err) cudaFree(f->d_err);
    delete f;
    p->fast = nullptr;
}

}  // namespace dd
