// Subband de-dispersion (Section 3.2): the two-stage approximation of the
// Section 3.1 sum.
//
// The fine DM list is split into consecutive groups of G trials, each with a
// nominal DM (the midpoint of the group's first and last trial); the channels
// into nsub equal subbands of consecutive channels.
//   stage 1: I[s][k][t] = sum_{c in s} in[c][t + d1(k,c)],
//            d1(k,c) = d(c, D_k) - d(ref(s), D_k), ref(s) = the subband's
//            highest-frequency channel (one partially de-dispersed series per
//            subband and nominal DM);
//   stage 2: out[j][t] = sum_s I[s][k(j)][t + d2(j,s)], d2(j,s) = d(ref(s), dm_j)
//            (brute force over the subbands at every fine DM of the group).
// d() is the plan's rounded Eq. 1 delay, so a fine DM whose delays equal its
// nominal DM's gets exactly the brute-force sum.  Work per output sample:
// C/G (stage 1, amortised over the group) + nsub (stage 2) adds instead of C.
//
// Both stages run one kernel: kernel 3's lane-interleaved body (one
// conflict-free shared word per add, TMA-staged rows, bounded waits) over a
// list of blocks, each naming its input rows, its channel count, its output
// rows and its delay records.  Stage 2 emits the statistics partials that the
// plan's search consumes.
#include "dd_lane_impl.cuh"

#include <algorithm>
#include <climits>
#include <cstring>
#include <new>

namespace dd {

struct SubBlock {
    int32_t in_row;   // input row of the block's channel 0
    int32_t nc;       // channels summed
    int32_t row0;     // first output row
    int32_t ntr;      // valid trials (output rows), <= DR*NW
    int32_t tab;      // first channel record of the block in base[] / offs[]
    int32_t pad_[3];
};
static_assert(sizeof(SubBlock) == 32, "SubBlock layout");

struct SubLaunch {
    const void *in;
    int64_t pitch;          // elements between consecutive input rows
    int64_t in_rstride;     // input rows between consecutive channels of a block
    int64_t nsamp_in_al;    // staged length limit of an input row (aligned)
    const SubBlock *blocks;
    const int32_t *offs;    // [record][DR*NW] offsets within the staged row
    const int32_t *base;    // [record] row start relative to the tile start (aligned)
    int nblk, rs, ch, bar_off;
    int64_t ntile;
    int dgroup;
    void *out;
    int64_t out_pitch, nout;
    void *partials;
    int *err;
    size_t smem;
};

// Kernel 3's tile shape: 16 samples per lane x 8 trials per warp; 3 or 4
// warps per block, chosen per stage so that blocks of 24 or 32 trials leave
// the fewest trial slots idle (e.g. groups of 24 fine DMs).
constexpr int kSubTI = 16, kSubDR = 8;

template <typename Tin, bool kInt, bool kStats, int TI, int DR, int NW>
__global__ void __launch_bounds__(NW * 32, 3) sub_kernel(SubLaunch a)
{
    constexpr int kTile = 32 * TI, kDmBlk = DR * NW;
    extern __shared__ __align__(128) unsigned char smem[];
    const Tin *__restrict__ in = static_cast<const Tin *>(a.in);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rs = a.rs, ch = a.ch;

    const int64_t lin = blockIdx.x;
    const int64_t per_group = (int64_t)a.dgroup * a.ntile;
    const int64_t grp = lin / per_group;
    const int64_t rr = lin - grp * per_group;
    const int gsize = min(a.dgroup, a.nblk - (int)grp * a.dgroup);
    const int blk = (int)grp * a.dgroup + (int)(rr % gsize);
    const int64_t t0 = (rr / gsize) * kTile;
    const SubBlock B = a.blocks[blk];
    const int nchans = B.nc;

    const size_t stage_elems = (size_t)ch * rs;
    Tin *rows = reinterpret_cast<Tin *>(smem);
    int32_t *soffs = reinterpret_cast<int32_t *>(smem + kStages * stage_elems * sizeof(Tin));
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + a.bar_off);
    const int32_t *boffs = a.offs + (size_t)B.tab * kDmBlk;
    const int32_t *bbase = a.base + B.tab;
    const int nst = (nchans + ch - 1) / ch;

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
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
        const int buf = s % kStages;
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
            const int64_t r = (int64_t)B.in_row + (int64_t)(c0 + cc) * a.in_rstride;
            if (nb)
                bulk_g2s(rows + (size_t)buf * stage_elems + (size_t)cc * rs, in + r * a.pitch + g, nb,
                         &bar[buf]);
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
        const int buf = s % kStages;
        if (ok) ok = mbar_wait(&bar[buf], (uint32_t)((s / kStages) & 1), a.err);
        const int cn = min(ch, nchans - s * ch);
        const Tin *srow = rows + (size_t)buf * stage_elems + lane;
        const int32_t *so = soffs + (size_t)buf * ch * kDmBlk + warp * DR;
        for (int cc = 0; cc < cn; ++cc) {
            const Tin *r = srow + (size_t)cc * rs;
            int o[DR];
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
    ok = __syncthreads_and(ok);
    if (!ok) return;

    const int64_t nout = a.nout;
    if constexpr (kInt) {
        long long n = 0, s = 0;
        unsigned long long q = 0;
        int32_t *out = reinterpret_cast<int32_t *>(a.out);
#pragma unroll
        for (int j = 0; j < DR; ++j) {
            const int jr = warp * DR + j;
#pragma unroll
            for (int i = 0; i < TI; ++i) {
                const int64_t t = t0 + lane + 32 * i;
                if (jr < B.ntr && t < nout) {
                    const long long v = __float2int_rn(acc[j][i]);
                    out[(size_t)(B.row0 + jr) * a.out_pitch + t] = (int32_t)v;
                    n++; s += v; q += (unsigned long long)(v * v);
                }
            }
        }
        if constexpr (kStats) block_stat_i(n, s, q, reinterpret_cast<StatI *>(a.partials) + lin);
    } else {
        int n = 0;
        float s = 0.f;
        float *out = reinterpret_cast<float *>(a.out);
#pragma unroll
        for (int j = 0; j < DR; ++j) {
            const int jr = warp * DR + j;
#pragma unroll
            for (int i = 0; i < TI; ++i) {
                const int64_t t = t0 + lane + 32 * i;
                if (jr < B.ntr && t < nout) {
                    out[(size_t)(B.row0 + jr) * a.out_pitch + t] = acc[j][i];
                    n++; s += acc[j][i];
                }
            }
        }
        if constexpr (kStats) {
            const float m = n ? s / (float)n : 0.f;
            float q = 0.f;
#pragma unroll
            for (int j = 0; j < DR; ++j) {
                const int jr = warp * DR + j;
#pragma unroll
                for (int i = 0; i < TI; ++i) {
                    const int64_t t = t0 + lane + 32 * i;
                    if (jr < B.ntr && t < nout) { const float d = acc[j][i] - m; q += d * d; }
                }
            }
            block_stat_f32(n, s, q, reinterpret_cast<StatF *>(a.partials) + lin);
        }
    }
}

// stage 1 (input dtype -> float series) and stage 2 (float series -> out)
template <typename Tin, bool kInt, bool kStats>
static cudaError_t sub_launch(const SubLaunch &a, int nw, cudaStream_t s)
{
    const unsigned grid = (unsigned)(a.ntile * a.nblk);
    if (nw == 3)
        sub_kernel<Tin, kInt, kStats, kSubTI, kSubDR, 3><<<grid, 3 * 32, a.smem, s>>>(a);
    else
        sub_kernel<Tin, kInt, kStats, kSubTI, kSubDR, 4><<<grid, 4 * 32, a.smem, s>>>(a);
    return cudaGetLastError();
}

template <typename Tin, bool kInt, bool kStats>
static cudaError_t sub_prepare_one(size_t optin)
{
    cudaError_t e = allow_max_dynamic_smem((const void *)sub_kernel<Tin, kInt, kStats, kSubTI, kSubDR, 3>, optin);
    if (e == cudaSuccess)
        e = allow_max_dynamic_smem((const void *)sub_kernel<Tin, kInt, kStats, kSubTI, kSubDR, 4>, optin);
    return e;
}

static cudaError_t sub_prepare(size_t optin)
{
    cudaError_t e = sub_prepare_one<float, false, false>(optin);
    if (e == cudaSuccess) e = sub_prepare_one<__half, false, false>(optin);
    if (e == cudaSuccess) e = sub_prepare_one<uint8_t, false, false>(optin);
    if (e == cudaSuccess) e = sub_prepare_one<float, false, true>(optin);
    if (e == cudaSuccess) e = sub_prepare_one<float, true, true>(optin);
    return e;
}

// Warps per block (3 or 4) for runs of n trials: fewest idle trial slots,
// ties to 4.
static int pick_nw(int n)
{
    auto idle = [&](int nw) { const int db = kSubDR * nw; return (n + db - 1) / db * db - n; };
    return idle(3) < idle(4) ? 3 : 4;
}

// One stage's block list and delay records, host and device.
struct SubStage {
    int nw = 4, db = 32;             // warps per block, trials per block
    std::vector<SubBlock> blocks;
    std::vector<int32_t> offs, base;
    SubBlock *d_blocks = nullptr;
    int32_t *d_offs = nullptr, *d_base = nullptr;
    int rs = 0, ch = 0, bar_off = 0;
    size_t smem = 0;

    void release()
    {
        if (d_blocks) cudaFree(d_blocks);
        if (d_offs) cudaFree(d_offs);
        if (d_base) cudaFree(d_base);
        d_blocks = nullptr; d_offs = nullptr; d_base = nullptr;
    }
};

// Append a block: delay(j, c) for j < ntr trials, c < nc channels.
template <typename F>
static void add_block(SubStage &st, int in_row, int nc, int row0, int ntr, int al, long long &need, F delay)
{
    SubBlock b{};
    b.in_row = in_row; b.nc = nc; b.row0 = row0; b.ntr = ntr;
    b.tab = (int32_t)st.base.size();
    st.blocks.push_back(b);
    for (int c = 0; c < nc; ++c) {
        int lo = INT_MAX, hi = 0;
        for (int j = 0; j < ntr; ++j) { const int d = delay(j, c); lo = std::min(lo, d); hi = std::max(hi, d); }
        const int r0 = lo - (lo % al);
        st.base.push_back(r0);
        for (int j = 0; j < st.db; ++j) st.offs.push_back(delay(std::min(j, ntr - 1), c) - r0);
        need = std::max<long long>(need, (long long)(hi - r0) + 32LL * kSubTI);
    }
}

static int finish_stage(SubStage &st, long long need, size_t eb, size_t optin)
{
    st.rs = (int)((need + 15) / 16 * 16);
    const size_t budget = std::min<size_t>(optin, (228 * 1024) / 3 - 1024) - 1024;
    const size_t per_ch = (size_t)st.rs * eb + (size_t)st.db * sizeof(int32_t);
    st.ch = (int)std::min<size_t>(16, budget / (kStages * per_ch));
    if (st.ch < 1) return set_error(DD_ERR_ARG, "subband rows too long for shared memory (%d samples)", st.rs);
    st.bar_off = (int)(((size_t)kStages * st.ch * per_ch + 15) / 16 * 16);
    st.smem = (size_t)st.bar_off + kStages * sizeof(uint64_t);
    cudaError_t e = cudaMalloc(&st.d_blocks, st.blocks.size() * sizeof(SubBlock));
    if (e == cudaSuccess) e = cudaMalloc(&st.d_offs, st.offs.size() * 4);
    if (e == cudaSuccess) e = cudaMalloc(&st.d_base, st.base.size() * 4);
    if (e == cudaSuccess)
        e = cudaMemcpy(st.d_blocks, st.blocks.data(), st.blocks.size() * sizeof(SubBlock), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(st.d_offs, st.offs.data(), st.offs.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(st.d_base, st.base.data(), st.base.size() * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { st.release(); return cuda_fail(e, "subband tables"); }
    return DD_OK;
}

}  // namespace dd

using namespace dd;

struct dd_subband_plan {
    dd_plan *fine = nullptr;          // fine-DM plan: delay table, search and statistics
    int G = 0, nsub = 0, cs = 0, K = 0;
    std::vector<double> nominal;      // [K]
    std::vector<int32_t> d1;          // [K][nchans]
    std::vector<int32_t> d2;          // [ndm][nsub]
    int64_t maxshift = 0, nsamp_out = 0, L = 0;
    SubStage st1, st2;
    float *d_inter = nullptr;         // [nsub][K][L] partially de-dispersed series
    int *d_err = nullptr;
};

static void free_subband(dd_subband_plan *p)
{
    if (!p) return;
    p->st1.release();
    p->st2.release();
    if (p->d_inter) cudaFree(p->d_inter);
    if (p->d_err) cudaFree(p->d_err);
    if (p->fine) dd_plan_destroy(p->fine);
    delete p;
}

extern "C" {

int dd_subband_plan_create(int32_t nchans, double fch1_mhz, double foff_mhz, double tsamp_s,
                           const double *dm_list, int32_t ndm, int32_t dms_per_nominal, int32_t nsub,
                           const int32_t *boxcar_widths, int32_t nwidths, double sigma,
                           int32_t in_dtype, int64_t nsamp_in, dd_subband_plan **plan_out)
{
    if (!plan_out) return set_error(DD_ERR_ARG, "plan_out is NULL");
    *plan_out = nullptr;
    if (dms_per_nominal < 1) return set_error(DD_ERR_ARG, "dms_per_nominal must be >= 1");
    if (nsub < 1 || nchans < 1 || nchans % nsub != 0)
        return set_error(DD_ERR_ARG, "nsub must be >= 1 and divide nchans");
    dd_subband_plan *p = new (std::nothrow) dd_subband_plan();
    if (!p) return set_error(DD_ERR_NOMEM, "host allocation failed");
    int rc = plan_create(nchans, fch1_mhz, foff_mhz, tsamp_s, dm_list, ndm, boxcar_widths, nwidths, sigma,
                         in_dtype, nsamp_in, false, &p->fine);
    if (rc) { free_subband(p); return rc; }
    dd_plan *f = p->fine;
    const int C = nchans, D = ndm, G = dms_per_nominal, S = nsub, cs = nchans / nsub;
    const int K = (D + G - 1) / G;
    p->G = G; p->nsub = S; p->cs = cs; p->K = K;
    auto ref = [&](int s) { return foff_mhz < 0.0 ? s * cs : s * cs + cs - 1; };

    // nominal DMs and the two stages' delays (Section 3.2)
    p->nominal.resize(K);
    std::vector<int32_t> dn((size_t)K * C);
    for (int k = 0; k < K; ++k) {
        const int j0 = k * G, j1 = std::min(j0 + G, D) - 1;
        p->nominal[k] = 0.5 * (dm_list[j0] + dm_list[j1]);
        for (int c = 0; c < C; ++c)
            dn[(size_t)k * C + c] = (int32_t)delay_samples(fch1_mhz, foff_mhz, C, tsamp_s, p->nominal[k], c);
    }
    p->d1.resize((size_t)K * C);
    for (int k = 0; k < K; ++k)
        for (int c = 0; c < C; ++c)
            p->d1[(size_t)k * C + c] = dn[(size_t)k * C + c] - dn[(size_t)k * C + ref(c / cs)];
    p->d2.resize((size_t)D * S);
    int d2max = 0;
    for (int j = 0; j < D; ++j)
        for (int s = 0; s < S; ++s) {
            p->d2[(size_t)j * S + s] = f->delays[(size_t)j * C + ref(s)];
            d2max = std::max(d2max, p->d2[(size_t)j * S + s]);
        }
    long long m = 0;
    for (int j = 0; j < D; ++j)
        for (int c = 0; c < C; ++c)
            m = std::max<long long>(m, (long long)p->d2[(size_t)j * S + c / cs] + p->d1[(size_t)(j / G) * C + c]);
    if (nsamp_in <= m) {
        free_subband(p);
        return set_error(DD_ERR_ARG, "nsamp_in (%lld) must exceed the subband maxshift (%lld)",
                         (long long)nsamp_in, m);
    }
    p->maxshift = m;
    p->nsamp_out = nsamp_in - m;
    for (int i = 0; i < nwidths; ++i)
        if (boxcar_widths[i] > p->nsamp_out) {
            free_subband(p);
            return set_error(DD_ERR_ARG, "boxcar width %d exceeds nsamp_out", boxcar_widths[i]);
        }
    f->maxshift = p->maxshift;          // the search runs over the subband output
    f->nsamp_out = p->nsamp_out;
    p->L = (p->nsamp_out + d2max + 3) / 4 * 4;

    // stage 1 blocks: per subband, nominal DMs in chunks of db
    const int al_in = (int)(16 / in_elem_bytes((dd_dtype)in_dtype));
    long long need1 = 0, need2 = 0;
    p->st1.nw = pick_nw(K); p->st1.db = kSubDR * p->st1.nw;
    p->st2.nw = pick_nw(G); p->st2.db = kSubDR * p->st2.nw;
    const int db1 = p->st1.db, db2 = p->st2.db;
    for (int s = 0; s < S; ++s)
        for (int k0 = 0; k0 < K; k0 += db1) {
            const int nt = std::min(db1, K - k0);
            add_block(p->st1, s * cs, cs, s * K + k0, nt, al_in, need1,
                      [&](int j, int c) { return p->d1[(size_t)(k0 + j) * C + s * cs + c]; });
        }
    // stage 2 blocks: per group, fine DMs in chunks of kSubDB; channel s of
    // group k is series row s*K + k
    for (int k = 0; k < K; ++k) {
        const int j0 = k * G, j1 = std::min(j0 + G, D);
        for (int jb = j0; jb < j1; jb += db2) {
            const int nt = std::min(db2, j1 - jb);
            add_block(p->st2, k, S, jb, nt, 4, need2,
                      [&](int j, int s) { return p->d2[(size_t)(jb + j) * S + s]; });
        }
    }
    rc = finish_stage(p->st1, need1, in_elem_bytes((dd_dtype)in_dtype), f->smem_optin);
    if (rc == DD_OK) rc = finish_stage(p->st2, need2, 4, f->smem_optin);
    if (rc) { free_subband(p); return rc; }
    cudaError_t e = sub_prepare(f->smem_optin);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(p->d_err, 0, sizeof(int));
    if (e != cudaSuccess) { rc = cuda_fail(e, "subband setup"); free_subband(p); return rc; }
    *plan_out = p;
    return DD_OK;
}

int dd_subband_plan_destroy(dd_subband_plan *plan)
{
    if (!plan) return DD_OK;
    cudaDeviceSynchronize();
    free_subband(plan);
    return DD_OK;
}

int dd_subband_plan_info(const dd_subband_plan *plan, int32_t *n_nominal, int64_t *maxshift,
                         int64_t *nsamp_out, double *nominal_dms, int32_t *stage1_delays,
                         int32_t *stage2_delays, int64_t *work_bytes)
{
    if (!plan) return set_error(DD_ERR_ARG, "plan is NULL");
    if (n_nominal) *n_nominal = plan->K;
    if (maxshift) *maxshift = plan->maxshift;
    if (nsamp_out) *nsamp_out = plan->nsamp_out;
    if (nominal_dms) memcpy(nominal_dms, plan->nominal.data(), plan->nominal.size() * sizeof(double));
    if (stage1_delays) memcpy(stage1_delays, plan->d1.data(), plan->d1.size() * sizeof(int32_t));
    if (stage2_delays) memcpy(stage2_delays, plan->d2.data(), plan->d2.size() * sizeof(int32_t));
    if (work_bytes) *work_bytes = (int64_t)plan->nsub * plan->K * plan->L * (int64_t)sizeof(float);
    return DD_OK;
}

int dd_subband_execute(dd_subband_plan *plan, const void *in_dev, int64_t in_pitch, void *out_dev,
                       void *stream)
{
    if (!plan) return set_error(DD_ERR_ARG, "plan is NULL");
    dd_plan *f = plan->fine;
    if (!in_dev || !out_dev) return set_error(DD_ERR_ARG, "NULL buffer");
    if (in_pitch < f->nsamp_in) return set_error(DD_ERR_ARG, "in_pitch < nsamp_in");
    const int al = (int)(16 / in_elem_bytes(f->dtype));
    if (((uintptr_t)in_dev & 15u) || (in_pitch % al))
        return set_error(DD_ERR_ARG, "subband input rows must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t inter = (size_t)plan->nsub * plan->K * plan->L * sizeof(float);
    if (!plan->d_inter) {
        cudaError_t e = cudaMalloc(&plan->d_inter, inter);
        if (e != cudaSuccess) { plan->d_inter = nullptr; return cuda_fail(e, "cudaMalloc(subband series)"); }
    }
    constexpr int kTile = 32 * kSubTI;

    // stage 1: input -> series [nsub][K][L]
    SubLaunch a{};
    a.in = in_dev; a.pitch = in_pitch; a.in_rstride = 1;
    a.nsamp_in_al = (f->nsamp_in + al - 1) / al * al;
    a.blocks = plan->st1.d_blocks; a.offs = plan->st1.d_offs; a.base = plan->st1.d_base;
    a.nblk = (int)plan->st1.blocks.size(); a.rs = plan->st1.rs; a.ch = plan->st1.ch;
    a.bar_off = plan->st1.bar_off; a.smem = plan->st1.smem;
    a.ntile = (plan->L + kTile - 1) / kTile; a.dgroup = 8;
    a.out = plan->d_inter; a.out_pitch = plan->L; a.nout = plan->L;
    a.partials = nullptr; a.err = plan->d_err;
    if (a.ntile * a.nblk > INT32_MAX) return set_error(DD_ERR_ARG, "subband stage 1 grid too large");
    const int nw1 = plan->st1.nw, nw2 = plan->st2.nw;
    cudaError_t e = f->dtype == DD_F32 ? sub_launch<float, false, false>(a, nw1, s)
                  : f->dtype == DD_F16 ? sub_launch<__half, false, false>(a, nw1, s)
                                       : sub_launch<uint8_t, false, false>(a, nw1, s);
    if (e != cudaSuccess) return cuda_fail(e, "launch subband stage 1");

    // stage 2: series -> out [ndm][nsamp_out], with statistics partials
    SubLaunch b{};
    b.in = plan->d_inter; b.pitch = plan->L; b.in_rstride = plan->K; b.nsamp_in_al = plan->L;
    b.blocks = plan->st2.d_blocks; b.offs = plan->st2.d_offs; b.base = plan->st2.d_base;
    b.nblk = (int)plan->st2.blocks.size(); b.rs = plan->st2.rs; b.ch = plan->st2.ch;
    b.bar_off = plan->st2.bar_off; b.smem = plan->st2.smem;
    b.ntile = (plan->nsamp_out + kTile - 1) / kTile; b.dgroup = 8;
    b.out = out_dev; b.out_pitch = plan->nsamp_out; b.nout = plan->nsamp_out;
    b.err = plan->d_err;
    const int64_t np = b.ntile * b.nblk;
    if (np > INT32_MAX) return set_error(DD_ERR_ARG, "subband stage 2 grid too large");
    int rc = ensure_partials_public(f, np);
    if (rc) return rc;
    b.partials = f->d_partials;
    e = f->dtype == DD_U8 ? sub_launch<float, true, true>(b, nw2, s) : sub_launch<float, false, true>(b, nw2, s);
    if (e != cudaSuccess) return cuda_fail(e, "launch subband stage 2");
    f->n_partials = np;
    f->stats_out = out_dev;
    return DD_OK;
}

int dd_subband_search(dd_subband_plan *plan, const void *out_dev, dd_candidate *cand_host,
                      int64_t capacity, int64_t *n_found, void *stream)
{
    if (!plan) return set_error(DD_ERR_ARG, "plan is NULL");
    const int rc = dd_search(plan->fine, out_dev, cand_host, capacity, n_found, stream);
    if (rc != DD_OK && rc != DD_ERR_OVERFLOW) return rc;
    int h = 0;
    cudaError_t e = cudaMemcpy(&h, plan->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read subband status");
    if (h) {
        cudaMemset(plan->d_err, 0, sizeof(int));
        return set_error(h, "subband kernel gave up waiting for its input copies (status %d)", h);
    }
    return rc;
}

int dd_subband_last_stats(const dd_subband_plan *plan, double *mu, double *sigma)
{
    if (!plan) return set_error(DD_ERR_ARG, "plan is NULL");
    return dd_last_stats(plan->fine, mu, sigma);
}

}  // extern "C"

// ===================================================================== survey
// Multi-pass survey plans (Section 3.2 with binning; the plans of Table 1 /
// Table 4): each pass bins the input by its factor N_b (average of N_b
// adjacent samples) and runs subband de-dispersion over its DM range at the
// binned sampling time.

namespace dd {

// out[c][i] = (1/nb) * sum_{q<nb} in[c][i*nb + q], float32 result.  Thread i
// of a row reads nb consecutive samples: a warp covers 32*nb consecutive
// inputs, so the reads are coalesced for any nb.
template <typename Tin>
__global__ void bin_kernel(const Tin *__restrict__ in, int64_t pitch, int64_t nbin, int nb,
                           float *__restrict__ out, int64_t out_pitch)
{
    const int64_t c = blockIdx.y;
    const float inv = 1.0f / (float)nb;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nbin;
         i += (int64_t)gridDim.x * blockDim.x) {
        const Tin *p = in + c * pitch + i * nb;
        float s = 0.f;
        for (int q = 0; q < nb; ++q) s += lane_ld<Tin>(p + q);
        out[c * out_pitch + i] = nb == 1 ? s : s * inv;
    }
}

}  // namespace dd

struct dd_survey_plan {
    int nchans = 0;
    dd_dtype dtype = DD_F32;
    int64_t nsamp_in = 0;
    std::vector<dd_subband_plan *> sub;   // one per pass
    std::vector<int> bin;
    std::vector<float *> d_bin;            // binned input per pass (bin > 1)
    std::vector<int64_t> bin_n, bin_pitch;
};

static void free_survey(dd_survey_plan *p)
{
    if (!p) return;
    for (auto *s : p->sub) free_subband(s);
    for (auto *b : p->d_bin) if (b) cudaFree(b);
    delete p;
}

extern "C" {

int dd_survey_plan_create(int32_t nchans, double fch1_mhz, double foff_mhz, double tsamp_s,
                          const dd_survey_pass *passes, int32_t npass, int32_t nsub,
                          const int32_t *boxcar_widths, int32_t nwidths, double sigma,
                          int32_t in_dtype, int64_t nsamp_in, dd_survey_plan **plan_out)
{
    if (!plan_out) return set_error(DD_ERR_ARG, "plan_out is NULL");
    *plan_out = nullptr;
    if (!passes || npass < 1) return set_error(DD_ERR_ARG, "need npass >= 1 passes");
    dd_survey_plan *p = new (std::nothrow) dd_survey_plan();
    if (!p) return set_error(DD_ERR_NOMEM, "host allocation failed");
    p->nchans = nchans; p->dtype = (dd_dtype)in_dtype; p->nsamp_in = nsamp_in;
    for (int i = 0; i < npass; ++i) {
        const dd_survey_pass &ps = passes[i];
        if (!(ps.dm_step > 0.0) || !(ps.high_dm > ps.low_dm) || ps.bin < 1 || !(ps.sub_dm_step > 0.0)) {
            free_survey(p);
            return set_error(DD_ERR_ARG, "pass %d: need dm_step > 0, high_dm > low_dm, bin >= 1, sub_dm_step > 0", i);
        }
        const long long ndm = llround((ps.high_dm - ps.low_dm) / ps.dm_step);
        const long long G = llround(ps.sub_dm_step / ps.dm_step);
        if (ndm < 1 || ndm > INT32_MAX || G < 1) {
            free_survey(p);
            return set_error(DD_ERR_ARG, "pass %d: fewer than one DM trial or trial per nominal DM", i);
        }
        std::vector<double> dms((size_t)ndm);
        for (long long j = 0; j < ndm; ++j) dms[(size_t)j] = ps.low_dm + (double)j * ps.dm_step;
        const int64_t nb = nsamp_in / ps.bin;
        dd_subband_plan *sp = nullptr;
        const int rc = dd_subband_plan_create(nchans, fch1_mhz, foff_mhz, tsamp_s * (double)ps.bin, dms.data(),
                                              (int32_t)ndm, (int32_t)G, nsub, boxcar_widths, nwidths, sigma,
                                              ps.bin == 1 ? in_dtype : (int32_t)DD_F32, nb, &sp);
        if (rc) { free_survey(p); return rc; }
        p->sub.push_back(sp);
        p->bin.push_back(ps.bin);
        p->d_bin.push_back(nullptr);
        p->bin_n.push_back(nb);
        p->bin_pitch.push_back((nb + 3) / 4 * 4);
    }
    *plan_out = p;
    return DD_OK;
}

int dd_survey_plan_destroy(dd_survey_plan *plan)
{
    if (!plan) return DD_OK;
    cudaDeviceSynchronize();
    free_survey(plan);
    return DD_OK;
}

int dd_survey_pass_info(const dd_survey_plan *plan, int32_t pass, int32_t *ndm, int32_t *bin,
                        int32_t *dms_per_nominal, int64_t *maxshift, int64_t *nsamp_out, double *dm_list)
{
    if (!plan) return set_error(DD_ERR_ARG, "plan is NULL");
    if (pass < 0 || pass >= (int)plan->sub.size()) return set_error(DD_ERR_ARG, "no pass %d", pass);
    const dd_subband_plan *sp = plan->sub[pass];
    if (ndm) *ndm = sp->fine->ndm;
    if (bin) *bin = plan->bin[pass];
    if (dms_per_nominal) *dms_per_nominal = sp->G;
    if (maxshift) *maxshift = sp->maxshift;
    if (nsamp_out) *nsamp_out = sp->nsamp_out;
    if (dm_list) memcpy(dm_list, sp->fine->dm_list.data(), sp->fine->dm_list.size() * sizeof(double));
    return DD_OK;
}

int dd_survey_execute(dd_survey_plan *plan, const void *in_dev, int64_t in_pitch, void *const *out_devs,
                      void *stream)
{
    if (!plan) return set_error(DD_ERR_ARG, "plan is NULL");
    if (!in_dev || !out_devs) return set_error(DD_ERR_ARG, "NULL buffer");
    if (in_pitch < plan->nsamp_in) return set_error(DD_ERR_ARG, "in_pitch < nsamp_in");
    cudaStream_t s = (cudaStream_t)stream;
    for (size_t i = 0; i < plan->sub.size(); ++i) {
        if (!out_devs[i]) return set_error(DD_ERR_ARG, "out_devs[%d] is NULL", (int)i);
        const void *src = in_dev;
        int64_t pitch = in_pitch;
        const int nb = plan->bin[i];
        if (nb > 1) {
            if (!plan->d_bin[i]) {
                cudaError_t e = cudaMalloc(&plan->d_bin[i], (size_t)plan->nchans * plan->bin_pitch[i] * sizeof(float));
                if (e != cudaSuccess) { plan->d_bin[i] = nullptr; return cuda_fail(e, "cudaMalloc(binned input)"); }
            }
            const int64_t n = plan->bin_n[i];
            const dim3 grid((unsigned)std::min<int64_t>((n + 255) / 256, 4096), (unsigned)plan->nchans);
            if (plan->dtype == DD_F32)
                bin_kernel<float><<<grid, 256, 0, s>>>((const float *)in_dev, in_pitch, n, nb, plan->d_bin[i], plan->bin_pitch[i]);
            else if (plan->dtype == DD_F16)
                bin_kernel<__half><<<grid, 256, 0, s>>>((const __half *)in_dev, in_pitch, n, nb, plan->d_bin[i], plan->bin_pitch[i]);
            else
                bin_kernel<uint8_t><<<grid, 256, 0, s>>>((const uint8_t *)in_dev, in_pitch, n, nb, plan->d_bin[i], plan->bin_pitch[i]);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail(e, "launch bin_kernel");
            src = plan->d_bin[i];
            pitch = plan->bin_pitch[i];
        }
        const int rc = dd_subband_execute(plan->sub[i], src, pitch, out_devs[i], stream);
        if (rc) return rc;
    }
    return DD_OK;
}

int dd_survey_search(dd_survey_plan *plan, int32_t pass, const void *out_dev, dd_candidate *cand_host,
                     int64_t capacity, int64_t *n_found, void *stream)
{
    if (!plan) return set_error(DD_ERR_ARG, "plan is NULL");
    if (pass < 0 || pass >= (int)plan->sub.size()) return set_error(DD_ERR_ARG, "no pass %d", pass);
    return dd_subband_search(plan->sub[pass], out_dev, cand_host, capacity, n_found, stream);
}

int dd_survey_last_stats(const dd_survey_plan *plan, int32_t pass, double *mu, double *sigma)
{
    if (!plan) return set_error(DD_ERR_ARG, "plan is NULL");
    if (pass < 0 || pass >= (int)plan->sub.size()) return set_error(DD_ERR_ARG, "no pass %d", pass);
    return dd_subband_last_stats(plan->sub[pass], mu, sigma);
}

}  // extern "C"
