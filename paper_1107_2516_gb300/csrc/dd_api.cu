// libdd C ABI: plan creation (Eq. 1 delay table in double on the host),
// execution and search entry points.  See include/dd.h for the contract.
#include "dd_internal.h"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

namespace dd {

static thread_local char g_err[512] = "";

int set_error(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return set_error(e == cudaErrorMemoryAllocation ? DD_ERR_NOMEM : DD_ERR_CUDA,
                     "%s: %s", what, cudaGetErrorString(e));
}

size_t in_elem_bytes(dd_dtype t)
{
    return t == DD_F32 ? 4 : (t == DD_F16 ? 2 : 1);
}

// Eq. 1 divided by the sampling time, relative to the highest channel centre.
// Evaluated as ((4.15e6*DM) * (1/f^2 - 1/f_top^2)) / (tsamp*1e3) in double,
// left to right; this file is compiled with FMA contraction off so the
// rounding of every step is fixed.  Rounded half away from zero.
long long delay_samples(double fch1, double foff, int nchans, double tsamp_s,
                        double dm, int c)
{
    const double f_top = (foff < 0.0) ? fch1 + 0.0 * foff : fch1 + (double)(nchans - 1) * foff;
    const double f = fch1 + (double)c * foff;
    const double tsamp_ms = tsamp_s * 1e3;
    const double k = 4.15e6 * dm;
    const double diff = 1.0 / (f * f) - 1.0 / (f_top * f_top);
    return llround((k * diff) / tsamp_ms);
}

// Largest delay over all channels at the deepest DM trial (the plan's
// maxshift), without building a plan; -1 for invalid arguments.
long long max_delay(int nchans, double fch1, double foff, double tsamp_s, const double *dm_list, int ndm)
{
    if (nchans < 1 || ndm < 1 || !dm_list || !(tsamp_s > 0.0)) return -1;
    double dmax = 0.0;
    for (int i = 0; i < ndm; ++i) {
        if (!(dm_list[i] >= 0.0)) return -1;
        dmax = std::max(dmax, dm_list[i]);
    }
    long long m = 0;
    for (int c = 0; c < nchans; ++c) m = std::max(m, delay_samples(fch1, foff, nchans, tsamp_s, dmax, c));
    return m;
}

static void free_plan(dd_plan *p)
{
    if (!p) return;
    fast_release(p);
    if (p->d_gen) cudaFree(p->d_gen);
    if (p->d_partials) cudaFree(p->d_partials);
    if (p->d_params) cudaFree(p->d_params);
    if (p->d_wsorted) cudaFree(p->d_wsorted);
    if (p->d_cands) cudaFree(p->d_cands);
    if (p->d_count) cudaFree(p->d_count);
    if (p->h_count) cudaFreeHost(p->h_count);
    if (p->h_params) cudaFreeHost(p->h_params);
    if (p->d_rowprm) cudaFree(p->d_rowprm);
    if (p->h_rowprm) cudaFreeHost(p->h_rowprm);
    if (p->d_in_stage) cudaFree(p->d_in_stage);
    if (p->d_out_stage) cudaFree(p->d_out_stage);
    delete p;
}

static int ensure_cands(dd_plan *p, int64_t cap)
{
    if (cap <= p->cand_cap) return DD_OK;
    if (p->d_cands) cudaFree(p->d_cands);
    p->d_cands = nullptr;
    p->cand_cap = 0;
    cudaError_t e = cudaMalloc(&p->d_cands, (size_t)cap * sizeof(dd_candidate));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(candidates)");
    p->cand_cap = cap;
    return DD_OK;
}

// Synchronise `s`, read the search results of the plan's last search_launch
// (dev_cap = the candidate capacity that launch used) and sort them.
int search_readback(dd_plan *plan, dd_candidate *cand_host, int64_t capacity, int64_t *n_found,
                    cudaStream_t s, int64_t dev_cap)
{
    cudaError_t e = cudaMemcpyAsync(plan->h_count, plan->d_count, sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(plan->h_params, plan->d_params, sizeof(SearchParams), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && plan->row_stats && plan->d_rowprm)
        e = cudaMemcpyAsync(plan->h_rowprm, plan->d_rowprm, (size_t)plan->ndm * sizeof(RowParams),
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "search readback");
    int rc = fast_error(plan, s);
    if (rc) return rc;
    const int64_t total = (int64_t)*plan->h_count;
    const int64_t n = std::min<int64_t>(std::min<int64_t>(total, dev_cap), capacity);
    plan->last_mu = plan->h_params->mu;
    plan->last_sigma = plan->h_params->sigma;
    if (n > 0) {
        e = cudaMemcpyAsync(cand_host, plan->d_cands, (size_t)n * sizeof(dd_candidate),
                            cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "candidate readback");
        std::sort(cand_host, cand_host + n, [](const dd_candidate &a, const dd_candidate &b) {
            if (a.dm_idx != b.dm_idx) return a.dm_idx < b.dm_idx;
            if (a.t != b.t) return a.t < b.t;
            return a.width_idx < b.width_idx;
        });
    }
    *n_found = total;
    if (total > capacity || total > dev_cap)
        return set_error(DD_ERR_OVERFLOW, "%lld candidates exceed capacity %lld",
                         (long long)total, (long long)std::min(capacity, dev_cap));
    return DD_OK;
}

}  // namespace dd

using namespace dd;

extern "C" {

const char *dd_last_error(void) { return g_err; }

const char *dd_version(void) { return "libdd 0.1 (sm_103a)"; }

int dd_plan_create(int32_t nchans, double fch1_mhz, double foff_mhz, double tsamp_s,
                   const double *dm_list, int32_t ndm,
                   const int32_t *boxcar_widths, int32_t nwidths, double sigma_k,
                   int32_t in_dtype, int64_t nsamp_in, dd_plan **plan_out)
{
    return dd::plan_create(nchans, fch1_mhz, foff_mhz, tsamp_s, dm_list, ndm, boxcar_widths, nwidths,
                           sigma_k, in_dtype, nsamp_in, true, plan_out);
}

}  // extern "C"

namespace dd {

int plan_create(int32_t nchans, double fch1_mhz, double foff_mhz, double tsamp_s,
                const double *dm_list, int32_t ndm, const int32_t *boxcar_widths, int32_t nwidths,
                double sigma_k, int32_t in_dtype, int64_t nsamp_in, bool kernels, dd_plan **plan_out)
{
    g_err[0] = 0;
    if (!plan_out) return set_error(DD_ERR_ARG, "plan_out is NULL");
    *plan_out = nullptr;
    if (nchans < 1) return set_error(DD_ERR_ARG, "nchans must be >= 1 (got %d)", nchans);
    if (in_dtype == DD_U8 && nchans > 65536)
        return set_error(DD_ERR_ARG, "uint8 input supports at most 65536 channels");
    if (ndm < 1 || !dm_list) return set_error(DD_ERR_ARG, "need ndm >= 1 DM trials");
    if (nwidths < 1 || nwidths > kMaxWidths || !boxcar_widths)
        return set_error(DD_ERR_ARG, "need 1..%d boxcar widths", kMaxWidths);
    if (!(tsamp_s > 0.0) || !std::isfinite(tsamp_s)) return set_error(DD_ERR_ARG, "tsamp must be > 0");
    if (!(fch1_mhz > 0.0) || !std::isfinite(fch1_mhz) || !std::isfinite(foff_mhz))
        return set_error(DD_ERR_ARG, "fch1 must be finite and > 0, foff finite");
    if (!(fch1_mhz + (double)(nchans - 1) * foff_mhz > 0.0))
        return set_error(DD_ERR_ARG, "lowest channel centre must be > 0 MHz");
    if (!std::isfinite(sigma_k)) return set_error(DD_ERR_ARG, "sigma must be finite");
    if (in_dtype != DD_F32 && in_dtype != DD_U8 && in_dtype != DD_F16)
        return set_error(DD_ERR_ARG, "unknown input dtype %d", in_dtype);
    if (nsamp_in < 1) return set_error(DD_ERR_ARG, "nsamp_in must be >= 1");
    for (int i = 0; i < ndm; ++i)
        if (!(dm_list[i] >= 0.0) || !std::isfinite(dm_list[i]))
            return set_error(DD_ERR_ARG, "dm_list[%d] must be finite and >= 0", i);

    dd_plan *p = new (std::nothrow) dd_plan();
    if (!p) return set_error(DD_ERR_NOMEM, "host allocation failed");
    p->nchans = nchans; p->ndm = ndm; p->nwidths = nwidths;
    p->dtype = (dd_dtype)in_dtype;
    p->fch1 = fch1_mhz; p->foff = foff_mhz; p->tsamp = tsamp_s; p->sigma_k = sigma_k;
    p->nsamp_in = nsamp_in;
    p->dm_list.assign(dm_list, dm_list + ndm);
    p->widths.assign(boxcar_widths, boxcar_widths + nwidths);

    // Eq. 1 delay table, once per plan, in double on the host.
    p->delays.resize((size_t)ndm * nchans);
    long long m = 0;
    for (int i = 0; i < ndm; ++i)
        for (int c = 0; c < nchans; ++c) {
            const long long d = delay_samples(fch1_mhz, foff_mhz, nchans, tsamp_s, dm_list[i], c);
            if (d < 0 || d > (long long)INT32_MAX / 2) {
                free_plan(p);
                return set_error(DD_ERR_ARG, "delay out of range at dm[%d], channel %d", i, c);
            }
            p->delays[(size_t)i * nchans + c] = (int32_t)d;
            m = std::max(m, d);
        }
    p->maxshift = m;
    if (nsamp_in <= m) {
        free_plan(p);
        return set_error(DD_ERR_ARG, "nsamp_in (%lld) must exceed maxshift (%lld)",
                         (long long)nsamp_in, m);
    }
    p->nsamp_out = nsamp_in - m;
    for (int i = 0; i < nwidths; ++i)
        if (boxcar_widths[i] < 1 || boxcar_widths[i] > 4096 || boxcar_widths[i] > p->nsamp_out) {
            free_plan(p);
            return set_error(DD_ERR_ARG, "boxcar width %d outside 1..min(4096, nsamp_out)",
                             boxcar_widths[i]);
        }

    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) { free_plan(p); return cuda_fail(e, "cudaGetDevice"); }
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, p->device);
    p->sm_count = v;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
    p->smem_optin = (size_t)v;

    // Search scratch: params, widths (sorted + original order), count.
    {
        std::vector<int32_t> idx(nwidths);
        for (int i = 0; i < nwidths; ++i) idx[i] = i;
        std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
            return boxcar_widths[a] < boxcar_widths[b];
        });
        std::vector<int32_t> ws(3 * (size_t)nwidths);
        for (int i = 0; i < nwidths; ++i) {
            ws[i] = boxcar_widths[idx[i]];
            ws[nwidths + i] = idx[i];
            ws[2 * nwidths + i] = boxcar_widths[i];
        }
        e = cudaMalloc(&p->d_wsorted, ws.size() * sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMemcpy(p->d_wsorted, ws.data(), ws.size() * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMalloc(&p->d_params, sizeof(SearchParams));
        if (e == cudaSuccess) e = cudaMalloc(&p->d_count, sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMallocHost(&p->h_count, sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMallocHost(&p->h_params, sizeof(SearchParams));
        if (e != cudaSuccess) { int rc = cuda_fail(e, "plan scratch"); free_plan(p); return rc; }
    }
    int rc = ensure_cands(p, 1 << 16);
    if (kernels) {
        if (rc == DD_OK) rc = generic_configure(p);
        if (rc == DD_OK) rc = fast_configure(p);   // may leave the tiled kernels unavailable
    }
    if (rc != DD_OK) { free_plan(p); return rc; }
    p->kernel = p->fast ? 2 : 1;
    *plan_out = p;
    return DD_OK;
}

}  // namespace dd

extern "C" {

int dd_plan_destroy(dd_plan *plan)
{
    if (!plan) return DD_OK;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(plan->device);
    cudaDeviceSynchronize();
    free_plan(plan);
    cudaSetDevice(prev);
    return DD_OK;
}

int dd_plan_info(const dd_plan *plan, int64_t *maxshift, int64_t *nsamp_out, int32_t *delays_host)
{
    if (!plan) return set_error(DD_ERR_ARG, "plan is NULL");
    if (maxshift) *maxshift = plan->maxshift;
    if (nsamp_out) *nsamp_out = plan->nsamp_out;
    if (delays_host) memcpy(delays_host, plan->delays.data(), plan->delays.size() * sizeof(int32_t));
    return DD_OK;
}

int dd_plan_set_kernel(dd_plan *plan, int32_t kernel)
{
    if (!plan) return set_error(DD_ERR_ARG, "plan is NULL");
    if (kernel == 0) { plan->kernel = plan->fast ? 2 : 1; plan->kernel_req = 0; return DD_OK; }
    if (kernel == 1) { plan->kernel = 1; plan->kernel_req = 1; return DD_OK; }
    if (kernel == 2) {
        if (!plan->fast) return set_error(DD_ERR_ARG, "kernel 2 is not available for this plan");
        if (fast_kernel_id(plan) != 2) {
            int rc = fast_set_tile(plan, 0, 8);
            if (rc) return rc;
        }
        plan->kernel = 2; plan->kernel_req = 2; return DD_OK;
    }
    if (kernel == 3 || kernel == 4 || kernel == 5) {
        // the kernel's tile configurations, fastest measured first
        static const int k3[] = {5, 3, 4, 6}, k4[] = {7, 8}, k5[] = {11, 9, 10};
        const int *cfg = kernel == 3 ? k3 : kernel == 4 ? k4 : k5;
        const int n = kernel == 3 ? 4 : kernel == 4 ? 2 : 3;
        int rc = set_error(DD_ERR_ARG, "kernel %d is not available for this plan", kernel);
        for (int i = 0; plan->fast && i < n && rc != DD_OK; ++i) {
            rc = fast_set_tile(plan, cfg[i], 8);
            if (rc != DD_OK) set_error(DD_ERR_ARG, "kernel %d is not available for this plan", kernel);
        }
        if (rc) return rc;
        plan->kernel = 2; plan->kernel_req = kernel; return DD_OK;
    }
    return set_error(DD_ERR_ARG, "unknown kernel %d", kernel);
}

int dd_plan_get_kernel(const dd_plan *plan, int32_t *kernel)
{
    if (!plan || !kernel) return set_error(DD_ERR_ARG, "NULL argument");
    *kernel = plan->kernel == 2 ? fast_kernel_id(plan) : plan->kernel;
    return DD_OK;
}

int dd_plan_autotune(dd_plan *plan, const void *in_dev, int64_t in_pitch, void *out_dev, void *stream)
{
    if (!plan) return set_error(DD_ERR_ARG, "plan is NULL");
    if (!in_dev || !out_dev) return set_error(DD_ERR_ARG, "NULL buffer");
    if (in_pitch < plan->nsamp_in) return set_error(DD_ERR_ARG, "in_pitch < nsamp_in");
    return fast_autotune(plan, in_dev, in_pitch, out_dev, (cudaStream_t)stream);
}

int dd_plan_set_tile(dd_plan *plan, int32_t config, int32_t raster_group)
{
    if (!plan) return set_error(DD_ERR_ARG, "plan is NULL");
    return fast_set_tile(plan, config, raster_group);
}

int dd_plan_get_tile(const dd_plan *plan, int32_t *config, int32_t *raster_group,
                     int32_t *samples_per_thread, int32_t *warps_per_block)
{
    if (!plan) return set_error(DD_ERR_ARG, "plan is NULL");
    int c = 0, g = 0, tr = 0, nw = 0;
    int rc = fast_get_tile(plan, &c, &g, &tr, &nw);
    if (rc) return rc;
    if (config) *config = c;
    if (raster_group) *raster_group = g;
    if (samples_per_thread) *samples_per_thread = tr;
    if (warps_per_block) *warps_per_block = nw;
    return DD_OK;
}

int dd_execute(dd_plan *plan, const void *in_dev, int64_t in_pitch, void *out_dev, void *stream)
{
    if (!plan) return set_error(DD_ERR_ARG, "plan is NULL");
    if (!in_dev || !out_dev) return set_error(DD_ERR_ARG, "NULL buffer");
    if (in_pitch < plan->nsamp_in) return set_error(DD_ERR_ARG, "in_pitch (%lld) < nsamp_in (%lld)",
                                                    (long long)in_pitch, (long long)plan->nsamp_in);
    cudaStream_t s = (cudaStream_t)stream;
    if (plan->kernel == 2) return fast_execute(plan, in_dev, in_pitch, out_dev, s);
    return generic_execute(plan, in_dev, in_pitch, out_dev, s);
}

int dd_search(dd_plan *plan, const void *out_dev, dd_candidate *cand_host, int64_t capacity,
              int64_t *n_found, void *stream)
{
    if (!plan) return set_error(DD_ERR_ARG, "plan is NULL");
    if (!out_dev || !n_found || capacity < 0 || (capacity > 0 && !cand_host))
        return set_error(DD_ERR_ARG, "bad search arguments");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = DD_OK;
    if (plan->stats_out != out_dev || plan->n_partials == 0) rc = stats_from_out(plan, out_dev, s);
    if (rc) return rc;
    rc = ensure_cands(plan, std::max<int64_t>(capacity, 1));
    if (rc) return rc;
    const int64_t saved_cap = plan->cand_cap;
    plan->cand_cap = std::max<int64_t>(capacity, 0);
    rc = search_launch(plan, out_dev, s);
    const int64_t dev_cap = plan->cand_cap;
    plan->cand_cap = saved_cap;
    if (rc) return rc;
    return search_readback(plan, cand_host, capacity, n_found, s, dev_cap);
}

int dd_plan_set_search_stats(dd_plan *plan, int32_t per_row)
{
    if (!plan) return set_error(DD_ERR_ARG, "plan is NULL");
    if (per_row != 0 && per_row != 1) return set_error(DD_ERR_ARG, "per_row must be 0 or 1");
    if (per_row && !plan->d_rowprm) {
        cudaError_t e = cudaMalloc(&plan->d_rowprm, (size_t)plan->ndm * sizeof(RowParams));
        if (e == cudaSuccess) e = cudaMallocHost(&plan->h_rowprm, (size_t)plan->ndm * sizeof(RowParams));
        if (e == cudaSuccess) memset(plan->h_rowprm, 0, (size_t)plan->ndm * sizeof(RowParams));
        if (e != cudaSuccess) {
            if (plan->d_rowprm) cudaFree(plan->d_rowprm);
            plan->d_rowprm = nullptr;
            plan->h_rowprm = nullptr;
            return cuda_fail(e, "per-row statistics scratch");
        }
    }
    plan->row_stats = per_row;
    return DD_OK;
}

int dd_last_row_stats(const dd_plan *plan, double *mu_rows, double *sigma_rows)
{
    if (!plan) return set_error(DD_ERR_ARG, "plan is NULL");
    if (!plan->row_stats || !plan->h_rowprm) return set_error(DD_ERR_ARG, "per-row statistics are not enabled");
    for (int i = 0; i < plan->ndm; ++i) {
        if (mu_rows) mu_rows[i] = plan->h_rowprm[i].mu;
        if (sigma_rows) sigma_rows[i] = plan->h_rowprm[i].sigma;
    }
    return DD_OK;
}

int dd_last_stats(const dd_plan *plan, double *mu, double *sigma)
{
    if (!plan) return set_error(DD_ERR_ARG, "plan is NULL");
    if (mu) *mu = plan->last_mu;
    if (sigma) *sigma = plan->last_sigma;
    return DD_OK;
}

int dd_process_host(dd_plan *plan, const void *in_host, int64_t in_pitch, dd_candidate *cand_host,
                    int64_t capacity, int64_t *n_found, void *stream)
{
    if (!plan) return set_error(DD_ERR_ARG, "plan is NULL");
    if (!in_host || in_pitch < plan->nsamp_in) return set_error(DD_ERR_ARG, "bad host input");
    const size_t eb = in_elem_bytes(plan->dtype);
    const size_t in_bytes = (size_t)plan->nchans * (size_t)in_pitch * eb;
    const size_t out_bytes = (size_t)plan->ndm * (size_t)plan->nsamp_out * 4;
    cudaError_t e;
    if (plan->in_stage_bytes < in_bytes) {
        if (plan->d_in_stage) cudaFree(plan->d_in_stage);
        plan->d_in_stage = nullptr; plan->in_stage_bytes = 0;
        e = cudaMalloc(&plan->d_in_stage, in_bytes);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(input staging)");
        plan->in_stage_bytes = in_bytes;
    }
    if (plan->out_stage_bytes < out_bytes) {
        if (plan->d_out_stage) cudaFree(plan->d_out_stage);
        plan->d_out_stage = nullptr; plan->out_stage_bytes = 0;
        e = cudaMalloc(&plan->d_out_stage, out_bytes);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(output staging)");
        plan->out_stage_bytes = out_bytes;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // kernels 3 and 5: input copied in column chunks, each chunk's output tiles
    // de-dispersed while the next chunk is in flight; otherwise copy, then execute
    int rc = plan->kernel == 2 ? fast_execute_host(plan, in_host, in_pitch, plan->d_in_stage, plan->d_out_stage, s)
                               : kNotPipelined;
    if (rc == kNotPipelined) {
        e = cudaMemcpyAsync(plan->d_in_stage, in_host, in_bytes, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "H2D input");
        rc = dd_execute(plan, plan->d_in_stage, in_pitch, plan->d_out_stage, stream);
    }
    if (rc) return rc;
    return dd_search(plan, plan->d_out_stage, cand_host, capacity, n_found, stream);
}

}  // extern "C"
