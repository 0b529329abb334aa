// Internal declarations shared by the libdd translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "dd.h"

namespace dd {

// Per-block partial statistics written by the de-dispersion kernels.
// Floating point: (count, mean, M2) merged with the pairwise update of
// Chan, Golub & LeVeque.  Integer: exact (count, sum, sum of squares).
struct StatF { double n, mean, m2; };
struct StatI { long long n, sum; unsigned long long sumsq; };

// Device-side result of the statistics finalisation.
struct SearchParams {
    double mu, sigma;
    int nw;                      // number of boxcar widths
    int pad_;
    float thr_f[64];             // largest float <= T_w (FP compare is then exact)
    long long thr_i[64];         // floor(T_w) (integer compare is then exact)
};

constexpr int kMaxWidths = 64;

// Per-DM-row statistics and thresholds (search option: statistics of each DM
// row instead of the whole buffer), same exact float / integer forms.
struct RowParams {
    double mu, sigma;
    float thr_f[kMaxWidths];
    long long thr_i[kMaxWidths];
};

// Tile shape of the generic kernel (kernel 1).
constexpr int kGenDms = 16;      // DM trials per block
constexpr int kGenThreads = 256; // threads per block
constexpr int kGenTimes = 2;     // samples per thread (strided by kGenThreads)
constexpr int kGenTile = kGenThreads * kGenTimes;

// Register-blocked kernel (kernel 2) constants live in dd_fast.cu.

}  // namespace dd

struct dd_plan {
    // problem
    int32_t nchans = 0, ndm = 0, nwidths = 0;
    dd_dtype dtype = DD_F32;
    double fch1 = 0, foff = 0, tsamp = 0, sigma_k = 0;
    int64_t nsamp_in = 0, maxshift = 0, nsamp_out = 0;
    std::vector<double> dm_list;
    std::vector<int32_t> widths;
    std::vector<int32_t> delays;           // host copy [ndm][nchans]
    int device = 0;
    int sm_count = 0;
    size_t smem_optin = 0;

    // kernel selection
    int32_t kernel_req = 0;                // 0 auto
    int32_t kernel = 1;                    // resolved

    // device data
    int32_t *d_gen = nullptr;              // kernel-1 tables: offsets | base | span
    // generic kernel geometry
    int gen_stride = 0;                    // smem row stride (floats)
    int gen_chunk = 0;                     // channels per smem stage (0: no smem)
    size_t gen_smem = 0;
    // statistics partials of the last dd_execute
    void *d_partials = nullptr;            // StatF or StatI per block
    int64_t n_partials_cap = 0;
    int64_t n_partials = 0;
    const void *stats_out = nullptr;       // out buffer the partials describe
    // search
    dd::SearchParams *d_params = nullptr;
    int32_t *d_wsorted = nullptr;          // widths sorted ascending: [nw] widths, [nw] indices
    dd_candidate *d_cands = nullptr;
    int64_t cand_cap = 0;
    unsigned long long *d_count = nullptr;
    unsigned long long *h_count = nullptr; // pinned
    dd::SearchParams *h_params = nullptr;  // pinned
    double last_mu = 0, last_sigma = 0;
    // per-DM-row statistics option
    int32_t row_stats = 0;                 // 0: whole buffer (Section 3), 1: per DM row
    dd::RowParams *d_rowprm = nullptr;     // [ndm]
    dd::RowParams *h_rowprm = nullptr;     // pinned [ndm], filled by the last search
    // end-to-end staging (dd_process_host)
    void *d_in_stage = nullptr;
    size_t in_stage_bytes = 0;
    void *d_out_stage = nullptr;
    size_t out_stage_bytes = 0;

    // register-blocked kernel data (kernel 2)
    void *fast = nullptr;
};

namespace dd {

int set_error(int code, const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);

// dd_api.cu: Eq. 1 delay in samples (rounded), and plan creation; with
// kernels == false the plan gets its delay table and search scratch only
// (no de-dispersion kernel tables), for composite plans that run their own
// kernels and reuse the search.
long long delay_samples(double fch1, double foff, int nchans, double tsamp_s, double dm, int c);
int plan_create(int32_t nchans, double fch1_mhz, double foff_mhz, double tsamp_s,
                const double *dm_list, int32_t ndm, const int32_t *boxcar_widths, int32_t nwidths,
                double sigma_k, int32_t in_dtype, int64_t nsamp_in, bool kernels, dd_plan **plan_out);

size_t in_elem_bytes(dd_dtype t);

// dd_kernels.cu
int generic_configure(dd_plan *p);
int generic_execute(dd_plan *p, const void *in, int64_t pitch, void *out, cudaStream_t s);
int stats_from_out(dd_plan *p, const void *out, cudaStream_t s);
int search_launch(dd_plan *p, const void *out, cudaStream_t s);
int ensure_partials_public(dd_plan *p, int64_t n);
// windows crossing from the previous chunk (`tail`: [ndm][L] outputs) into
// `out`, against the plan's current thresholds; hits in the plan's candidate
// buffer (read back with search_readback)
int boundary_search_launch(dd_plan *p, const void *tail, const void *out, int L, cudaStream_t s);
long long max_delay(int nchans, double fch1, double foff, double tsamp_s, const double *dm_list, int ndm);
int search_readback(dd_plan *plan, dd_candidate *cand_host, int64_t capacity, int64_t *n_found,
                    cudaStream_t s, int64_t dev_cap);
cudaError_t allow_max_dynamic_smem(const void *fn, size_t optin);

// dd_fast.cu
int fast_configure(dd_plan *p);
int fast_execute(dd_plan *p, const void *in, int64_t pitch, void *out, cudaStream_t s);
// dd_process_host's copy of in_host into in_dev pipelined with the
// de-dispersion (kernels 3 and 5); kNotPipelined if the plan's kernel has no
// such path (nothing is done then).
constexpr int kNotPipelined = -1;
int fast_execute_host(dd_plan *p, const void *in_host, int64_t pitch, void *in_dev, void *out, cudaStream_t s);
void fast_release(dd_plan *p);
int fast_error(dd_plan *p, cudaStream_t s);
int fast_autotune(dd_plan *p, const void *in, int64_t pitch, void *out, cudaStream_t s);
int fast_set_tile(dd_plan *p, int cfg, int dgroup);
int fast_get_tile(const dd_plan *p, int *cfg, int *dgroup, int *tr, int *nw);
int fast_kernel_id(const dd_plan *p);

}  // namespace dd
