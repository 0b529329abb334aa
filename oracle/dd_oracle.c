/*
 * dd_oracle.c -- plain, slow, obviously-correct CPU oracle for brute-force
 * incoherent de-dispersion and the boxcar single-pulse threshold search.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header, table or constant with the
 * CUDA path.
 *
 * Everything is computed in IEEE double (or exact 64-bit integers for 8-bit
 * input) with plain loops in the paper's order.  Build with FMA contraction
 * off (-ffp-contract=off) and without -ffast-math so every expression below is
 * evaluated exactly as written.
 *
 * Paper: Magro et al. 2011, "Real-time, fast radio transient searches with GPU
 * de-dispersion".
 *   - Eq. 1 (Section 1): cold-plasma delay 4.15e6 ms * (f1^-2 - f2^-2) * DM,
 *     f in MHz.
 *   - Section 3, "Maximum shift" (Eq. 2): n_samp outputs need n_samp + maxshift
 *     input samples.
 *   - Section 3.1: brute force, each output sample is the sum over all
 *     channels of the input shifted by that channel's delay.
 *   - Section 3.2: subband de-dispersion, the two-stage approximation (at the
 *     end of this file).
 *   - Section 3 (output thread): mean and standard deviation over the whole
 *     processed buffer, an n-sigma threshold, every value above it emitted as
 *     (time, DM, intensity).  The search generalises the single sample to
 *     boxcar sums of several widths.
 *
 * Readings where the paper is silent (each also recorded in the design notes):
 *   - channel frequencies are channel centres f_c = fch1 + c*foff; delays are
 *     relative to the highest frequency f_ref = max_c f_c;
 *   - the delay in samples is rounded half away from zero (C round());
 *   - maxshift is the exact max_{c,dm} d(c,dm), not the Eq. 2 approximation;
 *   - the output keeps n_out = n_in - maxshift samples, no padding;
 *   - mean and sigma are global over all n_dm * n_out values, population
 *     (1/N) normalisation;
 *   - "above the threshold" is strict: B_w > w*mu + k*sigma*sqrt(w);
 *   - a boxcar of width w starting at t covers t..t+w-1 and never crosses
 *     the end of the row.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_API __attribute__((visibility("default")))

/* Candidate record, in the oracle's own layout (not the library's). */
typedef struct {
    int64_t dm_idx;
    int64_t t;
    int64_t width_idx;
    double snr;
    double value;
} oracle_cand;

ORACLE_API int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

ORACLE_API void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0)
        omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Eq. 1: per-channel, per-DM delay in samples.                             */
/* ------------------------------------------------------------------------ */

/* Channel-centre frequency of channel c (MHz). */
static double chan_freq(double fch1, double foff, int64_t c)
{
    return fch1 + (double)c * foff;
}

/* Fractional delay x(c,dm) in samples, relative to the highest channel:
 *   x = ((4.15e6 * dm) * (1/(f_c*f_c) - 1/(f_ref*f_ref))) / tsamp_ms
 * evaluated left to right in double (Eq. 1 divided by the sample time). */
ORACLE_API double oracle_delay_exact(double fch1, double foff, int64_t nchans,
                                     double tsamp_s, double dm, int64_t c)
{
    double f_top = (foff < 0.0) ? chan_freq(fch1, foff, 0)
                                : chan_freq(fch1, foff, nchans - 1);
    double f = chan_freq(fch1, foff, c);
    double tsamp_ms = tsamp_s * 1e3;
    double inv_f = 1.0 / (f * f);
    double inv_top = 1.0 / (f_top * f_top);
    return ((4.15e6 * dm) * (inv_f - inv_top)) / tsamp_ms;
}

/* Integer delay table d[dm][c] = round(x(c,dm)) and maxshift = max d.
 * Returns 0, or -1 for invalid arguments. */
ORACLE_API int oracle_delays(int64_t nchans, double fch1, double foff, double tsamp_s,
                             const double *dm_list, int64_t ndm,
                             int64_t *delays, int64_t *maxshift)
{
    if (nchans < 1 || ndm < 1 || !(tsamp_s > 0.0) || !(fch1 > 0.0))
        return -1;
    if (!(chan_freq(fch1, foff, nchans - 1) > 0.0))
        return -1;
    int64_t m = 0;
    for (int64_t i = 0; i < ndm; ++i) {
        if (!(dm_list[i] >= 0.0))
            return -1;
        for (int64_t c = 0; c < nchans; ++c) {
            double x = oracle_delay_exact(fch1, foff, nchans, tsamp_s, dm_list[i], c);
            int64_t d = (int64_t)round(x);
            delays[i * nchans + c] = d;
            if (d > m)
                m = d;
        }
    }
    *maxshift = m;
    return 0;
}

/* Eq. 2 approximation of maxshift (derivative form), used only as a sanity
 * bound: 8.3e6 ms * bandwidth * f^-3 * DM_max / tsamp_ms, with the bandwidth
 * nchans*|foff| and f the centre of the band (mean of the channel centres). */
ORACLE_API double oracle_maxshift_eq2(int64_t nchans, double fch1, double foff,
                                      double tsamp_s, double dm_max)
{
    double f_a = chan_freq(fch1, foff, 0);
    double f_b = chan_freq(fch1, foff, nchans - 1);
    double bw = (double)nchans * fabs(foff);
    double f = 0.5 * (f_a + f_b);
    return 8.3e6 * bw * (1.0 / (f * f * f)) * dm_max / (tsamp_s * 1e3);
}

/* ------------------------------------------------------------------------ */
/* IEEE binary16 -> double, exact (every binary16 value is a double).       */
/* ------------------------------------------------------------------------ */
ORACLE_API double oracle_half_to_double(uint16_t h)
{
    int sign = (h >> 15) & 1;
    int e = (h >> 10) & 0x1f;
    int m = h & 0x3ff;
    double v;
    if (e == 0)
        v = ldexp((double)m, -24);                 /* zero / subnormal */
    else if (e == 31)
        v = (m == 0) ? INFINITY : NAN;
    else
        v = ldexp((double)(1024 + m), e - 25);     /* (1.m) * 2^(e-15) */
    return sign ? -v : v;
}

/* ------------------------------------------------------------------------ */
/* Section 3.1: brute-force de-dispersion                                    */
/*   out[dm][t] = sum_{c=0}^{C-1} in[c][t + d(c,dm)],  0 <= t < n_out        */
/* summed in ascending channel order.                                        */
/* ------------------------------------------------------------------------ */

ORACLE_API void oracle_dedisperse_f32(const float *in, int64_t pitch, int64_t nchans,
                                      const int64_t *delays, int64_t ndm,
                                      int64_t nout, double *out)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < ndm; ++i) {
        const int64_t *d = delays + i * nchans;
        for (int64_t t = 0; t < nout; ++t) {
            double s = 0.0;
            for (int64_t c = 0; c < nchans; ++c)
                s += (double)in[c * pitch + t + d[c]];
            out[i * nout + t] = s;
        }
    }
}

ORACLE_API void oracle_dedisperse_f16(const uint16_t *in, int64_t pitch, int64_t nchans,
                                      const int64_t *delays, int64_t ndm,
                                      int64_t nout, double *out)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < ndm; ++i) {
        const int64_t *d = delays + i * nchans;
        for (int64_t t = 0; t < nout; ++t) {
            double s = 0.0;
            for (int64_t c = 0; c < nchans; ++c)
                s += oracle_half_to_double(in[c * pitch + t + d[c]]);
            out[i * nout + t] = s;
        }
    }
}

ORACLE_API void oracle_dedisperse_u8(const uint8_t *in, int64_t pitch, int64_t nchans,
                                     const int64_t *delays, int64_t ndm,
                                     int64_t nout, int64_t *out)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < ndm; ++i) {
        const int64_t *d = delays + i * nchans;
        for (int64_t t = 0; t < nout; ++t) {
            int64_t s = 0;
            for (int64_t c = 0; c < nchans; ++c)
                s += (int64_t)in[c * pitch + t + d[c]];
            out[i * nout + t] = s;
        }
    }
}

/* One output sample, for sampled checks of outputs too large to compute whole. */
ORACLE_API double oracle_point_f32(const float *in, int64_t pitch, int64_t nchans,
                                   const int64_t *delay_row, int64_t t)
{
    double s = 0.0;
    for (int64_t c = 0; c < nchans; ++c)
        s += (double)in[c * pitch + t + delay_row[c]];
    return s;
}

/* One de-dispersed row (all t), for sampled row checks at large sizes. */
ORACLE_API void oracle_row_f32(const float *in, int64_t pitch, int64_t nchans,
                               const int64_t *delay_row, int64_t nout, double *row)
{
    for (int64_t t = 0; t < nout; ++t) {
        double s = 0.0;
        for (int64_t c = 0; c < nchans; ++c)
            s += (double)in[c * pitch + t + delay_row[c]];
        row[t] = s;
    }
}

/* ------------------------------------------------------------------------ */
/* Section 3 (output thread): statistics over the whole processed buffer.   */
/* Two passes in double: mu = (1/N) sum x, sigma = sqrt((1/N) sum (x-mu)^2). */
/* ------------------------------------------------------------------------ */
ORACLE_API void oracle_stats_f64(const double *x, int64_t n, double *mu, double *sigma)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i)
        s += x[i];
    double m = s / (double)n;
    double q = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double d = x[i] - m;
        q += d * d;
    }
    *mu = m;
    *sigma = sqrt(q / (double)n);
}

ORACLE_API void oracle_stats_i64(const int64_t *x, int64_t n, double *mu, double *sigma)
{
    int64_t s = 0;
    for (int64_t i = 0; i < n; ++i)
        s += x[i];
    double m = (double)s / (double)n;
    double q = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double d = (double)x[i] - m;
        q += d * d;
    }
    *mu = m;
    *sigma = sqrt(q / (double)n);
}

/* ------------------------------------------------------------------------ */
/* Boxcar threshold search (Section 3's n-sigma test applied to boxcar sums).*/
/* For every dm, t and width w (t + w <= n_out):                             */
/*   B_w(dm,t) = sum_{j<w} out[dm][t+j]                                      */
/*   T_w       = w*mu + k*sigma*sqrt(w)                                      */
/*   candidate iff B_w > T_w, S/N = (B_w - w*mu) / (sigma*sqrt(w)).          */
/* Candidates are written in (dm, t, width index) order; the return value is */
/* the total count (records beyond cap are counted but not written).         */
/* ------------------------------------------------------------------------ */
ORACLE_API double oracle_threshold(int64_t w, double mu, double sigma, double k)
{
    return (double)w * mu + k * sigma * sqrt((double)w);
}

ORACLE_API int64_t oracle_search_f64(const double *out, int64_t ndm, int64_t nout,
                                     const int32_t *widths, int64_t nw,
                                     double mu, double sigma, double k,
                                     oracle_cand *cands, int64_t cap)
{
    int64_t n = 0;
    for (int64_t i = 0; i < ndm; ++i) {
        const double *row = out + i * nout;
        for (int64_t t = 0; t < nout; ++t) {
            for (int64_t wi = 0; wi < nw; ++wi) {
                int64_t w = widths[wi];
                if (t + w > nout)
                    continue;
                double b = 0.0;
                for (int64_t j = 0; j < w; ++j)
                    b += row[t + j];
                double thr = oracle_threshold(w, mu, sigma, k);
                if (b > thr) {
                    if (n < cap) {
                        cands[n].dm_idx = i;
                        cands[n].t = t;
                        cands[n].width_idx = wi;
                        cands[n].snr = (b - (double)w * mu) / (sigma * sqrt((double)w));
                        cands[n].value = b;
                    }
                    ++n;
                }
            }
        }
    }
    return n;
}

ORACLE_API int64_t oracle_search_i64(const int64_t *out, int64_t ndm, int64_t nout,
                                     const int32_t *widths, int64_t nw,
                                     double mu, double sigma, double k,
                                     oracle_cand *cands, int64_t cap)
{
    int64_t n = 0;
    for (int64_t i = 0; i < ndm; ++i) {
        const int64_t *row = out + i * nout;
        for (int64_t t = 0; t < nout; ++t) {
            for (int64_t wi = 0; wi < nw; ++wi) {
                int64_t w = widths[wi];
                if (t + w > nout)
                    continue;
                int64_t b = 0;
                for (int64_t j = 0; j < w; ++j)
                    b += row[t + j];
                double thr = oracle_threshold(w, mu, sigma, k);
                if ((double)b > thr) {
                    if (n < cap) {
                        cands[n].dm_idx = i;
                        cands[n].t = t;
                        cands[n].width_idx = wi;
                        cands[n].snr = ((double)b - (double)w * mu) / (sigma * sqrt((double)w));
                        cands[n].value = (double)b;
                    }
                    ++n;
                }
            }
        }
    }
    return n;
}

/* ------------------------------------------------------------------------ */
/* Section 3.2: subband de-dispersion.                                       */
/*                                                                          */
/* The fine DM list is split into consecutive groups of G trials, each      */
/* centred on a nominal DM; the channels are split into nsub subbands of    */
/* nchans/nsub consecutive channels.                                        */
/*   stage 1: for every nominal DM k and subband s, the subband's channels  */
/*            are shifted by their delay at the nominal DM minus the delay  */
/*            of the subband's highest-frequency channel, and summed:       */
/*              I[k][s][t] = sum_{c in s} in[c][t + d1(k,c)],               */
/*              d1(k,c) = d(c, D_k) - d(ref(s), D_k);                       */
/*   stage 2: every fine DM j of group k is de-dispersed by brute force     */
/*            over the subband series, each subband shifted by the delay    */
/*            of its highest-frequency channel at the fine DM:              */
/*              out[j][t] = sum_s I[k][s][t + d2(j,s)],  d2(j,s) = d(ref(s), dm_j). */
/* Readings: the nominal DM of a group is the midpoint of its first and     */
/* last fine DM; subbands are equal groups of consecutive channels; d() is  */
/* the rounded Eq. 1 delay of the brute-force path, so at a fine DM whose   */
/* delays equal the nominal DM's the result is the brute-force sum.         */
/* ------------------------------------------------------------------------ */

/* Highest-frequency channel of subband s (cs channels per subband). */
static int64_t subband_ref(double foff, int64_t s, int64_t cs)
{
    return foff < 0.0 ? s * cs : s * cs + cs - 1;
}

/* Tables of the two stages.  nominal[K]; d1[K][nchans]; d2[ndm][nsub];
 * *maxshift = max over (j, c) of d2(j, sub(c)) + d1(k(j), c).
 * Returns 0, or -1 for invalid arguments. */
ORACLE_API int oracle_subband_tables(int64_t nchans, double fch1, double foff, double tsamp_s,
                                     const double *dm_list, int64_t ndm, int64_t G, int64_t nsub,
                                     double *nominal, int64_t *d1, int64_t *d2, int64_t *maxshift)
{
    if (G < 1 || nsub < 1 || nchans % nsub != 0)
        return -1;
    const int64_t cs = nchans / nsub;
    const int64_t K = (ndm + G - 1) / G;
    int64_t m_fine = 0, m_nom = 0;
    int64_t *fine = (int64_t *)malloc(sizeof(int64_t) * ndm * nchans);
    int64_t *nom = (int64_t *)malloc(sizeof(int64_t) * K * nchans);
    if (!fine || !nom) { free(fine); free(nom); return -1; }
    int rc = oracle_delays(nchans, fch1, foff, tsamp_s, dm_list, ndm, fine, &m_fine);
    if (rc == 0) {
        for (int64_t k = 0; k < K; ++k) {
            const int64_t j0 = k * G;
            const int64_t j1 = (j0 + G < ndm ? j0 + G : ndm) - 1;
            nominal[k] = 0.5 * (dm_list[j0] + dm_list[j1]);
        }
        rc = oracle_delays(nchans, fch1, foff, tsamp_s, nominal, K, nom, &m_nom);
    }
    if (rc == 0) {
        for (int64_t k = 0; k < K; ++k)
            for (int64_t c = 0; c < nchans; ++c) {
                const int64_t r = subband_ref(foff, c / cs, cs);
                d1[k * nchans + c] = nom[k * nchans + c] - nom[k * nchans + r];
            }
        for (int64_t j = 0; j < ndm; ++j)
            for (int64_t s = 0; s < nsub; ++s)
                d2[j * nsub + s] = fine[j * nchans + subband_ref(foff, s, cs)];
        int64_t m = 0;
        for (int64_t j = 0; j < ndm; ++j)
            for (int64_t c = 0; c < nchans; ++c) {
                const int64_t e = d2[j * nsub + c / cs] + d1[(j / G) * nchans + c];
                if (e > m)
                    m = e;
            }
        *maxshift = m;
    }
    free(fine);
    free(nom);
    return rc;
}

/* Stage 1 then stage 2 for one output sample of fine DM j: the subband sums
 * (ascending channel) and then their sum (ascending subband), in double. */
static double subband_point(const float *in_f32, const uint16_t *in_f16, int64_t pitch,
                            int64_t nchans, int64_t nsub, const int64_t *d1, const int64_t *d2,
                            int64_t G, int64_t j, int64_t t)
{
    const int64_t cs = nchans / nsub;
    const int64_t *r1 = d1 + (j / G) * nchans;
    double out = 0.0;
    for (int64_t s = 0; s < nsub; ++s) {
        const int64_t tt = t + d2[j * nsub + s];
        double sub = 0.0;
        for (int64_t c = s * cs; c < (s + 1) * cs; ++c) {
            const int64_t i = c * pitch + tt + r1[c];
            sub += in_f32 ? (double)in_f32[i] : oracle_half_to_double(in_f16[i]);
        }
        out += sub;
    }
    return out;
}

ORACLE_API void oracle_subband_f32(const float *in, int64_t pitch, int64_t nchans, int64_t nsub,
                                   const int64_t *d1, const int64_t *d2, int64_t G, int64_t ndm,
                                   int64_t nout, double *out)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t j = 0; j < ndm; ++j)
        for (int64_t t = 0; t < nout; ++t)
            out[j * nout + t] = subband_point(in, NULL, pitch, nchans, nsub, d1, d2, G, j, t);
}

ORACLE_API void oracle_subband_f16(const uint16_t *in, int64_t pitch, int64_t nchans, int64_t nsub,
                                   const int64_t *d1, const int64_t *d2, int64_t G, int64_t ndm,
                                   int64_t nout, double *out)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t j = 0; j < ndm; ++j)
        for (int64_t t = 0; t < nout; ++t)
            out[j * nout + t] = subband_point(NULL, in, pitch, nchans, nsub, d1, d2, G, j, t);
}

ORACLE_API void oracle_subband_u8(const uint8_t *in, int64_t pitch, int64_t nchans, int64_t nsub,
                                  const int64_t *d1, const int64_t *d2, int64_t G, int64_t ndm,
                                  int64_t nout, int64_t *out)
{
    const int64_t cs = nchans / nsub;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t j = 0; j < ndm; ++j) {
        const int64_t *r1 = d1 + (j / G) * nchans;
        for (int64_t t = 0; t < nout; ++t) {
            int64_t acc = 0;
            for (int64_t s = 0; s < nsub; ++s) {
                const int64_t tt = t + d2[j * nsub + s];
                int64_t sub = 0;
                for (int64_t c = s * cs; c < (s + 1) * cs; ++c)
                    sub += (int64_t)in[c * pitch + tt + r1[c]];
                acc += sub;
            }
            out[j * nout + t] = acc;
        }
    }
}

/* One output sample (float32 input), for sampled checks at full size. */
ORACLE_API double oracle_subband_point_f32(const float *in, int64_t pitch, int64_t nchans,
                                           int64_t nsub, const int64_t *d1, const int64_t *d2,
                                           int64_t G, int64_t j, int64_t t)
{
    return subband_point(in, NULL, pitch, nchans, nsub, d1, d2, G, j, t);
}

/* ------------------------------------------------------------------------ */
/* Section 3.2, binning: average of N_b adjacent samples,                    */
/*   out[c][i] = (1/N_b) sum_{q<N_b} in[c][N_b*i + q],  i < floor(n / N_b).   */
/* In double; the subband stages below then run on the binned series.        */
/* ------------------------------------------------------------------------ */
static double in_value(const void *in, int dtype, int64_t i)
{
    /* dtype: 0 float32, 1 uint8, 2 binary16 (the library's dd_dtype codes) */
    if (dtype == 0) return (double)((const float *)in)[i];
    if (dtype == 1) return (double)((const uint8_t *)in)[i];
    return oracle_half_to_double(((const uint16_t *)in)[i]);
}

ORACLE_API void oracle_bin(const void *in, int dtype, int64_t pitch, int64_t nchans, int64_t nsamp,
                           int64_t nb, double *out, int64_t out_pitch)
{
    const int64_t n = nsamp / nb;
    for (int64_t c = 0; c < nchans; ++c)
        for (int64_t i = 0; i < n; ++i) {
            double s = 0.0;
            for (int64_t q = 0; q < nb; ++q)
                s += in_value(in, dtype, c * pitch + i * nb + q);
            out[c * out_pitch + i] = s / (double)nb;
        }
}

/* Subband stages on double input (binned series), as oracle_subband_f32. */
ORACLE_API void oracle_subband_f64(const double *in, int64_t pitch, int64_t nchans, int64_t nsub,
                                   const int64_t *d1, const int64_t *d2, int64_t G, int64_t ndm,
                                   int64_t nout, double *out)
{
    const int64_t cs = nchans / nsub;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t j = 0; j < ndm; ++j) {
        const int64_t *r1 = d1 + (j / G) * nchans;
        for (int64_t t = 0; t < nout; ++t) {
            double acc = 0.0;
            for (int64_t s = 0; s < nsub; ++s) {
                const int64_t tt = t + d2[j * nsub + s];
                double sub = 0.0;
                for (int64_t c = s * cs; c < (s + 1) * cs; ++c)
                    sub += in[c * pitch + tt + r1[c]];
                acc += sub;
            }
            out[j * nout + t] = acc;
        }
    }
}
