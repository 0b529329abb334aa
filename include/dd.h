/*
 * dd.h -- C ABI of libdd: brute-force incoherent de-dispersion and a boxcar
 * single-pulse threshold search on one NVIDIA GB300 (sm_103a).
 *
 * Method: Magro et al. 2011, "Real-time, fast radio transient searches with
 * GPU de-dispersion".
 *   Eq. 1 (Section 1)   delay between frequencies f1, f2 (MHz):
 *                       4.15e6 ms * (f1^-2 - f2^-2) * DM
 *   Section 3, Eq. 2    n outputs need n + maxshift input samples
 *   Section 3.1         brute force: each output sample is the sum over all
 *                       channels of the input shifted by its delay
 *   Section 3           mean/std over the processed buffer, n-sigma threshold,
 *                       (time, DM, intensity) candidates
 *
 * Definitions used by every call (C = nchans, D = ndm):
 *   f_c      = fch1 + c*foff                     channel centre, MHz
 *   f_top    = max_c f_c
 *   d(c,dm)  = round(((4.15e6*DM) * (1/f_c^2 - 1/f_top^2)) / (tsamp*1e3))
 *              evaluated in IEEE double, FMA contraction off, rounded half
 *              away from zero                     (Eq. 1 over the sample time)
 *   maxshift = max_{c,dm} d(c,dm)                (the exact form of Eq. 2)
 *   nsamp_out = nsamp_in - maxshift
 *   out[dm][t] = sum_{c=0}^{C-1} in[c][t + d(c,dm)],  0 <= t < nsamp_out
 *   mu, sigma  = population mean / std over all D*nsamp_out values of out
 *   B_w(dm,t)  = sum_{j<w} out[dm][t+j]  for t + w <= nsamp_out
 *   candidate iff B_w > w*mu + sigma_k*sigma*sqrt(w)   (strict)
 *   snr        = (B_w - w*mu) / (sigma*sqrt(w))
 *
 * Layouts.  `in` is channel-major: in[c*in_pitch + t], t contiguous, element
 * type float32, uint8 or IEEE binary16 (DD_F32 / DD_U8 / DD_F16).  `out` is
 * row-major [D][nsamp_out] with no padding: float32 for DD_F32 and DD_F16
 * input (FP32 accumulation), int32 for DD_U8 input (exact integer sums).
 *
 * Ownership.  The caller owns `in`, `out` (device memory) and the host
 * candidate array.  A plan owns its delay table, its statistics and candidate
 * scratch on the device and its pinned host staging; dd_plan_destroy frees
 * them.  A plan lives on the device that was current when it was created.
 *
 * Errors.  Every call returns a dd_status; none aborts.  On failure
 * dd_last_error() returns a message for the calling thread.  Calls on one
 * plan must not run concurrently from several host threads.
 *
 * Units: MHz, seconds, pc cm^-3 (the paper's units, Eq. 1).
 */
#ifndef DD_H
#define DD_H

#include <stdint.h>

#if defined(__GNUC__)
#define DD_API __attribute__((visibility("default")))
#else
#define DD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dd_plan dd_plan;
typedef struct dd_batch dd_batch;

typedef enum { DD_F32 = 0, DD_U8 = 1, DD_F16 = 2 } dd_dtype;

typedef enum {
    DD_OK = 0,
    DD_ERR_ARG = 1,       /* invalid argument; nothing was launched          */
    DD_ERR_NOMEM = 2,     /* a device or pinned allocation failed            */
    DD_ERR_CUDA = 3,      /* a CUDA runtime call failed                      */
    DD_ERR_OVERFLOW = 4,  /* more candidates than the caller's capacity      */
    DD_ERR_TIMEOUT = 5,   /* a bounded device-side wait gave up              */
    DD_ERR_BUDGET = 6,    /* admission refused: the HBM budget is exhausted  */
    DD_PRIMING = 7,       /* server chunk accepted, no output yet: the beam's
                             resident history holds < maxshift samples       */
    DD_ERR_SEQ = 8,       /* server chunk refused: its seq repeats or precedes
                             the beam's last accepted chunk (nothing queued) */
    DD_SEQ_GAP = 9        /* server chunk accepted after a gap in seq: the
                             beam's stream restarts at it (history zeroed,
                             the beam primes again)                          */
} dd_status;

typedef struct dd_server dd_server;

/* Completion record of one served chunk (host steady-clock seconds). */
typedef struct {
    int32_t beam;
    int32_t status;       /* DD_OK, DD_PRIMING or an error status            */
    int64_t seq;          /* the caller's sequence number of the chunk       */
    int64_t n_candidates; /* search hits of this chunk                       */
    double t_submit;      /* dd_server_submit returned                       */
    double t_start;       /* a worker took the chunk                         */
    double t_done;        /* candidates on the host                          */
    double mu, sigma;     /* statistics of this chunk's output               */
} dd_chunk_result;

/* One search hit (32 bytes).  value is B_w exactly as summed on the device
 * (an integer for DD_U8 plans); snr as defined above, in double, rounded to
 * float. */
typedef struct {
    int32_t dm_idx;       /* index into the plan's dm_list                   */
    int32_t width_idx;    /* index into the plan's boxcar_widths             */
    int64_t t;            /* first sample of the boxcar, 0-based in out      */
    float snr;
    float reserved;
    double value;
} dd_candidate;

/* Create a plan (Eq. 1 delays, Eq. 2 maxshift, Section 3.1 sum, Section 3
 * search).  dm_list[ndm] (>= 0, any order) and boxcar_widths[nwidths]
 * (1 <= w <= nsamp_out) are copied.  sigma_k is the threshold multiple.
 * Requires nchans >= 1, ndm >= 1, tsamp_s > 0, fch1 > 0, the lowest channel
 * centre > 0, nsamp_in > maxshift.  The delay table is computed here once,
 * in double on the host, and uploaded as int32.  Returns DD_ERR_ARG for
 * invalid arguments, DD_ERR_NOMEM / DD_ERR_CUDA on allocation failure. */
DD_API int dd_plan_create(int32_t nchans, double fch1_mhz, double foff_mhz, double tsamp_s,
                   const double *dm_list, int32_t ndm,
                   const int32_t *boxcar_widths, int32_t nwidths, double sigma_k,
                   int32_t in_dtype, int64_t nsamp_in, dd_plan **plan_out);

/* Free everything the plan owns (synchronises the plan's device first).
 * NULL is accepted. */
DD_API int dd_plan_destroy(dd_plan *plan);

/* Report maxshift and nsamp_out; when delays_host is not NULL, copy the
 * int32 delay table d[dm][c] (ndm*nchans entries) into it.  Any output
 * pointer may be NULL. */
DD_API int dd_plan_info(const dd_plan *plan, int64_t *maxshift, int64_t *nsamp_out,
                 int32_t *delays_host);

/* Section 3.1: out[dm][t] = sum_c in[c][t + d(c,dm)] for all dm and
 * 0 <= t < nsamp_out, plus per-block partial statistics kept in the plan for
 * the next dd_search.  in_dev: device pointer, channel-major, in_pitch
 * elements per channel row (in_pitch >= nsamp_in).  out_dev: device pointer
 * to D*nsamp_out float32 (int32 for DD_U8).  stream: a cudaStream_t (NULL =
 * legacy default stream).  Asynchronous: returns after the launches are
 * queued.  The input buffers must not alias. */
DD_API int dd_execute(dd_plan *plan, const void *in_dev, int64_t in_pitch, void *out_dev,
               void *stream);

/* Section 3 output stage, generalised to boxcars: statistics over the whole
 * buffer, thresholds, boxcar sums, compaction.  out_dev is the buffer the
 * last dd_execute on this plan wrote (if it is another buffer the statistics
 * are recomputed from it).  Synchronises `stream`.  Writes up to `capacity`
 * candidates to cand_host sorted by (dm_idx, t, width_idx) and the true count
 * to *n_found.  If the true count exceeds capacity, the array holds an
 * unspecified subset of `capacity` hits (sorted) and DD_ERR_OVERFLOW is
 * returned. */
DD_API int dd_search(dd_plan *plan, const void *out_dev, dd_candidate *cand_host,
              int64_t capacity, int64_t *n_found, void *stream);

/* mu and sigma used by the last dd_search on this plan (Section 3; the
 * whole buffer's statistics also when per-row statistics are enabled). */
DD_API int dd_last_stats(const dd_plan *plan, double *mu, double *sigma);

/* Search variant: per_row = 1 makes dd_search (and the batch / server
 * searches of this plan) use each DM row's own mean and population standard
 * deviation instead of the whole buffer's (Section 3 uses the whole buffer):
 * T_w(row) = w*mu_row + k*sigma_row*sqrt(w), S/N = (B_w - w*mu_row) /
 * (sigma_row*sqrt(w)).  Robust to DM-dependent baselines (low-DM rows carry
 * more interference in real data).  One extra read of `out` per search.
 * per_row = 0 restores the whole-buffer statistics.  Allocates
 * ndm x 784 bytes of device and pinned host scratch on first enabling. */
DD_API int dd_plan_set_search_stats(dd_plan *plan, int32_t per_row);

/* Per-row mean and standard deviation used by the last dd_search (host
 * arrays of ndm doubles, either may be NULL); DD_ERR_ARG unless per-row
 * statistics are enabled. */
DD_API int dd_last_row_stats(const dd_plan *plan, double *mu_rows, double *sigma_rows);

/* End-to-end call with HOST buffers: copies in_host (pinned or pageable,
 * channel-major, in_pitch elements per row) to the device, runs dd_execute
 * and dd_search, and returns the candidates as dd_search does.  With
 * kernels 3 and 5 the copy goes in 8 column chunks on a stream of the plan,
 * and the output tiles each chunk completes are de-dispersed while the next
 * chunk is in flight (same results as the unsplit call).  The plan allocates
 * its device staging for `in` and `out` on the first call and keeps it until
 * dd_plan_destroy.  Synchronises `stream`. */
DD_API int dd_process_host(dd_plan *plan, const void *in_host, int64_t in_pitch,
                    dd_candidate *cand_host, int64_t capacity, int64_t *n_found,
                    void *stream);

/* Select the de-dispersion kernel for a plan: 0 = automatic (default: the
 * first available of tile configurations 12, 11, 9, 10, 5, 3, 6, 4, 1, 0, 2 —
 * kernel 5 shapes where their tables fit the plan, then kernel 3 and kernel 2
 * shapes, in the order of measured speed — or the autotuner's choice;
 * kernel 1 if no tiled configuration fits),
 * 1 = generic shared-memory kernel, 2 = register-blocked kernel (window
 * reused across 4 DM trials per thread), 3 = lane-interleaved kernel (one
 * conflict-free shared load per add, no branches), 4 = tensor-memory window
 * kernel (each staged input word copied once into TMEM and read back by every
 * DM trial of the warp at a runtime column offset), 5 = shared subband
 * partial sums (the DM trials of a block whose delays relative to a 4-channel
 * subband's reference coincide share that subband's partial sum: the exact
 * brute-force result with fewer adds; needs at most 16 such delay patterns
 * per block and subband).  Kernels 2-5 share the tile-configuration list of
 * dd_plan_set_tile.  Returns DD_ERR_ARG if the requested kernel cannot run
 * this plan. */
DD_API int dd_plan_set_kernel(dd_plan *plan, int32_t kernel);

/* Kernel that dd_execute will launch for this plan (1 to 5, see above). */
DD_API int dd_plan_get_kernel(const dd_plan *plan, int32_t *kernel);

/* Autotuner for the tiled kernels: runs the plan on the caller's buffers
 * once per compiled tile configuration of kernels 2, 3 and 5 (0-6, 9-12,
 * see dd_plan_set_tile) and raster group, times each with CUDA events on
 * `stream`, keeps the fastest for this plan and caches the choice
 * process-wide for plans of the same shape.  Kernel 4 is not timed (slower on
 * every plan measured); dd_plan_set_kernel(plan, 4) selects it.  Writes
 * out_dev (several full executions); synchronises `stream`.  A no-op (DD_OK)
 * when the tiled kernels cannot run the plan or the input rows are not
 * 16-byte aligned. */
DD_API int dd_plan_autotune(dd_plan *plan, const void *in_dev, int64_t in_pitch, void *out_dev,
                            void *stream);

/* Choose kernel 2's tile configuration explicitly.  config indexes the
 * compiled list {kernel 2 — 0: 36 samples x 4 DM trials per thread, 8 warps;
 * 1: 20 x 4, 12 warps; 2: 28 x 4, 8 warps; kernel 3 (samples per lane x
 * DM trials per warp, warps) — 3: 16 x 4, 8 warps; 4: 16 x 8, 8 warps;
 * 5: 16 x 8, 4 warps; 6: 8 x 16, 4 warps; kernel 4 (samples per lane x DM
 * trials per warp, warps) — 7: 20 x 4, 8 warps; 8: 12 x 8, 8 warps; kernel
 * 5 (samples per lane x DM trials per warp, warps; 4-channel subbands) — 9:
 * 16 x 8, 4 warps; 10: 8 x 8, 4 warps; 11: 16 x 8, 6 warps; 12: 16 x 8, 8
 * warps that add the partial sums beside 8 warps that form them (one block
 * per SM, the two groups joined by mbarriers; available where the GPU's
 * compiled register count covers the split)};
 * raster_group (>= 1) is the number of DM blocks whose time tiles are swept
 * together.  DD_ERR_ARG if the configuration cannot run this plan. */
DD_API int dd_plan_set_tile(dd_plan *plan, int32_t config, int32_t raster_group);

/* Current tiled-kernel choice: configuration index, raster group, samples
 * per thread (kernel 2) or per lane (kernels 3-5) and warps per block (any
 * pointer may be NULL).  DD_ERR_ARG if the tiled kernels cannot run this
 * plan. */
DD_API int dd_plan_get_tile(const dd_plan *plan, int32_t *config, int32_t *raster_group,
                            int32_t *samples_per_thread, int32_t *warps_per_block);

/* ---------------------------------------------------------------------
 * Batched beams.  The paper's kernel processes one buffer at a time
 * (Section 3.1); a batch runs the Section 3.1 sum for several plans (beams of
 * different channel counts, lengths, DM grids and input types) in ONE
 * persistent launch that pulls (beam, DM block, time tile) work items from a
 * device queue ordered heaviest first, followed by each beam's Section 3
 * search.  Each beam's output and candidates are those its plan alone would
 * produce (the same arithmetic in the same order).
 * ------------------------------------------------------------------- */

/* Group `nplans` plans (not owned; they must outlive the batch and live on
 * the current device).  Beams whose plan cannot use the register-blocked
 * kernel are still accepted and run by their own launch inside the batch. */
DD_API int dd_batch_create(dd_plan *const *plans, int32_t nplans, dd_batch **batch_out);

/* Free the batch (its graph, queue and descriptors; not the plans). */
DD_API int dd_batch_destroy(dd_batch *batch);

/* Asynchronous: de-disperse every beam (in_devs[i], in_pitches[i] ->
 * out_devs[i], layouts as dd_execute) and run every beam's search kernels on
 * `stream`.  Results are read with dd_batch_results. */
DD_API int dd_batch_execute(dd_batch *batch, const void *const *in_devs, const int64_t *in_pitches,
                            void *const *out_devs, void *stream);

/* Record dd_batch_execute's work for these buffers as a CUDA graph (stream
 * capture on `stream`); dd_batch_launch then replays it.  Allocates what the
 * launches need before capturing. */
DD_API int dd_batch_capture(dd_batch *batch, const void *const *in_devs, const int64_t *in_pitches,
                            void *const *out_devs, void *stream);

/* Replay the captured graph on `stream` (asynchronous). */
DD_API int dd_batch_launch(dd_batch *batch, void *stream);

/* Synchronise `stream` and return beam `beam`'s candidates of the last
 * execute/launch, as dd_search does. */
DD_API int dd_batch_results(dd_batch *batch, int32_t beam, dd_candidate *cand_host, int64_t capacity,
                            int64_t *n_found, void *stream);

/* Time the persistent launch with each compiled tile configuration that all
 * batched beams can use, keep the fastest (writes out_devs; synchronises). */
DD_API int dd_batch_autotune(dd_batch *batch, const void *const *in_devs, const int64_t *in_pitches,
                             void *const *out_devs, void *stream);

/* dd_process_host's pipeline schedule (host only) for nsamp_out outputs in
 * tiles of `tile` samples whose input columns lie below the tile's first
 * sample + reach, with rows of `pitch` elements: *n (<= 8) chunks; chunk c
 * copies input columns up to col_end[c] (non-decreasing; the last is the
 * pitch), then de-disperses tiles up to tile_end[c] (the last is every
 * tile).  col_end and tile_end hold at least 8 entries.  DD_ERR_ARG for
 * non-positive sizes. */
DD_API int dd_host_chunk_schedule(int64_t nsamp_out, int64_t pitch, int32_t tile, int64_t reach,
                                  int64_t *col_end, int64_t *tile_end, int32_t *n);

/* Kernel 5's tables for tile configuration `config` (9-12) of a delay table
 * delays[ndm][nchans] (dd_plan_info's copy), computed on the host (no device
 * needed), for inspection and tests.  info[6] receives {1 if the shape can
 * run the table (at most 16 delay patterns per block and subband) else 0,
 * DM blocks, subbands, staged row stride rs, largest partial-sum length,
 * record length kLen}.  If info[0] is 1 and rec_out / base_out are not NULL,
 * they receive the records int32 [blocks][subbands][kLen] — [0, trials):
 * each trial's partial-sum index of its first sample; [trials]: the
 * subband's partial-sum length E; from trials + 4, 8 words per pattern:
 * {end of its sums in the partial-sum buffer, then per channel c of the
 * subband the staged element of its first term minus its start} — and
 * int32 [2][blocks][nchans]: the staged row starts relative to a tile's
 * first output sample, then the staged row lengths (the elements the block's
 * trials read, in 16-byte units; at most rs).  foff's sign picks the subband
 * reference channel (the highest frequency).  DD_ERR_ARG for another
 * configuration or too small a capacity. */
DD_API int dd_share_tables(const int32_t *delays, int32_t ndm, int32_t nchans, double foff, int32_t dtype,
                           int32_t config, int32_t *info, int32_t *rec_out, int64_t rec_cap, int32_t *base_out,
                           int64_t base_cap);

/* Tile configuration the persistent launch uses (-1 if no beam uses it),
 * number of work items, and number of beams run by their own launch.  A new
 * batch starts with the first of configurations 9, 5, 3, 6, 4, 1, 0, 2 that
 * every tiled beam can use.  Configuration 9 in a batch is mixed: kernel 5's
 * 16 x 8, 4-warp shape for the beams whose kernel 5 tables exist and fit
 * three blocks per SM, kernel 3's shape 5 (the same block geometry) for the
 * others, in one persistent launch. */
DD_API int dd_batch_info(const dd_batch *batch, int32_t *config, int64_t *nitems, int32_t *n_separate);

/* Launch mode: 0 = one persistent grid over every beam's work items (the
 * default), 1 = each beam's own kernel launch on its batch configuration, in
 * turn (still one CUDA graph with dd_batch_capture).  Beams that each fill
 * the GPU run faster on their own launches; batches of small beams gain from
 * the persistent grid.  dd_batch_autotune times both and keeps the faster.
 * Setting the mode drops a captured graph. */
DD_API int dd_batch_set_launch_mode(dd_batch *batch, int32_t per_beam);
DD_API int dd_batch_launch_mode(const dd_batch *batch, int32_t *per_beam);

/* Tile configuration beam `beam` runs in the batch (a kernel 5 shape or 5
 * under the mixed configuration 9, else the batch's), -1 if it runs the
 * generic kernel by its own launch.  A plan set to that configuration alone
 * (dd_plan_set_tile) reproduces the beam's batched output bit for bit.  In
 * the per-beam launch mode every beam with kernel 5 tables runs its first
 * available kernel 5 shape of 12, 11, 9, 10 (the order a plan starts from);
 * in the persistent grid shape 9, for the beams whose tables fit three
 * blocks per SM. */
DD_API int dd_batch_beam_config(const dd_batch *batch, int32_t beam, int32_t *config);

/* Choose the persistent launch's tile configuration (0-6, dd_plan_set_tile's
 * kernel 2 and kernel 3 shapes, or the mixed configuration 9); beams that
 * cannot use it run by their own launch.  Drops a captured graph.  DD_ERR_ARG
 * for another index. */
DD_API int dd_batch_set_config(dd_batch *batch, int32_t config);

/* ---------------------------------------------------------------------
 * Streaming server.  The paper processes an unbounded stream buffer by
 * buffer and needs maxshift extra samples per buffer (Section 3, "Maximum
 * shift"; real-time pipeline, Section 5).  A server keeps, per beam, the last
 * maxshift samples resident on the device, so each chunk of `chunk` new
 * samples yields `chunk` de-dispersed samples per DM trial (stream output
 * times [k*chunk - maxshift, (k+1)*chunk - maxshift) for chunk k) followed by
 * a Section 3 search over them (statistics per chunk).  The first
 * ceil(maxshift/chunk) chunks of a beam only fill the history (DD_PRIMING).
 * Worker threads, each with its own CUDA stream, take the oldest ready chunk
 * of any beam as soon as they are free, so chunks of different beams overlap
 * on the device; chunks of one beam run in submission order.
 * ------------------------------------------------------------------- */

/* Create a server with `nworkers` worker threads/streams, a device-memory
 * budget for admitted beams, and room for `max_candidates` hits per chunk. */
DD_API int dd_server_create(int64_t hbm_budget_bytes, int32_t nworkers, int64_t max_candidates,
                            dd_server **server_out);

/* Stop the workers (after the chunk each is running) and free every beam. */
DD_API int dd_server_destroy(dd_server *server);

/* Admit a beam (plan parameters as dd_plan_create, `chunk` new samples per
 * submission).  The beam's device memory (one sample ring of nchans rows x
 * about maxshift + K*chunk columns, K = 2 + floor(maxshift/chunk); the
 * output; the plan) is reserved against the budget: DD_ERR_BUDGET if it does
 * not fit (nothing allocated).  Each chunk is de-dispersed in place from the
 * ring (its window's base moves by one chunk per submission); the last
 * maxshift samples are moved to the ring's front once every K chunks.  The
 * beam runs kernel 5 where its tables fit the plan, else the plan's default
 * kernel; with dd_server_set_autotune on, the autotuner's choice timed on
 * the beam's own buffers at admission (cached per plan shape). */
DD_API int dd_server_add_beam(dd_server *server, int32_t nchans, double fch1_mhz, double foff_mhz,
                              double tsamp_s, const double *dm_list, int32_t ndm,
                              const int32_t *boxcar_widths, int32_t nwidths, double sigma_k,
                              int32_t in_dtype, int64_t chunk, int32_t *beam_id);

/* Remove a beam; its memory returns to the budget once its running chunk (if
 * any) finishes.  Queued chunks of the beam are dropped. */
DD_API int dd_server_remove_beam(dd_server *server, int32_t beam);

/* Search variant for streaming beams: on = 1 also tests, for every searched
 * chunk after the first, the boxcars that start in the previous chunk's last
 * wmax - 1 outputs and end in this chunk (wmax = the beam's widest boxcar;
 * by default windows never cross a chunk boundary).  They are tested against
 * this chunk's thresholds (the chunk holding the window's last sample) and
 * reported among this chunk's candidates with t < 0: the window starts |t|
 * samples before the chunk's first output.  Keeps ndm x (wmax - 1) outputs
 * per beam on the device (not counted against the admission budget).  Set it
 * before the beam's first chunk; DD_ERR_ARG otherwise or if wmax - 1 >
 * chunk. */
DD_API int dd_server_set_boundary_search(dd_server *server, int32_t beam, int32_t on);

/* Queue one chunk: chunk_host holds nchans rows of `chunk` samples,
 * host_pitch elements apart (pinned or pageable).  It must stay valid and
 * unchanged until dd_server_poll reports the chunk.  Returns immediately.
 * Sequence numbers: the beam's first chunk may carry any seq; each later one
 * must carry the previous accepted seq + 1 (DD_OK).  A larger seq means
 * chunks were lost: the chunk is queued, and the beam's stream restarts at it
 * (its history is zeroed, no boxcar joins the two parts, and the next
 * ceil(maxshift/chunk) chunks report DD_PRIMING): returns DD_SEQ_GAP.  A
 * seq that repeats or precedes the last accepted one is refused with
 * DD_ERR_SEQ and nothing is queued (the caller keeps ownership at once). */
DD_API int dd_server_submit(dd_server *server, int32_t beam, const void *chunk_host, int64_t host_pitch,
                            int64_t seq);

/* Collect up to max_results completion records (waiting up to wait_ms for
 * the first one). */
DD_API int dd_server_poll(dd_server *server, dd_chunk_result *results, int32_t max_results, int32_t *n,
                          int32_t wait_ms);

/* Candidates of a completed chunk, sorted as dd_search returns them (the
 * server keeps them until fetched). */
DD_API int dd_server_candidates(dd_server *server, int32_t beam, int64_t seq, dd_candidate *cand_host,
                                int64_t capacity, int64_t *n_found);

/* A beam's maxshift, chunk, DM trials, reserved bytes and its device output
 * buffer ([ndm][chunk], the latest completed chunk's; overwritten when the
 * beam's next chunk runs).  Any output pointer may be NULL. */
DD_API int dd_server_beam_info(dd_server *server, int32_t beam, int64_t *maxshift, int64_t *chunk,
                               int64_t *ndm, void **out_dev, int64_t *device_bytes);

/* Beams admitted from now on: on = 1 runs dd_plan_autotune on each beam's
 * own buffers at admission (the choice is cached process-wide per plan
 * shape, so a beam shaped like an earlier one is not timed again); on = 0
 * (the default) takes kernel 5 where available without timing. */
DD_API int dd_server_set_autotune(dd_server *server, int32_t on);

/* The kernel (dd_plan_get_kernel) and tile configuration (dd_plan_get_tile;
 * -1 for kernel 1) a beam runs; either pointer may be NULL. */
DD_API int dd_server_beam_kernel(dd_server *server, int32_t beam, int32_t *kernel, int32_t *config);

/* The host-side schedule the server follows for one beam, computed alone
 * (host code, no device work), so that it can be checked without a GPU.
 * For n submissions with sequence numbers seq[i] on a beam of maxshift M
 * and `chunk` samples per submission: *span = the ring's columns in use
 * (M + K*chunk); submit_status[i] = DD_OK, DD_SEQ_GAP or DD_ERR_SEQ as
 * dd_server_submit returns it; restart[i] = 1 if the stream restarts at i;
 * move_src[i] = the column whose M samples move to columns [0, M) before
 * chunk i is written (-1: no move); write_col[i] = the column of chunk i's
 * first sample; window_col[i] = the column of its de-dispersion window's
 * first sample (window = [window_col, window_col + M + chunk)); priming[i] =
 * 1 if it reports DD_PRIMING.  Refused submissions get -1 columns and
 * priming 0.  All arrays hold n entries (caller-owned).  DD_ERR_ARG for
 * M < 0, chunk < 1 or NULL arrays. */
DD_API int dd_server_ring_schedule(int64_t maxshift, int64_t chunk, int32_t n, const int64_t *seq,
                                   int64_t *span, int32_t *submit_status, int32_t *restart,
                                   int64_t *move_src, int64_t *write_col, int64_t *window_col,
                                   int32_t *priming);

/* Bytes reserved by admitted beams and the budget. */
DD_API int dd_server_memory(dd_server *server, int64_t *used, int64_t *budget);

/* Self-test of the bounded device waits (no counterpart in the paper: the
 * failure path of the staged kernels).  Every kernel that stages its input
 * with TMA copies waits on an mbarrier with a time limit; if a copy never
 * completes it records DD_ERR_TIMEOUT and returns instead of hanging, and the
 * host reports that status.  This runs one block that arms an mbarrier for 16
 * bytes and waits with that same bounded wait, its limit shortened to
 * limit_ns (1 .. 2e9): with issue_copy = 0 no copy is issued, nothing is left
 * in flight, and the wait runs out (returns DD_ERR_TIMEOUT, *device_status =
 * DD_ERR_TIMEOUT); with issue_copy = 1 the 16-byte copy completes it
 * (DD_OK, *device_status = 0).  Synchronous on the legacy default stream;
 * allocates and frees 32 device bytes.  DD_ERR_ARG for a limit out of range. */
DD_API int dd_wait_selftest(int64_t limit_ns, int32_t issue_copy, int32_t *device_status);

/* Allocation-free statistics (no counterpart in the paper).  For callers that
 * cannot call cudaMalloc — e.g. a real-time pipeline whose device memory is
 * budgeted once at start-up, where an allocation could synchronise the device
 * and stall live streams, or code running where another runtime owns the
 * allocator.  Writes mu = mean and sigma = population standard deviation of
 * the n float32 values at x_dev (device) to mu_sigma_dev[0] and [1] (device,
 * caller-owned), asynchronously on `stream`.  Needs no plan and allocates
 * nothing: its per-block partials live in a fixed 1.5 MB device array that
 * every GPU loading the library holds until exit, which limits n to
 * 1 <= n <= 268435456 (2^28); larger n returns DD_ERR_ARG without launching.
 * The first call on each device looks up that array's device address (with
 * the device current); make that first call before any stream capture.  The
 * address is kept for the life of the process: do not use this call on a
 * device after cudaDeviceReset (the module is reloaded and the kept address
 * no longer names the array).
 * Every call on a device shares the array, so calls whose kernels overlap on
 * the GPU (different streams, no ordering between them) race and may return
 * wrong values; calls ordered on one stream are safe. */
DD_API int dd_stats_f32_noalloc(const float *x_dev, int64_t n, double *mu_sigma_dev, void *stream);

/* ---------------------------------------------------------------------
 * Candidate clustering (search variant, host side).  Section 3's test
 * reports every point above the threshold, so one pulse gives many
 * neighbouring (DM, time, width) points.  Friends-of-friends: candidates
 * whose DM indices differ by at most dm_link and times by at most t_link
 * (samples; any widths) are linked; clusters are the connected components.
 * Each cluster: its strongest member (largest S/N; ties: smallest
 * (dm_idx, t, width_idx)), member count and DM / time extent.  Clusters are
 * written sorted by their strongest member's (dm_idx, t, width_idx); labels
 * (optional, [n]) receives each candidate's cluster index in that order.
 * Host arrays, caller-owned; no device work.  DD_ERR_OVERFLOW (and the true
 * count in *n_clusters) if more than `capacity` clusters. */
typedef struct {
    int32_t dm_idx, width_idx;   /* strongest member */
    int64_t t;
    float snr;
    int32_t n_members;
    int32_t dm_lo, dm_hi;        /* extent, inclusive */
    int64_t t_lo, t_hi;
} dd_cluster;

DD_API int dd_cluster_candidates(const dd_candidate *cands, int64_t n, int32_t dm_link, int64_t t_link,
                                 dd_cluster *clusters, int64_t capacity, int64_t *n_clusters,
                                 int64_t *labels);

/* ---------------------------------------------------------------------
 * Subband de-dispersion (Section 3.2): the paper's two-stage approximation
 * of the Section 3.1 sum, for fewer adds per output.
 *
 * The fine DM list (dm_list, ndm trials) is split into consecutive groups of
 * dms_per_nominal trials (the last group may be shorter); each group's
 * nominal DM is the midpoint of its first and last trial.  The nchans
 * channels are split into nsub subbands of nchans/nsub consecutive channels
 * (nsub must divide nchans); ref(s) is subband s's highest-frequency channel.
 * With d(c, DM) the Eq. 1 delay of dd_plan_create:
 *   stage 1  I[s][k][t] = sum_{c in s} in[c][t + d(c, D_k) - d(ref(s), D_k)]
 *            (each subband partially de-dispersed at nominal DM D_k),
 *   stage 2  out[j][t]  = sum_s I[s][k(j)][t + d(ref(s), dm_j)]
 *            (brute force over the subbands at each fine DM of group k(j)).
 * A fine DM whose delays equal its nominal DM's gets exactly the brute-force
 * sum; elsewhere each channel's effective delay differs from d(c, dm_j) by at
 * most |dm_j - D_k| x (its delay per unit DM minus ref(s)'s) + 2 samples,
 * the smearing the paper trades for speed.  Work per output sample:
 * nchans/dms_per_nominal + nsub adds instead of nchans.
 *
 * maxshift = max over (j, c) of the effective delay; nsamp_out = nsamp_in -
 * maxshift.  Output layout and dtype are those of dd_execute.  The plan owns
 * the intermediate series (nsub x n_nominal x L float32, L = nsamp_out + the
 * largest stage-2 delay rounded up to 4; allocated on the first execute,
 * size from dd_subband_plan_info) and the search scratch.  Input rows must be
 * 16-byte aligned (pointer and pitch); other arguments are checked as in
 * dd_plan_create.  Errors: DD_ERR_ARG (arguments, rows too long for shared
 * memory), DD_ERR_NOMEM, DD_ERR_CUDA. */
typedef struct dd_subband_plan dd_subband_plan;

DD_API int dd_subband_plan_create(int32_t nchans, double fch1_mhz, double foff_mhz, double tsamp_s,
                                  const double *dm_list, int32_t ndm, int32_t dms_per_nominal,
                                  int32_t nsub, const int32_t *boxcar_widths, int32_t nwidths,
                                  double sigma, int32_t in_dtype, int64_t nsamp_in,
                                  dd_subband_plan **plan_out);

/* Synchronises the device, then frees everything the plan owns. */
DD_API int dd_subband_plan_destroy(dd_subband_plan *plan);

/* Plan geometry; every pointer may be NULL.  nominal_dms: [n_nominal];
 * stage1_delays: [n_nominal][nchans] (d(c,D_k) - d(ref(s),D_k));
 * stage2_delays: [ndm][nsub] (d(ref(s), dm_j)); work_bytes: the intermediate
 * series' device bytes.  Host buffers, caller-owned. */
DD_API int dd_subband_plan_info(const dd_subband_plan *plan, int32_t *n_nominal, int64_t *maxshift,
                                int64_t *nsamp_out, double *nominal_dms, int32_t *stage1_delays,
                                int32_t *stage2_delays, int64_t *work_bytes);

/* Both stages, asynchronously on `stream` (in: [nchans][in_pitch] device,
 * out: [ndm][nsamp_out] device, as dd_execute), plus the per-block
 * statistics partials of out that dd_subband_search uses. */
DD_API int dd_subband_execute(dd_subband_plan *plan, const void *in_dev, int64_t in_pitch,
                              void *out_dev, void *stream);

/* dd_search on the subband output (Section 3 output stage: global mu/sigma,
 * boxcar n-sigma test, candidates sorted by (dm, t, width)); synchronises
 * `stream`.  DD_ERR_OVERFLOW as dd_search; DD_ERR_TIMEOUT if a kernel of the
 * last execute gave up waiting for its input copies. */
DD_API int dd_subband_search(dd_subband_plan *plan, const void *out_dev, dd_candidate *cand_host,
                             int64_t capacity, int64_t *n_found, void *stream);

/* mu and sigma used by the last dd_subband_search. */
DD_API int dd_subband_last_stats(const dd_subband_plan *plan, double *mu, double *sigma);

/* ---------------------------------------------------------------------
 * Survey plans (Section 3.2 with binning; the plans of Table 1 / Table 4):
 * several passes over disjoint DM ranges, each binning the input by its
 * factor and running subband de-dispersion at the binned sampling time.
 *
 * A pass is one row of the paper's survey-plan table: fine DM trials
 * low_dm + i*dm_step for i < round((high_dm - low_dm) / dm_step), input
 * binned by `bin` (average of `bin` adjacent samples: x_b[c][i] =
 * (1/bin) sum_{q<bin} x[c][i*bin + q], i < nsamp_in/bin, float32), and
 * round(sub_dm_step / dm_step) fine DMs per nominal DM.  Each pass is a
 * dd_subband_plan with tsamp_s*bin, nsamp_in/bin samples and nsub subbands
 * (input dtype for bin 1, float32 otherwise).  Pass outputs are
 * [ndm][nsamp_out] at the pass's resolution, caller-owned.  The plan owns
 * the binned inputs (nchans x nsamp_in/bin float32 per pass with bin > 1)
 * and each pass's subband series.  Arguments as dd_subband_plan_create. */
typedef struct {
    double low_dm, high_dm, dm_step;   /* pc cm^-3 */
    int32_t bin;                       /* binning factor N_b >= 1 */
    int32_t reserved;
    double sub_dm_step;                /* DM step between nominal DMs */
} dd_survey_pass;

typedef struct dd_survey_plan dd_survey_plan;

DD_API int dd_survey_plan_create(int32_t nchans, double fch1_mhz, double foff_mhz, double tsamp_s,
                                 const dd_survey_pass *passes, int32_t npass, int32_t nsub,
                                 const int32_t *boxcar_widths, int32_t nwidths, double sigma,
                                 int32_t in_dtype, int64_t nsamp_in, dd_survey_plan **plan_out);

/* Synchronises the device, then frees everything the plan owns. */
DD_API int dd_survey_plan_destroy(dd_survey_plan *plan);

/* Geometry of pass `pass` (any pointer may be NULL; dm_list: [ndm] host). */
DD_API int dd_survey_pass_info(const dd_survey_plan *plan, int32_t pass, int32_t *ndm, int32_t *bin,
                               int32_t *dms_per_nominal, int64_t *maxshift, int64_t *nsamp_out,
                               double *dm_list);

/* Every pass, asynchronously on `stream`: in_dev [nchans][in_pitch] (16-byte
 * aligned rows), out_devs[npass] device buffers of [ndm][nsamp_out]. */
DD_API int dd_survey_execute(dd_survey_plan *plan, const void *in_dev, int64_t in_pitch,
                             void *const *out_devs, void *stream);

/* Search of one pass's output (dd_subband_search; its own mu/sigma). */
DD_API int dd_survey_search(dd_survey_plan *plan, int32_t pass, const void *out_dev,
                            dd_candidate *cand_host, int64_t capacity, int64_t *n_found, void *stream);

/* mu and sigma used by the last dd_survey_search of pass `pass`. */
DD_API int dd_survey_last_stats(const dd_survey_plan *plan, int32_t pass, double *mu, double *sigma);

/* ---------------------------------------------------------------------
 * Front end of the real-time pipeline (Section 5, Tables 5-6): channeliser,
 * intensity and corner turn in one pass.
 *
 * volt_dev: complex64 baseband voltages [npol][nsub][nsamp] (interleaved
 * float32 re, im; device, 16-byte aligned; nsamp even), each subband sampled
 * in upper sideband.  Each subband's stream is cut into blocks of nfft
 * samples (nfft in {2, 4, 8, 16, 32}; trailing samples dropped) and
 * transformed by an nfft-point forward FFT (the paper's channeliser); the
 * intensity |X|^2 is summed over the npol (1 or 2) polarisations; the result
 * is written channel-major ("corner turn") to out_dev [nsub*nfft][out_pitch]
 * float32 (device, caller-owned, out_pitch >= nsamp/nfft): row s*nfft + j
 * holds the subband's j-th channel in DEScending frequency (FFT bin
 * (nfft/2 - 1 - j) mod nfft), column b the b-th block.  With subbands ordered
 * from the top of the band down, the rows form a standard descending-band
 * filterbank ready for dd_execute (sampling time nfft x the subband's).
 * Asynchronous on `stream`.  DD_ERR_ARG for invalid arguments. */
DD_API int dd_channelise(const void *volt_dev, int32_t npol, int32_t nsub, int64_t nsamp, int32_t nfft,
                         float *out_dev, int64_t out_pitch, void *stream);

/* Message describing the last failure on the calling thread ("" if none). */
DD_API const char *dd_last_error(void);

/* Library version string. */
DD_API const char *dd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DD_H */
