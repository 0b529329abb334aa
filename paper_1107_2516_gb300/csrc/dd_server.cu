// Streaming server: beams submit chunks of new samples as they arrive; each
// beam keeps the last maxshift samples of its stream resident on the device
// (Section 3, "Maximum shift": n outputs need n + maxshift inputs), so every
// chunk of N new samples yields N de-dispersed samples per DM trial and a
// Section 3 search over them.  Worker threads, each with its own CUDA stream,
// take the next ready chunk of any beam as soon as they are free, so chunks
// that arrive while others are on the GPU start immediately and overlap on the
// device (continuous batching).  Beams are admitted against a device-memory
// budget.
//
// Each beam's samples live in one device ring of nchans rows x `span` =
// maxshift + K*chunk columns.  Chunk k is written behind the previous one and
// de-dispersed in place from the window [write - maxshift, write + chunk):
// the window's base moves by one chunk per submission, and only when the next
// chunk would run past `span` are the last maxshift samples moved to the front
// (once per K chunks; K = 2 + floor(maxshift / chunk) keeps the move's source
// and destination disjoint).  Sequence numbers are checked on submission: a
// chunk that repeats or precedes the last accepted one is refused, and a chunk
// after a gap restarts the beam's stream (zeroed history, priming again)
// instead of joining unrelated samples.
#include "dd_internal.h"
#include "dd_ring.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Pending {
    int64_t seq;
    const void *host;
    int64_t host_pitch;
    double t_submit;
    bool restart;        // first chunk after a gap in seq: the stream starts over
};

struct ServerBeam {
    int id = 0;
    dd_plan *plan = nullptr;
    int64_t chunk = 0, maxshift = 0, nin = 0, pitch = 0;
    size_t eb = 1;
    void *ring = nullptr;     // [nchans][pitch] samples; the window base moves (dd::Ring)
    dd::Ring r;
    dd::SeqCheck sq;
    void *out = nullptr;
    // boundary search (optional): the previous chunk's last L outputs per row
    bool carry = false, tail_valid = false;
    int L = 0;
    void *tail = nullptr;
    int64_t processed = 0;
    bool busy = false, removed = false;
    std::deque<Pending> queue;
    size_t bytes = 0;
};

}  // namespace

struct dd_server {
    int device = 0;
    int64_t budget = 0, used = 0;
    int64_t cand_cap = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::map<int, ServerBeam *> beams;
    int next_id = 0;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;
    std::deque<dd_chunk_result> done;
    std::map<std::pair<int, int64_t>, std::vector<dd_candidate>> cands;
    bool stop = false;
    bool autotune = false;
};

namespace dd {

static void free_beam(ServerBeam *b)
{
    if (b->plan) dd_plan_destroy(b->plan);
    if (b->ring) cudaFree(b->ring);
    if (b->out) cudaFree(b->out);
    if (b->tail) cudaFree(b->tail);
    delete b;
}

// Next beam with a pending chunk and no chunk in flight (oldest submission first).
static ServerBeam *pick(dd_server *S)
{
    ServerBeam *best = nullptr;
    for (auto &kv : S->beams) {
        ServerBeam *b = kv.second;
        if (b->busy || b->removed || b->queue.empty()) continue;
        if (!best || b->queue.front().t_submit < best->queue.front().t_submit) best = b;
    }
    return best;
}

static void process(dd_server *S, ServerBeam *b, const Pending &pc, cudaStream_t s, dd_chunk_result &r,
                    std::vector<dd_candidate> &found)
{
    r.beam = b->id;
    r.seq = pc.seq;
    r.t_submit = pc.t_submit;
    r.t_start = now_s();
    r.status = DD_OK;
    const size_t rowb = (size_t)b->pitch * b->eb;
    const size_t hist = (size_t)b->maxshift * b->eb;
    const size_t nch = (size_t)b->plan->nchans;
    char *ring = static_cast<char *>(b->ring);
    const Ring::Step st = b->r.next(pc.restart);
    if (st.zero_history) b->tail_valid = false;      // no boundary window joins the two streams
    cudaError_t e = cudaSuccess;
    if (st.zero_history && hist)
        e = cudaMemset2DAsync(ring, rowb, 0, hist, nch, s);
    // the last maxshift samples to the front (once per K chunks)
    if (e == cudaSuccess && st.move_src >= 0 && hist)
        e = cudaMemcpy2DAsync(ring, rowb, ring + (size_t)st.move_src * b->eb, rowb, hist, nch,
                              cudaMemcpyDeviceToDevice, s);
    // the new samples behind the history
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(ring + (size_t)st.write_col * b->eb, rowb, pc.host, (size_t)pc.host_pitch * b->eb,
                              (size_t)b->chunk * b->eb, nch, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        r.status = cuda_fail(e, "server copies");
    } else if (st.priming) {
        // the resident history does not yet hold maxshift real samples
        e = cudaStreamSynchronize(s);
        r.status = e == cudaSuccess ? DD_PRIMING : cuda_fail(e, "server sync");
    } else {
        int rc = dd_execute(b->plan, ring + (size_t)st.window_col * b->eb, b->pitch, b->out, s);
        int64_t n = 0;
        found.resize((size_t)S->cand_cap);
        if (rc == DD_OK) rc = dd_search(b->plan, b->out, found.data(), S->cand_cap, &n, s);
        found.resize((size_t)std::min(n, S->cand_cap));
        dd_last_stats(b->plan, &r.mu, &r.sigma);
        if ((rc == DD_OK || rc == DD_ERR_OVERFLOW) && b->carry && b->L > 0) {
            int rc2 = DD_OK;
            if (b->tail_valid) {
                // windows from the previous chunk's tail into this chunk
                std::vector<dd_candidate> bnd((size_t)S->cand_cap);
                int64_t nb = 0;
                rc2 = boundary_search_launch(b->plan, b->tail, b->out, b->L, s);
                if (rc2 == DD_OK)
                    rc2 = search_readback(b->plan, bnd.data(), S->cand_cap, &nb, s, b->plan->cand_cap);
                if (rc2 == DD_OK || rc2 == DD_ERR_OVERFLOW) {
                    const dd_plan *p = b->plan;
                    for (int64_t i = 0; i < std::min(nb, S->cand_cap); ++i) {
                        dd_candidate c = bnd[(size_t)i];
                        const double w = (double)p->widths[c.width_idx];
                        const double mu = p->row_stats ? p->h_rowprm[c.dm_idx].mu : r.mu;
                        const double sg = p->row_stats ? p->h_rowprm[c.dm_idx].sigma : r.sigma;
                        c.snr = (float)((c.value - w * mu) / (sg * std::sqrt(w)));
                        if ((int64_t)found.size() < S->cand_cap) found.push_back(c);
                    }
                    n += nb;
                    std::sort(found.begin(), found.end(), [](const dd_candidate &x, const dd_candidate &y) {
                        if (x.dm_idx != y.dm_idx) return x.dm_idx < y.dm_idx;
                        if (x.t != y.t) return x.t < y.t;
                        return x.width_idx < y.width_idx;
                    });
                    if (n > S->cand_cap) rc = DD_ERR_OVERFLOW;
                    rc2 = DD_OK;
                }
            }
            // this chunk's last L outputs of every row become the next tail
            if (rc2 == DD_OK) {
                cudaError_t e2 = cudaMemcpy2DAsync(b->tail, (size_t)b->L * 4, (const char *)b->out + (size_t)(b->chunk - b->L) * 4,
                                                   (size_t)b->chunk * 4, (size_t)b->L * 4, (size_t)b->plan->ndm,
                                                   cudaMemcpyDeviceToDevice, s);
                if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(s);
                if (e2 != cudaSuccess) rc2 = cuda_fail(e2, "boundary tail");
                b->tail_valid = rc2 == DD_OK;
            }
            if (rc2 != DD_OK) rc = rc2;
        }
        r.status = rc;
        r.n_candidates = n;
    }
    b->processed++;
    r.t_done = now_s();
}

static void worker(dd_server *S, int w)
{
    cudaSetDevice(S->device);
    cudaStream_t s = S->streams[w];
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        ServerBeam *b = nullptr;
        S->cv_work.wait(lk, [&] { return S->stop || (b = pick(S)) != nullptr; });
        if (S->stop) return;
        Pending pc = b->queue.front();
        b->queue.pop_front();
        b->busy = true;
        lk.unlock();
        dd_chunk_result r;
        memset(&r, 0, sizeof(r));
        std::vector<dd_candidate> found;
        process(S, b, pc, s, r, found);
        lk.lock();
        b->busy = false;
        if (!found.empty()) S->cands[{b->id, pc.seq}] = std::move(found);
        S->done.push_back(r);
        if (b->removed && b->queue.empty()) {
            S->used -= (int64_t)b->bytes;
            S->beams.erase(b->id);
            free_beam(b);
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
}

}  // namespace dd

using namespace dd;

extern "C" {

int dd_server_create(int64_t hbm_budget_bytes, int32_t nworkers, int64_t max_candidates, dd_server **out)
{
    if (!out) return set_error(DD_ERR_ARG, "server_out is NULL");
    *out = nullptr;
    if (hbm_budget_bytes <= 0 || nworkers < 1 || nworkers > 64 || max_candidates < 1)
        return set_error(DD_ERR_ARG, "bad server parameters");
    dd_server *S = new dd_server();
    cudaGetDevice(&S->device);
    S->budget = hbm_budget_bytes;
    S->cand_cap = max_candidates;
    for (int w = 0; w < nworkers; ++w) {
        cudaStream_t s;
        cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e != cudaSuccess) { dd_server_destroy(S); return cuda_fail(e, "cudaStreamCreate"); }
        S->streams.push_back(s);
    }
    for (int w = 0; w < nworkers; ++w) S->workers.emplace_back(worker, S, w);
    *out = S;
    return DD_OK;
}

int dd_server_destroy(dd_server *S)
{
    if (!S) return DD_OK;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (auto &t : S->workers) t.join();
    for (auto &kv : S->beams) free_beam(kv.second);
    for (cudaStream_t s : S->streams) cudaStreamDestroy(s);
    delete S;
    return DD_OK;
}

int dd_server_add_beam(dd_server *S, int32_t nchans, double fch1, double foff, double tsamp,
                       const double *dm_list, int32_t ndm, const int32_t *widths, int32_t nwidths,
                       double sigma, int32_t dtype, int64_t chunk, int32_t *beam_id)
{
    if (!S || !beam_id || chunk < 1) return set_error(DD_ERR_ARG, "bad arguments");
    cudaSetDevice(S->device);
    // maxshift first: it sizes the history ring and the plan's input length
    const long long M = max_delay(nchans, fch1, foff, tsamp, dm_list, ndm);
    if (M < 0) return set_error(DD_ERR_ARG, "invalid beam parameters");
    if (dtype != DD_F32 && dtype != DD_U8 && dtype != DD_F16) return set_error(DD_ERR_ARG, "unknown input dtype");
    int rc = DD_OK;
    const size_t eb = in_elem_bytes((dd_dtype)dtype);
    const int64_t nin = M + chunk;
    const int64_t al = 16 / (int64_t)eb;
    // ring pitch: the span, aligned, plus one aligned unit (the tiled kernels
    // stage an input row up to nsamp_in rounded up to that unit)
    const int64_t pitch = (Ring::span_of(M, chunk) + al - 1) / al * al + al;
    // device bytes: the ring, the output, and the plan's tables (delay-table sized estimate)
    const size_t ring_b = (size_t)nchans * (size_t)pitch * eb;
    const size_t out_b = (size_t)ndm * (size_t)chunk * 4;
    const size_t tab_b = (size_t)ndm * (size_t)nchans * 4 * 8;
    const size_t need = ring_b + out_b + tab_b;
    bool tune;
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (S->used + (int64_t)need > S->budget)
            return set_error(DD_ERR_BUDGET, "admission refused: beam needs %zu bytes, %lld of %lld in use",
                             need, (long long)S->used, (long long)S->budget);
        S->used += (int64_t)need;    // reserve before allocating
        tune = S->autotune;
    }
    ServerBeam *b = new ServerBeam();
    b->chunk = chunk; b->maxshift = M; b->nin = nin; b->pitch = pitch; b->eb = eb; b->bytes = need;
    b->r.init(M, chunk);
    rc = dd_plan_create(nchans, fch1, foff, tsamp, dm_list, ndm, widths, nwidths, sigma, dtype, nin, &b->plan);
    cudaError_t e = cudaSuccess;
    if (rc == DD_OK) e = cudaMalloc(&b->ring, ring_b);
    if (rc == DD_OK && e == cudaSuccess) e = cudaMalloc(&b->out, out_b);
    if (rc == DD_OK && e == cudaSuccess) e = cudaMemset(b->ring, 0, ring_b);
    if (rc == DD_OK && e != cudaSuccess) rc = cuda_fail(e, "beam buffers");
    if (rc == DD_OK) {
        // kernel 5 (shared subband partial sums) where its tables fit this
        // beam, else the plan's default; or, on request, the autotuner's pick
        // timed on the beam's own (zeroed) buffers, cached per plan shape
        if (tune) {
            cudaStream_t ts = nullptr;
            e = cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking);
            if (e == cudaSuccess) {
                rc = dd_plan_autotune(b->plan, b->ring, pitch, b->out, ts);
                cudaStreamDestroy(ts);
            } else {
                rc = cuda_fail(e, "admission stream");
            }
        } else if (dd_plan_set_kernel(b->plan, 5) != DD_OK) {
            set_error(DD_OK, "%s", "");
        }
    }
    std::lock_guard<std::mutex> g(S->mu);
    if (rc != DD_OK) {
        S->used -= (int64_t)need;
        free_beam(b);
        return rc;
    }
    b->id = S->next_id++;
    S->beams[b->id] = b;
    *beam_id = b->id;
    return DD_OK;
}

int dd_server_set_boundary_search(dd_server *S, int32_t beam, int32_t on)
{
    if (!S) return set_error(DD_ERR_ARG, "server is NULL");
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->beams.find(beam);
    if (it == S->beams.end() || it->second->removed) return set_error(DD_ERR_ARG, "no beam %d", beam);
    ServerBeam *b = it->second;
    if (b->busy || !b->queue.empty() || b->processed > 0)
        return set_error(DD_ERR_ARG, "set the boundary search before the beam's first chunk");
    int wmax = 1;
    for (int w : b->plan->widths) wmax = std::max(wmax, w);
    const int L = wmax - 1;
    if (on && L > b->chunk) return set_error(DD_ERR_ARG, "widest boxcar exceeds chunk + 1");
    if (on && L > 0 && !b->tail) {
        cudaSetDevice(S->device);
        cudaError_t e = cudaMalloc(&b->tail, (size_t)b->plan->ndm * L * 4);
        if (e != cudaSuccess) { b->tail = nullptr; return cuda_fail(e, "boundary tail"); }
    }
    b->carry = on != 0;
    b->L = L;
    b->tail_valid = false;
    return DD_OK;
}

int dd_server_remove_beam(dd_server *S, int32_t beam)
{
    if (!S) return set_error(DD_ERR_ARG, "server is NULL");
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->beams.find(beam);
    if (it == S->beams.end()) return set_error(DD_ERR_ARG, "no beam %d", beam);
    ServerBeam *b = it->second;
    b->removed = true;
    b->queue.clear();
    if (!b->busy) {
        S->used -= (int64_t)b->bytes;
        S->beams.erase(it);
        free_beam(b);
    }
    return DD_OK;
}

int dd_server_submit(dd_server *S, int32_t beam, const void *chunk_host, int64_t host_pitch, int64_t seq)
{
    if (!S || !chunk_host) return set_error(DD_ERR_ARG, "bad arguments");
    const double t = now_s();
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->beams.find(beam);
    if (it == S->beams.end() || it->second->removed) return set_error(DD_ERR_ARG, "no beam %d", beam);
    ServerBeam *b = it->second;
    if (host_pitch < b->chunk) return set_error(DD_ERR_ARG, "host_pitch < chunk");
    bool restart = false;
    const int64_t expect = b->sq.next;
    const int rc = b->sq.admit(seq, &restart);
    if (rc == DD_ERR_SEQ)
        return set_error(DD_ERR_SEQ, "beam %d: chunk seq %lld refused (next expected %lld): repeated or late",
                         beam, (long long)seq, (long long)expect);
    b->queue.push_back(Pending{seq, chunk_host, host_pitch, t, restart});
    S->cv_work.notify_one();
    if (rc == DD_SEQ_GAP)
        return set_error(DD_SEQ_GAP, "beam %d: chunks %lld..%lld missing; the stream restarts at %lld",
                         beam, (long long)expect, (long long)seq - 1, (long long)seq);
    return DD_OK;
}

int dd_server_poll(dd_server *S, dd_chunk_result *results, int32_t max_results, int32_t *n, int32_t wait_ms)
{
    if (!S || !n || (max_results > 0 && !results)) return set_error(DD_ERR_ARG, "bad arguments");
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->done.empty() && wait_ms > 0)
        S->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !S->done.empty(); });
    int k = 0;
    while (k < max_results && !S->done.empty()) {
        results[k++] = S->done.front();
        S->done.pop_front();
    }
    *n = k;
    return DD_OK;
}

int dd_server_candidates(dd_server *S, int32_t beam, int64_t seq, dd_candidate *cand_host, int64_t capacity,
                         int64_t *n_found)
{
    if (!S || !n_found || capacity < 0 || (capacity > 0 && !cand_host)) return set_error(DD_ERR_ARG, "bad arguments");
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->cands.find({beam, seq});
    if (it == S->cands.end()) { *n_found = 0; return DD_OK; }
    const int64_t n = (int64_t)it->second.size();
    memcpy(cand_host, it->second.data(), (size_t)std::min(n, capacity) * sizeof(dd_candidate));
    *n_found = n;
    S->cands.erase(it);
    return n > capacity ? set_error(DD_ERR_OVERFLOW, "capacity too small") : DD_OK;
}

int dd_server_beam_info(dd_server *S, int32_t beam, int64_t *maxshift, int64_t *chunk, int64_t *ndm,
                        void **out_dev, int64_t *device_bytes)
{
    if (!S) return set_error(DD_ERR_ARG, "server is NULL");
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->beams.find(beam);
    if (it == S->beams.end()) return set_error(DD_ERR_ARG, "no beam %d", beam);
    ServerBeam *b = it->second;
    if (maxshift) *maxshift = b->maxshift;
    if (chunk) *chunk = b->chunk;
    if (ndm) *ndm = b->plan->ndm;
    if (out_dev) *out_dev = b->out;
    if (device_bytes) *device_bytes = (int64_t)b->bytes;
    return DD_OK;
}

int dd_server_set_autotune(dd_server *S, int32_t on)
{
    if (!S) return set_error(DD_ERR_ARG, "server is NULL");
    std::lock_guard<std::mutex> g(S->mu);
    S->autotune = on != 0;
    return DD_OK;
}

int dd_server_beam_kernel(dd_server *S, int32_t beam, int32_t *kernel, int32_t *config)
{
    if (!S) return set_error(DD_ERR_ARG, "server is NULL");
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->beams.find(beam);
    if (it == S->beams.end()) return set_error(DD_ERR_ARG, "no beam %d", beam);
    int rc = DD_OK;
    if (kernel) rc = dd_plan_get_kernel(it->second->plan, kernel);
    if (rc == DD_OK && config) {
        int32_t grp = 0, ti = 0, nw = 0;
        if (dd_plan_get_tile(it->second->plan, config, &grp, &ti, &nw) != DD_OK) *config = -1;
    }
    return rc;
}

int dd_server_ring_schedule(int64_t maxshift, int64_t chunk, int32_t n, const int64_t *seq, int64_t *span,
                            int32_t *submit_status, int32_t *restart, int64_t *move_src, int64_t *write_col,
                            int64_t *window_col, int32_t *priming)
{
    if (maxshift < 0 || chunk < 1 || n < 0 || (n > 0 && (!seq || !submit_status || !restart || !move_src ||
                                                         !write_col || !window_col || !priming)))
        return set_error(DD_ERR_ARG, "bad arguments");
    SeqCheck sq;
    Ring r;
    r.init(maxshift, chunk);
    if (span) *span = r.span;
    for (int32_t i = 0; i < n; ++i) {
        bool rs = false;
        submit_status[i] = sq.admit(seq[i], &rs);
        restart[i] = rs ? 1 : 0;
        if (submit_status[i] == DD_ERR_SEQ) {
            move_src[i] = write_col[i] = window_col[i] = -1;
            priming[i] = 0;
            continue;
        }
        const Ring::Step st = r.next(rs);
        move_src[i] = st.move_src;
        write_col[i] = st.write_col;
        window_col[i] = st.window_col;
        priming[i] = st.priming ? 1 : 0;
    }
    return DD_OK;
}

int dd_server_memory(dd_server *S, int64_t *used, int64_t *budget)
{
    if (!S) return set_error(DD_ERR_ARG, "server is NULL");
    std::lock_guard<std::mutex> g(S->mu);
    if (used) *used = S->used;
    if (budget) *budget = S->budget;
    return DD_OK;
}

}  // extern "C"
