// fdd_serve.cu -- the serving runtime: continuous batching of real-time chunks
// from many compound beams onto one GPU.
//
// The paper's pipeline processes 1.024 s chunks of every compound beam as
// they arrive, each output needing the next max-delay of input (Sec. "AMBER";
// Sec. "Computing performance": real time over a whole observation).  Here:
//   * every beam owns two device window buffers [n_tab][n_chan][pitch]; a
//     window of n_in = chunk + max delay (+ D - 1) samples starting at w*chunk
//     is searched for the outputs whose first sample lies in
//     [w*chunk, (w+1)*chunk), with downsampling bins aligned to the beam's
//     stream (fdd_search_window), so the windows tile one search of the
//     whole stream.  When window w is complete its tail is copied device-to-device
//     to the other buffer, where window w+1 is assembled from the following
//     chunks (host-to-device 2-D copies on the copy stream);
//   * complete windows wait in a FIFO; "slots" (workspace + candidate buffer
//     + pinned host result buffer) are sized once from free HBM at start-up;
//   * whenever slots are free, every queued window (up to the free slots and
//     FDD_MAX_BATCH_JOBS) goes out in ONE fdd_search_batch on one of several
//     compute streams, so windows that arrive while others run are admitted
//     as soon as slots free up and their kernels overlap with the running
//     ones;
//   * GPU-side events order everything: a search waits for its window's
//     copies, a buffer is refilled only after the search that reads it has
//     finished, results are copied back to pinned memory behind the search.
// The host never blocks except in fdd_server_drain.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <new>
#include <vector>

#include "fdd_plan_impl.h"

using namespace fdd::host;

namespace {

double now_s() {
    using namespace std::chrono;
    return duration_cast<duration<double>>(steady_clock::now().time_since_epoch()).count();
}

constexpr int kComputeStreams = 3;

}  // namespace

struct ServeBeam {
    uint8_t* buf[2] = {nullptr, nullptr};   // window buffers
    cudaEvent_t ready[2] = {nullptr, nullptr};  // copies into buf[k] done
    cudaEvent_t freed[2] = {nullptr, nullptr};  // last search reading buf[k] done
    bool freed_valid[2] = {false, false};
    bool pending[2] = {false, false};  // buf[k] holds a queued, not yet launched window
    bool deferred = false;     // tail copy into the other buffer waits for that buffer's window to launch
    int cur = 0;               // buffer that receives the next chunk
    int64_t held = 0;          // samples of the current window present in buf[cur]
    int64_t next_seq = 0;      // expected chunk sequence number
    int64_t window = 0;        // index of the window being assembled in buf[cur]
};

struct ServeSlot {
    void* ws = nullptr;
    fdd_candidate* d_cands = nullptr;
    uint64_t* d_count = nullptr;
    fdd_candidate* d_sb_cands = nullptr;  // plain per-SB path: one SB's records before they are appended
    uint64_t* d_sb_count = nullptr;
    fdd_candidate* h_cands = nullptr;   // pinned
    uint64_t* h_count = nullptr;        // pinned
    bool busy = false;
};

struct ServeWindow {
    int32_t beam;
    int64_t window;
    int buf;
    double t_arrival;   // arrival of the chunk that completed the window
    double t_ready;     // when it entered the queue
    double t_launch = 0;
    int slot = -1;
    int batch_jobs = 0;
};

struct ServeBatch {
    std::vector<ServeWindow> wins;
    cudaEvent_t done = nullptr;
    int stream = 0;
};

struct fdd_server {
    fdd_plan* plan = nullptr;
    fdd_server_desc d{};
    int64_t n_in = 0, pitch = 0, buf_len = 0, rows = 0;
    size_t ws_bytes = 0;
    std::vector<ServeBeam> beams;
    std::vector<ServeSlot> slots;
    std::deque<ServeWindow> queue;
    std::deque<ServeBatch> inflight;
    std::vector<fdd_window_result> results;
    std::vector<fdd_candidate> result_cands;
    std::vector<cudaEvent_t> event_pool;
    cudaStream_t copy_stream = nullptr;
    cudaStream_t compute[kComputeStreams] = {};
    int next_stream = 0;
    int64_t n_launched = 0, n_done = 0, n_batches = 0, max_queue = 0;
    std::vector<fdd_plan*> sb_plans;  // non-empty: the plain per-SB path (fdd_server_set_plain)
};

namespace {

cudaEvent_t take_event(fdd_server* s) {
    if (!s->event_pool.empty()) {
        cudaEvent_t e = s->event_pool.back();
        s->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    return e;
}

void destroy_server(fdd_server* s) {
    if (!s) return;
    if (s->copy_stream) cudaStreamSynchronize(s->copy_stream);
    for (cudaStream_t st : s->compute)
        if (st) cudaStreamSynchronize(st);
    for (ServeBeam& b : s->beams)
        for (int k = 0; k < 2; k++) {
            if (b.buf[k]) cudaFree(b.buf[k]);
            if (b.ready[k]) cudaEventDestroy(b.ready[k]);
            if (b.freed[k]) cudaEventDestroy(b.freed[k]);
        }
    for (ServeSlot& sl : s->slots) {
        if (sl.ws) cudaFree(sl.ws);
        if (sl.d_cands) cudaFree(sl.d_cands);
        if (sl.d_count) cudaFree(sl.d_count);
        if (sl.d_sb_cands) cudaFree(sl.d_sb_cands);
        if (sl.d_sb_count) cudaFree(sl.d_sb_count);
        if (sl.h_cands) cudaFreeHost(sl.h_cands);
        if (sl.h_count) cudaFreeHost(sl.h_count);
    }
    for (ServeBatch& b : s->inflight)
        if (b.done) cudaEventDestroy(b.done);
    for (cudaEvent_t e : s->event_pool) cudaEventDestroy(e);
    if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
    for (cudaStream_t st : s->compute)
        if (st) cudaStreamDestroy(st);
    delete s;
}

// Carry the last buf_len - chunk samples of beam b's current buffer into the
// other buffer (after the search that last read it), making it current.
int tail_copy(fdd_server* s, ServeBeam& b) {
    cudaStream_t cs = s->copy_stream;
    const int src = b.cur, dst = 1 - b.cur;
    const int64_t L = s->d.chunk_len;
    cudaError_t e;
    if (b.freed_valid[dst] && (e = cudaStreamWaitEvent(cs, b.freed[dst], 0)) != cudaSuccess)
        return cuda_fail(e, "cudaStreamWaitEvent");
    e = cudaMemcpy2DAsync(b.buf[dst], s->pitch, b.buf[src] + L, s->pitch, s->buf_len - L, s->rows,
                          cudaMemcpyDeviceToDevice, cs);
    if (e != cudaSuccess) return cuda_fail(e, "window tail copy");
    b.cur = dst;
    b.held = s->buf_len - L;
    b.deferred = false;
    return FDD_OK;
}

// Retire finished batches: copy results out of the pinned slot buffers.
int retire(fdd_server* s, double t) {
    for (auto it = s->inflight.begin(); it != s->inflight.end();) {
        ServeBatch& b = *it;
        const cudaError_t q = cudaEventQuery(b.done);
        if (q == cudaErrorNotReady) {
            ++it;
            continue;
        }
        if (q != cudaSuccess) return cuda_fail(q, "server batch");
        for (ServeWindow& w : b.wins) {
            ServeSlot& sl = s->slots[w.slot];
            fdd_window_result r{};
            r.beam = w.beam;
            r.window = w.window;
            r.t0_native = w.window * s->d.chunk_len;
            r.t_arrival = w.t_arrival;
            r.t_ready = w.t_ready;
            r.t_launch = w.t_launch;
            r.t_done = t;
            r.n_cands = static_cast<int64_t>(*sl.h_count);
            r.batch_jobs = w.batch_jobs;
            const int64_t keep = std::min<int64_t>(r.n_cands, s->d.cap_per_window);
            r.cand_offset = static_cast<int64_t>(s->result_cands.size());
            r.n_cands_kept = keep;
            s->result_cands.insert(s->result_cands.end(), sl.h_cands, sl.h_cands + keep);
            s->results.push_back(r);
            sl.busy = false;
            s->n_done++;
        }
        s->event_pool.push_back(b.done);
        it = s->inflight.erase(it);
    }
    return FDD_OK;
}

// Plain per-SB path: append the records of single-SB search `sb` (sb field 0)
// to the window's list, relabelled with the compound beam's SB index.  The
// launches of one window are ordered on one stream, so *count is the number
// of records (true total) appended so far; the first cap are kept.
__global__ void k_append_sb(const fdd_candidate* __restrict__ src, const uint64_t* __restrict__ src_count,
                            int64_t src_cap, fdd_candidate* __restrict__ dst, uint64_t* __restrict__ count,
                            int64_t cap, int32_t sb) {
    const uint64_t base = *count;
    const uint64_t n_true = *src_count;
    const uint64_t n_src = n_true < static_cast<uint64_t>(src_cap) ? n_true : static_cast<uint64_t>(src_cap);
    for (uint64_t k = threadIdx.x; k < n_src && base + k < static_cast<uint64_t>(cap); k += blockDim.x) {
        fdd_candidate c = src[k];
        c.sb = sb;
        dst[base + k] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) *count = base + n_true;
}

// One window through the plain per-SB path on stream cs: n_sb single-SB
// searches one after another, each appending its records to the slot's list.
int launch_plain(fdd_server* s, const ServeWindow& w, ServeSlot& sl, cudaStream_t cs) {
    const ServeBeam& b = s->beams[w.beam];
    cudaError_t e = cudaMemsetAsync(sl.d_count, 0, sizeof(uint64_t), cs);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    for (size_t k = 0; k < s->sb_plans.size(); k++) {
        const int rc = search_impl(s->sb_plans[k], b.buf[w.buf], s->n_in, s->pitch, s->d.chunk_len,
                                   w.window * s->d.chunk_len, true, sl.ws, s->ws_bytes, sl.d_sb_cands,
                                   s->d.cap_per_window, sl.d_sb_count, nullptr, cs);
        if (rc != FDD_OK) return rc;
        k_append_sb<<<1, 256, 0, cs>>>(sl.d_sb_cands, sl.d_sb_count, s->d.cap_per_window, sl.d_cands, sl.d_count,
                                       s->d.cap_per_window, static_cast<int32_t>(k));
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "k_append_sb");
    }
    return FDD_OK;
}

// Launch every queued window that finds a free slot, as one batch.
int schedule(fdd_server* s, double t) {
    while (!s->queue.empty()) {
        std::vector<int> free_slots;
        for (int k = 0; k < static_cast<int>(s->slots.size()); k++)
            if (!s->slots[k].busy) free_slots.push_back(k);
        if (free_slots.empty()) return FDD_OK;
        // the plain per-SB path takes one window per launch group (no batching)
        const int n = std::min<int>({static_cast<int>(free_slots.size()), static_cast<int>(s->queue.size()),
                                     s->sb_plans.empty() ? FDD_MAX_BATCH_JOBS : 1});
        ServeBatch batch;
        // SB-factored batches (and the plain path) are independent of one another and rotate over the
        // compute streams; the persistent modes share the plan's work counters, so their batches stay
        // in order on one stream
        const bool shared_counters = s->sb_plans.empty() && !s->plan->batch.sbf;
        batch.stream = shared_counters ? 0 : s->next_stream;
        if (!shared_counters) s->next_stream = (s->next_stream + 1) % kComputeStreams;
        cudaStream_t cs = s->compute[batch.stream];
        std::vector<fdd_job> jobs(n);
        for (int k = 0; k < n; k++) {
            ServeWindow w = s->queue.front();
            s->queue.pop_front();
            ServeBeam& b = s->beams[w.beam];
            ServeSlot& sl = s->slots[free_slots[k]];
            w.slot = free_slots[k];
            w.t_launch = t;
            w.batch_jobs = n;
            sl.busy = true;
            cudaError_t e = cudaStreamWaitEvent(cs, b.ready[w.buf], 0);
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
            fdd_job& j = jobs[k];
            j.d_tabs = b.buf[w.buf];
            j.n_in = s->n_in;
            j.pitch = s->pitch;
            j.t_offset_native = w.window * s->d.chunk_len;
            j.d_workspace = sl.ws;
            j.workspace_bytes = s->ws_bytes;
            j.d_cands = sl.d_cands;
            j.cap = s->d.cap_per_window;
            j.d_count = sl.d_count;
            j.d_series = nullptr;
            j.bins_absolute = 1;
            batch.wins.push_back(w);
        }
        int rc = s->sb_plans.empty()
                     ? fdd_search_batch(s->plan, jobs.data(), n, s->d.chunk_len, reinterpret_cast<fdd_stream_t>(cs))
                     : launch_plain(s, batch.wins[0], s->slots[batch.wins[0].slot], cs);
        if (rc != FDD_OK) return rc;
        for (const ServeWindow& w : batch.wins) {
            ServeSlot& sl = s->slots[w.slot];
            cudaError_t e = cudaMemcpyAsync(sl.h_count, sl.d_count, sizeof(uint64_t), cudaMemcpyDeviceToHost, cs);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(sl.h_cands, sl.d_cands, sizeof(fdd_candidate) * s->d.cap_per_window,
                                    cudaMemcpyDeviceToHost, cs);
            if (e != cudaSuccess) return cuda_fail(e, "result copy");
            // the buffer this window read may be refilled once this stream gets here
            ServeBeam& b = s->beams[w.beam];
            if ((e = cudaEventRecord(b.freed[w.buf], cs)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
            b.freed_valid[w.buf] = true;
            b.pending[w.buf] = false;
            if (b.deferred && b.cur != w.buf) {
                const int rc2 = tail_copy(s, b);
                if (rc2 != FDD_OK) return rc2;
            }
        }
        batch.done = take_event(s);
        if (!batch.done) return fail(FDD_ERR_CUDA, "cudaEventCreate");
        cudaError_t e = cudaEventRecord(batch.done, cs);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        s->n_launched += n;
        s->n_batches++;
        s->inflight.push_back(std::move(batch));
    }
    return FDD_OK;
}

}  // namespace

extern "C" {

double fdd_now(void) { return now_s(); }

int fdd_server_create(fdd_plan* plan, const fdd_server_desc* desc, fdd_server** out) {
    if (!plan || !desc || !out || desc->n_beams < 1 || desc->chunk_len < 1 || desc->cap_per_window < 1 ||
        desc->max_slots < 0 || desc->hbm_reserve_frac < 0 || desc->hbm_reserve_frac >= 1)
        return fail(FDD_ERR_INVALID_ARG, "bad server description");
    *out = nullptr;
    fdd_server* s = new (std::nothrow) fdd_server();
    if (!s) return fail(FDD_ERR_NO_MEMORY, "host allocation");
    s->plan = plan;
    s->d = *desc;
    s->rows = static_cast<int64_t>(plan->n_tab) * plan->n_chan;
    // A window holds chunk + max delay samples; chunks arrive whole, so the
    // buffer holds a whole number of chunks.
    s->n_in = window_input_len(plan, desc->chunk_len);
    const int64_t chunks_per_window = (s->n_in + desc->chunk_len - 1) / desc->chunk_len;
    s->buf_len = chunks_per_window * desc->chunk_len;
    s->pitch = static_cast<int64_t>(align_up(static_cast<size_t>(s->buf_len), 16));
    int rc = FDD_OK;
    s->ws_bytes = make_layout(plan, s->n_in, desc->chunk_len, true, true).total;
    const size_t ring_bytes = static_cast<size_t>(s->rows) * s->pitch;
    const size_t slot_bytes = s->ws_bytes + sizeof(fdd_candidate) * desc->cap_per_window + 256;
    // Admission by free HBM: rings for every beam first, then as many slots
    // as the rest allows (minus the reserve), capped by max_slots.
    size_t free_b = 0, total_b = 0;
    cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) {
        destroy_server(s);
        return cuda_fail(e, "cudaMemGetInfo");
    }
    if (desc->hbm_budget_bytes > 0) free_b = std::min(free_b, static_cast<size_t>(desc->hbm_budget_bytes));
    const double usable = static_cast<double>(free_b) * (1.0 - desc->hbm_reserve_frac);
    const double after_rings = usable - 2.0 * ring_bytes * desc->n_beams;
    int64_t n_slots = after_rings > 0 ? static_cast<int64_t>(after_rings / slot_bytes) : 0;
    if (desc->max_slots > 0) n_slots = std::min<int64_t>(n_slots, desc->max_slots);
    n_slots = std::min<int64_t>(n_slots, 4 * FDD_MAX_BATCH_JOBS);
    if (n_slots < 1) {
        destroy_server(s);
        return fail(FDD_ERR_NO_MEMORY, "free HBM does not hold the beams' rings and one search slot");
    }
    if ((rc = batch_prepare_mode(plan, desc->chunk_len, true)) != FDD_OK) {
        destroy_server(s);
        return rc;
    }
    if ((e = cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking)) != cudaSuccess) {
        destroy_server(s);
        return cuda_fail(e, "cudaStreamCreate");
    }
    for (cudaStream_t& st : s->compute)
        if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) {
            destroy_server(s);
            return cuda_fail(e, "cudaStreamCreate");
        }
    s->beams.resize(desc->n_beams);
    for (ServeBeam& b : s->beams)
        for (int k = 0; k < 2; k++) {
            if ((e = cudaMalloc(&b.buf[k], ring_bytes)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&b.ready[k], cudaEventDisableTiming)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&b.freed[k], cudaEventDisableTiming)) != cudaSuccess) {
                destroy_server(s);
                return cuda_fail(e, "beam ring allocation");
            }
            if ((e = cudaMemset(b.buf[k], 0, ring_bytes)) != cudaSuccess) {
                destroy_server(s);
                return cuda_fail(e, "cudaMemset");
            }
        }
    s->slots.resize(n_slots);
    for (ServeSlot& sl : s->slots) {
        if ((e = cudaMalloc(&sl.ws, s->ws_bytes)) != cudaSuccess ||
            (e = cudaMalloc(&sl.d_cands, sizeof(fdd_candidate) * desc->cap_per_window)) != cudaSuccess ||
            (e = cudaMalloc(&sl.d_count, sizeof(uint64_t))) != cudaSuccess ||
            (e = cudaMallocHost(&sl.h_cands, sizeof(fdd_candidate) * desc->cap_per_window)) != cudaSuccess ||
            (e = cudaMallocHost(&sl.h_count, sizeof(uint64_t))) != cudaSuccess) {
            destroy_server(s);
            return cuda_fail(e, "slot allocation");
        }
    }
    *out = s;
    return FDD_OK;
}

int fdd_server_set_plain(fdd_server* s, fdd_plan* const* sb_plans, int32_t n_sb) {
    if (!s || !sb_plans || n_sb != s->plan->n_sb) return fail(FDD_ERR_INVALID_ARG, "need one plan per SB");
    if (s->n_launched > 0 || !s->queue.empty()) return fail(FDD_ERR_INVALID_ARG, "server already in use");
    for (int32_t k = 0; k < n_sb; k++) {
        const fdd_plan* q = sb_plans[k];
        if (!q || q->n_sb != 1 || q->n_tab != s->plan->n_tab || q->n_chan != s->plan->n_chan ||
            window_input_len(q, s->d.chunk_len) > s->n_in)
            return fail(FDD_ERR_INVALID_ARG, "each plan must be a single-SB plan of the server's TABs and channels, "
                                             "with no larger delay");
        if (make_layout(q, s->n_in, s->d.chunk_len, true, true).total > s->ws_bytes)
            return fail(FDD_ERR_WORKSPACE, "a single-SB plan needs more workspace than a slot has");
    }
    for (ServeSlot& sl : s->slots) {
        cudaError_t e;
        if (!sl.d_sb_cands &&
            ((e = cudaMalloc(&sl.d_sb_cands, sizeof(fdd_candidate) * s->d.cap_per_window)) != cudaSuccess ||
             (e = cudaMalloc(&sl.d_sb_count, sizeof(uint64_t))) != cudaSuccess))
            return cuda_fail(e, "slot allocation");
    }
    s->sb_plans.assign(sb_plans, sb_plans + n_sb);
    return FDD_OK;
}

int fdd_server_destroy(fdd_server* s) {
    destroy_server(s);
    return FDD_OK;
}

int fdd_server_push(fdd_server* s, int32_t beam, int64_t seq, const uint8_t* host_chunk, double t_arrival) {
    if (!s || !host_chunk || beam < 0 || beam >= static_cast<int32_t>(s->beams.size()))
        return fail(FDD_ERR_INVALID_ARG, "bad push argument");
    ServeBeam& b = s->beams[beam];
    if (seq != b.next_seq)
        return fail(FDD_ERR_SEQUENCE, "chunk out of sequence (dropped, late, duplicate or reordered); "
                                      "fdd_server_reset_beam resynchronises the beam");
    if (b.deferred)
        return fail(FDD_ERR_BUSY, "beam backlogged: its previous window is still waiting for a search slot");
    cudaStream_t cs = s->copy_stream;
    cudaError_t e;
    const int64_t L = s->d.chunk_len;
    if (b.held == 0 && b.freed_valid[b.cur]) {
        // buf[cur] is refilled from scratch: wait until the last search reading it is done
        if ((e = cudaStreamWaitEvent(cs, b.freed[b.cur], 0)) != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
    }
    e = cudaMemcpy2DAsync(b.buf[b.cur] + b.held, s->pitch, host_chunk, L, L, s->rows, cudaMemcpyHostToDevice, cs);
    if (e != cudaSuccess) return cuda_fail(e, "chunk copy");
    b.held += L;
    b.next_seq++;
    if (b.held == s->buf_len) {
        // window complete: queue it, then carry its tail into the other buffer
        if ((e = cudaEventRecord(b.ready[b.cur], cs)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        ServeWindow w;
        w.beam = beam;
        w.window = b.window;
        w.buf = b.cur;
        w.t_arrival = t_arrival;
        w.t_ready = now_s();
        s->queue.push_back(w);
        s->max_queue = std::max<int64_t>(s->max_queue, static_cast<int64_t>(s->queue.size()));
        b.pending[b.cur] = true;
        b.window++;
        if (b.pending[1 - b.cur]) {
            b.deferred = true;  // the other buffer's window has not been launched yet
        } else {
            const int rc = tail_copy(s, b);
            if (rc != FDD_OK) return rc;
        }
    }
    return FDD_OK;
}

int fdd_server_reset_beam(fdd_server* s, int32_t beam, int64_t next_seq) {
    if (!s || beam < 0 || beam >= static_cast<int32_t>(s->beams.size()) || next_seq < 0)
        return fail(FDD_ERR_INVALID_ARG, "bad reset argument");
    ServeBeam& b = s->beams[beam];
    // Drop the partial window; windows already queued or running are kept.
    int k = b.cur;
    if (b.pending[k]) k = 1 - k;
    if (b.pending[k]) return fail(FDD_ERR_BUSY, "both buffers of the beam hold queued windows");
    b.cur = k;
    b.deferred = false;
    b.held = 0;
    b.next_seq = next_seq;
    b.window = next_seq;  // window index = index of its first chunk
    return FDD_OK;
}

int fdd_server_poll(fdd_server* s) {
    if (!s) return fail(FDD_ERR_INVALID_ARG, "null server");
    const double t = now_s();
    int rc = retire(s, t);
    if (rc != FDD_OK) return rc;
    return schedule(s, t);
}

int fdd_server_drain(fdd_server* s) {
    if (!s) return fail(FDD_ERR_INVALID_ARG, "null server");
    for (;;) {
        int rc = fdd_server_poll(s);
        if (rc != FDD_OK) return rc;
        if (s->queue.empty() && s->inflight.empty()) return FDD_OK;
        if (!s->inflight.empty()) {
            const cudaError_t e = cudaEventSynchronize(s->inflight.front().done);  // then re-poll all
            if (e != cudaSuccess) return cuda_fail(e, "server drain");
        }
    }
}

int fdd_server_results(fdd_server* s, fdd_window_result* out, int32_t max_results, fdd_candidate* cands,
                       int64_t cands_cap, int32_t* n_results, int64_t* n_cands) {
    if (!s || !n_results || (max_results > 0 && !out) || (cands_cap > 0 && !cands))
        return fail(FDD_ERR_INVALID_ARG, "bad results argument");
    int32_t n = 0;
    int64_t nc = 0;
    size_t used = 0;
    for (; used < s->results.size() && n < max_results; used++) {
        fdd_window_result r = s->results[used];
        if (nc + r.n_cands_kept > cands_cap && r.n_cands_kept > 0) break;
        if (r.n_cands_kept > 0)
            std::memcpy(cands + nc, s->result_cands.data() + r.cand_offset, sizeof(fdd_candidate) * r.n_cands_kept);
        r.cand_offset = nc;
        nc += r.n_cands_kept;
        out[n++] = r;
    }
    s->results.erase(s->results.begin(), s->results.begin() + used);
    if (s->results.empty()) {
        s->result_cands.clear();
    } else if (used > 0) {
        // compact: keep only the candidates of the results not handed out yet
        std::vector<fdd_candidate> rest;
        for (fdd_window_result& r : s->results) {
            const int64_t off = static_cast<int64_t>(rest.size());
            rest.insert(rest.end(), s->result_cands.begin() + r.cand_offset,
                        s->result_cands.begin() + r.cand_offset + r.n_cands_kept);
            r.cand_offset = off;
        }
        s->result_cands.swap(rest);
    }
    *n_results = n;
    if (n_cands) *n_cands = nc;
    return FDD_OK;
}

int fdd_server_info(const fdd_server* s, fdd_server_stats* st) {
    if (!s || !st) return fail(FDD_ERR_INVALID_ARG, "bad argument");
    st->n_slots = static_cast<int32_t>(s->slots.size());
    int busy = 0;
    for (const ServeSlot& sl : s->slots) busy += sl.busy ? 1 : 0;
    st->slots_busy = busy;
    st->queued = static_cast<int32_t>(s->queue.size());
    st->max_queued = s->max_queue;
    st->launched = s->n_launched;
    st->done = s->n_done;
    st->batches = s->n_batches;
    st->window_len = s->n_in;
    st->ring_bytes_per_beam = 2 * static_cast<int64_t>(s->rows) * s->pitch;
    st->slot_bytes = static_cast<int64_t>(s->ws_bytes + sizeof(fdd_candidate) * s->d.cap_per_window);
    return FDD_OK;
}

}  // extern "C"
