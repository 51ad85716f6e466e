// fdd_stream.cu -- per-beam streaming search (fdd_stream_*): one compound
// beam's chunks are pushed from device memory as they arrive; the stream
// keeps the beam's delay overlap on the device and searches every window as
// soon as its last needed chunk is in.
//
// The paper's pipeline searches each 1.024 s chunk of a compound beam with
// the following max-delay of data appended (Sec. "AMBER"; Sec. "Computing
// performance").  Here window w searches the outputs of the beam whose first
// native sample lies in [w*L, (w+1)*L) (L = chunk length), from the samples
// that start at w*L, with every range's downsampling bins aligned to the
// beam's stream (fdd_search_window), so the windows tile one search of the
// whole stream.  Two device buffers of a whole number of chunks alternate: when the
// current one is full its window is searched, then its last buf_len - L
// samples are copied to the other buffer, which continues the stream.  All
// work of a push is enqueued on the caller's CUDA stream; an event recorded
// at the end of each push orders the next push after it even when the
// caller switches streams.
#include <algorithm>
#include <new>

#include "fdd_plan_impl.h"

using namespace fdd::host;

struct fdd_stream {
    fdd_plan* plan = nullptr;
    int32_t beam = 0;
    int64_t L = 0, n_in = 0, buf_len = 0, pitch = 0, rows = 0;
    uint8_t* buf[2] = {nullptr, nullptr};
    int cur = 0;
    int64_t held = 0, next_seq = 0, window = 0;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    fdd_candidate* d_cands = nullptr;
    uint64_t* d_count = nullptr;
    int64_t cap = 0;
    cudaEvent_t last = nullptr;
    bool last_valid = false;
    cudaStream_t last_stream = nullptr;
    int64_t result_t0 = -1;  // first output sample of the window searched last
    bool result_new = false;
};

namespace {

// Copy the first min(true count, src_cap, dst_cap) records of the stream's
// candidate buffer to the caller's and the true count to *dst_count.
__global__ void k_take_cands(const fdd_candidate* __restrict__ src, const uint64_t* __restrict__ src_count,
                             int64_t src_cap, fdd_candidate* __restrict__ dst, int64_t dst_cap,
                             uint64_t* __restrict__ dst_count) {
    const uint64_t n_true = *src_count;
    const uint64_t cap = static_cast<uint64_t>(src_cap < dst_cap ? src_cap : dst_cap);
    const int64_t n = static_cast<int64_t>(n_true < cap ? n_true : cap);
    const int64_t words = n * static_cast<int64_t>(sizeof(fdd_candidate) / sizeof(uint4));
    const uint4* s = reinterpret_cast<const uint4*>(src);
    uint4* d = reinterpret_cast<uint4*>(dst);
    for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < words;
         k += static_cast<int64_t>(gridDim.x) * blockDim.x)
        d[k] = s[k];
    if (blockIdx.x == 0 && threadIdx.x == 0) *dst_count = n_true;
}

void destroy_stream(fdd_stream* st) {
    if (!st) return;
    if (st->last_valid) cudaEventSynchronize(st->last);
    for (uint8_t* b : st->buf)
        if (b) cudaFree(b);
    if (st->ws) cudaFree(st->ws);
    if (st->d_cands) cudaFree(st->d_cands);
    if (st->d_count) cudaFree(st->d_count);
    if (st->last) cudaEventDestroy(st->last);
    delete st;
}

}  // namespace

extern "C" {

int fdd_stream_open(fdd_plan* plan, int32_t beam_id, int64_t chunk_len, int64_t cap, fdd_stream** out) {
    if (!plan || !out || chunk_len < 1 || cap < 1) return fail(FDD_ERR_INVALID_ARG, "bad stream argument");
    *out = nullptr;
    fdd_stream* st = new (std::nothrow) fdd_stream();
    if (!st) return fail(FDD_ERR_NO_MEMORY, "host allocation");
    st->plan = plan;
    st->beam = beam_id;
    st->L = chunk_len;
    st->cap = cap;
    st->rows = static_cast<int64_t>(plan->n_tab) * plan->n_chan;
    st->n_in = window_input_len(plan, chunk_len);
    st->buf_len = (st->n_in + chunk_len - 1) / chunk_len * chunk_len;
    st->pitch = static_cast<int64_t>(align_up(static_cast<size_t>(st->buf_len), 16));
    st->ws_bytes = make_layout(plan, st->n_in, chunk_len, true, true, 1).total;  // plain window searches
    const size_t buf_bytes = static_cast<size_t>(st->rows) * st->pitch;
    cudaError_t e;
    for (uint8_t*& b : st->buf)
        if ((e = cudaMalloc(&b, buf_bytes)) != cudaSuccess) {
            destroy_stream(st);
            return cuda_fail(e, "cudaMalloc(stream buffer)");
        }
    if ((e = cudaMalloc(&st->ws, st->ws_bytes)) != cudaSuccess ||
        (e = cudaMalloc(&st->d_cands, sizeof(fdd_candidate) * cap)) != cudaSuccess ||
        (e = cudaMalloc(&st->d_count, sizeof(uint64_t))) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&st->last, cudaEventDisableTiming)) != cudaSuccess) {
        destroy_stream(st);
        return cuda_fail(e, "stream allocation");
    }
    *out = st;
    return FDD_OK;
}

int fdd_stream_push(fdd_stream* st, const uint8_t* d_chunk, int64_t chunk_pitch, int64_t seq, fdd_stream_t stream) {
    if (!st || !d_chunk || chunk_pitch < st->L) return fail(FDD_ERR_INVALID_ARG, "bad push argument");
    if (seq != st->next_seq)
        return fail(FDD_ERR_SEQUENCE, "beam " + std::to_string(st->beam) + ": chunk " + std::to_string(seq) +
                                          " pushed, chunk " + std::to_string(st->next_seq) + " expected");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (st->last_valid && st->last_stream != s && (e = cudaStreamWaitEvent(s, st->last, 0)) != cudaSuccess)
        return cuda_fail(e, "cudaStreamWaitEvent");
    e = cudaMemcpy2DAsync(st->buf[st->cur] + st->held, st->pitch, d_chunk, chunk_pitch, st->L, st->rows,
                          cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "chunk copy");
    st->held += st->L;
    st->next_seq++;
    if (st->held == st->buf_len) {
        const int rc = search_impl(st->plan, st->buf[st->cur], st->n_in, st->pitch, st->L, st->window * st->L, true,
                                   st->ws, st->ws_bytes, st->d_cands, st->cap, st->d_count, nullptr, s);
        if (rc != FDD_OK) return rc;
        st->result_t0 = st->window * st->L;
        st->result_new = true;
        st->window++;
        const int dst = 1 - st->cur;
        e = cudaMemcpy2DAsync(st->buf[dst], st->pitch, st->buf[st->cur] + st->L, st->pitch, st->buf_len - st->L,
                              st->rows, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "window tail copy");
        st->cur = dst;
        st->held = st->buf_len - st->L;
    }
    if ((e = cudaEventRecord(st->last, s)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    st->last_valid = true;
    st->last_stream = s;
    return FDD_OK;
}

int fdd_stream_results(fdd_stream* st, fdd_candidate* d_cands, int64_t cap, uint64_t* d_count, int64_t* t0_native) {
    if (!st || !t0_native || !d_count || cap < 0 || (cap > 0 && !d_cands))
        return fail(FDD_ERR_INVALID_ARG, "bad results argument");
    if (!st->result_new) {
        *t0_native = -1;
        return FDD_OK;
    }
    k_take_cands<<<148, 256, 0, st->last_stream>>>(st->d_cands, st->d_count, st->cap, d_cands, cap, d_count);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_take_cands");
    *t0_native = st->result_t0;
    st->result_new = false;
    return FDD_OK;
}

int fdd_stream_close(fdd_stream* st) {
    destroy_stream(st);
    return FDD_OK;
}

int fdd_copy_rows(void* dst, int64_t dst_pitch, const void* src, int64_t src_pitch, int64_t width, int64_t rows,
                  fdd_stream_t stream) {
    if (!dst || !src || width < 0 || rows < 0 || dst_pitch < width || src_pitch < width)
        return fail(FDD_ERR_INVALID_ARG, "bad row copy");
    if (width == 0 || rows == 0) return FDD_OK;
    const cudaError_t e = cudaMemcpy2DAsync(dst, static_cast<size_t>(dst_pitch), src, static_cast<size_t>(src_pitch),
                                            static_cast<size_t>(width), static_cast<size_t>(rows), cudaMemcpyDefault,
                                            reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? FDD_OK : cuda_fail(e, "row copy");
}

}  // extern "C"
