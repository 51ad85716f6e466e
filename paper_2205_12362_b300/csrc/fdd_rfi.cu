// fdd_rfi.cu -- RFI mitigation on the TAB filterbanks, in place (Sec.
// "AMBER", "RFI mitigation (optional)": a time-domain filter for bright
// wide-band low-DM RFI and a frequency-domain filter for bright narrowband
// RFI, each iterated -- three times each in ARTS, Sec. "Fraction of data lost
// to RFI" -- on ever cleaner samples).  The paper leaves the statistics to
// another publication; this library's reading, per TAB:
//   time domain: zero-DM series z[t] = sum_c x[c][t]; each iteration takes
//     mu, sigma of z over unflagged samples and flags z[t] - mu > thr_t sigma;
//     flagged samples of every channel become the channel's mean over the
//     unflagged samples (rounded half up);
//   frequency domain, on the time-cleaned data: channel sums b[c]; each
//     iteration flags |b[c] - mu| > thr_f sigma over unflagged channels;
//     flagged channels are filled with the mean level of the others.
// Moments are exact 64-bit sums; mu = S1/n, var = S2/n - mu^2, sigma =
// sqrt(var) in FP64 with explicit round-to-nearest operations, so every flag
// decision is the same FP64 computation a CPU performs.
//
// Kernels: k_rfi_zdm (zero-DM series, 4 samples per thread), k_rfi_flag (one
// block per TAB, the iterations), k_rfi_time_fix (per channel: masked sum,
// replacement, cleaned channel sum), k_rfi_chan_fix (fills flagged channels).
#include "fdd_plan_impl.h"

using namespace fdd::host;

namespace {

constexpr int kFlagThreads = 1024;

__global__ void k_rfi_zdm(const uint8_t* __restrict__ x, int32_t n_chan, int64_t n_in, int64_t pitch,
                          uint32_t* __restrict__ z) {
    const int tab = blockIdx.y;
    const int64_t t = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) * 4;
    if (t >= n_in) return;
    const uint8_t* rows = x + static_cast<int64_t>(tab) * n_chan * pitch;
    uint32_t s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    for (int c = 0; c < n_chan; c++) {
        const uint32_t w = __ldg(reinterpret_cast<const uint32_t*>(rows + c * pitch + t));  // t + 3 < pitch
        s0 += w & 0xFFu;
        s1 += (w >> 8) & 0xFFu;
        s2 += (w >> 16) & 0xFFu;
        s3 += w >> 24;
    }
    uint32_t* zt = z + static_cast<int64_t>(tab) * n_in + t;
    zt[0] = s0;
    if (t + 1 < n_in) zt[1] = s1;
    if (t + 2 < n_in) zt[2] = s2;
    if (t + 3 < n_in) zt[3] = s3;
}

// FP64 moments of the unflagged values (same operations as a CPU's IEEE
// double arithmetic, no contraction).
__device__ void flag_moments(uint64_t s1, uint64_t s2, uint64_t k, double* mu, double* sigma) {
    *mu = __ddiv_rn(__ull2double_rn(s1), __ull2double_rn(k));
    const double m2 = __ddiv_rn(__ull2double_rn(s2), __ull2double_rn(k));
    const double var = __dsub_rn(m2, __dmul_rn(*mu, *mu));
    *sigma = var > 0.0 ? __dsqrt_rn(var) : 0.0;
}

// One block per TAB: `iters` rounds of flagging values v[j] (j < n) whose
// deviation exceeds thr * sigma (one-sided: v - mu; two-sided: |v - mu|).
// Values are uint32 (zero-DM series) or uint64 (channel sums).
template <typename V, bool TWO_SIDED>
__global__ void __launch_bounds__(kFlagThreads) k_rfi_flag(const V* __restrict__ vals, int64_t n, double thr, int iters,
                                                           uint8_t* __restrict__ flags, unsigned long long* __restrict__ ok) {
    const int tab = blockIdx.x;
    const V* v = vals + static_cast<int64_t>(tab) * n;
    uint8_t* fl = flags + static_cast<int64_t>(tab) * n;
    __shared__ unsigned long long s_s1[kFlagThreads / 32], s_s2[kFlagThreads / 32], s_k[kFlagThreads / 32];
    __shared__ double s_mu, s_sigma;
    __shared__ int s_stop;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t j = threadIdx.x; j < n; j += kFlagThreads) fl[j] = 0;
    __syncthreads();
    for (int it = 0; it <= iters; it++) {
        unsigned long long s1 = 0, s2 = 0, k = 0;
        for (int64_t j = threadIdx.x; j < n; j += kFlagThreads)
            if (!fl[j]) {
                const unsigned long long x = v[j];
                s1 += x;
                s2 += x * x;
                k++;
            }
        for (int o = 16; o > 0; o >>= 1) {
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            k += __shfl_xor_sync(0xffffffffu, k, o);
        }
        if (lane == 0) {
            s_s1[warp] = s1;
            s_s2[warp] = s2;
            s_k[warp] = k;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long a1 = 0, a2 = 0, ak = 0;
            for (int w = 0; w < kFlagThreads / 32; w++) {
                a1 += s_s1[w];
                a2 += s_s2[w];
                ak += s_k[w];
            }
            s_stop = (ak == 0) || (it == iters);
            if (ak > 0) flag_moments(a1, a2, ak, &s_mu, &s_sigma);
            if (s_stop) ok[tab] = ak;  // unflagged count after the last round
        }
        __syncthreads();
        if (s_stop) break;
        const double mu = s_mu, lim = __dmul_rn(thr, s_sigma);
        for (int64_t j = threadIdx.x; j < n; j += kFlagThreads) {
            if (fl[j]) continue;
            const double d = __dsub_rn(__ull2double_rn(static_cast<unsigned long long>(v[j])), mu);
            if ((TWO_SIDED ? fabs(d) : d) > lim) fl[j] = 1;
        }
        __syncthreads();
    }
}

// Per (channel, TAB): sum over the unflagged samples, replace the flagged ones
// by the rounded mean, and leave the cleaned channel sum in b.
__global__ void k_rfi_time_fix(uint8_t* __restrict__ x, int32_t n_chan, int64_t n_in, int64_t pitch,
                               const uint8_t* __restrict__ tflags, const unsigned long long* __restrict__ ok,
                               unsigned long long* __restrict__ b) {
    const int c = blockIdx.x, tab = blockIdx.y;
    uint8_t* row = x + (static_cast<int64_t>(tab) * n_chan + c) * pitch;
    const uint8_t* fl = tflags ? tflags + static_cast<int64_t>(tab) * n_in : nullptr;
    __shared__ unsigned long long s_part[8];
    __shared__ unsigned long long s_all[8];
    unsigned long long s = 0, all = 0;
    for (int64_t t = threadIdx.x; t < n_in; t += blockDim.x) {
        const unsigned v = row[t];
        all += v;
        if (!fl || !fl[t]) s += v;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        all += __shfl_xor_sync(0xffffffffu, all, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s_part[threadIdx.x >> 5] = s;
        s_all[threadIdx.x >> 5] = all;
    }
    __syncthreads();
    unsigned long long tot = 0, tot_all = 0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); w++) {
        tot += s_part[w];
        tot_all += s_all[w];
    }
    const unsigned long long n_ok = fl ? ok[tab] : static_cast<unsigned long long>(n_in);
    const bool replace = fl && n_ok > 0 && n_ok < static_cast<unsigned long long>(n_in);
    unsigned long long cleaned = tot_all;
    if (replace) {
        const unsigned long long m = (2 * tot + n_ok) / (2 * n_ok);
        for (int64_t t = threadIdx.x; t < n_in; t += blockDim.x)
            if (fl[t]) row[t] = static_cast<uint8_t>(m);
        cleaned = tot + (static_cast<unsigned long long>(n_in) - n_ok) * m;
    }
    if (threadIdx.x == 0) b[static_cast<int64_t>(tab) * n_chan + c] = cleaned;
}

// Fill flagged channels with the rounded mean level of the unflagged ones.
__global__ void k_rfi_chan_fix(uint8_t* __restrict__ x, int32_t n_chan, int64_t n_in, int64_t pitch,
                               const uint8_t* __restrict__ cflags, const unsigned long long* __restrict__ b,
                               const unsigned long long* __restrict__ ok) {
    const int c = blockIdx.x, tab = blockIdx.y;
    const unsigned long long n_ok = ok[tab];
    if (!cflags[static_cast<int64_t>(tab) * n_chan + c] || n_ok == 0 || n_ok >= static_cast<unsigned long long>(n_chan))
        return;
    __shared__ unsigned long long s_level;
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int k = 0; k < n_chan; k++)
            if (!cflags[static_cast<int64_t>(tab) * n_chan + k]) s += b[static_cast<int64_t>(tab) * n_chan + k];
        const unsigned long long den = n_ok * static_cast<unsigned long long>(n_in);
        s_level = (2 * s + den) / (2 * den);
    }
    __syncthreads();
    uint8_t* row = x + (static_cast<int64_t>(tab) * n_chan + c) * pitch;
    for (int64_t t = threadIdx.x; t < n_in; t += blockDim.x) row[t] = static_cast<uint8_t>(s_level);
}

struct RfiLayout {
    size_t z = 0, b = 0, tf = 0, cf = 0, ok_t = 0, ok_c = 0, total = 0;
};

RfiLayout rfi_layout(int32_t n_tab, int32_t n_chan, int64_t n_in) {
    RfiLayout L;
    size_t cur = 0;
    auto take = [&](size_t bytes) {
        const size_t at = cur;
        cur = align_up(cur + bytes, 256);
        return at;
    };
    L.z = take(sizeof(uint32_t) * n_tab * static_cast<size_t>(n_in));
    L.b = take(sizeof(unsigned long long) * n_tab * static_cast<size_t>(n_chan));
    L.tf = take(static_cast<size_t>(n_tab) * n_in);
    L.cf = take(static_cast<size_t>(n_tab) * n_chan);
    L.ok_t = take(sizeof(unsigned long long) * n_tab);
    L.ok_c = take(sizeof(unsigned long long) * n_tab);
    L.total = cur;
    return L;
}

}  // namespace

extern "C" {

int fdd_rfi_workspace_size(int32_t n_tab, int32_t n_chan, int64_t n_in, size_t* bytes) {
    if (!bytes || n_tab < 1 || n_chan < 1 || n_in < 0) return fail(FDD_ERR_INVALID_ARG, "bad argument");
    *bytes = rfi_layout(n_tab, n_chan, n_in).total;
    return FDD_OK;
}

int fdd_rfi_clean(const fdd_rfi_desc* desc, uint8_t* d_tabs, int32_t n_tab, int32_t n_chan, int64_t n_in,
                  int64_t pitch, void* d_workspace, size_t workspace_bytes, uint8_t* d_time_flags,
                  uint8_t* d_chan_flags, fdd_stream_t stream) {
    if (!desc || !d_tabs || !d_workspace || n_tab < 1 || n_chan < 1 || n_chan > FDD_MAX_CHANNELS || n_in < 1 ||
        pitch < n_in || desc->time_iters < 0 || desc->freq_iters < 0)
        return fail(FDD_ERR_INVALID_ARG, "bad RFI argument");
    if ((reinterpret_cast<uintptr_t>(d_tabs) & 15) || (pitch & 15) || (reinterpret_cast<uintptr_t>(d_workspace) & 255))
        return fail(FDD_ERR_MISALIGNED, "d_tabs/pitch must be 16-byte aligned, workspace 256-byte aligned");
    const RfiLayout L = rfi_layout(n_tab, n_chan, n_in);
    if (workspace_bytes < L.total) return fail(FDD_ERR_WORKSPACE, "workspace smaller than fdd_rfi_workspace_size()");
    // exact 64-bit second moments: n * max^2 below 2^64
    const double zmax = 255.0 * n_chan, bmax = 255.0 * static_cast<double>(n_in);
    if (static_cast<double>(n_in) * zmax * zmax >= 1.8e19 || static_cast<double>(n_chan) * bmax * bmax >= 1.8e19)
        return fail(FDD_ERR_UNSUPPORTED, "chunk too long for exact 64-bit RFI moments");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    uint8_t* ws = static_cast<uint8_t*>(d_workspace);
    uint32_t* z = reinterpret_cast<uint32_t*>(ws + L.z);
    auto* b = reinterpret_cast<unsigned long long*>(ws + L.b);
    uint8_t* tf = d_time_flags ? d_time_flags : ws + L.tf;
    uint8_t* cf = d_chan_flags ? d_chan_flags : ws + L.cf;
    auto* ok_t = reinterpret_cast<unsigned long long*>(ws + L.ok_t);
    auto* ok_c = reinterpret_cast<unsigned long long*>(ws + L.ok_c);
    cudaError_t e;
    const bool time_on = desc->time_thresh > 0, freq_on = desc->freq_thresh > 0;
    if ((e = cudaMemsetAsync(tf, 0, static_cast<size_t>(n_tab) * n_in, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(cf, 0, static_cast<size_t>(n_tab) * n_chan, s)) != cudaSuccess)
        return cuda_fail(e, "cudaMemsetAsync(RFI flags)");
    if (time_on) {
        const unsigned gx = static_cast<unsigned>((n_in + 4 * 256 - 1) / (4 * 256));
        k_rfi_zdm<<<dim3(gx, n_tab), 256, 0, s>>>(d_tabs, n_chan, n_in, pitch, z);
        k_rfi_flag<uint32_t, false><<<n_tab, kFlagThreads, 0, s>>>(z, n_in, desc->time_thresh, desc->time_iters, tf, ok_t);
    }
    k_rfi_time_fix<<<dim3(n_chan, n_tab), 256, 0, s>>>(d_tabs, n_chan, n_in, pitch, time_on ? tf : nullptr, ok_t, b);
    if (freq_on) {
        k_rfi_flag<unsigned long long, true><<<n_tab, kFlagThreads, 0, s>>>(b, n_chan, desc->freq_thresh,
                                                                            desc->freq_iters, cf, ok_c);
        k_rfi_chan_fix<<<dim3(n_chan, n_tab), 256, 0, s>>>(d_tabs, n_chan, n_in, pitch, cf, b, ok_c);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "RFI launch");
    return FDD_OK;
}

}  // extern "C"
