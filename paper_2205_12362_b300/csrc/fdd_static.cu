// fdd_static.cu -- fdd_search_static: the search with its scratch memory in a
// fixed, file-scope device array instead of a caller-allocated workspace.
//
// For callers that cannot allocate device memory when they search: a
// real-time thread that must not block in the allocator, a process whose GPU
// memory is handed out by an external arbiter after start-up, or code audited
// to allocate only at initialisation.  Those callers still own the input,
// candidate, counter and (optional) series buffers; only the workspace moves
// into the library.
#include <mutex>
#include <string>

#include "fdd_internal.cuh"

namespace {

// The scratch array.  Every GPU that loads this library's device code holds
// FDD_STATIC_SCRATCH_BYTES of it until the process exits.
__device__ __align__(256) uint8_t g_fdd_static_scratch[FDD_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 128;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};  // device address of the array, per device

thread_local std::string g_static_error;

}  // namespace

extern "C" int fdd_search_static(fdd_plan* plan, const uint8_t* d_tabs, int64_t n_in, int64_t pitch, int64_t n_out,
                                 int64_t t_offset_native, fdd_candidate* d_cands, int64_t cap, uint64_t* d_count,
                                 int32_t* d_series, fdd_stream_t stream) {
    if (!plan) return FDD_ERR_INVALID_ARG;
    if (fdd::plan_timing_enabled(plan)) {
        // stage timing creates CUDA events on first use: not allocation-free
        fdd::set_last_error("fdd_search_static: disable stage timing (fdd_plan_set_timing(plan, 0)) first");
        return FDD_ERR_INVALID_ARG;
    }
    size_t need = 0;
    int rc = fdd_workspace_size(plan, n_in, n_out, d_series == nullptr, &need);
    if (rc != FDD_OK) return rc;
    if (need > FDD_STATIC_SCRATCH_BYTES) {
        fdd::set_last_error("fdd_search_static: this search needs " + std::to_string(need) +
                            " bytes of scratch, more than the static array's " +
                            std::to_string(static_cast<size_t>(FDD_STATIC_SCRATCH_BYTES)) +
                            " (pass d_series, shorten the chunk, or use fdd_search with a workspace)");
        return FDD_ERR_WORKSPACE;
    }
    // One-time set-up per device, with that device current: resolve the
    // array's device address (the host-side symbol is only a stand-in).
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        fdd::set_last_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return FDD_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        fdd::set_last_error("fdd_search_static: device index beyond the supported range");
        return FDD_ERR_UNSUPPORTED;
    }
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_fdd_static_scratch);
            if (e != cudaSuccess) {
                fdd::set_last_error(std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
                return FDD_ERR_CUDA;
            }
            g_scratch_addr[dev] = p;
        }
        scratch = g_scratch_addr[dev];
    }
    // fdd_search zeroes the parts of the workspace that must start at zero
    // (series moments) on `stream` before its kernels run.
    return fdd_search(plan, d_tabs, n_in, pitch, n_out, t_offset_native, scratch, FDD_STATIC_SCRATCH_BYTES, d_cands,
                      cap, d_count, d_series, stream);
}
