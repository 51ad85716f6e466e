// fdd_static.cu -- fdd_search_static: the search with its scratch memory in a
// fixed, file-scope device array instead of a caller-allocated workspace.
//
// For callers that cannot allocate device memory when they search: a
// real-time thread that must not block in the allocator, a process whose GPU
// memory is handed out by an external arbiter after start-up, or code audited
// to allocate only at initialisation.  Those callers still own the input,
// candidate, counter and (optional) series buffers; only the workspace moves
// into the library.
#include <string>

#include "fdd_internal.cuh"

namespace {

// The scratch array.  The build links every .cu file as its own module and
// CUDA loads modules lazily, so the array is committed on a device when this
// file's module is first loaded there -- at the latest by the first
// fdd_search_static call on that device -- and held until the process exits.
__device__ __align__(256) uint8_t g_fdd_static_scratch[FDD_STATIC_SCRATCH_BYTES];

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
    if (n_in < 0 || n_out < 0) return FDD_ERR_INVALID_ARG;
    const size_t need = fdd::plain_workspace_bytes(plan, n_in, n_out, d_series == nullptr);
    if (need > FDD_STATIC_SCRATCH_BYTES) {
        fdd::set_last_error("fdd_search_static: this search needs " + std::to_string(need) +
                            " bytes of scratch, more than the static array's " +
                            std::to_string(static_cast<size_t>(FDD_STATIC_SCRATCH_BYTES)) +
                            " (pass d_series, shorten the chunk, or use fdd_search with a workspace)");
        return FDD_ERR_WORKSPACE;
    }
    // Resolve the array's device address with the calling device current
    // (the host-side symbol is only a stand-in).  It is resolved on every
    // call rather than cached: after a context is torn down and re-created
    // (cudaDeviceReset) the module is loaded afresh at another address.  The
    // first call on a device loads the module, which commits the array.
    void* scratch = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&scratch, g_fdd_static_scratch);
    if (e != cudaSuccess) {
        fdd::set_last_error(std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
        return FDD_ERR_CUDA;
    }
    // fdd_search zeroes the parts of the workspace that must start at zero
    // (series moments) on `stream` before its kernels run.
    return fdd_search(plan, d_tabs, n_in, pitch, n_out, t_offset_native, scratch, FDD_STATIC_SCRATCH_BYTES, d_cands,
                      cap, d_count, d_series, stream);
}
