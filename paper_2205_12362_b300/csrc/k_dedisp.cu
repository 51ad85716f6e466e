// k_dedisp.cu -- per-range dedispersion launches: one grid per DM range,
// (time tiles x DM blocks x SBs), each block running one dedisp_tile (see
// dedisp_tile.cuh for the algorithm), and the table of compiled variants.
#include <mutex>

#include "dedisp_tile.cuh"

namespace fdd {

namespace {

template <int E, int NW, int DPW, int WARPS, int MAXIT>
__global__ void __launch_bounds__(WARPS * 32) k_dedisp(const DedispArgs a) {
    detail::dedisp_tile<E, NW, DPW, WARPS, MAXIT>(a, blockIdx.x, blockIdx.y, blockIdx.z);
}

using KernelFn = void (*)(const DedispArgs);

struct Entry {
    DedispVariant v;
    KernelFn fn;
};

#define FDD_V(E, NW, DPW, WARPS, MAXIT) {{E, NW, DPW, WARPS, MAXIT}, k_dedisp<E, NW, DPW, WARPS, MAXIT>}
const Entry kEntries[] = {
    // uint8 input (native-rate ranges)
    FDD_V(1, 4, 2, 8, 4),    // BD 16, T 512, 256 threads
    FDD_V(1, 4, 2, 16, 4),   // BD 32, T 512, 512 threads
    FDD_V(1, 4, 4, 8, 4),    // BD 32, T 512, 256 threads
    FDD_V(1, 2, 4, 8, 4),    // BD 32, T 256, 256 threads
    FDD_V(1, 2, 2, 16, 4),   // BD 32, T 256, 512 threads
    FDD_V(1, 4, 1, 16, 4),   // BD 16, T 512, 512 threads
    FDD_V(1, 2, 4, 16, 4),   // BD 64, T 256, 512 threads
    FDD_V(1, 1, 4, 16, 4),   // BD 64, T 128, 512 threads
    // uint16 input (downsampled ranges)
    FDD_V(2, 4, 2, 8, 4),    // BD 16, T 256
    FDD_V(2, 4, 2, 16, 4),   // BD 32, T 256
    FDD_V(2, 4, 4, 8, 4),    // BD 32, T 256
    FDD_V(2, 8, 2, 8, 4),    // BD 16, T 512
    FDD_V(2, 2, 4, 16, 4),   // BD 64, T 128
};
#undef FDD_V

}  // namespace

int num_dedisp_variants() { return static_cast<int>(sizeof(kEntries) / sizeof(kEntries[0])); }

const DedispVariant& dedisp_variant(int idx) { return kEntries[idx].v; }

size_t dedisp_smem_bytes(const DedispVariant& v, int Lw, int CC) {
    return static_cast<size_t>(CC) * (4 / v.E) * Lw * 4 + static_cast<size_t>(CC) * v.bd() * 4;
}

bool dedisp_cc_ok(const DedispVariant& v, int Lw, int CC, size_t smem_budget) {
    if (CC < 1 || CC > 256) return false;
    if (static_cast<int64_t>(CC) * (Lw / 4) > static_cast<int64_t>(v.MAXIT) * v.threads()) return false;
    if (CC * (v.bd() / 4) > v.threads()) return false;
    return dedisp_smem_bytes(v, Lw, CC) <= smem_budget;
}

cudaError_t allow_dynamic_smem(const void* fn, size_t smem) {
    static std::mutex mu;  // read and raise as one step when several host threads launch
    std::lock_guard<std::mutex> lock(mu);
    cudaFuncAttributes fa;
    cudaError_t err = cudaFuncGetAttributes(&fa, fn);
    if (err != cudaSuccess) return err;
    if (smem <= static_cast<size_t>(fa.maxDynamicSharedSizeBytes)) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
}

cudaError_t launch_dedisp(int variant, const DedispArgs& a, cudaStream_t s) {
    const Entry& e = kEntries[variant];
    const size_t smem = dedisp_smem_bytes(e.v, a.Lw, a.CC);
    cudaError_t err = allow_dynamic_smem(reinterpret_cast<const void*>(e.fn), smem);
    if (err != cudaSuccess) return err;
    const int T = e.v.tile(), BD = e.v.bd();
    dim3 grid((a.n_out + T - 1) / T, (a.n_dm + BD - 1) / BD, a.n_sb);
    e.fn<<<grid, e.v.threads(), smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace fdd
