// k_sbf.cu -- SB-factored dedispersion kernels.
//
// Every SB of a compound beam takes, channel by channel, the data of one of
// the TABs (Sec. "Hierarchical beam forming"); on a segment of channels where
// every SB keeps one TAB, the SB's dedispersed sum over the segment is the
// same number as that TAB's sum over the segment.  So, with segments u,
//     S[s][i][t] = sum_u P[tab(s, u)][u][i][t],
//     P[k][u][i][t] = sum_{c in u} X[k][c][t + d[i][c]],
// exactly (integer sums regrouped).  Per (trial, sample) brute force needs
// n_sb * n_chan channel-adds; this needs n_tab * n_chan for P plus n_sb * n_seg
// for S -- for 12 TABs, 71 SBs and 16-channel segments about 4.3x fewer.
//
// k_sbf_part computes P for a slab of DM trials: the brute-force block tile
// of dedisp_tile.cuh (staged byte-shifted rows, SWAR adds), run per TAB with
// channel stages made of whole segments, storing each segment's 16-bit sums
// instead of summing all channels.  k_sbf_comb reads P (L1/L2-resident
// rows, 4 samples per lane) and adds, for each SB, the rows its TABs select,
// in 16-bit lanes folded into int32 every `flush` segments, then writes the
// series and its moments like the brute-force epilogue.
#include "sbf_part.cuh"
#include "tma.cuh"

namespace fdd {

namespace {

template <int E, int NW, int DPW, int WARPS, int MAXIT>
__global__ void __launch_bounds__(WARPS * 32) k_sbf_part(const SbfPartArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    detail::sbf_part_tile<E, NW, DPW, WARPS, MAXIT>(a, blockIdx.x, blockIdx.y, blockIdx.z, smem);
}

// Comb: block = CW warps x CSB SBs per warp, one DM trial, CT = 128 samples
// (4 per lane).  The partial rows of every TAB for UC segments at a time are
// one tile of P -- CT samples x UC segments x n_tab TABs -- which thread 0
// requests with a single TMA tensor copy (cp.async.bulk.tensor) into shared
// memory, double-buffered and completed on an mbarrier; each row is read from
// L2/HBM once per block and then serves every SB that selects it.  Segments
// past n_seg fall outside the tensor and arrive as zeros.  A warp whose SBs
// run past n_sb repeats its last valid SB (results discarded), so the inner
// loop has no per-SB branches.
constexpr int CW = 12, CSB = 6, CT = 128, UC = 8;
constexpr int kRowBytes = CT * 2;            // one partial row in shared memory
constexpr int kTabBytes = UC * kRowBytes;    // UC rows of one TAB
static_assert(kTabBytes == 1 << 11, "the TAB offset is formed as tab << 11");
constexpr int kSmemAlign = 128;              // TMA destination alignment

__device__ __forceinline__ uint2 lds64(uint32_t addr) {
    uint2 v;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(addr));
    return v;
}
__global__ void __launch_bounds__(CW * 32, 2) k_sbf_comb(const __grid_constant__ SbfCombArgs a) {
    extern __shared__ __align__(16) uint8_t smem_raw[];  // [2][n_tab][UC][CT] uint16, then 2 mbarriers
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i_s = blockIdx.y;
    const int i = a.i0 + i_s;
    const int t0 = blockIdx.x * CT;
    const int sb0 = blockIdx.z * (CW * CSB) + warp * CSB;
    const int nsb = max(0, min(CSB, a.n_sb - sb0));  // warp-uniform
    const int n_chunks = (a.n_seg + UC - 1) / UC;
    const uint32_t s_raw = static_cast<uint32_t>(__cvta_generic_to_shared(smem_raw));
    const uint32_t s_base = (s_raw + (kSmemAlign - 1)) & ~static_cast<uint32_t>(kSmemAlign - 1);
    const uint32_t buf_bytes = static_cast<uint32_t>(a.n_tab) * kTabBytes;
    const uint32_t s_bar = s_base + 2u * buf_bytes;  // two 8-byte mbarriers
    // the SBs of this warp (invalid slots repeat SB sb0 + nsb - 1, or SB 0 for an idle warp)
    const uint8_t* tab_row[CSB];
#pragma unroll
    for (int j = 0; j < CSB; j++) {
        const int sj = nsb > 0 ? sb0 + min(j, nsb - 1) : 0;
        tab_row[j] = a.seg_tab + static_cast<int64_t>(sj) * a.seg_pitch;
    }

    // chunk ch (UC segments of every TAB) into buffer ch & 1: one tensor copy by thread 0
    auto issue = [&](int ch) {
        const uint32_t bar = s_bar + 8u * (ch & 1);
        tma::mbar_expect_tx(bar, buf_bytes);
        tma::load_4d(s_base + (ch & 1) * buf_bytes, &a.tmap, t0, i_s, ch * UC, 0, bar);
    };
    if (threadIdx.x == 0) {
        tma::mbar_init(s_bar, 1);
        tma::mbar_init(s_bar + 8u, 1);
        tma::mbar_init_fence();
    }
    __syncthreads();

    uint32_t acc[CSB][2], tot[CSB][4];
#pragma unroll
    for (int j = 0; j < CSB; j++) {
        acc[j][0] = acc[j][1] = 0u;
        tot[j][0] = tot[j][1] = tot[j][2] = tot[j][3] = 0u;
    }
    auto fold = [&]() {
#pragma unroll
        for (int j = 0; j < CSB; j++) {
            tot[j][0] += acc[j][0] & 0xFFFFu;
            tot[j][1] += acc[j][0] >> 16;
            tot[j][2] += acc[j][1] & 0xFFFFu;
            tot[j][3] += acc[j][1] >> 16;
            acc[j][0] = acc[j][1] = 0u;
        }
    };

    if (threadIdx.x == 0) issue(0);
    int since = 0;
    for (int ch = 0; ch < n_chunks; ch++) {
        const int buf = ch & 1;
        if (threadIdx.x == 0 && ch + 1 < n_chunks) issue(ch + 1);  // buffer buf ^ 1 was released below
        const bool ok = tma::mbar_wait_bounded(s_bar + 8u * buf, static_cast<uint32_t>(ch >> 1) & 1u);
        if (__syncthreads_or(!ok)) {
            // a copy did not land: flag it, let thread 0 wait (bounded) for this block's copies, stop
            if (threadIdx.x == 0) {
                atomicOr(a.status, 1u);
                tma::mbar_wait_bounded(s_bar + 8u * buf, static_cast<uint32_t>(ch >> 1) & 1u);
                if (ch + 1 < n_chunks) tma::mbar_wait_bounded(s_bar + 8u * (buf ^ 1), static_cast<uint32_t>((ch + 1) >> 1) & 1u);
            }
            return;
        }
        const int u0 = ch * UC;
        const int nu = min(UC, a.n_seg - u0);
        const uint32_t s_buf = s_base + buf * buf_bytes + 8u * lane;
        // segment du of the chunk for every SB of the warp: the TAB (byte dq of tabs4; PRMT zero-fills
        // the rest) times kTabBytes (2^11) picks the row
        auto add_segment = [&](const uint32_t (&tabs4)[CSB], int dq, int du) {
#pragma unroll
            for (int j = 0; j < CSB; j++) {
                const uint32_t tab = __byte_perm(tabs4[j], 0u, 0x4440u + dq);
                const uint2 v = lds64(s_buf + (tab << 11) + du * kRowBytes);
                acc[j][0] += v.x;
                acc[j][1] += v.y;
            }
        };
        if (nu == UC && a.flush % UC == 0) {  // block-uniform: a whole chunk, folds only at its end
#pragma unroll
            for (int q = 0; q < UC; q += 4) {
                uint32_t tabs4[CSB];
#pragma unroll
                for (int j = 0; j < CSB; j++) tabs4[j] = __ldg(reinterpret_cast<const uint32_t*>(tab_row[j] + u0 + q));
#pragma unroll
                for (int dq = 0; dq < 4; dq++) add_segment(tabs4, dq, q + dq);
            }
            since += UC;
            if (since == a.flush) {
                fold();
                since = 0;
            }
        } else {
#pragma unroll
            for (int q = 0; q < UC; q += 4) {
                uint32_t tabs4[CSB];
#pragma unroll
                for (int j = 0; j < CSB; j++) tabs4[j] = __ldg(reinterpret_cast<const uint32_t*>(tab_row[j] + u0 + q));
#pragma unroll
                for (int dq = 0; dq < 4; dq++) {
                    const int du = q + dq;
                    if (du < nu) {  // block-uniform
                        add_segment(tabs4, dq, du);
                        if (++since == a.flush) {
                            fold();
                            since = 0;
                        }
                    }
                }
            }
        }
        __syncthreads();  // buffer free for the copy issued next iteration
    }
    fold();
    const int t = t0 + 4 * lane;
#pragma unroll
    for (int j = 0; j < CSB; j++) {
        unsigned long long s1 = 0, s2 = 0;
        if (j < nsb) {
            int32_t* row = a.series + (static_cast<int64_t>(sb0 + j) * a.n_dm + i) * a.n_out;
#pragma unroll
            for (int e = 0; e < 4; e++) {
                if (t + e < a.n_emit) {
                    const uint32_t v = tot[j][e];
                    row[t + e] = static_cast<int32_t>(v);
                    s1 += v;
                    s2 += static_cast<unsigned long long>(v) * v;
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        if (lane == 0 && j < nsb) {
            const int64_t qq = static_cast<int64_t>(sb0 + j) * a.n_dm + i;
            atomicAdd(a.stat + 2 * qq, s1);
            atomicAdd(a.stat + 2 * qq + 1, s2);
        }
    }
}

using PartFn = void (*)(const SbfPartArgs);

struct Entry {
    DedispVariant v;
    PartFn fn;
    int fact;  // >= 0: the partial sums come from this pattern-factored variant in part mode
};

#define FDD_S(E, NW, DPW, WARPS, MAXIT) {{E, NW, DPW, WARPS, MAXIT}, k_sbf_part<E, NW, DPW, WARPS, MAXIT>, -1}
// pattern-factored part: tile 64 * NWF samples = 128 * (NWF / 2) of a DedispVariant with E = 1,
// = 64 * NWF of one with E = 2
#define FDD_SF(NWF, DPW, WARPS, FV) {{1, (NWF) / 2, DPW, WARPS, 0}, nullptr, FV}
#define FDD_SF2(NWF, DPW, WARPS, FV) {{2, NWF, DPW, WARPS, 0}, nullptr, FV}
const Entry kEntries[] = {
    FDD_S(1, 4, 2, 8, 4),   // BD 16, T 512
    FDD_S(1, 4, 4, 8, 4),   // BD 32, T 512
    FDD_S(1, 2, 4, 8, 4),   // BD 32, T 256
    FDD_S(1, 4, 2, 16, 4),  // BD 32, T 512, 512 threads
    FDD_S(1, 4, 2, 8, 8),   // BD 16, T 512, stages of up to 48-60 channels
    FDD_S(2, 4, 2, 8, 4),   // BD 16, T 256
    FDD_S(2, 4, 4, 8, 4),   // BD 32, T 256
    FDD_S(2, 8, 2, 8, 4),   // BD 16, T 512
    FDD_S(2, 2, 2, 8, 4),   // BD 16, T 128: short rows, stages of up to 48 channels
    FDD_S(2, 4, 2, 16, 4),  // BD 32, T 256, 512 threads: stages of up to 48 channels
    FDD_SF(4, 4, 16, 2),    // pattern-factored part, G 4, BD 64, T 256
    FDD_SF(4, 4, 16, 0),    // pattern-factored part, G 8, BD 64, T 256
    FDD_SF(4, 4, 8, 7),     // pattern-factored part, G 4, BD 32, T 256, 256 threads
    FDD_SF2(4, 4, 16, 2),   // pattern-factored part of 16-bit (downsampled) rows, G 4, BD 64, T 256
    FDD_SF2(4, 4, 16, 0),   // the same with G 8
    FDD_SF2(4, 4, 8, 7),    // the same, G 4, BD 32, 256 threads
    FDD_SF(4, 4, 8, 9),     // pattern-factored part with two pattern-row buffers (one barrier per
    FDD_SF2(4, 4, 8, 9),    // stage), G 4, BD 32, 256 threads: 8-bit and 16-bit rows
};
#undef FDD_S
#undef FDD_SF
#undef FDD_SF2

}  // namespace

int num_sbf_variants() { return static_cast<int>(sizeof(kEntries) / sizeof(kEntries[0])); }

const DedispVariant& sbf_variant(int idx) { return kEntries[idx].v; }

int sbf_fact_variant(int idx) { return kEntries[idx].fact; }

size_t sbf_smem_bytes(const DedispVariant& v, int Lw, int CC) {
    return static_cast<size_t>(CC) * (4 / v.E) * Lw * 4 + static_cast<size_t>(CC) * v.bd() * 4;
}

bool sbf_cc_ok(const DedispVariant& v, int Lw, int CC, size_t smem_budget) {
    if (CC < 1 || CC > 256) return false;
    if (static_cast<int64_t>(CC) * (Lw / 4) > static_cast<int64_t>(v.MAXIT) * v.threads()) return false;
    if (CC * (v.bd() / 4) > v.threads()) return false;
    return sbf_smem_bytes(v, Lw, CC) <= smem_budget;
}

cudaError_t launch_sbf_part(int idx, const SbfPartArgs& a, int n_tab, cudaStream_t s) {
    const Entry& e = kEntries[idx];
    if (!e.fn) return cudaErrorInvalidValue;  // pattern-factored parts launch through launch_sbf_part_fact
    const size_t smem = sbf_smem_bytes(e.v, a.Lw, a.CC);
    cudaError_t err = allow_dynamic_smem(reinterpret_cast<const void*>(e.fn), smem);
    if (err != cudaSuccess) return err;
    const int T = e.v.tile(), BD = e.v.bd();
    dim3 grid((a.n_out + T - 1) / T, (a.n_slab + BD - 1) / BD, n_tab);
    e.fn<<<grid, e.v.threads(), smem, s>>>(a);
    return cudaGetLastError();
}

int sbf_comb_sbs_per_block() { return CW * CSB; }

int sbf_comb_uc(int) { return UC; }

size_t sbf_comb_smem_bytes(int n_tab) { return 2ull * n_tab * kTabBytes + 16 + kSmemAlign; }

EncodeTiledFn encode_tiled_fn() {
    static const EncodeTiledFn fn = []() -> EncodeTiledFn {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<EncodeTiledFn>(ptr);
    }();
    return fn;
}

// P of a slab as a 4-D uint16 tensor: (t: Np, trial: slab rows, segment:
// n_seg, TAB: n_tab), box (CT, 1, UC, n_tab) = one comb chunk.
cudaError_t encode_comb_map(SbfCombArgs& a) {
    const EncodeTiledFn enc = encode_tiled_fn();
    if (!enc) return cudaErrorNotSupported;
    if (a.Np <= 0 || a.seg_stride % a.Np != 0 || a.tab_stride != a.seg_stride * a.n_seg || a.n_tab > 256 ||
        (reinterpret_cast<uintptr_t>(a.P) & 15u) != 0)
        return cudaErrorInvalidValue;
    const cuuint64_t dims[4] = {static_cast<cuuint64_t>(a.Np), static_cast<cuuint64_t>(a.seg_stride / a.Np),
                                static_cast<cuuint64_t>(a.n_seg), static_cast<cuuint64_t>(a.n_tab)};
    const cuuint64_t strides[3] = {static_cast<cuuint64_t>(a.Np) * 2, static_cast<cuuint64_t>(a.seg_stride) * 2,
                                   static_cast<cuuint64_t>(a.tab_stride) * 2};
    const cuuint32_t box[4] = {CT, 1, UC, static_cast<cuuint32_t>(a.n_tab)};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = enc(&a.tmap, CU_TENSOR_MAP_DATA_TYPE_UINT16, 4, const_cast<uint16_t*>(a.P), dims, strides, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_sbf_comb(const SbfCombArgs& a, cudaStream_t s) {
    const int per_block = CW * CSB;
    const int n_valid = a.n_dm - a.i0 < a.n_slab ? a.n_dm - a.i0 : a.n_slab;
    const size_t smem = sbf_comb_smem_bytes(a.n_tab);
    cudaError_t err = allow_dynamic_smem(reinterpret_cast<const void*>(k_sbf_comb), smem);
    if (err != cudaSuccess) return err;
    dim3 grid((a.n_out + CT - 1) / CT, n_valid, (a.n_sb + per_block - 1) / per_block);
    k_sbf_comb<<<grid, CW * 32, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace fdd
