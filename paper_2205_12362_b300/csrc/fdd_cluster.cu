// fdd_cluster.cu -- DM-width clustering of a candidate list on the GPU
// (Sec. "AMBER", "Clustering (optional)"): among candidates of one SB at the
// same time and DM keep the highest S/N over widths; then every group of
// neighbouring DM trials at that SB and time keeps its highest-S/N member.
//
// Both steps together keep exactly the maximum of each connected group of
// candidates sharing (sb, t_native) whose DM indices form a run without gaps,
// ordered by S/N, then smaller dm_index, smaller width, earlier record.
// On the device:
//   k_cl_init    empty the hash table (open addressing, linear probing,
//                capacity a power of two >= 2 * cap_in), zero the counters;
//   k_cl_tmin    smallest t_native of the list (keys hold t - t_min);
//   k_cl_insert  one slot per (sb, dm, t): atomicMax of (S/N, -width);
//   k_cl_winner  the step-1 winner of each slot: smallest record index
//                whose (S/N, -width) equals the slot's maximum;
//   k_cl_emit    each winner walks its DM neighbours (dm-1, dm-2, ... then
//                dm+1, ...) while their slots exist and stops at the first
//                better one; a winner that meets none is the group's maximum
//                and is written out (warp-aggregated append).
// Records whose sb, dm_index or t_native - t_min do not fit the key
// (sb >= 2^13, dm_index >= 2^21, t - t_min >= 2^30 - 1) are passed through
// unclustered.
#include "fdd_plan_impl.h"

using namespace fdd::host;

namespace {

constexpr uint64_t kEmpty = ~0ull;
constexpr int kSbBits = 13, kDmBits = 21, kTBits = 30;

struct ClSlot {
    unsigned long long key;
    unsigned long long best;  // (ordered S/N bits << 32) | (0xFFFFFFFF - width)
    unsigned int win;         // smallest record index holding `best`
    unsigned int pad;
};

struct ClHeader {
    long long t_min;
    unsigned long long reserved[7];
};

__host__ __device__ inline uint64_t cl_capacity(int64_t cap_in) {
    uint64_t p = 1024;
    while (p < 2ull * static_cast<uint64_t>(cap_in)) p <<= 1;
    return p;
}

// Float -> uint32 with the same order (negative values reversed).
__device__ inline uint32_t ord_bits(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ inline uint64_t pack_best(const fdd_candidate& c) {
    return (static_cast<uint64_t>(ord_bits(c.snr)) << 32) | (0xFFFFFFFFu - static_cast<uint32_t>(c.width_native));
}

// 64-bit finaliser of the SplitMix64 generator (Steele, Lea, Flood 2014),
// used as the hash of a key.
__device__ inline uint64_t mix64(uint64_t x) {
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebull;
    x ^= x >> 31;
    return x;
}

__device__ inline bool make_key(int32_t sb, int32_t dm, int64_t t_rel, uint64_t* key) {
    if (sb < 0 || sb >= (1 << kSbBits) || dm < 0 || dm >= (1 << kDmBits) || t_rel < 0 ||
        t_rel >= (1ll << kTBits) - 1)
        return false;
    *key = (static_cast<uint64_t>(sb) << (kDmBits + kTBits)) | (static_cast<uint64_t>(dm) << kTBits) |
           static_cast<uint64_t>(t_rel);
    return true;
}

// t - t_min without signed overflow (a difference >= 2^63 comes out negative
// and is rejected by make_key).
__device__ inline int64_t t_diff(int64_t t, long long t_min) {
    return static_cast<int64_t>(static_cast<uint64_t>(t) - static_cast<uint64_t>(t_min));
}

__device__ inline ClSlot* find_slot(ClSlot* tab, uint64_t mask, uint64_t key) {
    uint64_t h = mix64(key) & mask;
    for (uint64_t probe = 0; probe <= mask; probe++) {
        const unsigned long long k = tab[h].key;
        if (k == key) return tab + h;
        if (k == kEmpty) return nullptr;
        h = (h + 1) & mask;
    }
    return nullptr;
}

__device__ inline int64_t n_records(const uint64_t* count, int64_t cap_in) {
    const uint64_t c = *count;
    return static_cast<int64_t>(c < static_cast<uint64_t>(cap_in) ? c : static_cast<uint64_t>(cap_in));
}

#define FDD_GRID_LOOP(i, n) \
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < (n); \
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)

__global__ void k_cl_init(ClSlot* tab, uint64_t cap, ClHeader* hdr, uint64_t* out_count) {
    FDD_GRID_LOOP(i, static_cast<int64_t>(cap)) {
        tab[i].key = kEmpty;
        tab[i].best = 0;
        tab[i].win = 0xFFFFFFFFu;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        hdr->t_min = 0x7FFFFFFFFFFFFFFFll;
        *out_count = 0;
    }
}

__global__ void k_cl_tmin(const fdd_candidate* __restrict__ in, const uint64_t* __restrict__ count, int64_t cap_in,
                          ClHeader* hdr) {
    const int64_t n = n_records(count, cap_in);
    long long m = 0x7FFFFFFFFFFFFFFFll;
    FDD_GRID_LOOP(i, n) m = min(m, static_cast<long long>(in[i].t_native));
    for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
    if ((threadIdx.x & 31) == 0 && m != 0x7FFFFFFFFFFFFFFFll) atomicMin(&hdr->t_min, m);
}

__global__ void k_cl_insert(const fdd_candidate* __restrict__ in, const uint64_t* __restrict__ count,
                            int64_t cap_in, ClSlot* tab, uint64_t mask, const ClHeader* hdr) {
    const int64_t n = n_records(count, cap_in);
    const long long t_min = hdr->t_min;
    FDD_GRID_LOOP(i, n) {
        const fdd_candidate c = in[i];
        uint64_t key;
        if (!make_key(c.sb, c.dm_index, t_diff(c.t_native, t_min), &key)) continue;
        uint64_t h = mix64(key) & mask;
        for (uint64_t probe = 0; probe <= mask; probe++) {
            const unsigned long long prev = atomicCAS(&tab[h].key, kEmpty, key);
            if (prev == kEmpty || prev == key) {
                atomicMax(&tab[h].best, pack_best(c));
                break;
            }
            h = (h + 1) & mask;
        }
    }
}

__global__ void k_cl_winner(const fdd_candidate* __restrict__ in, const uint64_t* __restrict__ count,
                            int64_t cap_in, ClSlot* tab, uint64_t mask, const ClHeader* hdr) {
    const int64_t n = n_records(count, cap_in);
    const long long t_min = hdr->t_min;
    FDD_GRID_LOOP(i, n) {
        const fdd_candidate c = in[i];
        uint64_t key;
        if (!make_key(c.sb, c.dm_index, t_diff(c.t_native, t_min), &key)) continue;
        ClSlot* s = find_slot(tab, mask, key);
        if (s && s->best == pack_best(c)) atomicMin(&s->win, static_cast<unsigned int>(i));
    }
}

__global__ void k_cl_emit(const fdd_candidate* __restrict__ in, const uint64_t* __restrict__ count, int64_t cap_in,
                          const ClSlot* tab, uint64_t mask, const ClHeader* hdr, fdd_candidate* __restrict__ out,
                          int64_t cap_out, unsigned long long* out_count) {
    const int64_t n = n_records(count, cap_in);
    const long long t_min = hdr->t_min;
    const int lane = threadIdx.x & 31;
    // every lane runs the same number of iterations so the warp vote below is complete
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t first = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    const int64_t warp_first = first - lane;
    for (int64_t base = warp_first; base < n; base += stride) {
        const int64_t i = base + lane;
        bool keep = false;
        if (i < n) {
            const fdd_candidate c = in[i];
            const int64_t t_rel = t_diff(c.t_native, t_min);
            uint64_t key;
            if (!make_key(c.sb, c.dm_index, t_rel, &key)) {
                keep = true;  // outside the key range: passed through
            } else {
                const ClSlot* s = find_slot(const_cast<ClSlot*>(tab), mask, key);
                if (s && s->win == static_cast<unsigned int>(i)) {
                    const uint32_t mine = static_cast<uint32_t>(s->best >> 32);
                    keep = true;
                    for (int32_t d = c.dm_index - 1; keep && d >= 0; d--) {  // lower DMs win ties
                        uint64_t k2;
                        if (!make_key(c.sb, d, t_rel, &k2)) break;
                        const ClSlot* q = find_slot(const_cast<ClSlot*>(tab), mask, k2);
                        if (!q) break;
                        if (static_cast<uint32_t>(q->best >> 32) >= mine) keep = false;
                    }
                    for (int32_t d = c.dm_index + 1; keep; d++) {
                        uint64_t k2;
                        if (!make_key(c.sb, d, t_rel, &k2)) break;
                        const ClSlot* q = find_slot(const_cast<ClSlot*>(tab), mask, k2);
                        if (!q) break;
                        if (static_cast<uint32_t>(q->best >> 32) > mine) keep = false;
                    }
                }
            }
        }
        const unsigned ballot = __ballot_sync(0xFFFFFFFFu, keep);
        if (ballot == 0) continue;
        unsigned long long slot0 = 0;
        if (lane == 0) slot0 = atomicAdd(out_count, static_cast<unsigned long long>(__popc(ballot)));
        slot0 = __shfl_sync(0xFFFFFFFFu, slot0, 0);
        if (keep) {
            const unsigned long long o = slot0 + __popc(ballot & ((1u << lane) - 1u));
            if (o < static_cast<unsigned long long>(cap_out)) out[o] = in[i];
        }
    }
}

#undef FDD_GRID_LOOP

size_t cl_workspace(int64_t cap_in) { return sizeof(ClHeader) + cl_capacity(cap_in) * sizeof(ClSlot); }

}  // namespace

extern "C" {

int fdd_cluster_workspace_size(int64_t cap_in, size_t* bytes) {
    if (!bytes || cap_in < 0 || cap_in > (1ll << 31)) return fail(FDD_ERR_INVALID_ARG, "bad argument");
    *bytes = cl_workspace(cap_in);
    return FDD_OK;
}

int fdd_cluster(const fdd_candidate* d_in, const uint64_t* d_in_count, int64_t cap_in, void* d_workspace,
                size_t workspace_bytes, fdd_candidate* d_out, int64_t cap_out, uint64_t* d_out_count,
                fdd_stream_t stream) {
    if (!d_in_count || !d_out_count || !d_workspace || cap_in < 0 || cap_in > (1ll << 31) || cap_out < 0 ||
        (cap_in > 0 && !d_in) || (cap_out > 0 && !d_out))
        return fail(FDD_ERR_INVALID_ARG, "bad cluster argument");
    if (reinterpret_cast<uintptr_t>(d_workspace) % 16 != 0 || reinterpret_cast<uintptr_t>(d_in) % 16 != 0 ||
        reinterpret_cast<uintptr_t>(d_out) % 16 != 0)
        return fail(FDD_ERR_MISALIGNED, "cluster buffers must be 16-byte aligned");
    if (workspace_bytes < cl_workspace(cap_in)) return fail(FDD_ERR_WORKSPACE, "cluster workspace too small");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    ClHeader* hdr = static_cast<ClHeader*>(d_workspace);
    ClSlot* tab = reinterpret_cast<ClSlot*>(hdr + 1);
    const uint64_t cap = cl_capacity(cap_in), mask = cap - 1;
    const int threads = 256, grid = 148 * 4;
    auto* out_count = reinterpret_cast<unsigned long long*>(d_out_count);
    k_cl_init<<<grid, threads, 0, s>>>(tab, cap, hdr, d_out_count);
    k_cl_tmin<<<grid, threads, 0, s>>>(d_in, d_in_count, cap_in, hdr);
    k_cl_insert<<<grid, threads, 0, s>>>(d_in, d_in_count, cap_in, tab, mask, hdr);
    k_cl_winner<<<grid, threads, 0, s>>>(d_in, d_in_count, cap_in, tab, mask, hdr);
    k_cl_emit<<<grid, threads, 0, s>>>(d_in, d_in_count, cap_in, tab, mask, hdr, d_out, cap_out, out_count);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "cluster launch");
    return FDD_OK;
}

}  // extern "C"
