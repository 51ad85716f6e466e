// k_sbf_persist.cu -- persistent SB-factored batched dedispersion.
//
// Every SB takes, per channel segment, one TAB (Sec. "Hierarchical beam
// forming"), so its dedispersed series is a sum of per-(TAB, segment)
// partial sums P (exact integers, regrouped; see k_sbf.cu).  Here ONE launch
// runs all of a batch: for every job (chunk), DM range and slab of DM trials,
// the part tasks (one TAB x BD trials x T samples: P of every segment, the
// tile of sbf_part.cuh) and the comb tasks (one trial x 256 samples x 40 SBs:
// each SB adds the partial rows of the TABs it takes).  Resident blocks take
// tasks from a global counter in a fixed order in which every task depends
// only on tasks issued before it:
//   - a job's scratch holds kSbfSlots slab buffers; its groups (range, slab)
//     use them in turn;
//   - issue order per job: P(0) .. P(S-1), C(0), P(S), C(1), P(S+1), ... with
//     S = kSbfSlots, so comb tasks of group g wait (bounded) until the part
//     tasks of g are done, and part tasks of group g wait until the comb
//     tasks of group g - S have read the buffer they overwrite.
// A task is taken only by a running block, so the oldest unfinished task
// always has its inputs: progress does not depend on how many blocks are
// resident.  Every wait polls a bounded number of times; a wait that gives
// up sets bit 0 of the plan's status word and an abort flag that makes every
// block stop taking tasks (the search's output is then incomplete).
//
// The comb task copies its partial rows with 1-D bulk copies
// (cp.async.bulk, 256 bytes per TAB and segment row, completion counted on
// an mbarrier per buffer; NB buffers of 8-segment chunks, NB - 1 chunks in
// flight ahead of the one being added), one copy per thread.
#include "sbf_part.cuh"
#include "tma.cuh"

namespace fdd {

namespace {

constexpr int PW = 8;                            // warps per block
constexpr int P_NW = 4, P_DPW = 4, P_MAXIT = 4;  // part tile: BD = 32 trials, T = 512 (uint8) / 256 (uint16)
constexpr int PBD = PW * P_DPW;
constexpr int CSB = 5;                           // SBs per warp of a comb task (40 per task)
constexpr int CT = 128, UC = 8;                  // comb: samples per sub-tile, segments per chunk
constexpr int CSUB = 2;                          // comb sub-tiles per task (CT * CSUB samples)
constexpr int NB = 4;                            // comb chunk buffers (NB - 1 chunks in flight ahead)
constexpr int kRowBytes = CT * 2;                // one partial row (uint16) in shared memory
constexpr int kTabBytes = UC * kRowBytes;        // UC rows of one TAB
static_assert(kTabBytes == 1 << 11, "the TAB offset is formed as tab << 11");

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ uint2 lds64(uint32_t addr) {
    uint2 v;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(addr));
    return v;
}

// Thread 0: wait until *count >= need; false after the poll limit or when
// another block has aborted the launch.
__device__ bool wait_count(const unsigned* count, unsigned need, const unsigned long long* abort) {
    for (int it = 0; it < tma::kSpinLimit; it++) {
        if (ld_acquire(count) >= need) return true;
        if ((it & 63) == 63 && *reinterpret_cast<const volatile unsigned long long*>(abort) != 0ULL) return false;
        if (it >= 32) __nanosleep(512);
    }
    return false;
}

struct Task {
    int kind;  // -1 stop, 0 part, 1 comb
    int job, group, idx;
};

__global__ void __launch_bounds__(PW * 32, 2) k_sbf_persist(const __grid_constant__ BatchParams p) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    __shared__ SbfPartArgs s_pa;
    __shared__ Task s_task;
    __shared__ __align__(8) unsigned long long s_bar[NB];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint8_t* smem = smem_raw + ((128 - (reinterpret_cast<uintptr_t>(smem_raw) & 127)) & 127);
    const uint32_t s_base = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
    const uint32_t bar0 = static_cast<uint32_t>(__cvta_generic_to_shared(&s_bar[0]));
    unsigned long long* abort_flag = p.counter + 3;
    if (tid == 0) {
        for (int b = 0; b < NB; b++) tma::mbar_init(bar0 + 8u * b, 1);
        tma::mbar_init_fence();
    }
    // comb stages this block has run so far (the same in every thread): stage g uses buffer g % NB, the
    // (g / NB)-th use of that buffer's barrier
    uint32_t stage0 = 0;
    const unsigned long long total = static_cast<unsigned long long>(p.sp_tasks_per_job) * p.n_jobs;
    // thread 0 takes its next task while the block works on the current one (a block holding a task it
    // has not started still lets the oldest unfinished task proceed: that task is either running or
    // the next one of a block whose current task is done)
    unsigned long long t_next = 0;
    int seg_job = -1, seg = 0;  // thread 0: segment of its last task (task indices only grow within a job)
    if (tid == 0) t_next = atomicAdd(p.counter + 2, 1ULL);

    for (;;) {
        __syncthreads();  // the previous task's shared-memory use is over
        if (tid == 0) {
            Task tk{-1, 0, 0, 0};
            const unsigned long long t = t_next;
            if (t < total) t_next = atomicAdd(p.counter + 2, 1ULL);
            if (t < total && *reinterpret_cast<const volatile unsigned long long*>(abort_flag) == 0ULL) {
                const int job = static_cast<int>(t / static_cast<unsigned long long>(p.sp_tasks_per_job));
                const int local = static_cast<int>(t - static_cast<unsigned long long>(job) * p.sp_tasks_per_job);
                if (job != seg_job) {
                    seg_job = job;
                    seg = 0;
                }
                while (seg + 1 < p.sp_n_segs && p.sp_segs[seg + 1].start <= local) seg++;
                const SbfPersistSeg sg = p.sp_segs[seg];
                const unsigned* done = p.sp_done + static_cast<size_t>(job) * p.sp_n_groups * 2;
                bool ok = true;
                if (sg.kind == 1)
                    ok = wait_count(done + 2 * sg.group, static_cast<unsigned>(p.sp_groups[sg.group].n_part),
                                    abort_flag);
                else if (sg.group >= kSbfSlots)
                    ok = wait_count(done + 2 * (sg.group - kSbfSlots) + 1,
                                    static_cast<unsigned>(p.sp_groups[sg.group - kSbfSlots].n_comb), abort_flag);
                if (!ok) {
                    atomicOr(p.status, 1u);
                    atomicExch(abort_flag, 1ULL);
                } else {
                    tk = Task{sg.kind, job, sg.group, local - sg.start};
                    if (sg.kind == 0) {
                        const SbfPersistGroup G = p.sp_groups[sg.group];
                        const SbfPersistRange& R = p.sp_ranges[G.range];
                        const BatchJob& J = p.jobs[job];
                        SbfPartArgs& a = s_pa;  // written in place by thread 0
                        const int phase_in = R.ds_index < 0 ? 0 : J.ds_phase[R.ds_index];
                        a.in = R.ds_index < 0 ? J.tabs : reinterpret_cast<const uint8_t*>(J.ds[R.ds_index]);
                        a.pitch_bytes = R.ds_index < 0 ? J.tab_pitch : J.ds_pitch[R.ds_index] * 2;
                        a.n_valid = (J.n_in - phase_in) / R.D;
                        a.base = R.base;
                        a.off = R.off;
                        a.stages = R.stages;
                        a.segs = R.segs;
                        a.P = J.sbf_scratch + static_cast<int64_t>(G.slot) * R.slot_elems;
                        a.seg_stride = static_cast<int64_t>(R.slab) * R.Np;
                        a.tab_stride = a.seg_stride * R.n_seg;
                        a.Np = R.Np;
                        a.n_chan = p.n_chan;
                        a.n_dm = R.n_dm;
                        a.n_out = R.n_out;
                        a.Lw = R.Lw;
                        a.CC = R.CC;
                        a.n_stages = R.n_stages;
                        a.i0 = G.i0;
                        a.n_slab = G.n_slab;
                    }
                }
            }
            s_task = tk;
        }
        __syncthreads();
        const Task tk = s_task;
        if (tk.kind < 0) break;
        const SbfPersistGroup G = p.sp_groups[tk.group];
        const SbfPersistRange& R = p.sp_ranges[G.range];
        unsigned* done = p.sp_done + (static_cast<size_t>(tk.job) * p.sp_n_groups + tk.group) * 2;

        if (tk.kind == 0) {
            // ---- part task: TAB x BD trials x T samples of every segment
            const int n_blk = (G.n_slab + PBD - 1) / PBD;
            const int tile = tk.idx % R.part_tiles;
            const int rest = tk.idx / R.part_tiles;
            const int blk_rel = rest % n_blk;
            const int tab = rest / n_blk;
            if (R.E == 1)
                detail::sbf_part_tile<1, P_NW, P_DPW, PW, P_MAXIT>(s_pa, tile, blk_rel, tab, smem);
            else
                detail::sbf_part_tile<2, P_NW, P_DPW, PW, P_MAXIT>(s_pa, tile, blk_rel, tab, smem);
            __threadfence();             // every thread's partials are visible device-wide ...
            fence_proxy_async_global();  // ... and to the bulk copies of the comb tasks that read them
            __syncthreads();
            if (tid == 0) atomicAdd(done, 1u);
            continue;
        }

        // ---- comb task: one trial x CSUB * CT samples x PW*CSB SBs.  Its stages (sub-tile, chunk of UC
        // segments) run as one pipeline over NB chunk buffers, NB - 1 chunks in flight ahead.
        const BatchJob& J = p.jobs[tk.job];
        // the SB groups of one (trial, tile) are consecutive tasks, so the second reads its rows from L2
        const int z = tk.idx % R.sb_groups;
        const int rest = tk.idx / R.sb_groups;
        const int y = rest % R.comb_tiles;
        const int i_s = rest / R.comb_tiles;
        const int i = G.i0 + i_s;
        const int r = G.range;
        const int emit = J.emit[r];
        const int n_sub = max(0, min(CSUB, (emit - y * CSUB * CT + CT - 1) / CT));  // sub-tiles with outputs
        const int n_tab = p.n_tab;
        const int n_seg = R.n_seg;
        const int n_chunks = (n_seg + UC - 1) / UC;
        const int n_stages = n_sub * n_chunks;
        const int64_t seg_stride = static_cast<int64_t>(R.slab) * R.Np;
        const int64_t tab_stride = seg_stride * R.n_seg;
        const uint16_t* P_trial =
            J.sbf_scratch + static_cast<int64_t>(G.slot) * R.slot_elems + static_cast<int64_t>(i_s) * R.Np;
        const uint32_t buf_bytes = static_cast<uint32_t>(n_tab) * kTabBytes;
        const int sb0 = z * (PW * CSB) + warp * CSB;
        const int nsb = max(0, min(CSB, p.n_sb - sb0));  // warp-uniform
        const uint8_t* seg_tab = R.seg_tab;
        uint32_t tab_row[CSB];  // byte offsets of this warp's SB rows in seg_tab
#pragma unroll
        for (int j = 0; j < CSB; j++) {
            const int sj = nsb > 0 ? sb0 + min(j, nsb - 1) : 0;
            tab_row[j] = static_cast<uint32_t>(sj) * static_cast<uint32_t>(R.seg_pitch);
        }
        // stage q: chunk q % n_chunks of sub-tile q / n_chunks into buffer (stage0 + q) % NB, one
        // 256-byte bulk copy per (TAB, segment) row, spread over the block's threads (one copy per
        // thread for up to 256 rows); thread 0 arms the barrier with the chunk's byte count (copies
        // that land first only lower its pending count: the phase needs thread 0's arrival too)
        auto issue = [&](int q) {
            const uint32_t b = (stage0 + static_cast<uint32_t>(q)) % NB;
            const uint32_t bar = bar0 + 8u * b;
            const int sub = q / n_chunks, ch = q - sub * n_chunks;
            const int u0 = ch * UC;
            const int nu = min(UC, n_seg - u0);
            const uint16_t* src0 = P_trial + (y * CSUB + sub) * CT;
            if (tid == 0) tma::mbar_expect_tx(bar, static_cast<uint32_t>(n_tab * nu * kRowBytes));
            const uint32_t dst0 = s_base + b * buf_bytes;
            for (int it = tid; it < n_tab * nu; it += PW * 32) {
                const int k = it / nu, du = it - k * nu;
                fence_proxy_async_shared();
                bulk_copy(dst0 + static_cast<uint32_t>(k * kTabBytes + du * kRowBytes),
                          src0 + k * tab_stride + static_cast<int64_t>(u0 + du) * seg_stride, kRowBytes, bar);
            }
        };
        uint32_t acc[CSB][2], tot[CSB][4];
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
        fence_proxy_async_global();  // the partials were written through the generic proxy
        for (int q = 0; q < NB - 1 && q < n_stages; q++) issue(q);
        int since = 0;
        bool failed = false;
        for (int q = 0; q < n_stages; q++) {
            const int sub = q / n_chunks, ch = q - sub * n_chunks;
            // the buffer of stage q + NB - 1 was released at the end of stage q - 1
            if (q + NB - 1 < n_stages) issue(q + NB - 1);
            const uint32_t g = stage0 + static_cast<uint32_t>(q);
            const bool ok = tma::mbar_wait_bounded(bar0 + 8u * (g % NB), (g / NB) & 1u);
            if (__syncthreads_or(!ok)) {
                // a copy did not land: flag it, wait (bounded) for this block's copies in flight, stop
                if (tid == 0) {
                    atomicOr(p.status, 1u);
                    atomicExch(abort_flag, 1ULL);
                    for (int w2 = q; w2 < n_stages && w2 < q + NB - 1; w2++) {
                        const uint32_t g2 = stage0 + static_cast<uint32_t>(w2);
                        tma::mbar_wait_bounded(bar0 + 8u * (g2 % NB), (g2 / NB) & 1u);
                    }
                }
                failed = true;
                break;
            }
            if (ch == 0) {
#pragma unroll
                for (int j = 0; j < CSB; j++) {
                    acc[j][0] = acc[j][1] = 0u;
                    tot[j][0] = tot[j][1] = tot[j][2] = tot[j][3] = 0u;
                }
                since = 0;
            }
            const int u0 = ch * UC;
            const int nu = min(UC, n_seg - u0);
            const uint32_t s_buf = s_base + (g % NB) * buf_bytes + 8u * lane;
#pragma unroll
            for (int qq = 0; qq < UC; qq += 4) {
                uint32_t tabs4[CSB];
#pragma unroll
                for (int j = 0; j < CSB; j++)
                    tabs4[j] = __ldg(reinterpret_cast<const uint32_t*>(seg_tab + tab_row[j] + u0 + qq));
#pragma unroll
                for (int dq = 0; dq < 4; dq++) {
                    const int du = qq + dq;
                    if (du < nu) {  // block-uniform
#pragma unroll
                        for (int j = 0; j < CSB; j++) {
                            // byte dq of tabs4 (the TAB; PRMT zero-fills the rest) times kTabBytes (2^11)
                            const uint32_t tab = __byte_perm(tabs4[j], 0u, 0x4440u + dq);
                            const uint2 v = lds64(s_buf + (tab << 11) + du * kRowBytes);
                            acc[j][0] += v.x;
                            acc[j][1] += v.y;
                        }
                        if (++since == R.flush) {
                            fold();
                            since = 0;
                        }
                    }
                }
            }
            __syncthreads();  // buffer free for the copy issued at the next stage
            if (ch == n_chunks - 1) {
                // sub-tile complete: write its series samples and fold the moments
                fold();
                const int t = (y * CSUB + sub) * CT + 4 * lane;
                int32_t* series = J.series + R.series_elem_off;
                unsigned long long* stat = J.stat + 2 * R.stat_off;
#pragma unroll
                for (int j = 0; j < CSB; j++) {
                    unsigned long long s1 = 0, s2 = 0;
                    if (j < nsb) {
                        int32_t* row = series + (static_cast<int64_t>(sb0 + j) * R.n_dm + i) * R.n_out;
#pragma unroll
                        for (int e = 0; e < 4; e++) {
                            if (t + e < emit) {
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
                        const int64_t qs = static_cast<int64_t>(sb0 + j) * R.n_dm + i;
                        atomicAdd(stat + 2 * qs, s1);
                        atomicAdd(stat + 2 * qs + 1, s2);
                    }
                }
            }
        }
        if (failed) break;
        stage0 += static_cast<uint32_t>(n_stages);
        if (tid == 0) {
            __threadfence();
            atomicAdd(done + 1, 1u);
        }
    }
}

}  // namespace

DedispVariant sbf_persist_part_variant(int E) { return DedispVariant{E, P_NW, P_DPW, PW, P_MAXIT}; }

size_t sbf_persist_smem_bytes(size_t part_smem_max, int n_tab) {
    const size_t comb = static_cast<size_t>(NB) * static_cast<size_t>(n_tab) * kTabBytes;
    return (part_smem_max > comb ? part_smem_max : comb) + 128;  // + alignment of the base to 128 bytes
}

cudaError_t sbf_persist_occupancy(size_t smem, int* blocks_per_sm) {
    cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void*>(k_sbf_persist), smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_sbf_persist, PW * 32, smem);
}

cudaError_t launch_sbf_persist(const BatchParams& p, int grid, size_t smem, cudaStream_t s) {
    cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void*>(k_sbf_persist), smem);
    if (e != cudaSuccess) return e;
    k_sbf_persist<<<grid, PW * 32, smem, s>>>(p);
    return cudaGetLastError();
}

int sbf_persist_comb_sbs() { return PW * CSB; }

int sbf_persist_comb_tile() { return CT * CSUB; }

}  // namespace fdd
