/*
 * fdd.h -- C ABI of the B300 single-pulse (FRB) search hot path.
 *
 * The library implements, as CUDA kernels for sm_103a, the per-chunk search
 * the paper's AMBER pipeline runs on each compound beam (Sec. "AMBER"):
 * downsampling, brute-force incoherent dedispersion with synthesized-beam
 * (SB) formation, boxcar integration over pulse widths, S/N evaluation and
 * candidate selection.  Inputs follow the paper's data description: 8-bit
 * Stokes-I filterbank per tied-array beam (TAB), time the fastest index
 * (Sec. "Data formats"; Sec. "Dedicated ARTS TABF on Central Uniboards").
 * The output record carries the fields the paper's candidate files hold:
 * beam, downsampling factor, arrival time, width, DM and S/N (Sec. "DARC").
 *
 * Conventions shared by every call:
 *   - Pointers named d_* are DEVICE pointers (cudaMalloc / torch CUDA
 *     tensors) owned by the caller; everything else is host memory.
 *   - Calls that take a cudaStream_t only enqueue work on that stream and
 *     return; results are valid once the stream has been synchronised.
 *   - Return value: FDD_OK (0) or a negative FDD_ERR_* code.  Argument
 *     errors are detected on the host before anything is enqueued.  A CUDA
 *     runtime failure returns FDD_ERR_CUDA; fdd_last_error_message() then
 *     holds the runtime's text (per thread).
 *   - The library owns the plan's device tables (delay offsets, SB map) and
 *     frees them in fdd_plan_destroy.  It never allocates per-call memory:
 *     scratch ("workspace") is a caller buffer sized by fdd_workspace_size.
 *   - A plan may be used from one host thread at a time.  Searches on
 *     different streams may overlap if each has its own workspace,
 *     candidate buffer and counter.
 */
#ifndef FDD_H
#define FDD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* fdd_stream_t; /* same type as cudaStream_t; NULL = legacy default stream */

enum {
    FDD_OK = 0,
    FDD_ERR_INVALID_ARG = -1,  /* bad size, pointer, plan field or sb_map entry */
    FDD_ERR_SHORT_INPUT = -2,  /* n_in < n_out + max delay of some range (native samples) */
    FDD_ERR_NO_MEMORY = -3,    /* device or host allocation of plan tables failed */
    FDD_ERR_MISALIGNED = -4,   /* device pointer or row pitch not 16-byte aligned */
    FDD_ERR_UNSUPPORTED = -5,  /* plan outside the kernels' limits (see FDD_MAX_*) */
    FDD_ERR_CUDA = -6,         /* CUDA runtime error; see fdd_last_error_message() */
    FDD_ERR_WORKSPACE = -7,    /* workspace smaller than fdd_workspace_size() */
    FDD_ERR_SEQUENCE = -8,     /* serving: chunk out of sequence (dropped/late/duplicate/reordered) */
    FDD_ERR_BUSY = -9,         /* serving: beam backlogged, retry after fdd_server_poll */
    FDD_ERR_TIMEOUT = -10      /* a kernel's bounded wait for a tile copy gave up (fdd_plan_status) */
};

#define FDD_MAX_WIDTHS 16      /* boxcar widths per DM range */
#define FDD_MAX_WIDTH 1024     /* largest boxcar width, in range samples; also, per range,
                                  n_chan * 255 * downsamp * widest width must stay below 2^31 (the
                                  box sums are exact 32-bit differences), else FDD_ERR_UNSUPPORTED */
#define FDD_MAX_CHANNELS 16384
#define FDD_MAX_TABS 256
#define FDD_MAX_RANGES 8       /* DM ranges per plan in batched searches */
#define FDD_MAX_BATCH_JOBS 64  /* chunks per batched search */

/* One range of the DM plan (paper Table "dedispersion setup": each GPU
 * covers a DM range with its own step; Sec. "Downsampling" lets a range run
 * at a reduced time resolution).  Trial i of the range has
 * DM_i = dm0 + i * ddm (formed afresh, not accumulated). */
typedef struct {
    double dm0;            /* first trial DM, pc cm^-3, >= 0 */
    double ddm;            /* DM step, > 0 */
    int32_t n_dm;          /* number of trials, >= 1 */
    int32_t downsamp;      /* D >= 1: the range works on sums of D native samples */
    int32_t n_width;       /* 1..FDD_MAX_WIDTHS */
    const int32_t* widths; /* host [n_width]: boxcar widths in range samples, 1..FDD_MAX_WIDTH */
} fdd_range;

/* Plan description.  Channel order is free; the highest frequency is the
 * dedispersion reference (its delay is 0 for every DM). */
typedef struct {
    int32_t n_tab;                /* TABs per compound beam (12 in ARTS), 1..FDD_MAX_TABS */
    int32_t n_chan;               /* channels (1536 in ARTS), 1..FDD_MAX_CHANNELS */
    int32_t n_sb;                 /* synthesized beams to search (71 in ARTS), >= 1 */
    const double* chan_freq_mhz;  /* host [n_chan]: channel centre frequencies, > 0 */
    double t_samp_s;              /* native sampling time (81.92e-6 in ARTS), > 0 */
    int32_t n_range;              /* >= 1 */
    const fdd_range* ranges;      /* host [n_range] */
    float snr_thresh;             /* candidate when S/N > snr_thresh (strict) */
} fdd_plan_desc;

/* One candidate (32 bytes, POD).  Fields after Sec. "DARC" candidate files:
 * SB index, DM-trial index (global over the concatenated ranges), the range's
 * downsampling factor, boxcar width and window start in NATIVE samples (start
 * = t * D + t_offset_native of the search call), trial DM and S/N. */
typedef struct {
    int32_t sb;
    int32_t dm_index;
    int32_t downsamp;
    int32_t width_native;
    int64_t t_native;
    float dm;
    float snr;
} fdd_candidate;

typedef struct fdd_plan fdd_plan;

/* Build a plan: computes every range's integer delay table on the host in
 * FP64,
 *     d[i][c] = llround(4148.808 * DM_i * (f_c^-2 - f_top^-2) / (D * t_samp)),
 * (Sec. "Dedispersion"; the cold-plasma constant is not printed in the paper)
 * and uploads it, with the SB map, to the current CUDA device.
 * sb_map_host: host int16 [n_sb][n_chan]; SB s takes channel c from TAB
 * sb_map_host[s*n_chan + c], which must lie in [0, n_tab) (Sec.
 * "Hierarchical beam forming": SBs are per-channel selections of TABs).
 * On success *out receives the plan (free with fdd_plan_destroy).
 * Errors: INVALID_ARG, UNSUPPORTED, NO_MEMORY, CUDA. */
int fdd_plan_create(const fdd_plan_desc* desc, const int16_t* sb_map_host, fdd_plan** out);

/* Free the plan and its device tables (library bookkeeping; no counterpart in
 * the paper).  NULL is accepted.  The caller makes
 * sure no enqueued search still uses it. */
int fdd_plan_destroy(fdd_plan* plan);

/* Largest delay over all ranges, in native samples (max_r D_r * max d_r; the
 * overlap each chunk needs, Sec. "Dedispersion"):
 * a search of n_out output samples needs n_in >= n_out + max_delay_native
 * input samples per channel. */
int fdd_plan_max_delay(const fdd_plan* plan, int64_t* max_delay_native);

/* Plan summary (library bookkeeping) for a search of n_out native output
 * samples: the largest
 * delay (as fdd_plan_max_delay) and the workspace bytes of a search with
 * n_in = n_out + max_delay_native whose series stay in the workspace (as
 * fdd_workspace_size(plan, n_in, n_out, 1, ...)). */
int fdd_plan_info(const fdd_plan* plan, int64_t n_out, int64_t* max_delay_native, int64_t* workspace_bytes);

/* Number of DM trials summed over all ranges (the DM plan of Table
 * "dedispersion setup"; the length of the global
 * dm_index axis). */
int fdd_plan_total_dms(const fdd_plan* plan, int64_t* n_dm_total);

/* Copy range r's integer delay table (Sec. "Dedispersion"; int32
 * [n_dm][n_chan], units of D_r
 * native samples) to host memory dst (n_dm * n_chan entries). */
int fdd_plan_delays(const fdd_plan* plan, int32_t r, int32_t* dst);

/* Bytes of device workspace a search of (n_in, n_out) needs (library
 * bookkeeping; no counterpart in the paper).
 * If the caller passes d_series to fdd_search, the series live there and the
 * workspace shrinks by fdd_series_size().  For plans with two or more SBs and
 * DM ranges the size holds two lanes of SB-factored partial-sum scratch, which
 * a batched search runs concurrently (fdd_search_batch); a plain search uses
 * one of them. */
int fdd_workspace_size(const fdd_plan* plan, int64_t n_in, int64_t n_out, int32_t with_series,
                       size_t* bytes);

/* Bytes of the dedispersed-series buffer (the dedispersed time series of
 * Sec. "Dedispersion"): int32, packed per range as
 * [range][sb][dm][floor(n_out / D_r)]. */
int fdd_series_size(const fdd_plan* plan, int64_t n_out, size_t* bytes);

/* Search one chunk of every SB of the plan: the per-chunk AMBER search of
 * Sec. "AMBER" ("Downsampling", "Dedispersion", "Integration", "S/N
 * evaluation", "Candidate selection").
 *   d_tabs        device uint8 [n_tab][n_chan][pitch]: TAB filterbanks; the
 *                 first n_in samples of each row are data.  16-byte aligned.
 *   pitch         row pitch in samples (bytes), multiple of 16, >= n_in.
 *   n_out         output samples (native) to search; range r produces
 *                 floor(n_out / D_r) samples per series, and downsampling
 *                 bins start at input sample 0.
 *   t_offset_native  added to every candidate's t_native (stream position).
 *   d_workspace   >= fdd_workspace_size(plan, n_in, n_out, d_series == NULL).
 *   d_cands       device [cap] candidate records (order unspecified).
 *   d_count       device uint64: set to the TRUE number of candidates; only
 *                 the first min(count, cap) records are written, so
 *                 count > cap signals an overflow.
 *   d_series      NULL, or device int32 buffer of fdd_series_size() bytes that
 *                 receives every dedispersed series (for verification).
 * Stages per range: downsample (D > 1), SB-gather + dedispersion with exact
 * int32 sums, series statistics, boxcar S/N over the range's widths, warp-
 * ballot threshold and compaction.  Asynchronous on stream.
 * Errors (host-side, nothing enqueued): INVALID_ARG, SHORT_INPUT, MISALIGNED,
 * WORKSPACE; CUDA on a launch failure. */
int fdd_search(fdd_plan* plan, const uint8_t* d_tabs, int64_t n_in, int64_t pitch, int64_t n_out,
               int64_t t_offset_native, void* d_workspace, size_t workspace_bytes,
               fdd_candidate* d_cands, int64_t cap, uint64_t* d_count, int32_t* d_series,
               fdd_stream_t stream);

/* Streaming form of fdd_search (Sec. "Downsampling" with bins aligned to the
 * beam's stream, so that consecutive windows tile one search of the whole
 * stream): input sample 0 is native sample t0_native (>= 0) of the stream,
 * and range r's downsampling bins are aligned to stream sample 0 (bin J
 * covers stream samples [J D_r, (J+1) D_r)).  The window searches, per
 * range, the bins whose first sample lies in [t0_native, t0_native + n_out):
 *     n_r = ceil((t0 + n_out)/D_r) - ceil(t0/D_r) bins, read from input
 *     sample phase_r = ceil(t0/D_r) D_r - t0 on
 * (for D_r = 8 and 12500-sample chunks, n_r alternates 1563 and 1562); a
 * candidate's t_native is its bin's first stream sample.  Everything else as
 * fdd_search, except the sizes: n_in >= phase_r + D_r (n_r + max delay_r)
 * for every range (fdd_window_sizes gives an n_in that fits every t0), the
 * workspace and d_series (if given) as fdd_window_sizes reports, and d_series
 * packed [range][sb][dm][ceil(n_out / D_r)] with the first n_r samples of
 * each row written.  Errors as fdd_search; INVALID_ARG for t0_native < 0. */
int fdd_search_window(fdd_plan* plan, const uint8_t* d_tabs, int64_t n_in, int64_t pitch, int64_t n_out,
                      int64_t t0_native, void* d_workspace, size_t workspace_bytes, fdd_candidate* d_cands,
                      int64_t cap, uint64_t* d_count, int32_t* d_series, fdd_stream_t stream);

/* Sizes of fdd_search_window for n_out outputs, valid for every window
 * start: *n_in = n_out + max_r (D_r (max delay_r + 1) - 1) input samples, the
 * workspace (series in the workspace) and the d_series buffer.  Any output
 * pointer may be NULL (library bookkeeping; no counterpart in the paper). */
int fdd_window_sizes(const fdd_plan* plan, int64_t n_out, int64_t* n_in, size_t* workspace_bytes,
                     size_t* series_bytes);

/* Stage entry point (Sec. "Downsampling"): d_out[row][j] =
 * sum_{k<D} d_in[row][j*D + k] for j < floor(n_in / D), rows = n_rows.
 * d_in uint8 rows at in_pitch bytes; d_out uint16 rows at out_pitch
 * elements (multiple of 8).  Both 16-byte aligned.  1 <= D <= 257. */
int fdd_downsample_u8(const uint8_t* d_in, int64_t n_rows, int64_t n_in, int64_t in_pitch,
                      int32_t downsamp, uint16_t* d_out, int64_t out_pitch, fdd_stream_t stream);

/* Kernel configuration of one DM range's dedispersion launch (the paper's
 * AMBER picks its kernel configuration per platform and observation by
 * auto-tuning, Sec. "AMBER"; this library does the same with its own tuner).
 * Fields: variant index, DM trials per block, output samples per block,
 * channels per shared-memory stage, threads per block, 32-bit words per
 * staged row copy, the mean launch time the tuner measured (ms, 0 if the
 * range was not tuned), and the kernel's adds per brute-force channel-add. */
typedef struct {
    int32_t variant;
    int32_t dm_per_block;
    int32_t tile;
    int32_t chan_per_stage;
    int32_t threads;
    int32_t row_words;
    float tuned_ms;
    float work_ratio;  /* integer adds the configured kernel performs per brute-force channel-add (1 for
                          brute force; < 1 for the pattern-factored kernel: pattern builds + per-trial adds) */
} fdd_kernel_config;

/* Number of compiled dedispersion kernel variants (valid variant indices are
 * 0 .. n-1).  *bytes_per_sample of variant v is 1 (native-rate ranges) or 2
 * (downsampled ranges); *group is 0 for brute-force variants and the channel
 * group size G of pattern-factored variants (exact: within a block of
 * trials, channel groups with equal relative delays share one partial sum;
 * native-rate ranges only).  Any output pointer may be NULL. */
int fdd_num_variants(int32_t* n);
/* Kind of variant v: 0 brute force; 1 pattern-factored (native-rate ranges);
 * 2 SB-factored (plans with >= 2 SBs: per DM-trial slab, every TAB is
 * dedispersed over channel segments on which every SB keeps one TAB, and
 * each SB adds the segment partials of the TABs it takes -- exact; the
 * search workspace then holds a scratch of at most 4 GiB for the partials,
 * counted by fdd_workspace_size); 3 SB-factored whose segment partials come
 * from the pattern-factored kernel (native-rate ranges whose channel segments
 * are runs of whole channel groups of size *group; FDD_ERR_UNSUPPORTED
 * from fdd_plan_set_config otherwise). */
int fdd_variant_kind(int32_t variant, int32_t* kind);
int fdd_variant_info(int32_t variant, int32_t* bytes_per_sample, int32_t* dm_per_block, int32_t* tile,
                     int32_t* threads, int32_t* group);

/* Diagnostics: the tables of pattern-factored variant `variant` (a global
 * variant index with *group > 0) for native-rate range r of a plan
 * description, built on the host only (no GPU), for inspection and CPU
 * checks of the kernel's shared-memory addressing.  info[0..14] receives Lw
 * (raw row words; < 0 if the layout does not fit), bytes of one pattern-row
 * buffer, groups, stages, ints per descriptor, shared-memory bytes,
 * descriptors, DM blocks, then the byte offsets (from the kernel's
 * 128-byte-aligned shared-memory base) of the zero row, the raw-row buffers,
 * one raw slot's size, the pattern region and the two mbarriers, and the
 * number of pattern-row buffers (2: stage s + 1 is built into the other
 * buffer while stage s accumulates; the descriptor and offset tables then
 * hold the buffer's address), and in info[14] the channels per TMA copy R
 * (8 or 4: the rows of R consecutive channels travel as one box of slot-size
 * rows from the box's least staged start, bbase [n_blk][ceil(n_chan / R)], each
 * channel's data shifted by its start's distance to it, as the descriptors
 * record; 1: one copy per row).  Array arguments may be NULL (sizes first, then data): base
 * [n_blk][n_chan], goff [n_blk][n_groups][BD], pdesc [n_desc][desc_ints],
 * pd_idx [n_blk][n_stages][2], delays [n_dm][n_chan]. */
int fdd_fact_tables_host(const fdd_plan_desc* desc, const int16_t* sb_map_host, int32_t range, int32_t variant,
                         int32_t chan_per_stage, int64_t* info, int32_t* base, int32_t* goff, int32_t* pdesc,
                         int32_t* pd_idx, int32_t* delays, int32_t* bbase);

/* Current kernel configuration of range r. */
int fdd_plan_get_config(const fdd_plan* plan, int32_t r, fdd_kernel_config* out);

/* Set range r's kernel variant and channels per stage (0 = largest that
 * fits); rebuilds the range's device tables.  Synchronous.  Errors:
 * INVALID_ARG (variant for the other sample width), UNSUPPORTED (does not
 * fit), NO_MEMORY / CUDA. */
int fdd_plan_set_config(fdd_plan* plan, int32_t r, int32_t variant, int32_t chan_per_stage);

/* Auto-tune every range: time each compatible (variant, channels per stage)
 * on the given chunk, `reps` launches each, and keep the fastest.  Arguments
 * as fdd_search; the workspace must be sized with_series = 1.  Synchronous
 * (returns after the stream has drained); results are reproducible only up
 * to timing noise. */
int fdd_plan_autotune(fdd_plan* plan, const uint8_t* d_tabs, int64_t n_in, int64_t pitch, int64_t n_out,
                      void* d_workspace, size_t workspace_bytes, int32_t reps, fdd_stream_t stream);

/* ---------------------------------------------------------------------
 * Batched search (the paper runs one AMBER instance per DM range on each of
 * three GPUs per compound beam, Sec. "Computing performance"; here one GPU
 * searches many chunks, all ranges and all SBs in one persistent launch).
 * One job = one chunk of one compound beam; all jobs of a batch share the
 * plan and n_out. */
typedef struct {
    const uint8_t* d_tabs;    /* device uint8 [n_tab][n_chan][pitch], 16-byte aligned */
    int64_t n_in;             /* samples of data per row, >= n_out + max delay */
    int64_t pitch;            /* multiple of 16 */
    int64_t t_offset_native;  /* added to the job's candidate t_native */
    void* d_workspace;        /* >= fdd_workspace_size(plan, n_in, n_out, d_series == NULL), 256-aligned */
    size_t workspace_bytes;
    fdd_candidate* d_cands;   /* device [cap] */
    int64_t cap;
    uint64_t* d_count;        /* device: true candidate count of this job */
    int32_t* d_series;        /* NULL, or fdd_series_size() bytes for this job's series */
    int32_t bins_absolute;    /* 0: as fdd_search; 1: as fdd_search_window (t_offset_native is the
                                 window's stream position; workspace and series sized by
                                 fdd_window_sizes).  All jobs of a batch share the mode. */
} fdd_job;

/* Batch variant value selecting SB-factored mode: instead of the persistent
 * launches, every job's ranges run their SB-factored kernels (2 launches per
 * DM slab per range per job), with each range's SB-factored configuration
 * (set where a range has none).  Plans with >= 2 SBs only. */
#define FDD_BATCH_SB_FACTORED 1000

/* Batch variant value selecting persistent SB-factored mode: ONE launch runs
 * the SB-factored part and combine work of every job, range and DM slab
 * (blocks take tasks in an order in which each task depends only on earlier
 * ones; a job's scratch holds three slab buffers used in turn), then one
 * boxcar launch.  Same results as FDD_BATCH_SB_FACTORED.  Plans with >= 2
 * SBs whose scratch (fdd_plan_set_scratch_limit) holds three slabs of 32 DM
 * trials of every range; FDD_ERR_UNSUPPORTED otherwise. */
#define FDD_BATCH_SB_PERSISTENT 1001

/* Prepare the plan's batched tables for chunks of n_out native samples with
 * persistent-kernel variant `variant` (-1: keep the current, possibly tuned,
 * configuration; variant 0 if none; FDD_BATCH_SB_FACTORED: SB-factored mode).
 * Allocates and synchronises; must precede any capture of fdd_search_batch.
 * Errors: UNSUPPORTED (more than FDD_MAX_RANGES ranges or 4 distinct D). */
int fdd_batch_prepare(fdd_plan* plan, int64_t n_out, int32_t variant);

/* Search n_jobs (1..FDD_MAX_BATCH_JOBS) chunks in at most five launches:
 * prep, downsample, persistent dedispersion over every (job, range, SB, DM
 * block, time tile) -- one launch for the native-rate ranges and one for the
 * downsampled ranges -- and one boxcar/threshold launch.  Results per job are
 * identical to fdd_search on that job alone.  Prepares on first use of an
 * n_out (not allowed while the stream is capturing).  In the persistent
 * modes, batched searches of one plan must not overlap on the GPU (they share
 * the plan's work counters); SB-factored batches of one plan may run at the
 * same time on different streams (the serving runtime overlaps them).
 * In SB-factored mode the part / combine launches of the range with the most
 * trial-samples run on one library-owned side stream and those of the other
 * ranges on a second (a pair per caller stream, created on first use and
 * freed with the plan), forked from and joined back into `stream` before the
 * boxcar launch: `stream` still orders the whole search, and a CUDA graph
 * captured from it holds the two branches. */
int fdd_search_batch(fdd_plan* plan, const fdd_job* jobs, int32_t n_jobs, int64_t n_out, fdd_stream_t stream);

/* Time every persistent variant on these jobs (`reps` batches each) and, for
 * plans with >= 2 SBs, SB-factored mode with each range's SB-factored
 * variant chosen greedily; keep the fastest.  Synchronous.  Ranges keep
 * their previous per-range configuration unless SB-factored mode wins. */
int fdd_batch_autotune(fdd_plan* plan, const fdd_job* jobs, int32_t n_jobs, int64_t n_out, int32_t reps,
                       fdd_stream_t stream);

/* Current persistent configuration: variant, resident grid, threads per
 * block, DM trials per block, tuned batch time (ms, 0 if untuned).  In
 * SB-factored mode: variant FDD_BATCH_SB_FACTORED, grid/threads/dm 0. */
int fdd_batch_config(const fdd_plan* plan, int32_t* variant, int32_t* grid, int32_t* threads,
                     int32_t* dm_per_block, float* tuned_ms);

/* A CUDA graph of fdd_search_batch for fixed jobs (no counterpart in the
 * paper; launch-overhead removal for the batched search): create captures and
 * instantiates it; launch replays it on a stream; update re-captures for new
 * job buffers/offsets (same n_jobs) and updates the executable graph in
 * place; destroy frees it.  The plan must outlive the graph.  Graphs carry
 * no stage-timing events (time a graph launch as a whole). */
typedef struct fdd_graph fdd_graph;
int fdd_graph_create(fdd_plan* plan, const fdd_job* jobs, int32_t n_jobs, int64_t n_out, fdd_graph** out);
int fdd_graph_update(fdd_graph* graph, const fdd_job* jobs, int32_t n_jobs);
int fdd_graph_launch(fdd_graph* graph, fdd_stream_t stream);
int fdd_graph_destroy(fdd_graph* graph);

/* ---------------------------------------------------------------------
 * Serving runtime (the paper's real-time operation: every compound beam's
 * 1.024 s chunks are searched as they arrive, each output needing the next
 * max-delay of input; Sec. "AMBER", Sec. "Computing performance").
 * One server, one plan, many beams.  Per beam the server keeps two device
 * window buffers of n_in samples (fdd_window_sizes, rounded up to whole chunks);
 * a complete window is queued; "slots" (workspace + candidate buffers) are
 * allocated once from free HBM; fdd_server_poll launches every queued
 * window that finds a free slot as one batched search (continuous
 * batching), retires finished ones and copies their candidates to host.
 * Window w of a beam searches, like fdd_search_window, the outputs whose
 * first native sample lies in [w*chunk, (w+1)*chunk) with downsampling bins
 * aligned to the beam's stream (t_native of its candidates is absolute), and
 * is complete once the chunk holding its last needed sample (n_in of
 * fdd_window_sizes) has arrived. */
typedef struct fdd_server fdd_server;

typedef struct {
    int32_t n_beams;           /* compound beams */
    int64_t chunk_len;         /* native samples per arriving chunk (12500 in ARTS) */
    int32_t max_slots;         /* cap on in-flight windows; 0 = as many as HBM allows */
    double hbm_reserve_frac;   /* part of free HBM left unused, in [0, 1) */
    int64_t hbm_budget_bytes;  /* > 0: treat free HBM as at most this (admission tests) */
    int64_t cap_per_window;    /* candidate records kept per window */
} fdd_server_desc;

typedef struct {
    int32_t beam;
    int64_t window;            /* window index of the beam */
    int64_t t0_native;         /* first output sample (absolute) */
    double t_arrival;          /* caller's arrival time of the completing chunk (fdd_now clock) */
    double t_ready;            /* window queued */
    double t_launch;           /* window launched */
    double t_done;             /* results seen by fdd_server_poll */
    int64_t n_cands;           /* true candidate count */
    int64_t n_cands_kept;      /* records returned (<= cap_per_window) */
    int64_t cand_offset;       /* offset of this window's records in the candidate array */
    int32_t batch_jobs;        /* windows in the batch it ran in */
} fdd_window_result;

typedef struct {
    int32_t n_slots, slots_busy, queued;
    int64_t max_queued, launched, done, batches;
    int64_t window_len;        /* input samples per window */
    int64_t ring_bytes_per_beam, slot_bytes;
} fdd_server_stats;

/* Monotonic clock (seconds) used for all server timestamps (no counterpart in
 * the paper). */
double fdd_now(void);

/* Create a server.  Allocates every beam's buffers, then slots from free HBM
 * (FDD_ERR_NO_MEMORY if not even one slot fits: admission refused), and
 * prepares the plan's batched search for chunk_len. */
int fdd_server_create(fdd_plan* plan, const fdd_server_desc* desc, fdd_server** out);
int fdd_server_destroy(fdd_server* server);

/* Switch a new server (before its first push) to the plain per-SB path, the
 * comparison point of the batched one: every window is searched by n_sb
 * single-SB plans, one fdd_search each, one after another on one stream,
 * one window per launch group (windows still overlap across the server's
 * compute streams); plan k searches SB k (its records are relabelled sb = k,
 * appended to the window's list, the true total counted).  sb_plans: n_sb =
 * the server plan's SB count, each with n_sb = 1, the same TABs and channels
 * and no larger max delay; they must outlive the server.  Errors:
 * INVALID_ARG, WORKSPACE (a plan needs more workspace than a slot holds),
 * CUDA. */
int fdd_server_set_plain(fdd_server* server, fdd_plan* const* sb_plans, int32_t n_sb);

/* Deliver chunk `seq` (0, 1, 2, ... per beam) of `beam`: host memory
 * uint8 [n_tab][n_chan][chunk_len] (pinned for asynchronous copies; it may be
 * reused once the call returns only if pageable).  FDD_ERR_SEQUENCE for a
 * dropped/late/duplicate/reordered chunk (state unchanged); FDD_ERR_BUSY if
 * the beam's previous window still waits for a slot (call fdd_server_poll,
 * then retry). */
int fdd_server_push(fdd_server* server, int32_t beam, int64_t seq, const uint8_t* host_chunk, double t_arrival);

/* Drop a beam's partial window and expect chunk next_seq next (after a gap). */
int fdd_server_reset_beam(fdd_server* server, int32_t beam, int64_t next_seq);

/* Retire finished searches and launch queued windows on free slots.  Never
 * blocks. */
int fdd_server_poll(fdd_server* server);

/* Poll until nothing is queued or running (blocks). */
int fdd_server_drain(fdd_server* server);

/* Hand out finished windows in completion order: up to max_results records
 * and their candidates (at most cands_cap records in total). */
int fdd_server_results(fdd_server* server, fdd_window_result* out, int32_t max_results, fdd_candidate* cands,
                       int64_t cands_cap, int32_t* n_results, int64_t* n_cands);

int fdd_server_info(const fdd_server* server, fdd_server_stats* stats);

/* ---------------------------------------------------------------------
 * Per-beam streaming search (the paper's real-time search of one compound
 * beam: every 1.024 s chunk is searched with the following max delay of
 * data appended; Sec. "AMBER", Sec. "Computing performance").  The caller
 * pushes the beam's chunks from DEVICE memory in order; the stream keeps the
 * delay overlap in two device buffers of ceil((chunk + max delay) / chunk)
 * chunks each (owned by the stream, freed by fdd_stream_close) and searches
 * window w -- the outputs whose first native sample lies in
 * [w*chunk, (w+1)*chunk), candidate t_native absolute -- with
 * fdd_search_window (downsampling bins aligned to the beam's stream, so the
 * windows tile one search of the whole stream) as soon as its last needed
 * chunk is pushed (window 0 after chunk ceil(n_in / chunk) - 1 with n_in
 * from fdd_window_sizes, then one window per chunk).  For many beams on one GPU with batching and admission control,
 * use the fdd_server_* runtime below.  Not thread-safe per stream object. */
typedef struct fdd_stream fdd_stream;

/* Open a stream for compound beam beam_id (a label used in error messages)
 * with chunks of chunk_len native samples; cap = candidate records kept per
 * window.  Allocates the buffers, a search workspace and the candidate
 * buffer on the current device.  Errors: INVALID_ARG, CUDA (allocation). */
int fdd_stream_open(fdd_plan* plan, int32_t beam_id, int64_t chunk_len, int64_t cap, fdd_stream** out);

/* Push chunk `seq` (0, 1, 2, ...): device uint8 [n_tab][n_chan] rows of
 * chunk_len samples at chunk_pitch bytes (>= chunk_len, any alignment).
 * Enqueues on `stream` the copy into the stream's buffer and, when the push
 * completes a window, that window's search and the carry of its overlap;
 * the chunk buffer may be reused once those have run.  A push is ordered
 * after the previous push of the same object even on another CUDA stream.
 * Errors: SEQUENCE (seq is not the next chunk; nothing enqueued),
 * INVALID_ARG, CUDA. */
int fdd_stream_push(fdd_stream* st, const uint8_t* d_chunk, int64_t chunk_pitch, int64_t seq, fdd_stream_t stream);

/* (No counterpart in the paper: window assembly for a caller that streams
 * chunks into its own window buffers.)  Enqueue on `stream` a copy of `rows`
 * rows of `width` bytes from src (row r at src + r * src_pitch) to dst (row
 * r at dst + r * dst_pitch); either side may be device or page-locked host
 * memory (the direction follows from the pointers).  Runs on a copy engine,
 * not on the SMs.  Errors: INVALID_ARG (null pointer, negative size, a
 * pitch below the width), CUDA. */
int fdd_copy_rows(void* dst, int64_t dst_pitch, const void* src, int64_t src_pitch, int64_t width, int64_t rows,
                  fdd_stream_t stream);

/* Results of the window searched last, if no fdd_stream_results call has
 * taken them yet: enqueues, on the CUDA stream of the last push, a copy of
 * the first min(true count, cap, stream cap) candidate records to device
 * d_cands and of the window's TRUE candidate count to device *d_count, and
 * sets host *t0_native to the window's first output sample.  With no new
 * window, enqueues nothing and sets *t0_native = -1.  Each window that
 * completes replaces the previous window's results: call after every push
 * to see every window. */
int fdd_stream_results(fdd_stream* st, fdd_candidate* d_cands, int64_t cap, uint64_t* d_count, int64_t* t0_native);

/* Wait for the stream's last push, free everything it owns.  NULL accepted. */
int fdd_stream_close(fdd_stream* st);

/* Host helper (no counterpart in the paper; the records are those of
 * Sec. "DARC"): sort n host candidate records in place by (sb, dm_index,
 * width_native, t_native), the order used to compare candidate sets (the
 * search itself emits them in no particular order). */
int fdd_sort_candidates(fdd_candidate* cands, int64_t n);

/* DM-width clustering of a candidate list (Sec. "AMBER", "Clustering
 * (optional)"): among candidates of one SB at the same time (t_native) and
 * DM trial, keep the highest S/N over widths; then every group of
 * neighbouring DM trials (consecutive dm_index, no gap, possibly across a
 * DM-range boundary) at that SB and time keeps only its highest-S/N
 * candidate.  Ties keep the smaller width, then the earlier record of the
 * input list (step 1), and the smaller dm_index (step 2).
 *   d_in, d_in_count  device candidate list as written by fdd_search: the
 *                     first min(*d_in_count, cap_in) records are clustered.
 *   d_workspace       >= fdd_cluster_workspace_size(cap_in) bytes, 16-byte
 *                     aligned (a hash table of about 48 * cap_in bytes).
 *   d_out, cap_out    device output records (order unspecified); *d_out_count
 *                     receives the TRUE number kept (> cap_out: overflow, the
 *                     first cap_out written).
 * Records with sb >= 8192, dm_index >= 2^21, or t_native more than 2^30 - 2
 * samples after the list's earliest are passed through unclustered.
 * Asynchronous on stream (five small launches).  cap_in <= 2^31.
 * Errors: INVALID_ARG, MISALIGNED, WORKSPACE, CUDA. */
int fdd_cluster_workspace_size(int64_t cap_in, size_t* bytes);
int fdd_cluster(const fdd_candidate* d_in, const uint64_t* d_in_count, int64_t cap_in, void* d_workspace,
                size_t workspace_bytes, fdd_candidate* d_out, int64_t cap_out, uint64_t* d_out_count,
                fdd_stream_t stream);

/* Two-step subband dedispersion for range r (APPROXIMATE; the paper's AMBER
 * can dedisperse "using a more efficient two step process including
 * subbanding", Sec. "AMBER", "Dedispersion"; Table "dedispersion setup": 32
 * subbands, subbanding DM step 32x the fine step).  Subbands of
 * chan_per_subband channels are first aligned to their top channel at the
 * midpoint DM of each block of dm_per_coarse fine trials, then the subbands
 * are aligned at every fine DM:
 *   d1[q][c] = llround(K*DMc_q*(f_c^-2 - f_b^-2)/(D t)),
 *   d2[i][b] = llround(K*DM_i*(f_b^-2 - f_top^-2)/(D t)),
 *   S[s][i][t] = sum_b sum_{c in b} y[tab(s,b)][c][t + d2[i][b] + d1[i/K'][c]]
 * (f_b = top channel of subband b, DMc_q = dm0 + (q K' + (K'-1)/2) ddm,
 * K' = dm_per_coarse).  About (n_chan/K' + n_sub) adds per trial and sample
 * instead of n_chan; S/N of pulses narrower than the intra-subband smearing
 * drops.  The SB map must keep one TAB per subband (FDD_ERR_UNSUPPORTED
 * otherwise); chan_per_subband <= 64 and <= 65535 / (255 D).  Applies to
 * fdd_search, fdd_search_static and streams; batched searches refuse plans
 * with a range in this mode.  May raise fdd_plan_max_delay and
 * fdd_workspace_size (re-query after the call).  chan_per_subband = 0
 * restores exact dedispersion. */
int fdd_plan_set_subband(fdd_plan* plan, int32_t r, int32_t chan_per_subband, int32_t dm_per_coarse);
int fdd_plan_get_subband(const fdd_plan* plan, int32_t r, int32_t* chan_per_subband, int32_t* dm_per_coarse);

/* (No counterpart in the paper: failure reporting of the device-side waits.)
 * Device status word of the plan, read with a blocking copy after the
 * searches it covers have been synchronised (clear != 0 resets it).  Bit 0
 * (FDD_STATUS_TILE_WAIT): a kernel's wait for an asynchronous tile copy
 * gave up after its poll limit (about a second); that block stopped without
 * writing its series, so the affected search's output is incomplete.  0 in
 * normal operation.  Returns FDD_ERR_TIMEOUT (with *status filled) when the
 * word is not 0, FDD_OK when it is: this is how device-side wait failures
 * reach a caller that checks return codes, since searches are asynchronous. */
#define FDD_STATUS_TILE_WAIT 1
int fdd_plan_status(fdd_plan* plan, int32_t* status, int32_t clear);

/* Self-test of the bounded wait that every TMA-staged kernel uses for its
 * tile copies (the paper has no counterpart): one block waits on an
 * mbarrier that nothing arrives on, giving up after `polls` polls (1 ..
 * 2^22; each poll after the 64th sleeps ~256 ns).  *gave_up = 1 when the
 * wait ended by its limit and the kernel returned normally, which is the
 * expected outcome.  Blocking; uses the current device. */
int fdd_selftest_bounded_wait(int32_t polls, int32_t* gave_up);

/* (Tracing; no counterpart in the paper.)  Number of kernels the last
 * fdd_search or fdd_search_batch on this plan
 * enqueued (graph launches replay the last captured batch's kernels). */
int fdd_plan_last_launches(const fdd_plan* plan, int64_t* n);

/* (No counterpart in the paper: a memory knob of the SB-factored kernels.)
 * Cap (bytes) on the scratch the SB-factored kernel keeps in the search
 * workspace for its partial sums (0 = default, 4 GiB).  The partials of a
 * slab of DM trials must fit: a smaller cap means smaller slabs and more
 * launches, never a different result; at least one DM block's worth is
 * always reserved.  Changes fdd_workspace_size for plans with >= 2 SBs. */
int fdd_plan_set_scratch_limit(fdd_plan* plan, int64_t bytes);

/* Per-stage GPU timing (tracing; the paper reports AMBER's time per stage,
 * Sec. "Computing performance").  With timing enabled, fdd_search records a
 * CUDA event pair around every kernel it enqueues; the pairs are reused by
 * the next search.  Enabling creates the events on the current device. */
int fdd_plan_set_timing(fdd_plan* plan, int32_t enable);

/* Elapsed time of each stage of the last timed fdd_search on this plan,
 * in enqueue order (also of the last batched search or graph launch).  Call
 * after that search's stream has been synchronised (FDD_ERR_CUDA "not ready"
 * otherwise).  For stage k: kind[k] = 0 downsample, 1 SB-gather +
 * dedispersion, 2 boxcar S/N + threshold, 3 batch prep; range[k] = DM range
 * index (downsample: its factor D; batched stages: -1); ms[k] milliseconds.
 * Writes min(max_n, stages) entries; *n_stages receives the stage count. */
int fdd_plan_stage_times(fdd_plan* plan, int32_t max_n, int32_t* kind, int32_t* range, float* ms,
                         int32_t* n_stages);

/* Allocation-free search (no counterpart in the paper: it exists for callers
 * of this library that cannot allocate device memory at search time -- a
 * real-time thread that must not block in the CUDA allocator, a process whose
 * GPU memory is granted by an external arbiter only at start-up, code
 * certified to allocate only during initialisation).
 * Same as fdd_search, except that the workspace is a file-scope device array
 * of FDD_STATIC_SCRATCH_BYTES inside the library instead of a caller buffer;
 * the caller still passes inputs, candidates, counter and optional series.
 *   - The call makes no cudaMalloc/cudaFree and calls no allocating routine.
 *     Stage timing must be off on the plan (it creates CUDA events), else
 *     FDD_ERR_INVALID_ARG.
 *   - Every call resolves the array's device address with
 *     cudaGetSymbolAddress on the current device.  The library's device code
 *     is loaded per device on first use, so the FIRST call on a device loads
 *     this array's module and commits the FDD_STATIC_SCRATCH_BYTES there (it
 *     can fail for lack of memory); make that first call at initialisation,
 *     before any stream capture.  Later calls allocate nothing.
 *   - Searches whose fdd_workspace_size(..., d_series == NULL) exceeds
 *     FDD_STATIC_SCRATCH_BYTES return FDD_ERR_WORKSPACE with a message.
 *   - All calls on a device share the one array, which keeps the previous
 *     call's contents (the call re-zeroes what must start at zero).  Calls
 *     whose GPU work overlaps (other streams, other host threads) race on it:
 *     serialise them.
 *   - Once committed on a device, the array stays until the process exits. */
#define FDD_STATIC_SCRATCH_BYTES (64u * 1024u * 1024u)
int fdd_search_static(fdd_plan* plan, const uint8_t* d_tabs, int64_t n_in, int64_t pitch, int64_t n_out,
                      int64_t t_offset_native, fdd_candidate* d_cands, int64_t cap, uint64_t* d_count,
                      int32_t* d_series, fdd_stream_t stream);

/* SB table from the array geometry (appendix "Tied-array beam simulations",
 * "Synthesized Beams"): host int16 sb_map_out[n_sb][n_chan] (the plan's SB
 * map), entry = TAB row n_TAB + n_tab/2 with n_TAB in [-n_tab/2, n_tab/2 - 1].
 * SB s has index n_SB = s - n_sb/2 (0 = compound-beam centre); at f_max it
 * takes TAB n_TAB = n_SB mod N (less N above N/2 - 1) of grating response
 * n_gr = (n_SB - n_TAB)/N, and below f_max it switches to the neighbouring TAB
 * k_{j+1} = k_j - sgn(n_SB) between the frequencies f_j at which successive TABs
 * land on the SB's position, f_j = f_max (n_gr B_max + k_j alpha B_cq) /
 * (n_gr B_max + n_TAB alpha B_cq), at 0.75 f_j + 0.25 f_{j+1} (even |n_SB|) or
 * 0.25 f_j + 0.75 f_{j+1} (odd).  chan_per_subband > 1 makes every block of
 * that many channels take the TAB chosen at the block's mean frequency (the
 * system combines TABs in whole subbands).  Apertif-10: n_tab 12, alpha 0.80,
 * B_max 1296 m, B_cq 144 m, f_max 1500 MHz, 71 SBs.  Host only; needs no GPU.
 * Errors: INVALID_ARG (odd n_tab among others). */
int fdd_sb_table(int32_t n_tab, int32_t n_sb, int32_t n_chan, const double* chan_freq_mhz, double f_max_mhz,
                 double alpha, double b_max_m, double b_cq_m, int32_t chan_per_subband, int16_t* sb_map_out);

/* RFI mitigation on TAB filterbanks, IN PLACE (Sec. "AMBER", "RFI mitigation
 * (optional)": a time-domain filter for bright wide-band low-DM RFI and a
 * frequency-domain filter for bright narrowband RFI, each applied
 * iteratively -- three iterations each in ARTS, Sec. "Fraction of data lost
 * to RFI").  The paper leaves the statistics to another publication; here,
 * per TAB:
 *   time domain: z[t] = sum_c x[c][t]; each iteration flags unflagged t with
 *     z[t] - mu > time_thresh * sigma (mu, sigma over unflagged samples);
 *     flagged samples of every channel become the channel's mean over the
 *     unflagged samples, rounded half up;
 *   frequency domain (after it): b[c] = sum_t x[c][t]; each iteration flags
 *     unflagged channels with |b[c] - mu| > freq_thresh * sigma; flagged
 *     channels are filled with the unflagged channels' mean level, rounded
 *     half up.
 * mu = S1/n, var = S2/n - mu^2, sigma = sqrt(var) in FP64 from exact 64-bit
 * sums (the population standard deviation; equal to the exact
 * sqrt((n S2 - S1^2)/n^2) to ~1e-11 relative, so a decision can differ from
 * one taken with the exact numerator only for a value that sits on the
 * threshold).  A threshold <= 0 disables that filter.  Run before fdd_search. */
typedef struct {
    double time_thresh;   /* sigmas, zero-DM filter (e.g. 4); <= 0: off */
    int32_t time_iters;   /* 3 in ARTS */
    double freq_thresh;   /* sigmas, channel filter (e.g. 4); <= 0: off */
    int32_t freq_iters;   /* 3 in ARTS */
} fdd_rfi_desc;

/* Workspace bytes of fdd_rfi_clean for n_tab x n_chan x n_in. */
int fdd_rfi_workspace_size(int32_t n_tab, int32_t n_chan, int64_t n_in, size_t* bytes);

/* d_tabs: device uint8 [n_tab][n_chan][pitch], first n_in samples per row
 * cleaned in place (16-byte aligned, pitch a multiple of 16).  d_time_flags
 * (device uint8 [n_tab][n_in]) and d_chan_flags ([n_tab][n_chan]) receive 1
 * for flagged samples / channels; either may be NULL.  Asynchronous on
 * stream.  Errors: INVALID_ARG, MISALIGNED, WORKSPACE, UNSUPPORTED (moments
 * would not fit 64 bits), CUDA. */
int fdd_rfi_clean(const fdd_rfi_desc* desc, uint8_t* d_tabs, int32_t n_tab, int32_t n_chan, int64_t n_in,
                  int64_t pitch, void* d_workspace, size_t workspace_bytes, uint8_t* d_time_flags,
                  uint8_t* d_chan_flags, fdd_stream_t stream);

/* Issue-rate probe (no counterpart in the paper; it measures the roofline
 * denominators of this integer shift-and-add path on the current device).
 * Launches blocks_per_sm (1..8) x SMs blocks of 256 threads, each thread
 * running 16 independent dependency chains for `iters` (1..2^30) loop
 * iterations of 4 rounds, once for warm-up and once timed with CUDA events.
 *   kind 0: chains of a = a + b + c (32-bit): *per_second = integer adds/s
 *           (two adds per three-input add);
 *   kind 1: chains of byte permutes (ALU pipe only): *per_second = permutes/s;
 *   kind 2: conflict-free 32-bit shared-memory loads: *per_second = bytes
 *           loaded/s;
 *   kind 3: chains of a = a * b + c (32-bit): *per_second = adds/s (one per
 *           multiply-add);
 *   kind 4: three-input-add and multiply-add chains interleaved one to one:
 *           *per_second = adds/s of both integer pipes together.
 * *ms receives the timed launch's duration, *n_sm (may be NULL) the SM count.
 * Blocking; allocates a 4-byte device word.  Errors: INVALID_ARG, CUDA. */
int fdd_probe_issue_rate(int32_t kind, int32_t blocks_per_sm, int64_t iters, double* per_second, float* ms,
                         int32_t* n_sm);

/* Human-readable text of an FDD_* code (static string; no counterpart in the paper). */
const char* fdd_error_string(int code);

/* Text of the last CUDA error seen by this thread inside the library (no
 * counterpart in the paper). */
const char* fdd_last_error_message(void);

/* Library version string (no counterpart in the paper). */
const char* fdd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FDD_H */
