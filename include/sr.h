/*
 * sr.h — C ABI of the GB300 (sm_103a) device-wide sum reduction library.
 *
 * The operation is the case study of Zhang, Wahib, Zhang and Matsuoka, "A
 * Study of Single and Multi-device Synchronization Methods in Nvidia GPUs"
 * (arXiv 2004.05371), Section VII: summing the elements of an array,
 * S = sum_{i<n} x_i, computed by stages joined by a barrier at each level of
 * the GPU hierarchy (Section III-A): per-thread accumulation (Fig.
 * "Basic function of device wide reduction", summing()), a warp shuffle tree
 * (Section VII-D, Table V), a shared-memory block tree joined by the block
 * barrier (block_reduce(), same figure), a thread-block-cluster merge through
 * distributed shared memory (sm_90+; no counterpart in the paper), and a grid
 * stage in one of the forms the paper compares (Section VII-E): the implicit
 * kernel-boundary barrier of a two-kernel reduction (Fig. "Code example of
 * reduction with implicit device synchronization"), a cooperative persistent
 * kernel with grid.sync() (Fig. "Code example of reduction with explicit
 * device synchronization"), plus two non-barrier finishes (atomics, and a
 * __threadfence last-block-done ticket).
 *
 * Conventions for every entry point:
 *  - Pointers named x, offsets, out are DEVICE pointers owned by the caller;
 *    the library never frees or retains them past the call.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Reductions are
 *    stream-ordered and asynchronous: `out` is valid once the stream has
 *    reached the end of the call's work (e.g. after cudaStreamSynchronize).
 *  - The library owns a small workspace per (device, stream) pair (partials,
 *    ticket counters, an error word).  It is allocated with cudaMalloc on the
 *    first call that uses that pair, so the first call on a stream must not be
 *    made while the stream is being captured into a CUDA graph.  Calls on
 *    different streams never share a workspace.
 *  - Arguments are validated before anything is launched; an invalid call
 *    returns an error status and launches nothing.
 *  - Return value: an sr_status.  SR_ERR_CUDA means a CUDA runtime call failed;
 *    sr_last_cuda_error() returns its cudaError_t for the calling thread.
 *  - No entry point falls back to the CPU.
 */
#ifndef SR_H
#define SR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* sr_stream_t; /* identical to cudaStream_t */

/* ------------------------------------------------------------ enums */

typedef enum {
    SR_F32 = 0,      /* binary32 in, binary32 out (binary64 with SR_F_FP64_COMBINE) */
    SR_I32 = 1,      /* int32 in, int64 out, exact (bit-exact with the definition) */
    SR_BF16 = 2,     /* bfloat16 in, binary32 accumulation and out */
    SR_FP8E4M3 = 3   /* FP8 E4M3 (OCP E4M3FN) codes in, binary32 accumulation;
                        the result is multiplied once by sr_config.scale */
} sr_dtype;

/* Grid stage: bits 0-3 of a variant. */
typedef enum {
    SR_AUTO = 0,           /* library chooses stage, cluster and launch shape */
    SR_TWO_KERNEL = 1,     /* implicit barrier: kernel 1 writes one partial per unit,
                              kernel 2 (one block) reduces them (Section III-B-2, VII-E) */
    SR_ATOMIC = 2,         /* each unit atomically adds its partial into out (out is
                              zeroed first by a one-line kernel on the same stream);
                              FP order is not deterministic */
    SR_LAST_BLOCK = 3,     /* partial store, __threadfence, ticket; the last unit to
                              arrive reduces all partials (one kernel, no spin) */
    SR_GRID_SYNC = 4,      /* cooperative persistent kernel: partials, grid.sync(),
                              block 0 reduces (Section III-A-3, VII-E) */
    SR_SINGLE_CLUSTER = 5  /* one cluster (or one CTA) covers the whole array: no grid
                              stage at all; for small n */
} sr_stage;

#define SR_STAGE_MASK 0xF
/* Cluster size of a unit, bits 4-6: 0 -> 1 CTA per unit (no cluster stage),
 * k in 1..4 -> 2^k CTAs per cluster, merged through distributed shared
 * memory before the grid stage.  16 uses the non-portable cluster size. */
#define SR_CLUSTER_SHIFT 4
#define SR_CLUSTER_MASK 0x70
#define SR_CLUSTER(log2c) (((log2c) & 7) << SR_CLUSTER_SHIFT)
/* Flags. */
#define SR_F_KAHAN 0x100        /* two-sum compensated accumulation, (sum, correction)
                                   pairs carried through every tree level */
#define SR_F_FP64_COMBINE 0x200 /* unit partials converted to binary64 and combined in
                                   binary64; `out` is then a double */
#define SR_F_BULK 0x400         /* load path: TMA bulk copies (cp.async.bulk) into a
                                   shared-memory ring instead of 128/256-bit LDG */
#define SR_F_FP64_AUTO 0x1000   /* compensated accumulation (implies SR_F_KAHAN) whose
                                   cross-unit combine switches to binary64 only when the
                                   binary32 pair combine's error bound (units * 2^-48 *
                                   sum|unit partials|) could exceed 1e-6 |S|; `out`
                                   stays binary32.  Ignored under SR_F_FP64_COMBINE.
                                   Single-array stages with a cross-unit combine
                                   (two-kernel, last-block, grid-sync); not segmented. */
#define SR_F_DENSE_SEGMENTS 0x2000 /* segmented only: rows of vectors in which three or
                                   more segments end are resolved in one warp-wide
                                   segmented scan instead of one warp reduction per
                                   segment (4.6-6.6x faster at 16-element segments,
                                   1.6-1.9x at 64); up to 17 % slower where few rows
                                   qualify.  512-thread CTAs by default; runs at most 4 rows in
                                   flight per warp (unroll 8 is lowered to 4; sr_plan_
                                   segmented reports it).  Same results contract. */
#define SR_F_WARP_SEGMENTS 0x4000 /* segmented only: each warp sums whole segments
                                   (blocks of up to 32 consecutive segments per warp,
                                   one coalesced offsets load per block, one warp
                                   reduction and one store per segment).  No segment
                                   crosses a warp, so the grid stage is not used and
                                   nothing is zeroed or finished; deterministic.  For
                                   many segments with no very long one: a long segment
                                   is summed by one warp alone.  Segments go in pairs,
                                   both first batches of loads in flight together; a
                                   batch is `unroll` 16/32-byte vectors per lane
                                   (default 16 bytes x 2; unroll 1/2/4/8).  Segments of
                                   at most 512 bytes are summed by a single lane.  Not
                                   with another form flag (SR_ERR_UNSUPPORTED).  The
                                   paper has no counterpart. */
#define SR_F_LANE_SEGMENTS 0x8000 /* segmented only: each thread sums whole segments
                                   alone (thread t takes segments t, t + T, ...), so a
                                   warp covers 32 consecutive segments with coalesced
                                   offsets and results; vector loads of each segment's
                                   aligned body (vec_bytes 16/32, default 16), `unroll`
                                   (1/2/4/8, default 4) per step.  For very short segments.  No grid stage;
                                   deterministic.  Not with another form flag
                                   (SR_ERR_UNSUPPORTED).  The paper has no counterpart. */
#define SR_F_ADAPTIVE_SEGMENTS 0x10000 /* segmented only: one cooperative launch for any
                                   layout.  The segments are partitioned by length on the
                                   device: segments of at most 512 bytes are summed by
                                   single lanes, longer ones up to one chunk by whole warps
                                   (as SR_F_WARP_SEGMENTS), and each longer segment is cut
                                   into chunks (at least 64 KiB of input, at least 2 x
                                   the total / 98304) queued in the workspace; after
                                   grid.sync() every warp takes chunks from the queue and
                                   the last chunk of a segment to finish combines its
                                   partials in chunk order.  No grid-stage variant is
                                   used; deterministic.  Shape fields other than grid
                                   must be 0 or the defaults (16-byte vectors, unroll 2,
                                   256 threads; else SR_ERR_UNSUPPORTED); an explicit grid
                                   that cannot be co-resident -> SR_ERR_LAUNCH.  Not with
                                   another form flag.  The paper has no counterpart (its
                                   grid.sync, Section III-A-3, joins the two phases). */
#define SR_F_HOST_DIRECT 0x800  /* sr_reduce_sum_host only: the kernel reads the host
                                   array in place over the CPU-GPU link (page-locked
                                   memory, or any memory where the device accesses
                                   pageable memory) instead of staging copies */

typedef enum {
    SR_OK = 0,
    SR_ERR_ARG = 1,         /* bad pointer, size, alignment or config value */
    SR_ERR_DTYPE = 2,       /* unknown dtype, or dtype not allowed for this call */
    SR_ERR_LAUNCH = 3,      /* launch shape impossible (e.g. a cooperative grid that
                               cannot be co-resident); nothing was launched */
    SR_ERR_CUDA = 4,        /* a CUDA runtime call failed: see sr_last_cuda_error() */
    SR_ERR_TIMEOUT = 5,     /* a bounded device-side wait expired (reported by
                               sr_stream_status) */
    SR_ERR_UNSUPPORTED = 6  /* valid but unsupported combination of options */
} sr_status;

/* Barrier levels of sr_barrier_bench (Section V, Fig. "Hierarchy of
 * synchronizations in CUDA"; the cluster level is sm_90+ only). */
typedef enum {
    SR_LEVEL_WARP = 0,       /* tile (warp) sync, bar.warp.sync */
    SR_LEVEL_COALESCED = 1,  /* coalesced-group sync over the active lanes */
    SR_LEVEL_BLOCK = 2,      /* __syncthreads */
    SR_LEVEL_CLUSTER = 3,    /* barrier.cluster arrive/wait */
    SR_LEVEL_GRID = 4,       /* cooperative grid.sync() */
    SR_LEVEL_KERNEL = 5,     /* implicit kernel-boundary barrier: launch overhead by
                                the kernel-fusion method (Eq. 6) */
    SR_LEVEL_SHUFFLE = 6,    /* dependent __shfl_xor_sync chain (Table II "Shuffle") */
    SR_LEVEL_FADD = 7,       /* dependent FP32 add chain: the methods' self-check
                                (Section IX-D; 4 cycles on V100, 6 on P100) */
    SR_LEVEL_WARP_REDUCE = 8 /* one warp sums 32 FP64 (or, with SR_WR_FP32, binary32)
                                values by sr_warp_reduce_method (Table V); one "sync"
                                = one whole reduction */
} sr_level;

/* How a warp sums 32 values for SR_LEVEL_WARP_REDUCE (the columns of Table V).
 * The shared-memory trees halve the active lanes (16, 8, 4, 2, 1) with the
 * named synchronisation between steps; the shuffle forms use the group's
 * shfl_down. */
typedef enum {
    SR_WR_SERIAL = 0,            /* lane 0 adds the 32 shared-memory values in order */
    SR_WR_NOSYNC = 1,            /* shared-memory tree, no synchronisation (racy: the
                                    paper reports its result as incorrect) */
    SR_WR_VOLATILE_TILE = 2,     /* volatile shared-memory tree + tile(32).sync() */
    SR_WR_TILE = 3,              /* shared-memory tree + tile(32).sync() */
    SR_WR_COALESCED = 4,         /* shared-memory tree + coalesced_group.sync() */
    SR_WR_TILE_SHUFFLE = 5,      /* tile(32).shfl_down tree */
    SR_WR_COALESCED_SHUFFLE = 6, /* coalesced_group.shfl_down tree */
    SR_WR_FP32 = 16              /* flag: binary32 values instead of Table V's FP64 */
} sr_warp_reduce_method;

/* Launch function measured by SR_LEVEL_KERNEL (Table I's rows; the paper's
 * multi-device cooperative launch no longer exists in CUDA 12+, and the
 * thread-block-cluster launch of sm_90+ takes its place). */
typedef enum {
    SR_LAUNCH_TRADITIONAL = 0,  /* cudaLaunchKernel, the <<<>>> launch */
    SR_LAUNCH_COOPERATIVE = 1,  /* cudaLaunchCooperativeKernel */
    SR_LAUNCH_CLUSTER = 2       /* cudaLaunchKernelEx with a cluster-dimension attribute */
} sr_launch_kind;

/* Launch configuration.  Zero in any field means "library default". */
typedef struct {
    int variant;        /* stage | SR_CLUSTER(k) | flags */
    int block_threads;  /* threads per CTA (multiple of 32, <= 1024) */
    int ctas_per_sm;    /* resident CTAs per SM the grid is sized for */
    int grid;           /* explicit CTA count (overrides ctas_per_sm); rounded up to a
                           multiple of the cluster size */
    int vec_bytes;      /* LDG path: bytes per vector load, 16 or 32 */
    int unroll;         /* LDG path: independent vector loads in flight per thread, 1..8 */
    int tile_bytes;     /* BULK path: bytes per TMA copy / ring stage (multiple of 1024) */
    int stages;         /* BULK path: ring depth, 2..8 */
    float scale;        /* FP8: factor applied once to the final sum (0 -> 1) */
    int reserved[3];
} sr_config;

/* --------------------------------------------------- single-array sum */

/* S = sum_{i<n} x_i (Section VII).  x: device array of n elements of `dtype`,
 * aligned to the element size.  out: device scalar — int64 for SR_I32, float
 * otherwise, double when SR_F_FP64_COMBINE is set.  n == 0 writes 0.
 * Errors: SR_ERR_ARG (n < 0, NULL x with n > 0, NULL out, misaligned x or out),
 * SR_ERR_DTYPE, SR_ERR_LAUNCH, SR_ERR_UNSUPPORTED, SR_ERR_CUDA.
 * variant SR_AUTO leaves the choice to the library: SR_AUTO's own rule, or the
 * variant the environment variable SR_VARIANT names (sr_parse_variant's
 * syntax, read once per process; one that does not parse makes these calls
 * return SR_ERR_ARG). */
int sr_reduce_sum(const void* x, int64_t n, int dtype, void* out, int variant,
                  sr_stream_t stream);

/* End-to-end form: x and out are HOST pointers (x preferably page-locked, e.g.
 * cudaHostAlloc / cudaHostRegister, so copies run asynchronously).  The input
 * is copied to the device in 64 MiB chunks through two library-owned staging
 * buffers on two copy streams, each chunk reduced on `stream` while the next
 * one is copied (the chunk units' partials go to disjoint workspace slots),
 * one final kernel combines all partials in order, and the result is copied
 * back to *out.  Blocks until the result is in *out.  cfg: NULL, or stage
 * SR_AUTO / SR_TWO_KERNEL with optional SR_F_KAHAN / SR_F_FP64_COMBINE and
 * launch-shape fields; other stages or SR_F_BULK -> SR_ERR_UNSUPPORTED.
 * The first call on a stream allocates the staging buffers (128 MiB).
 * With SR_F_HOST_DIRECT there is no staging: one reduction (LDG path, stage
 * SR_LAST_BLOCK) reads x through its device mapping; SR_ERR_UNSUPPORTED when x
 * is neither page-locked nor accessible as pageable memory on this device.
 * Errors: as sr_reduce_sum_ex. */
int sr_reduce_sum_host(const void* x, int64_t n, int dtype, void* out, const sr_config* cfg,
                       sr_stream_t stream);

/* Same with an explicit launch configuration (NULL cfg = the library's
 * choice: SR_AUTO, or the variant SR_VARIANT names as for sr_reduce_sum; a
 * configuration passed in is used as given, SR_VARIANT set or not). */
int sr_reduce_sum_ex(const void* x, int64_t n, int dtype, void* out,
                     const sr_config* cfg, sr_stream_t stream);

/* Synchronise `stream` and report (and clear) device-side error flags raised
 * by this library's kernels on it since the last call: SR_ERR_TIMEOUT when a
 * bounded wait expired, else SR_OK (or SR_ERR_CUDA).  Reporting an error also
 * clears it and resets the stream's tickets, so the next call starts clean;
 * results of the calls before it are void. */
int sr_stream_status(sr_stream_t stream);

/* Synchronise `stream`, then free the library's workspace and host-entry
 * staging buffers for (current device, stream); a later call on the stream
 * allocates them again.  Call it before destroying a stream the library
 * was used on (otherwise they live until the process exits).  Pending
 * error flags of the stream are discarded with the workspace.  A CUDA graph
 * captured from calls on this stream holds pointers into the freed
 * workspace: destroy such graphs first. */
int sr_stream_release(sr_stream_t stream);

/* Resolve the launch shape the library would use for this call on the
 * current device, without launching: fills *resolved (variant with the
 * stage, cluster and load path chosen, block_threads, grid, vec_bytes,
 * unroll, tile_bytes, stages).
 * Needs a device; returns the same errors sr_reduce_sum_ex would.  cfg ==
 * NULL plans the library's choice (SR_VARIANT when set, as sr_reduce_sum_ex). */
int sr_plan(int64_t n, int dtype, const sr_config* cfg, sr_config* resolved);

/* ------------------------------------------------------ segmented sum */

/* Batched sum over CSR segments: out[s] = sum x[offsets[s] .. offsets[s+1])
 * for s < nseg — the paper's reduction (Section VII) applied to many arrays
 * in one launch.  x: device array (element-aligned) holding at least
 * offsets[nseg] elements; offsets: device int64 array of nseg + 1 entries,
 * non-decreasing (the caller guarantees it; it is not checked); out: device
 * array of nseg results (int64 for SR_I32, float, or double with
 * SR_F_FP64_COMBINE).  Empty segments give 0.  nseg == 0 launches nothing.
 * The concatenated range is split evenly over the warps of one persistent
 * grid whatever the segment lengths; segments crossing a warp boundary are
 * finished by the configured grid stage: SR_TWO_KERNEL, SR_GRID_SYNC,
 * SR_LAST_BLOCK (per-segment tickets; the SR_AUTO default for floating-point
 * inputs) or SR_ATOMIC (out zeroed first; FP order not deterministic; the
 * SR_AUTO default for SR_I32, whose int64 sums are exact in any order).  All
 * other forms are deterministic.
 * Load path: rows of 16/32-byte vectors loaded into registers (LDG), or with
 * SR_F_BULK each warp streams its piece through its own ring of `stages`
 * (2..8, default 2) chunks of `unroll` rows (2, 4 or 8; default 4) in shared
 * memory, one cp.async.bulk per chunk (the TMA form; every wait bounded, an
 * expired one reported as SR_ERR_TIMEOUT by sr_stream_status).  Without an
 * explicit shape (vec_bytes, unroll, block_threads and stages all 0) calls
 * with 32768 or more segments take the TMA form, fewer the LDG one.
 * With SR_F_WARP_SEGMENTS whole segments go to single warps instead, with
 * SR_F_LANE_SEGMENTS to single threads (see the flags): no segment is split,
 * the stage bits are ignored and the results are deterministic.  With
 * SR_F_ADAPTIVE_SEGMENTS one cooperative launch partitions the segments by
 * length on the device (lanes, warps, queued chunks; see the flag): the stage
 * bits are ignored and the results are deterministic.
 * cfg fields used: variant (stage, SR_F_KAHAN, SR_F_FP64_COMBINE, SR_F_BULK,
 * SR_F_DENSE_SEGMENTS, SR_F_WARP_SEGMENTS, SR_F_LANE_SEGMENTS, SR_F_ADAPTIVE_SEGMENTS),
 * block_threads (at most 512), ctas_per_sm, grid (at most 65536 warps in
 * total), vec_bytes, unroll, stages (TMA form), scale (FP8).
 * SR_SINGLE_CLUSTER, cluster bits, and any two of SR_F_BULK,
 * SR_F_DENSE_SEGMENTS, SR_F_WARP_SEGMENTS, SR_F_LANE_SEGMENTS and
 * SR_F_ADAPTIVE_SEGMENTS ->
 * SR_ERR_UNSUPPORTED; a ring larger than a CTA's shared memory ->
 * SR_ERR_LAUNCH.
 * Errors: SR_ERR_ARG (nseg < 0, NULL pointer with nseg > 0, misalignment,
 * bad config), SR_ERR_DTYPE, SR_ERR_LAUNCH, SR_ERR_UNSUPPORTED, SR_ERR_CUDA. */
int sr_reduce_sum_segmented(const void* x, const int64_t* offsets, int64_t nseg, int dtype, void* out,
                            sr_stream_t stream);
int sr_reduce_sum_segmented_ex(const void* x, const int64_t* offsets, int64_t nseg, int dtype, void* out,
                               const sr_config* cfg, sr_stream_t stream);

/* The same sum with the offsets checked on the device first: n_elems is the
 * number of elements x holds (x may be NULL when n_elems == 0).  A small
 * kernel verifies offsets[0] >= 0, that every offset is >= its predecessor
 * and offsets[nseg] <= n_elems; if any fails, the summing kernels read
 * nothing (out is left as it was, or zero for SR_ATOMIC without a
 * whole-segment form flag) and the next sr_stream_status(stream) reports
 * SR_ERR_ARG.  The plain entry points trust
 * the caller with this contract; this one costs one extra kernel (8 bytes
 * read per segment).  The paper has no counterpart.  Host-side errors as
 * sr_reduce_sum_segmented_ex, plus SR_ERR_ARG for n_elems < 0 or x == NULL
 * with n_elems > 0. */
int sr_reduce_sum_segmented_checked(const void* x, int64_t n_elems, const int64_t* offsets, int64_t nseg,
                                    int dtype, void* out, const sr_config* cfg, sr_stream_t stream);

/* Resolved launch shape of a segmented call (as sr_plan).  Needs a device. */
int sr_plan_segmented(int64_t nseg, int dtype, const sr_config* cfg, sr_config* resolved);

/* A segmented sum captured once into a CUDA graph owned by the library and
 * replayed with one graph launch (no per-call host work).  The pointers are
 * baked into the graph: x, offsets and out must stay valid and keep their
 * addresses until sr_graph_destroy.  The graph has its own workspace (created
 * at capture time), so replays must not overlap each other on the GPU.
 * Capture errors: as sr_reduce_sum_segmented_ex, nseg == 0 -> SR_ERR_ARG. */
typedef struct sr_graph_s* sr_graph;
int sr_graph_capture_segmented(const void* x, const int64_t* offsets, int64_t nseg, int dtype, void* out,
                               const sr_config* cfg, sr_graph* graph);
int sr_graph_launch(sr_graph graph, sr_stream_t stream);
int sr_graph_destroy(sr_graph graph);

/* ------------------------------------------------- barrier benchmark */

/* One measurement of a synchronisation level (Section V; methods of Section
 * IX).  Zero fields take defaults. */
typedef struct {
    int level;      /* sr_level */
    int64_t iters;  /* r1: back-to-back syncs per kernel (default 100000; r2 = r1/10) */
    int blocks;     /* CTAs (default: 1; cluster size for SR_LEVEL_CLUSTER; SMs for SR_LEVEL_GRID) */
    int threads;    /* threads per CTA (default: 32 for warp-level levels, 1024 block and
                       cluster, 256 grid) */
    int cluster;    /* CTAs per cluster, power of two <= 16 (SR_LEVEL_CLUSTER and
                       SR_LAUNCH_CLUSTER: default 2; 0 or 1 elsewhere) */
    int group;      /* tile size (power of two) or coalesced-group size, 1..32 (default 32) */
    int reps;       /* N runs per repeat count for Eqs. 7-8 (default 10) */
    int method;     /* SR_LEVEL_WARP_REDUCE: sr_warp_reduce_method; SR_LEVEL_KERNEL:
                       sr_launch_kind (CTAs of 32 threads; `blocks` per launch, default 1,
                       the cluster size for SR_LAUNCH_CLUSTER); 0 elsewhere */
} sr_barrier_config;

typedef struct {
    double cycles_per_sync;        /* clock64 method (Wong): slowest warp, cycles per sync */
    double ns_per_sync;            /* Eq. 7: (L(r1) - L(r2)) / (r1 - r2), host clock; for
                                      SR_LEVEL_KERNEL the launch overhead O of Eq. 6 */
    double ns_sigma;               /* Eq. 8 (SR_LEVEL_KERNEL: sample s.d. of O) */
    double syncs_per_cycle_per_sm; /* warp syncs completed per SM per cycle */
    double clock_mhz;              /* SM clock seen by the run (clock64 / %globaltimer) */
    double null_kernel_total_ns;   /* SR_LEVEL_KERNEL: null-kernel total latency */
    int blocks, threads;           /* the shape measured */
    int correct;                   /* SR_LEVEL_WARP_REDUCE: 1 if every reduction of the
                                      clock64 run produced the exact sum (528), else 0;
                                      -1 for the other levels */
} sr_barrier_result;

/* Measure `level` with `iters` back-to-back syncs and default shape; the
 * result is kept for sr_barrier_bench_last (per calling thread).  Runs
 * synchronously on a private stream; allocates and frees its own buffers.
 * A grid-level shape that cannot be co-resident, or a cluster shape that
 * cannot be scheduled, returns SR_ERR_LAUNCH without launching (a partial
 * grid would wait forever: Section VIII-B).
 * Errors: SR_ERR_ARG (unknown level or method, iters < 10, bad shape),
 * SR_ERR_LAUNCH, SR_ERR_CUDA. */
int sr_barrier_bench(int level, int64_t iters);
int sr_barrier_bench_ex(const sr_barrier_config* cfg, sr_barrier_result* result);
int sr_barrier_bench_last(sr_barrier_result* result);

/* Eq. 7 and Eq. 8 on host data: t = (mean(L1) - mean(L2)) / (r1 - r2),
 * sigma = sqrt(s1^2 + s2^2) / |r1 - r2| (s = sample standard deviation of the
 * n1, n2 kernel total latencies).  Host only; SR_ERR_ARG if n < 2 or r1 == r2. */
int sr_differential_latency(const double* L1, int64_t n1, const double* L2, int64_t n2, int64_t r1, int64_t r2,
                            double* t, double* sigma);

/* ---------------------------------------------- autotuner and selection */

/* The candidate launch configurations: grid stage {SR_TWO_KERNEL, SR_ATOMIC,
 * SR_LAST_BLOCK, SR_GRID_SYNC} x grid {8 CTAs, 1, 2, 4, 8 CTAs per SM} of 256
 * threads x vector width {16, 32} bytes = 40 (unroll 4); with `full`, also x
 * unroll {1, 2, 4, 8} = 160.  `sms` is the device's SM count.  With out ==
 * NULL returns the count; else fills out[0..count) (cap entries available)
 * and returns the count.  Negative return = -sr_status.  Host only. */
int sr_candidates(int full, int sms, sr_config* out, int cap);

/* Exhaustive autotuning: times every candidate on the caller's data with
 * CUDA events on `stream` (one untimed warm-up call, then `reps` calls back
 * to back) and writes the mean microseconds per call to us[i]; a candidate
 * that cannot run (SR_ERR_LAUNCH / SR_ERR_UNSUPPORTED / SR_ERR_ARG) gets
 * +infinity.  offsets == NULL: single array of n elements (sr_reduce_sum_ex);
 * else segmented over nseg segments (sr_reduce_sum_segmented_ex, n unused).
 * out receives the last result.  Synchronises `stream`.
 * Errors: SR_ERR_ARG (bad arrays / reps), or the first CUDA error. */
int sr_autotune(const void* x, int64_t n, const int64_t* offsets, int64_t nseg, int dtype, void* out,
                const sr_config* cands, int ncand, int reps, float* us, sr_stream_t stream);

/* Parameters of the performance model (Section VII-A) for one GPU. */
typedef struct {
    int sms;
    double hbm_bytes_per_ns;  /* device-memory throughput at saturation (GB/s) */
    double mem_latency_ns;    /* T: latency of a device-memory access (Little's law) */
    double launch_ns;         /* implicit kernel-boundary barrier (Eq. 6 overhead) */
    double grid_sync_ns;      /* one grid.sync() */
    double last_block_ns;     /* fence + ticket + final reduction of the last unit */
    double atomic_ns;         /* one global atomic finish */
    double per_cta_ns;        /* partial-result cost per CTA per SM */
    double per_segment_ns;    /* per-segment cost of the segmented kernel, per warp */
} sr_model_params;

/* The model evaluated over candidate configurations: for each candidate,
 * throughput Thr = min(peak, bytes in flight / T) (Eq. 1 read as the
 * concurrency a launch shape sustains), C = T * Thr, and predicted time
 * launch + T + T_sync(stage) + max(0, N - C) / Thr (Eqs. 2-3) plus the
 * per-CTA and per-segment terms; N = n * sizeof(dtype).  A candidate that
 * sr_plan (nseg == 1) or sr_plan_segmented (nseg > 1) rejects on the current
 * device with SR_ERR_LAUNCH / SR_ERR_UNSUPPORTED / SR_ERR_ARG (for instance a
 * grid.sync() grid larger than the co-resident CTAs, Section VIII-B) is never
 * chosen and is predicted +infinity; with no device visible the planner is not
 * consulted.  Writes the predictions (microseconds) to predicted_us when
 * non-NULL and returns the index of the cheapest candidate, -SR_ERR_LAUNCH if
 * every candidate is rejected, or -SR_ERR_ARG.  Launches nothing. */
int sr_select_analytic(const sr_model_params* params, int64_t n, int dtype, int64_t nseg, const sr_config* cands,
                       int ncand, float* predicted_us);

/* Feature vector of one call for the learned selector (host only): 9 floats
 * = log2 n, one-hot dtype (4), log2 nseg, log2(1 + mean), log2(1 + std),
 * log2(1 + max) of the segment lengths (a single array: nseg = 1, mean = max
 * = n, std = 0).  SR_ERR_ARG on negative sizes, nseg < 1 or a bad dtype. */
#define SR_SELECTOR_FEATURES 9
int sr_selector_features(int64_t n, int dtype, int64_t nseg, double len_mean, double len_std, double len_max,
                         float* out);

/* ----------------------------------------------------- learned selector */

/* A small MLP cost model that picks a candidate configuration per call (no
 * counterpart in the paper): in_dim features -> hidden (ReLU) -> hidden (ReLU)
 * -> out_dim logits, trained on autotuner timings with a softmax
 * cross-entropy against soft target distributions, by this library's own
 * forward / backward / Adam kernels.  Parameters and Adam state live on the
 * device.  Limits: in_dim <= 32, hidden <= 64, 2 <= out_dim <= 64.
 * Parameter layout (one float array, row-major): W1[in][hidden], b1[hidden],
 * W2[hidden][hidden], b2[hidden], W3[hidden][out], b3[out]. */
typedef struct sr_mlp_s* sr_mlp;
int sr_mlp_create(int in_dim, int hidden, int out_dim, sr_mlp* mlp);   /* parameters start at 0 */
int sr_mlp_destroy(sr_mlp mlp);
int64_t sr_mlp_param_count(sr_mlp mlp);
int sr_mlp_dims(sr_mlp mlp, int* in_dim, int* hidden, int* out_dim);
/* Host copies of the parameters (count must equal sr_mlp_param_count);
 * set also resets the Adam state.  Synchronous. */
int sr_mlp_set_params(sr_mlp mlp, const float* host_params, int64_t count);
int sr_mlp_get_params(sr_mlp mlp, float* host_params, int64_t count);
/* One training step on a device batch: X [batch][in_dim], Q [batch][out_dim]
 * (each row a probability distribution).  Computes the mean cross-entropy
 * -1/B sum_b sum_o Q log softmax(z) and its gradient; writes the loss to
 * *loss (device float, optional) and the gradient to grad (device, param_count
 * floats, optional), then applies one Adam step (beta1 0.9, beta2 0.999,
 * eps 1e-8) with learning rate lr — none when lr == 0.  The per-CTA gradient
 * partials are summed in a fixed order: results are deterministic. */
int sr_mlp_train_step(sr_mlp mlp, const float* X, const float* Q, int batch, float lr, float* loss, float* grad,
                      sr_stream_t stream);
/* Inference kernel: cls[b] = argmax_o logits (lowest index on ties) for a
 * device batch X [batch][in_dim]; logits (device, optional) receives z. */
int sr_mlp_predict(sr_mlp mlp, const float* X, int batch, int* cls, float* logits, sr_stream_t stream);

/* Per-call selection.  A selector wraps a trained MLP (in_dim must be
 * SR_SELECTOR_FEATURES, out_dim = ncand), its feature normalisation
 * (x - mu) / sd and the candidate list its classes index (normally
 * sr_candidates(0, sms, ...)).  The MLP stays owned by the caller and must
 * outlive the selector. */
typedef struct sr_selector_s* sr_selector;
int sr_selector_create(sr_mlp mlp, const float* mu, const float* sd, const sr_config* cands, int ncand,
                       sr_selector* selector);
int sr_selector_destroy(sr_selector selector);
/* The configuration for a call shape: memoised per (device, n, dtype, nseg,
 * segment statistics at 1/16-octave resolution); on a miss the inference
 * kernel runs on `stream` and the call waits for its one-int result. */
int sr_selector_choose(sr_selector selector, int64_t n, int dtype, int64_t nseg, double len_mean, double len_std,
                       double len_max, sr_config* cfg, sr_stream_t stream);
/* Sums whose launch configuration is chosen per call: by `selector`, or —
 * selector == NULL, the fallback — by exhaustive autotuning over the 40
 * candidates on the call's own data the first time its shape is seen
 * (memoised; that first call synchronises `stream`).  Other arguments and
 * errors as sr_reduce_sum_ex / sr_reduce_sum_segmented_ex; the segmented form
 * takes the segment-length statistics from the caller (n = mean * nseg) and
 * applies the form sr_segmented_layout_flags gives for them: it adds
 * SR_F_DENSE_SEGMENTS to the chosen configuration, or replaces the chosen
 * configuration's shape with SR_F_WARP_SEGMENTS or SR_F_LANE_SEGMENTS at its
 * default shape (the lane form with 32-byte vectors from 128 bytes per
 * segment on average).  This layout rule runs after the selector (or the
 * autotuner) and overrides its shape: the selector's candidates, and so its
 * regret against exhaustive autotuning, cover the grid stage, grid size and
 * vector width of the plain and dense forms only. */
int sr_reduce_sum_selected(sr_selector selector, const void* x, int64_t n, int dtype, void* out,
                           sr_stream_t stream);
/* The segmented form for a layout, from the caller's segment-length
 * statistics (mean, standard deviation, maximum; len_max <= 0 when unknown,
 * then mean + 4 std stands in) and the device's SM count, in this order:
 * SR_F_LANE_SEGMENTS for 2^19 or more uniform segments (std <= mean / 2) of
 * at most 1 KiB on average and none above 4x the mean;
 * SR_F_DENSE_SEGMENTS for uniformly very short segments (mean * element size
 * <= 128 bytes, std <= mean / 2); SR_F_WARP_SEGMENTS for 2^19 or more
 * segments none longer than twice a warp's even share of the elements
 * (2 * mean * nseg / (32 * sms)); SR_F_DENSE_SEGMENTS for uniformly short
 * segments (<= 512 bytes, std <= mean / 2); else 0 (the plain form).
 * Host-only and pure (no device call).  The paper has no counterpart: the
 * thresholds come from this library's own measurements of the forms.
 * The statistics must describe the layout actually passed: they are trusted,
 * not checked against the offsets.  A len_max below the true longest segment
 * can route a layout with a very long segment to the lane or warp form, where
 * one thread or one warp sums that segment alone (still correct, but up to
 * hundreds of times slower than the plain form).  Callers without reliable
 * statistics should use SR_F_ADAPTIVE_SEGMENTS, which partitions the segments
 * from the offsets on the device.
 * Returns the flag, or a negated status: -SR_ERR_DTYPE, -SR_ERR_ARG (sms < 1,
 * nseg < 0, negative or NaN statistics). */
int sr_segmented_layout_flags(int sms, int dtype, int64_t nseg, double len_mean, double len_std, double len_max);
int sr_reduce_sum_segmented_selected(sr_selector selector, const void* x, const int64_t* offsets, int64_t nseg,
                                     int dtype, void* out, double len_mean, double len_std, double len_max,
                                     sr_stream_t stream);

/* --------------------------------- persisted selection and configuration */

/* Reads a variant from text: a decimal or 0x-hexadecimal number, or names
 * joined by '+': at most one grid stage (auto, two_kernel, atomic,
 * last_block, grid_sync, single_cluster), at most one cluster size (cluster2,
 * cluster4, cluster8, cluster16) and the flags kahan, fp64_combine,
 * fp64_auto, bulk, each at most once — e.g. "last_block+bulk" = 0x403.
 * Surrounding blanks are ignored.  Host-only and pure.  Only the syntax is
 * checked here; a call validates the combination as for any variant.
 * Errors: SR_ERR_ARG (NULL argument, empty text, unknown name, repeated
 * stage, cluster or flag, number out of range). */
int sr_parse_variant(const char* text, int* variant);

/* The autotuner fallback of sr_reduce_sum_selected /
 * sr_reduce_sum_segmented_selected memoises its choice per device identity
 * and call shape (n, dtype, segment count, segment statistics at 1/16-octave
 * resolution).  The memo can be kept across processes in a versioned text
 * file ("sr-tune 1"): sections headed "device <SMs> <driver version>
 * <name>", one line per shape.  A device's identity is its name, its SM count
 * and the CUDA driver version (cudaDriverGetVersion): entries are used only
 * on a device with the same identity and carried along otherwise.
 * When the environment variable SR_TUNE_FILE names a file, the memo is read
 * from it at its first use (a missing file is created at the first new
 * entry; a file that does not parse is neither used nor overwritten) and the
 * file is rewritten, whole, after every new entry.  Files are written to a
 * temporary name and renamed, so a reader never sees a partial file; of
 * concurrent writers the last rename wins.  Host-only; no device call.
 * sr_tune_save: writes the memo (every identity) to `path`.
 * sr_tune_load: merges the entries of `path` into the memo (an entry of the
 *   file replaces one with the same key); *entries (may be NULL) = entries
 *   read.  The whole file is parsed first: a malformed file (SR_ERR_ARG)
 *   changes nothing.
 * sr_tune_size: entries in the memo; sr_tune_clear: empties it.
 * Errors: SR_ERR_ARG (NULL or empty path, unreadable, unwritable or
 * malformed file). */
int sr_tune_save(const char* path);
int sr_tune_load(const char* path, int64_t* entries);
int64_t sr_tune_size(void);
int sr_tune_clear(void);

/* A trained selector (its MLP's dimensions and parameters, the feature
 * normalisation and the candidate list) as a versioned text file
 * ("sr-selector 1"), stamped with the identity of the device it was saved on.
 * sr_selector_save: writes `selector` to `path` (needs the current device for
 *   its identity).
 * sr_selector_load: reads `path` and creates a selector for the current
 *   device that owns its own MLP (sr_selector_destroy frees both).  The file
 *   is parsed before any device call: malformed -> SR_ERR_ARG; made on a
 *   device with another identity -> SR_ERR_UNSUPPORTED.
 * When the environment variable SR_MODEL_FILE names a selector file, the
 * selected entry points called with selector == NULL use the selector loaded
 * from it (once per device, kept until the process exits) instead of the
 * autotuner; if that load fails they return its status. */
int sr_selector_save(sr_selector selector, const char* path);
int sr_selector_load(const char* path, sr_selector* selector);

/* ------------------------------------------------- allocation-free sum */

/* The last-block-done sum (SR_LAST_BLOCK, LDG load path) for callers that must
 * not allocate device memory: code running where cudaMalloc is unavailable or
 * forbidden — inside a host function or callback that may not call the CUDA
 * allocator, in a process whose device memory is fully reserved by another
 * allocator, or under a policy that allows no allocation after start-up.
 * The paper has no counterpart.
 *
 * Instead of the per-stream workspace it uses one file-scope device array of
 * 64 KiB + 256 bytes (a ticket, an error word and 4096 unit-partial slots),
 * which every GPU that loads this library holds until the process exits.  It
 * calls no cudaMalloc, cudaFree or other allocating routine.  The caller
 * passes x and out exactly as for sr_reduce_sum_ex.
 *  - cfg: NULL, or a configuration whose stage is SR_AUTO or SR_LAST_BLOCK
 *    (other stages and SR_F_BULK -> SR_ERR_UNSUPPORTED); cluster bits and the
 *    SR_F_KAHAN / SR_F_FP64_COMBINE flags are honoured.
 *  - At most 4096 units (CTAs, or clusters when a cluster size is set): a
 *    larger explicit grid, or a plan needing more units, returns SR_ERR_ARG
 *    and launches nothing.
 *  - The first call on each device looks up the device address of the array
 *    (cudaGetSymbolAddress, with that device current); make that first call
 *    before any stream capture.
 *  - All calls share the one array, which keeps the last call's contents; each
 *    call resets the ticket on `stream` before its kernel.  Calls whose work
 *    overlaps on the GPU (different streams, no ordering between them) race on
 *    the array and give wrong results: order them on one stream.
 * Errors: the host-side statuses of sr_reduce_sum_ex (argument, dtype, launch
 * and CUDA errors), returned by the call.  There are no device-side errors to
 * report: the kernel it runs (vector loads, last-block-done finish) has no
 * bounded wait and sets no error word, which is why SR_F_BULK (whose copy
 * ring waits on mbarriers) is refused here; sr_stream_status reports nothing
 * about these calls. */
int sr_reduce_sum_noalloc(const void* x, int64_t n, int dtype, void* out, const sr_config* cfg,
                          sr_stream_t stream);

/* ------------------------------------------------------------ self-test */

/* Failure-detection self-test (no counterpart in the paper): launches on
 * `stream` one CTA that waits on an mbarrier nothing ever completes.  The
 * wait is bounded by limit_ns of %globaltimer time (0 < limit_ns <= 10 s);
 * when it gives up the kernel records SR_ERR_TIMEOUT in the stream's error
 * word and returns, so the next sr_stream_status(stream) reports
 * SR_ERR_TIMEOUT (and clears it) and the context stays usable.  This is the
 * same bounded-wait path every mbarrier wait of the TMA load path takes
 * (its limit: SR_SPIN_LIMIT_NS, default 2 s). */
int sr_selftest_bounded_wait(uint64_t limit_ns, sr_stream_t stream);

/* ------------------------------------------------------ host helpers */

const char* sr_status_string(int status);
int sr_last_cuda_error(void);
const char* sr_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SR_H */
