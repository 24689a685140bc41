/*
 * ddm.h -- C ABI of the GB300 (sm_103a) Sort-Based Matching library.
 *
 * The library solves the Data Distribution Management matching problem of
 * Marzolla and D'Angelo, "Parallel Sort-Based Matching for Data Distribution
 * Management on Shared-Memory Multiprocessors" (DS-RT 2017), Section 3: given
 * subscription extents S_0..S_{n-1} and update extents U_0..U_{m-1}, which are
 * d-dimensional axis-parallel rectangles with closed sides, report every pair
 * (i, j) such that S_i and U_j intersect.  Two closed intervals intersect iff
 * x.low <= y.high and y.low <= x.high (Algorithm 1); two rectangles intersect
 * iff their projections intersect in every dimension (Section 3).
 *
 * Method (Algorithm 4, Sort-Based Matching, re-planned for one GPU): the
 * endpoints of dimension 0 are turned into order-preserving integer keys and
 * radix sorted, with every lower endpoint placed before every upper endpoint
 * at equal coordinates (so that touching extents are reported, as closed
 * intervals require); one scan over the sorted stream yields the sizes of the
 * paper's active sets SubSet/UpdSet, and from them the exact number of matches
 * of every subscription; an exclusive scan turns these counts into output
 * offsets; the pairs are then written, with dimensions 1..d-1 filtered per
 * candidate.  All work runs in the library's CUDA kernels; there is no CPU
 * fallback.
 *
 * Conventions for every entry point:
 *   - Ids are 0-based indices into the caller's arrays.
 *   - Coordinates are IEEE float32.  -0 equals +0; +-inf are allowed; NaN,
 *     or lo > hi in any dimension, makes the call fail with DDM_ERR_INVALID.
 *   - Limits: 1 <= d <= DDM_MAX_DIMS; n >= 0, m >= 0, n + m <= DDM_MAX_REGIONS.
 *   - Pointers marked "device" must be device memory of the context's GPU
 *     (cudaMalloc, or torch tensors); pointers marked "host" are ordinary or
 *     pinned host memory.  The caller owns all of them; the library only reads
 *     inputs and writes outputs, and keeps no pointer after the call returns.
 *   - Calls on one context are not thread-safe; use one context per thread and
 *     stream.  Different contexts may run concurrently.
 *   - On error the outputs are unspecified, except *K_out for
 *     DDM_ERR_CAPACITY.  ddm_last_error() returns a message.
 */
#ifndef DDM_H
#define DDM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DDM_OK                  0
#define DDM_ERR_INVALID       (-1)  /* bad argument, NaN coordinate, or lo > hi   */
#define DDM_ERR_CAPACITY      (-2)  /* more pairs than the output can hold        */
#define DDM_ERR_NOMEM         (-3)  /* device memory or the context budget exhausted */
#define DDM_ERR_DEVICE_TIMEOUT (-4) /* a bounded device-side wait expired         */
#define DDM_ERR_CUDA          (-5)  /* a CUDA runtime call failed                 */
#define DDM_ERR_INTERNAL      (-6)  /* a device-side consistency check failed     */

#define DDM_MAX_DIMS      8
#define DDM_MAX_REGIONS   ((int64_t)1 << 29)   /* n + m; keeps 2(n+m) < 2^30 */

typedef struct ddm_ctx ddm_ctx;

/*
 * One matching instance (Section 3 problem statement).  sub_lo, sub_hi,
 * upd_lo and upd_hi are HOST arrays of d pointers; sub_lo[k] points to n
 * floats, the lower bounds of S_0..S_{n-1} along dimension k (likewise for the
 * others).  Whether the d pointers themselves are device or host memory is
 * fixed by the entry point (see each).
 */
typedef struct {
    int d;
    int64_t n, m;
    const float *const *sub_lo;
    const float *const *sub_hi;
    const float *const *upd_lo;
    const float *const *upd_hi;
} ddm_regions;

/*
 * Creates a context on CUDA device `device`, bound to `cuda_stream` (a
 * cudaStream_t; NULL means the legacy default stream).  All of the context's
 * kernels run on that stream.  mem_budget_bytes caps the device memory the
 * context may hold (0 = no cap): its pipeline workspace and the staging
 * buffers of ddm_match_host, together; scratch is kept between calls and
 * grows on demand.  A call whose scratch would exceed the cap fails with
 * DDM_ERR_NOMEM before any launch.  Returns DDM_OK and *out, or an error code
 * (then *out is NULL).
 */
int ddm_create(ddm_ctx **out, int device, void *cuda_stream, size_t mem_budget_bytes);

/* Frees the context and its scratch memory.  ddm_destroy(NULL) is a no-op. */
int ddm_destroy(ddm_ctx *ctx);

/* Text of the last error on this context (never NULL; empty after success). */
const char *ddm_last_error(const ddm_ctx *ctx);

/*
 * Exact number K of intersecting (S_i, U_j) pairs; the pairs are not stored
 * (the paper's measured mode, Section 5, "Experimental setup").  Coordinate
 * pointers are DEVICE memory.  Synchronous: returns after the work on the
 * context's stream has finished.
 */
int ddm_count(ddm_ctx *ctx, const ddm_regions *regions, uint64_t *K_out);

/*
 * All intersecting pairs (Section 3), as K interleaved int32 pairs
 * pairs[2k] = i (subscription id), pairs[2k+1] = j (update id), sorted
 * lexicographically by (i, j); each pair appears once.  `pairs` is DEVICE
 * memory for 2 * cap int32 values, 8-byte aligned (else DDM_ERR_INVALID).
 * If K > cap nothing is written, *K_out = K
 * and DDM_ERR_CAPACITY is returned, so the caller can retry with a larger
 * buffer.  Synchronous, like ddm_count.
 */
int ddm_match(ddm_ctx *ctx, const ddm_regions *regions, int32_t *pairs, uint64_t cap,
              uint64_t *K_out);

/*
 * ddm_match with HOST buffers: the coordinates are read from host memory and
 * the pairs written to host memory (`pairs` holds 2 * cap int32).  The
 * library copies through its own device buffers (on GB300 pinned and pageable
 * host memory measured the same, about 193 GB/s device to host, which bounds
 * this call for large outputs).  Same result and errors as ddm_match.
 */
int ddm_match_host(ddm_ctx *ctx, const ddm_regions *regions, int32_t *pairs, uint64_t cap,
                   uint64_t *K_out);

/*
 * The paper's two other matchers, as GPU comparison baselines with the result
 * contract of ddm_match (DEVICE coordinates, K sorted int32 pairs into
 * `pairs`, 8-byte aligned, DEVICE memory for 2 * cap int32; K > cap writes
 * nothing and returns DDM_ERR_CAPACITY with *K_out = K).  With pairs == NULL
 * and cap == 0 only K is computed.  Synchronous.  Errors as for ddm_match.
 *
 *   ddm_match_bruteforce  Brute-Force matching (Algorithm 2, Section 2): all
 *                         n * m pairs tested in every dimension with
 *                         Algorithm 1; O(n m d) work, for moderate sizes (a
 *                         second, independent check of the sort-based path).
 *   ddm_match_itm         Interval-Tree matching (Algorithm 3, Section 2): a
 *                         static balanced interval tree (nodes ordered by lower
 *                         bound, with each subtree's minimum lower and maximum
 *                         upper bound) over the updates' dimension 0, queried
 *                         by every subscription; dimensions 1..d-1 filtered
 *                         per reported pair.  The paper's tree holds S and is
 *                         queried by U; the roles are exchanged here, which
 *                         the symmetry of Algorithm 1 allows.
 */
int ddm_match_bruteforce(ddm_ctx *ctx, const ddm_regions *regions, int32_t *pairs, uint64_t cap,
                         uint64_t *K_out);
int ddm_match_itm(ddm_ctx *ctx, const ddm_regions *regions, int32_t *pairs, uint64_t cap,
                  uint64_t *K_out);

/*
 * Grid-Based matching (Section 2), the paper's third comparison method, with
 * the same result contract: a regular mesh of cells over the first min(d, 3)
 * dimensions of the instance's bounding box (other dimensions are filtered per
 * pair); every extent is registered in each cell it overlaps and brute force
 * runs inside each cell; a pair that shares several cells is reported once,
 * by the cell that holds max(S.lo, U.lo).  cells_per_dim > 0 fixes the cells
 * along each gridded dimension (clamped to 2^24, 2^12 or 2^8 for 1, 2 or 3
 * gridded dimensions; above 2^24: DDM_ERR_INVALID); 0 lets
 * the library choose (cells about as wide as the mean extent side, at least
 * about one extent per cell).  The paper leaves the grid size to the user or a
 * heuristic.  grid_out (HOST, 3 values, may be NULL) receives the cells used
 * per gridded dimension (1 for the others).  The memberships need 4 bytes per
 * (extent, cell) pair of device memory.
 */
int ddm_match_grid(ddm_ctx *ctx, const ddm_regions *regions, uint32_t cells_per_dim,
                   int32_t *pairs, uint64_t cap, uint64_t *K_out, uint32_t *grid_out);

/*
 * ddm_count without any allocation.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory -- code that
 * runs where cudaMalloc is unavailable or forbidden (a custom allocator that
 * owns all device memory, a simulation loop that must not allocate after
 * start-up, a process whose device memory is pinned down by other users).
 * It needs no context: it runs on the CURRENT device and on `cuda_stream`
 * (NULL = legacy default stream), and returns the same K as ddm_count for the
 * same DEVICE coordinates.
 *
 * All scratch lives in one fixed 24 MiB __device__ array inside the library,
 * held by every GPU that loads the library until the process exits.  The call
 * makes no cudaMalloc/cudaFree and no other allocation.  Limit: n + m <=
 * DDM_NOALLOC_MAX_REGIONS, for every d up to DDM_MAX_DIMS; larger instances
 * (and bad arguments) return DDM_ERR_INVALID without touching the GPU.  Every
 * call looks up the array's device address on the current device
 * (cudaGetSymbolAddress, which allocates nothing), so no address is kept
 * across calls.  All calls share the array: calls that overlap on the GPU
 * (two streams, two threads) race and give wrong results, so serialise them.
 * Synchronous: the call waits for its stream (cudaStreamSynchronize), so it
 * must not be made from a host function running on a stream
 * (cudaLaunchHostFunc, stream callbacks), where CUDA calls are not allowed.
 * Errors as for ddm_count.
 */
#define DDM_NOALLOC_MAX_REGIONS ((int64_t)1 << 17)
int ddm_count_noalloc(const ddm_regions *regions, void *cuda_stream, uint64_t *K_out);

/*
 * Tunables of a context (read by the autotuner; defaults are used otherwise).
 *   DDM_PARAM_WIN_SHIFT   log2 of the window length of the d = 1 emission, in
 *                         sorted-stream positions: 6 .. 10 (default 10).
 * Returns DDM_ERR_INVALID for an unknown parameter or a value out of range.
 *   DDM_PARAM_ND_PATH     strategy for d > 1: 0 = automatic (default: the tiled
 *                         join with dimension-1 pruning, measured faster on
 *                         GB300 for d = 2 and 3), 1 = tiled join, 2 = range
 *                         expansion.  Results are identical; only speed differs.
 *   DDM_PARAM_PDL         1 (default) = launch the kernels of a call with
 *                         programmatic dependent launch, so that each grid is
 *                         scheduled while its predecessor finishes; 0 = plain
 *                         stream order.  Results are identical.
 *   DDM_PARAM_SWEEP_DIM   0 (default) = sweep dimension 0 and filter the others
 *                         in the given order; 1 = choose the order: before a
 *                         d > 1 ddm_count / ddm_match / ddm_match_host call the
 *                         library counts, for every dimension k alone, the pairs
 *                         whose extents intersect in k (the d = 1 pipeline on
 *                         that dimension: d extra synchronous count passes), then
 *                         sweeps the dimension with the fewest and prunes on the
 *                         next (the paper's Section 3 reduction makes every order
 *                         correct).  Results are identical; the order used is
 *                         reported in ddm_stats.dim_order.  Sessions and batched
 *                         calls always use the given order.
 *   DDM_PARAM_SORT_ITEMS  keys per thread of the 32-bit endpoint sort: 12, 16 or 18
 *                         (default 18), i.e. tiles of 3072, 4096 or 4608 keys.
 *   DDM_PARAM_JOIN_SHIFT  log2 of the window length, in sorted-stream positions, of
 *                         the tiled join for d > 1: 9 .. 11 (default 11).
 *   DDM_PARAM_ND_WRITE    how ddm_match and ddm_match_batch write the pairs for d > 1
 *                         with the tiled join: 1 = a second filter pass into each
 *                         subscription's segment, then a per-segment sort; 2 = the
 *                         count pass also records every surviving pair as a 64-bit
 *                         key and one radix sort of those keys gives the list (no
 *                         second filter pass; needs 16 bytes per pair and per slot of
 *                         room, room sized by the K of the context's last d > 1 count
 *                         or match; falls back to 1 when a window's share overflows);
 *                         0 (default) = 2 for d >= 3, and for a batched call at
 *                         d = 2 when that last K is at most 4 (n + m); else 1
 *                         (measured).
 * Results never depend on any tunable; only speed does.
 */
#define DDM_PARAM_WIN_SHIFT 1
#define DDM_PARAM_ND_PATH 2
#define DDM_PARAM_PDL 3
#define DDM_PARAM_SWEEP_DIM 4
#define DDM_PARAM_SORT_ITEMS 5
#define DDM_PARAM_JOIN_SHIFT 6
#define DDM_PARAM_ND_WRITE 7
int ddm_set_param(ddm_ctx *ctx, int param, int64_t value);

/*
 * Counters and per-stage timing.  With profiling enabled (ddm_set_profiling),
 * every call records CUDA events on the context's stream at the stage
 * boundaries, and stage_ms[] holds the device time of each stage of the last
 * call: 0 key build (a1), 1 radix sort (a2), 2 sweep scan (a3), 3 counts --
 * rank arithmetic for d = 1, filter count for d > 1 (a4/a7), 4 offsets scan
 * (a5), 5 emission set-up -- window lists and rank table (a6), 6 pair emission
 * (a6/a7: the window kernel for d = 1, the range kernels for d > 1), 7 range
 * path of flagged subscriptions and per-segment sort (a6).
 * `launches` counts every kernel the context has launched since creation.
 * ddm_set_profiling modes: 0 = off; 1 = events at every stage boundary;
 * 2 + k (0 <= k < DDM_STAGES) = events only around stage k, so that a single
 * stage can be timed with the least disturbance of the others (each event
 * between two kernels also ends the overlap of programmatic dependent launch
 * there); the other stage_ms entries are then 0.  DDM_ERR_INVALID for any
 * other mode.
 */
#define DDM_STAGES 8
typedef struct {
    uint64_t launches;
    uint64_t calls;
    float stage_ms[DDM_STAGES];
    /* Dimension order of the last plain call: dim_order[0] is the swept
     * dimension, dim_order[1] the pruning one (identity unless
     * DDM_PARAM_SWEEP_DIM = 1 reordered a d > 1 call). */
    uint32_t dim_order[DDM_MAX_DIMS];
    /* d > 1 ddm_match calls whose pairs came from the survivors recorded by the
     * count pass (one sort, no second filter pass); the others ran the general
     * write pass (the first call of a context has no size hint; windows that
     * overflowed; no memory for the keys). */
    uint64_t survivor_calls;
} ddm_stats;

int ddm_set_profiling(ddm_ctx *ctx, int enable);
int ddm_get_stats(const ddm_ctx *ctx, ddm_stats *out);

/*
 * Batched matching: `num` independent instances inst[0..num-1] (a HOST array
 * of descriptors whose coordinate pointers are DEVICE memory), all with the
 * same d, matched together in one pass of the pipeline.  The instances are
 * concatenated on the device and the instance number becomes the high bits of
 * the 64-bit sort key, so one sort, one scan, one count and one emission serve
 * all of them, with no per-instance launches.  Instance b's pairs, with ids
 * local to instance b and sorted lexicographically, occupy pairs[2*o[b] ..
 * 2*o[b+1]) where o = inst_offsets, a HOST array of num + 1 values (o[0] = 0,
 * o[num] = K).  `pairs` is DEVICE memory for 2 * cap int32, 8-byte aligned
 * (else DDM_ERR_INVALID); with pairs == NULL only the counts (inst_offsets and
 * K) are computed.  Capacity rule as in ddm_match.  Limits: 0 <= num <= DDM_MAX_BATCH; the instances' regions
 * together obey DDM_MAX_REGIONS.  Synchronous.
 */
#define DDM_MAX_BATCH (1 << 20)
int ddm_match_batch(ddm_ctx *ctx, int num, const ddm_regions *inst, int32_t *pairs, uint64_t cap,
                    uint64_t *inst_offsets, uint64_t *K_out);

/*
 * Served mode: a session keeps one simulation's extents RESIDENT on the device
 * across timesteps, together with its own pipeline workspace (the sorted
 * endpoint stream and rank records of the last step stay there), so a request
 * for the next timestep moves no coordinates between host and device.
 *
 *   ddm_session_create   copies `initial` (DEVICE coordinate pointers) into
 *                        session-owned device memory on `device`.
 *   ddm_session_regions  a view of the resident coordinates (device pointers,
 *                        valid until the session is destroyed).
 *   ddm_session_drift    moves every extent by delta ~ N(0, sigma) per
 *                        dimension (lo and hi by the same delta; rounding keeps
 *                        lo <= hi); the draws are a counter-based SplitMix64
 *                        stream (seed, step), reproducible bit for bit.
 *   ddm_session_count    runs the pipeline up to the exact K (sort, sweep scan,
 *                        counts, offsets) and keeps that state; returns K.
 *   ddm_session_emit     after ddm_session_count: writes the K sorted pairs into
 *                        `pairs` (DEVICE, 2 * cap int32, 8-byte aligned) from
 *                        the kept state, without sorting again.
 *                        K > cap -> DDM_ERR_CAPACITY.
 *
 * mem_budget_bytes (0 = no cap) caps ALL device memory the session holds:
 * its resident coordinates, its pipeline workspace and the pair lists and
 * offsets of ddm_session_emit_delta; a call that would exceed it fails with
 * DDM_ERR_NOMEM (ddm_session_create too, if the coordinates alone exceed it).
 *
 * Between count and emit a caller can reserve exactly 8 K bytes of output
 * (admission by memory).  Every call takes the CUDA stream to run on (NULL =
 * legacy default stream) and is synchronous.  A session must not be used by
 * two threads at once; different sessions may run concurrently on different
 * streams.  The paper has no serving layer: dynamic extents are its future
 * work (Section 6, "Conclusions"; Pan et al. 2011).
 */
typedef struct ddm_session ddm_session;
int ddm_session_create(ddm_session **out, int device, const ddm_regions *initial,
                       size_t mem_budget_bytes);
int ddm_session_destroy(ddm_session *s);
const ddm_regions *ddm_session_regions(const ddm_session *s);
const char *ddm_session_last_error(const ddm_session *s);
int ddm_session_drift(ddm_session *s, void *cuda_stream, uint64_t seed, uint64_t step,
                      double sigma);
int ddm_session_count(ddm_session *s, void *cuda_stream, uint64_t *K_out);
int ddm_session_emit(ddm_session *s, void *cuda_stream, int32_t *pairs, uint64_t cap,
                     uint64_t *K_out);

/*
 * Incremental matching: the change report of one timestep.  Reports the
 * pairs whose status changed since the last successful ddm_session_emit_delta
 * call (the first call, which needs ddm_session_count first, reports every
 * pair as added).  A later report of a timestep not yet counted runs the count
 * phase itself, on the same stream with no synchronisation in between (K is
 * not needed for a report):
 *   added   (DEVICE, 2 * cap_added int32)   pairs present now and not then,
 *   removed (DEVICE, 2 * cap_removed int32) pairs present then and not now,
 * both sorted lexicographically; *n_added / *n_removed receive their numbers.
 * Nothing is recomputed in full: the session keeps the coordinates of the
 * last report, measures how far any endpoint has moved since (per
 * dimension), and tests only the pairs of endpoints that have come within
 * twice that distance of each other -- the only ones whose comparisons, and
 * so whose intersection, can have changed (the dimension-0 candidates come
 * from the sorted endpoint stream of the count phase).  The work therefore
 * follows the motion, not K.  If either list does not fit, returns
 * DDM_ERR_CAPACITY with both numbers set; calling again without a new count
 * writes the same report into larger buffers.  A delivered report consumes
 * the count: the next timestep is counted again (by ddm_session_count or by
 * the report itself).  Device memory (counted against the
 * session budget): a copy of the coordinates, and 16 bytes per changed pair
 * plus sort scratch; for d > 1 also the updates' bounds of dimensions 1..d-1
 * sorted per dimension (16 bytes per update and dimension).  Synchronous.
 * Other errors as for ddm_session_emit.  The paper recomputes the full match
 * every timestep; reporting changes is the dynamic DDM it names as future work
 * (Section 6).
 */
int ddm_session_emit_delta(ddm_session *s, void *cuda_stream, int32_t *added, uint64_t cap_added,
                           int32_t *removed, uint64_t cap_removed, uint64_t *n_added,
                           uint64_t *n_removed);

/*
 * K of the session's last count phase (run by ddm_session_count or by a
 * change report that counted its timestep itself); 0 before the first.
 * DDM_ERR_INVALID when s or K_out is NULL.  Host only, no device work.
 */
int ddm_session_K(ddm_session *s, uint64_t *K_out);

/*
 * Diagnostic view of the sweep stages for dimension 0 (the sorted endpoint
 * list T of Algorithm 4 and the active-set sizes it maintains), for tests.
 * All outputs are DEVICE memory, E = 2(n+m) entries unless noted:
 *   sorted_who[t]   endpoint t of the sorted list: (kind << 30) | id, kind 0 =
 *                   S lower, 1 = U lower, 2 = S upper, 3 = U upper;
 *   subset_size[t]  |SubSet| right after endpoint t is processed;
 *   updset_size[t]  |UpdSet| right after endpoint t is processed;
 *   sub_count[i]    number of updates intersecting S_i along dimension 0 (n);
 *   upd_count[j]    number of subscriptions intersecting U_j along dim 0 (m).
 * Any output pointer may be NULL to skip it.
 */
int ddm_debug_sweep(ddm_ctx *ctx, const ddm_regions *regions, uint32_t *sorted_who,
                    uint32_t *subset_size, uint32_t *updset_size, uint32_t *sub_count,
                    uint32_t *upd_count);

/*
 * Self-test of the bounded device-side waits (for tests).  Every wait in the
 * library's kernels gives up after a bounded number of polls, records
 * DDM_ERR_DEVICE_TIMEOUT and returns, so that a lost hand-off cannot hang the
 * GPU.  This call runs one of those wait helpers against a hand-off that never
 * happens, with at most `spin_limit` polls (1 .. 65536, a few milliseconds):
 *   which = 0  the decoupled look-back of the scans, waiting for a
 *              predecessor tile that never publishes;
 *   which = 1  the mbarrier wait of the bulk copies, waiting for transaction
 *              bytes that never arrive (no copy is issued).
 * Expected result: DDM_ERR_DEVICE_TIMEOUT, with the context still usable for
 * the next call.  DDM_ERR_INVALID for other `which` or limits.  Synchronous.
 * The paper has no counterpart (its multicore algorithm has no device waits).
 */
int ddm_debug_wait_timeout(ddm_ctx *ctx, int which, uint32_t spin_limit);

/*
 * Measurement aid: the write pattern of the window emission without its
 * filter, as the ceiling against which the emission's bandwidth is read.
 * nseg segments of 8-byte pairs, segment lengths drawn (hash of the segment
 * id) uniformly from mean_len/2 .. mean_len/2 + mean_len, laid out back to
 * back like the sorted pair list; one warp writes a segment in steps of 32
 * consecutive pairs with streaming stores.  scattered = 0: warps take the
 * segments in id order (concurrent segments adjacent in memory); scattered
 * != 0: in the order g * step mod nseg, step coprime to nseg near 0.618 nseg
 * (concurrent segments far apart, as the emission's windows meet
 * subscriptions of unrelated ids).  Runs reps + 1 times (the first warms up),
 * writing 256 MiB between runs to flush L2, and stores the fastest CUDA-event
 * time in *ms_out (ms) and the bytes written per run in *bytes_out (may be
 * NULL).  nseg 1 .. 2^26, mean_len 1 .. 4096, reps 1 .. 100, else
 * DDM_ERR_INVALID.  Allocates its buffers for the call with cudaMalloc,
 * outside the context's memory budget (DDM_ERR_NOMEM when that fails), and
 * frees them before returning.  Synchronous, on the context's stream.  Not
 * part of the paper's method.
 */
int ddm_debug_write_pattern(ddm_ctx *ctx, uint32_t nseg, uint32_t mean_len, int scattered,
                            int reps, double *ms_out, uint64_t *bytes_out);

#ifdef __cplusplus
}
#endif

#endif /* DDM_H */
