/*
 * cc.h -- C ABI of the GB300 (sm_103a) pair-collision library.
 *
 * The library counts, exactly, the unordered pairs that collide inside a set of N
 * objects, and can add a pairwise interaction term over the colliding pairs. It
 * implements the balanced cyclic enumeration of Saldanha and de Souza, "High
 * Performance Algorithms for Counting Collisions and Pairwise Interactions" (ICCS
 * 2019, arXiv 1901.11204), Section 4: object i evaluates objects (i+s) mod N for
 * s = 1..(N-1)/2, and for even N the objects i < N/2 also evaluate i + N/2, so every
 * unordered pair is evaluated exactly once and every object does the same work.
 *
 * Conventions shared by every call below
 * --------------------------------------
 * Pointers. Arguments named d_* and the coordinate arrays in cc_points are DEVICE
 *   pointers (memory of the current CUDA device). They are owned by the caller; the
 *   library keeps no pointer after a call returns, except the server's own copies of
 *   registered sets. Arrays must be 4-byte aligned; offsets arrays 8-byte aligned.
 * Streams. `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *   stream). Every compute call is asynchronous and stream-ordered: it enqueues work
 *   and returns; results are valid once the stream has been synchronised.
 * Errors. Argument errors are detected on the host before anything is enqueued and
 *   return CC_ERR_INVALID_ARG. Launch errors return CC_ERR_CUDA. Conditions that only
 *   the device can see (integer span beyond the supported range, a bounded wait that
 *   ran out) are recorded in a device status word of the stream's workspace: the call's
 *   output count is then set to CC_COUNT_INVALID (its sum, if any, to NaN) by the call's
 *   last kernel, and cc_stream_status() returns the code.
 *   cc_last_error() gives a message for the last failing call of the calling thread.
 * Workspace. The single-set calls keep one scratch buffer per stream, grown on demand
 *   with stream-ordered allocation (cudaMallocAsync) on that stream. The first call on
 *   a stream with a larger N than before allocates; call cc_reserve() first when the
 *   calls are to be captured in a CUDA graph. Calls on different streams never share
 *   scratch; calls on one stream are ordered by the stream.
 *
 * Collision predicates (the interact() of the paper's Section 4 listings)
 * ------------------------------------------------------------------------
 * CC_I32: integer points collide when dx*dx + dy*dy + dz*dz <= r2 (exact). r2 = 0 is
 *   the same-site collision of the paper's Section 3. Precondition: on every axis
 *   max - min <= 32767 (then d2 < 2^32); beyond it the device reports CC_ERR_RANGE.
 * CC_F32: spheres (centre, radius) collide when (dx*dx + dy*dy) + dz*dz <= (ri+rj)^2,
 *   every operation rounded to nearest in FP32 in exactly this order, no contraction
 *   (the predicate is then symmetric bit for bit). NaN never collides. r2 is ignored.
 * Interaction term: 1 / max(d, 1e-6) over colliding pairs, with d = sqrt(d2) correctly
 *   rounded in FP32 and an IEEE FP32 divide; the sum is accumulated in FP64 and
 *   returned as FP32.
 */
#ifndef CC_H
#define CC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CC_OK = 0,
    CC_ERR_INVALID_ARG = 1,  /* null pointer, n < 0, bad dtype, misaligned pointer ... */
    CC_ERR_RANGE = 2,        /* integer span above 32767 on some axis (device-detected) */
    CC_ERR_NOMEM = 3,        /* an allocation failed or the memory budget is exceeded */
    CC_ERR_CUDA = 4,         /* a CUDA runtime call failed; see cc_last_error() */
    CC_ERR_TIMEOUT = 5,      /* a bounded device-side wait ran out */
    CC_ERR_BUSY = 6,         /* resource temporarily unavailable (server full) */
    CC_ERR_NOT_FOUND = 7     /* unknown set id / request */
} cc_status;

typedef enum { CC_I32 = 0, CC_F32 = 1 } cc_dtype;

/* Count written to the output when the device detected an error for that call. */
#define CC_COUNT_INVALID 0xFFFFFFFFFFFFFFFFull

/* One set of N objects in structure-of-arrays form. For CC_I32, x, y, z point to
 * int32_t[N] and r is ignored (may be NULL). For CC_F32, x, y, z, r point to float[N]. */
typedef struct {
    int32_t dtype;           /* cc_dtype */
    const void *x, *y, *z;
    const float *r;
} cc_points;

/* ---- single set (Section 4, proposed algorithm) ------------------------------------ */

/* Exact number of colliding unordered pairs among the n objects of *p, written to
 * d_count[0] (device, unsigned 64-bit). n = 0 or 1 gives 0. */
cc_status cc_count_pairs(const cc_points *p, int64_t n, uint32_t r2,
                         unsigned long long *d_count, void *stream);

/* Interaction sum over the colliding pairs, written to d_sum[0] (device, FP32); the
 * count of colliding pairs goes to d_count[0] when d_count is not NULL. For CC_I32 the
 * distance is sqrtf((float)d2) of the exact integer d2 and each term 1/max(d, 1e-6) is
 * rounded to FP32; terms are accumulated in FP64 (FP32 pipe) or in Kahan-compensated
 * FP32 per thread then FP64 (tensor-core kernel), in a fixed order per launch shape. */
cc_status cc_interaction_sum(const cc_points *p, int64_t n, uint32_t r2,
                             float *d_sum, unsigned long long *d_count, void *stream);

/* The same count with the straightforward schedule the paper compares against
 * (Section 5): each group of 1024 objects is tested against all later objects, so the
 * work per group falls linearly along the set. Same records and inner loop as
 * cc_count_pairs; provided to measure what the balanced cyclic schedule gains. */
cc_status cc_count_pairs_straightforward(const cc_points *p, int64_t n, uint32_t r2,
                                         unsigned long long *d_count, void *stream);

/* ---- linear-time counts for integer beads (Section 3, Algorithms 1 and 2) ------------- */

/* Algorithm 1 (countColls): the number of unordered pairs of beads on the same lattice
 * site, in O(N) through a per-site count (dense over the bounding box when it is small,
 * else a hash table in the stream's workspace). Equals cc_count_pairs with r2 = 0.
 * CC_I32 only; per-axis spans up to 2^21 - 3 (else CC_ERR_RANGE via cc_stream_status and
 * the count set to CC_COUNT_INVALID). */
cc_status cc_count_same_site(const cc_points *p, int64_t n, unsigned long long *d_count, void *stream);

/* Algorithm 2 (countContacts): the number of unordered pairs of beads on face-adjacent
 * sites (squared distance exactly 1), in O(N). Same storage and limits as above. */
cc_status cc_count_contacts(const cc_points *p, int64_t n, unsigned long long *d_count, void *stream);

/* Checks the integer range precondition on the device and WAITS for the answer
 * (synchronises the stream): CC_OK, or CC_ERR_RANGE when some axis spans more than
 * 32767. FP32 points always pass. */
cc_status cc_validate_points(const cc_points *p, int64_t n, void *stream);

/* Grows the workspace of `stream` so that single-set calls with up to max_n objects
 * allocate nothing. */
cc_status cc_reserve(int64_t max_n, void *stream);

/* Releases the workspace of `stream` (stream-ordered free). */
cc_status cc_release(void *stream);

/* Synchronises `stream`, returns the device status recorded by the calls enqueued on
 * it since the previous cc_stream_status(), and clears it. */
cc_status cc_stream_status(void *stream);

/* Diagnostic: synchronises `stream` and writes to *mode which pair kernel the device
 * chose for the last cc_count_pairs / cc_interaction_sum call on it:
 *   CC_MODE_FP32_EXACT   integer points, expanded-square form exact in FP32 (FP32 pipe)
 *   CC_MODE_INT_WIDE     integer points, int32 difference form (spans up to 32767);
 *                        for sets below 8192 objects (one launch, each unit of work
 *                        centred on its own objects) some units needed this form
 *   CC_MODE_RANGE_ERROR  span above 32767: nothing was counted
 *   CC_MODE_FP32_SPHERES FP32 spheres
 *   CC_MODE_TENSOR       integer points, the same exact form as a TF32 tensor-core
 *                        contraction (n >= 8192, and only while the absolute values
 *                        of its eight terms sum to less than 2^24)
 *   CC_MODE_TENSOR_SPHERES FP32 spheres, n >= 8192: an exact integer screen of
 *                        quantised coordinates on the tensor cores passes every pair
 *                        that can collide, and the FP32 predicate above decides each
 *                        screened pair (all coordinates and radii finite, and the
 *                        largest 2|r| at most 2.2 % of the largest coordinate span)
 * CC_ERR_NOT_FOUND when no call has run on `stream` yet. */
enum {
    CC_MODE_FP32_EXACT = 0,
    CC_MODE_INT_WIDE = 1,
    CC_MODE_RANGE_ERROR = 2,
    CC_MODE_FP32_SPHERES = 3,
    CC_MODE_TENSOR = 4,
    CC_MODE_TENSOR_SPHERES = 5
};
cc_status cc_stream_mode(void *stream, int32_t *mode);

/* Enables (1, the default) or disables (0) the tensor-core kernel for later
 * cc_count_pairs / cc_interaction_sum calls of this process; when disabled every integer
 * set runs on the FP32 pipe. Counts are identical either way (both are exact; sums agree
 * to the rounding of their accumulation order); the switch exists to
 * compare the two kernels and to keep the tensor cores free for other work. The initial
 * value comes from the environment variable CC_TC (0 disables). Always CC_OK. */
cc_status cc_set_tensor_cores(int32_t enable);

/* Same result as cc_count_pairs, for callers that must not allocate device memory while
 * they run: code recording into a CUDA graph, engines whose single allocator forbids side
 * allocations, services with a fixed memory budget that must not fail mid-run on an
 * allocation. The paper has no counterpart; this is a deployment variant of the
 * single-set path. Scratch is one static device array of 8 MiB inside the library,
 * held by every GPU that loads the library until the process exits; it fits sets of
 * about 349 thousand objects, and larger n is rejected with CC_ERR_INVALID_ARG and a
 * message that states the exact limit. The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) for that device; make that first call before
 * any stream capture. All calls share the one array, so calls that overlap on the GPU
 * (for example on two streams) race and give wrong counts; serialise them. Each call
 * clears the state it needs. The count is CC_COUNT_INVALID when the device rejects the
 * integer range or a bounded wait runs out; this call has no stream workspace, so
 * cc_stream_status() does not report it: the count is the only report. Allocates
 * nothing: no cudaMalloc, cudaFree or allocating library call. */
cc_status cc_count_pairs_noalloc(const cc_points *p, int64_t n, uint32_t r2,
                                 unsigned long long *d_count, void *stream);

/* ---- batched sets (one persistent, graph-captured launch) --------------------------- */

typedef struct cc_plan cc_plan;

/* Creates a batching plan: the work shape per size band (from tune_table_json, a JSON
 * object as written by the autotuner, {"bands": [{"n_max": N, "r": R, "sc": S}, ...]},
 * or built-in defaults when NULL: R objects per lane in warp tiles of 32*R objects and S
 * stages of 64 objects per work item, or R = 0 for one warp per set, allowed for bands
 * of at most 256 objects and not for the last band) and device work-queue storage.
 * max_sets and max_points bound the batches it accepts. A table that breaks these rules
 * gives CC_ERR_INVALID_ARG (cc_last_error() says why). */
cc_status cc_plan_create(cc_plan **plan, const char *tune_table_json,
                         int32_t max_sets, int64_t max_points);
void cc_plan_destroy(cc_plan *plan);

/* Per-set exact counts for n_sets sets. Set k holds objects [d_offsets[k],
 * d_offsets[k+1]) of *p (d_offsets: device int64[n_sets+1], non-decreasing, from 0).
 * Counts go to d_counts[k]; when d_sums is not NULL the interaction sums go to
 * d_sums[k]. One captured CUDA graph is replayed per call (no per-set launches). */
cc_status cc_count_pairs_batched(cc_plan *plan, const cc_points *p, const int64_t *d_offsets,
                                 int32_t n_sets, uint32_t r2, unsigned long long *d_counts,
                                 float *d_sums, void *stream);

/* Number of work items the last batched call on this plan produced (synchronises). */
cc_status cc_plan_last_items(cc_plan *plan, int64_t *items);

/* ---- serving (continuous batching over device-resident sets) ------------------------- */

typedef struct cc_server cc_server;

enum { CC_OP_COUNT = 0, CC_OP_SUM = 1 };

typedef struct {
    uint64_t req_id;
    int32_t set_id;
    int32_t op;
    int32_t status;              /* cc_status of this request */
    int32_t pad;
    unsigned long long count;
    float sum;
    float pad2;
    double t_arrive_s;           /* host steady-clock seconds at submit */
    double t_done_s;             /* host steady-clock seconds when the result was seen */
} cc_result;

/* Creates a server with a device-memory budget for resident sets plus per-batch scratch
 * and at most max_slots requests admitted (in flight) at once. It owns two streams and
 * one scheduler thread; its batching plans use the built-in tile table. */
cc_status cc_server_create(cc_server **srv, size_t mem_budget_bytes, int32_t max_slots);

/* The same, with the batching plans built from tune_table_json (the autotuner's JSON, as
 * for cc_plan_create; NULL = built-in defaults). CC_ERR_INVALID_ARG for a malformed
 * table. */
cc_status cc_server_create_tuned(cc_server **srv, size_t mem_budget_bytes, int32_t max_slots,
                                 const char *tune_table_json);

/* Copies a set into device memory (host or device source pointers, detected) and
 * registers it; its id goes to *set_id. Fails with CC_ERR_NOMEM beyond the budget. */
cc_status cc_server_register_set(cc_server *srv, const cc_points *p, int64_t n,
                                 int32_t *set_id);

/* Removes a registered set once no admitted request uses it. */
cc_status cc_server_unregister_set(cc_server *srv, int32_t set_id);

/* Queues a request (thread-safe, non-blocking). op: CC_OP_COUNT or CC_OP_SUM. */
cc_status cc_server_submit(cc_server *srv, int32_t set_id, int32_t op, uint32_t r2,
                           uint64_t req_id);

/* Moves up to max finished results to out[]; *n_out receives how many. A result's status
 * is CC_OK, or the device-detected condition of its request (CC_ERR_RANGE: integer span
 * beyond the supported range; CC_ERR_TIMEOUT: a bounded wait ran out), with the count
 * CC_COUNT_INVALID and the sum NaN; CC_ERR_CUDA when its batch could not be launched. */
cc_status cc_server_poll(cc_server *srv, cc_result *out, int32_t max, int32_t *n_out);

/* Blocks until every submitted request has finished or timeout_s passed. */
cc_status cc_server_drain(cc_server *srv, double timeout_s);

/* Server counters: batches launched, requests admitted, peak in-flight requests, peak
 * device bytes in use (budget accounting). Any pointer may be NULL. */
cc_status cc_server_stats(cc_server *srv, int64_t *batches, int64_t *admitted,
                          int64_t *peak_inflight, int64_t *peak_bytes);

void cc_server_destroy(cc_server *srv);

/* ---- misc ------------------------------------------------------------------------------- */

const char *cc_status_string(cc_status s);
const char *cc_last_error(void);          /* thread-local message of the last failure */

/* Kernel timing for benchmarks. While enabled, every launch of the single-set pair
 * kernel is bracketed by a CUDA event pair recorded on its launching stream. */
void cc_profile_enable(int on);

/* Waits for the recorded events and returns the summed elapsed milliseconds and the
 * number of timed launches since the previous read; then clears both. */
cc_status cc_profile_read(double *total_ms, int64_t *launches);

/* Library build identification: "cc <version> sm_103a". */
const char *cc_version(void);

/* Bound for device-side waits (nanoseconds); the default is 2 s. Waits that exceed it
 * make the kernel record CC_ERR_TIMEOUT and return. */
void cc_set_wait_limit_ns(uint64_t ns);

/* Test hook for the bounded-wait path: when stall != 0 the single-set kernels' copy
 * issuer holds back every copy, so the consumers' waits run out and the kernel returns
 * CC_ERR_TIMEOUT through the stream status. No memory is accessed out of bounds and
 * nothing faults. 0 restores normal operation. */
void cc_debug_stall_copies(int stall);

#ifdef __cplusplus
}
#endif

#endif /* CC_H */
