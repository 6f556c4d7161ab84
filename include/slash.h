/*
 * slash.h -- C ABI of the SLASH similarity-search hot path on one B300 GPU.
 *
 * Method: Meisburger & Shrivastava, "Distributed Tera-Scale Similarity Search
 * with MPI" (arXiv 2008.03260).  The library indexes very sparse binary
 * vectors with densified one-permutation MinHash (DOPH, Sec. 2.2) in a
 * (K, L)-parameterised LSH structure (Sec. 2.3), stores ids in fixed-size
 * sub-sampled buckets (Sec. 3, "Avoid Skewed buckets"), and answers a query by
 * counting the ids of its L buckets in a count-min sketch and ranking them by
 * estimated frequency (Sec. 2.3 "Cheap Frequency based Filtering and K-NN";
 * Algorithm 2) -- no distance is ever computed.  The paper's m machine
 * partitions D_i (Sec. 3, Design) become `shards` on-device partitions whose
 * sketches are summed in device memory (Algorithm 2, merge across machines).
 *
 * Conventions for every entry point:
 *   - Return value: SLASH_OK (0) or a negative SLASH_E* code; slash_strerror()
 *     names it.  A call that fails validation changes nothing.
 *   - Pointers named d_* are caller-owned DEVICE memory on the index's device;
 *     the library never frees or retains them past the call's stream work.
 *     Pointers named h_* are caller-owned host memory.
 *   - `cuda_stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *     enqueued on it and the call returns without waiting, except where a call
 *     says it synchronises.  Caller buffers must stay valid until that stream
 *     work completes.
 *   - Errors the device finds in the data (a column id >= dim, decreasing
 *     offsets) do not fault: the offending feature (or row) is skipped, a
 *     sticky error word is set, and the next slash_sync() returns SLASH_EDATA
 *     and clears it.
 *   - An index is not thread-safe: serialise calls on one index.  Inserts, plain
 *     queries (SLASH_QUERY_PLAIN, SLASH_QUERY_WARP_PLAIN) and debug calls use
 *     per-index workspace, so issue them on one stream at a time.  Fused queries
 *     (SLASH_QUERY_FUSED, the default schedule, and SLASH_QUERY_WARP_FUSED) use no
 *     shared workspace: up to 4096 of them may be in flight at once on different
 *     streams, as long as no insert or reset runs meanwhile.
 *   - CSR input: row i's feature ids are d_cols[d_offs[i] .. d_offs[i+1]), ids
 *     in [0, dim); d_offs holds n+1 entries (d_offs[0] need not be 0).  Order
 *     and duplicates within a row do not matter (MinHash is a set function);
 *     a row with no features is valid (all its codes are empty, it still
 *     occupies one bucket per table).
 */
#ifndef SLASH_H
#define SLASH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SLASH_OK        0
#define SLASH_EINVAL   (-1)  /* bad argument or parameter                          */
#define SLASH_ENOMEM   (-2)  /* device allocation failed (index left unchanged)    */
#define SLASH_ECUDA    (-3)  /* a CUDA runtime call failed                         */
#define SLASH_EFULL    (-4)  /* insert would exceed `capacity`                     */
#define SLASH_EBUSY    (-5)  /* admission refused (serving layer)                  */
#define SLASH_ETIMEOUT (-6)  /* a bounded device wait gave up                      */
#define SLASH_EDATA    (-7)  /* the device found invalid input data (see above)    */
#define SLASH_EIO      (-8)  /* a checkpoint file could not be opened, written or read */

#define SLASH_EMPTY 0xFFFFFFFFu /* an unused bucket slot */

/* Limits of this implementation (checked by slash_build_index). */
#define SLASH_MAX_L     128u   /* tables                                  */
#define SLASH_MAX_NB    1024u  /* K * L DOPH bins                         */
#define SLASH_MAX_R     512u   /* reservoir slots per bucket              */
#define SLASH_MAX_CMROWS 8u    /* count-min rows d                        */
#define SLASH_MAX_TOPK  256u   /* k of a query                            */

typedef struct slash_index slash_index; /* opaque; owned by the library */

/* Index parameters.  Sec. 4 "Initialization": L x K hash functions from one
 * shared seed; every shard (the paper's machine partition) uses the same
 * functions, so the shards form one logical index. */
typedef struct {
  uint32_t dim;           /* D: feature ids must be < dim                          */
  uint32_t K;             /* codes concatenated per table address (>= 1)           */
  uint32_t L;             /* tables (1..SLASH_MAX_L); K*L <= SLASH_MAX_NB          */
  uint32_t log2_buckets;  /* B: 2^B buckets per table (1..30)                      */
  uint32_t reservoir;     /* R: ids kept per bucket (1..SLASH_MAX_R)               */
  uint32_t cm_rows;       /* d: count-min rows (1..SLASH_MAX_CMROWS)               */
  uint32_t cm_width;      /* w: counters per row, a power of two (>= 32)           */
  uint32_t shards;        /* S: on-device partitions (1 = single index)            */
  uint64_t seed;          /* the shared random seed                                */
  uint64_t capacity;      /* max ids ever inserted (1..2^31-1; ids are int32)      */
  uint32_t densify;       /* DOPH densification: SLASH_DENSIFY_SIDE or _OPTIMAL    */
  uint32_t reserved;      /* must be 0                                             */
} slash_params;

/* Densification rules for the empty DOPH bins (Sec. 2.2).  SIDE: the nearest
 * non-empty bin on a fixed per-bin side (left or right), circularly.  OPTIMAL:
 * optimal densification (Shrivastava, ICML 2017; the densified variant Sec. 6
 * says SLASH implements): empty bin j copies the first non-empty bin of the
 * probe sequence umulhi(mix32(mix32(j ^ od) + a), K*L), a = 1, 2, ..., with od
 * the seed word drawn after the count-min (or sketch-row) seeds; after
 * 32*K*L probes without a non-empty bin the SIDE rule decides.  Lower-variance
 * codes for sparse rows, at roughly K*L / (non-empty bins) probes per empty bin. */
#define SLASH_DENSIFY_SIDE    0u
#define SLASH_DENSIFY_OPTIMAL 1u

/* Allocate and clear an index on the current CUDA device: buckets
 * uint32 [S][L][2^B][R] (SLASH_EMPTY) and fill counts uint32 [S][L][2^B] (0).
 * Sec. 4 "Initialization".  Synchronises `cuda_stream`.
 * Errors: SLASH_EINVAL (limits above), SLASH_ENOMEM, SLASH_ECUDA. */
int slash_build_index(const slash_params *p, void *cuda_stream, slash_index **out);

/* Pre-processing (Algorithm 1): rows get ids [*first_id_out, +n_rows) in
 * order; each id enters one bucket per table of shard floor(id*S/capacity).
 * A bucket keeps the R ids of smallest seeded priority among all ids ever
 * inserted into it, in ascending priority -- independent of insertion order
 * and of how rows are split into calls.  n_rows = 0 is a no-op.
 * Errors: SLASH_EINVAL (NULL pointers with n_rows > 0), SLASH_EFULL,
 * SLASH_ENOMEM (workspace growth), SLASH_ECUDA. */
int slash_insert(slash_index *ix, const uint64_t *d_offs, const uint32_t *d_cols, uint32_t n_rows,
                 uint64_t *first_id_out, void *cuda_stream);

/* slash_insert from HOST memory: h_offs (n_rows+1 offsets into h_cols, checked on
 * the host: decreasing offsets give SLASH_EINVAL) and h_cols.  Pieces of up to 2M
 * rows are copied to two library-owned device staging slots on an internal copy
 * stream while the previous piece is hashed on `cuda_stream`; the per-bucket
 * merge then runs once per chunk.  Page-locked host buffers give overlapped
 * copies; pageable ones still work.  The caller keeps both buffers unchanged
 * until `cuda_stream`'s work completes.  Same results and errors as slash_insert
 * (plus SLASH_ENOMEM for the staging slots). */
int slash_insert_host(slash_index *ix, const uint64_t *h_offs, const uint32_t *h_cols, uint32_t n_rows,
                      uint64_t *first_id_out, void *cuda_stream);

/* Querying (Algorithm 2): for each query, hash it into its L buckets, gather
 * the ids they hold in every shard, count them in a d x w count-min sketch
 * (shard sketches summed), estimate each distinct candidate's frequency as the
 * minimum over rows, and write the top-k candidates by (estimate descending,
 * id ascending).  Outputs, row-major [n_queries][topk]: d_ids_out int32 (-1
 * padding when fewer than topk candidates exist) and d_scores_out uint32 (the
 * estimates, 0 padding).  1 <= topk <= SLASH_MAX_TOPK; n_queries = 0 is a no-op.
 * Errors: SLASH_EINVAL, SLASH_ENOMEM, SLASH_ECUDA. */
int slash_query(slash_index *ix, const uint64_t *d_offs, const uint32_t *d_cols, uint32_t n_queries,
                uint32_t topk, int32_t *d_ids_out, uint32_t *d_scores_out, void *cuda_stream);

/* Query schedules.  All give bit-identical results. */
#define SLASH_QUERY_FUSED 0u       /* one persistent launch: hash -> gather -> count -> top-k per CTA team   */
#define SLASH_QUERY_PLAIN 1u       /* one launch per stage: hash kernel, then gather/count/top-k kernel      */
#define SLASH_QUERY_WARP_FUSED 2u  /* one warp per query (hash included); for queries with few candidates:
                                      up to 32 counted by warp matches, up to 512 in a per-warp table, more
                                      by the team engine of SLASH_QUERY_FUSED where the index has one, else
                                      by the general kernel.  topk <= 10 and cm_width <= 32768 only          */
#define SLASH_QUERY_WARP_PLAIN 3u  /* the same after the hash kernel; queries above 512 candidates by the
                                      general kernel                                                        */

typedef struct {
  uint32_t mode;         /* SLASH_QUERY_FUSED, _PLAIN, _WARP_FUSED or _WARP_PLAIN                   */
  uint32_t threads;      /* threads per CTA (team): 256, 512 or 1024 (0 = the index's default);
                            the warp schedules always run 8 warps per CTA                             */
  uint32_t ctas_per_sm;  /* cap on resident CTAs per SM (0 = as many as fit)                          */
  uint32_t max_sms;      /* the launch's persistent CTAs fill at most this many SMs' worth of slots
                            (grid <= max_sms x resident CTAs per SM), leaving the rest of the GPU to
                            work on other streams; 0 or >= the SM count = the whole GPU.  The answers
                            do not depend on it                                                       */
} slash_query_opts;

/* slash_query with an explicit schedule (opts == NULL: the index's default,
 * initially {FUSED, smallest CTA holding S*L*R ids at 8 per thread, 0}, replaced
 * by slash_autotune).  Same outputs and
 * errors as slash_query; SLASH_EINVAL also when the schedule does not fit. */
int slash_query_ex(slash_index *ix, const uint64_t *d_offs, const uint32_t *d_cols, uint32_t n_queries,
                   uint32_t topk, int32_t *d_ids_out, uint32_t *d_scores_out, const slash_query_opts *opts,
                   void *cuda_stream);

/* Autotuner: time every query schedule (mode x threads x CTAs/SM; the warp
 * schedules suit batches of queries with few candidates, the team schedules
 * those with many) on the given
 * sample batch (each twice after a warm-up, CUDA events on `cuda_stream`), make
 * the fastest the index's default, and report it (*best_out, *best_ms_out may be
 * NULL).  The outputs buffers receive the sample's results.  Synchronises. */
int slash_autotune(slash_index *ix, const uint64_t *d_offs, const uint32_t *d_cols, uint32_t n_queries,
                   uint32_t topk, int32_t *d_ids_out, uint32_t *d_scores_out, void *cuda_stream,
                   slash_query_opts *best_out, float *best_ms_out);

/* Allocation-free query (this entry point has no counterpart in the paper).
 * Same results and errors as slash_query_ex with {SLASH_QUERY_PLAIN, 512, 0},
 * for callers that cannot call cudaMalloc at query time, such as hosts that
 * hand out all device memory from their own pool at start-up.
 * Its only scratch, the batch's table addresses, lives in a fixed 16 MiB
 * array inside the library's device image (held by every GPU that loads the
 * library, until the process exits), so n_queries * L must be <= 4194304
 * (else SLASH_EINVAL, nothing launched).  The index's device must be current
 * (else SLASH_EINVAL).  The first call on a device looks up the array's device
 * address (no allocation).
 * Every call shares the array and nothing in it needs clearing: calls whose
 * work overlaps on the GPU (other streams, or without ordering) race on it. */
int slash_query_static(slash_index *ix, const uint64_t *d_offs, const uint32_t *d_cols, uint32_t n_queries,
                       uint32_t topk, int32_t *d_ids_out, uint32_t *d_scores_out, void *cuda_stream);

/* ---- One logical index over several processes (Sec. 3 partitions; Algorithm 2's
 * merge across machines as one exchange of candidates).  Process r indexes the
 * ids [ceil(r*N/W), ceil((r+1)*N/W)) of N rows (W processes, one index each
 * with shards = 1, capacity = N and the shared seed).  A query batch, the same
 * on every process, is answered by: slash_query_candidates on each process; an
 * all-gather of the counts and ids; slash_query_cells on each process; a sum
 * over processes of the cells; slash_rank_candidates.  Because partitions hold
 * disjoint ids, the summed cells are those of the one index whose shards are
 * the partitions, and the ranking is identical to its slash_query. */

/* Rows inserted next get ids from next_id on (the first global id of this
 * process's partition).  next_id may not be below the index's next id nor above
 * its capacity (else SLASH_EINVAL). */
int slash_set_next_id(slash_index *ix, uint64_t next_id);

/* Each query's distinct candidates in this index (the ids of its S*L buckets):
 * d_counts int32 [n_queries], d_ids int32 [n_queries][m] in the order of their
 * first occurrence in the query's buckets (shard-major, then table, then slot),
 * -1 past the count; m >= S*L*R.  Uses the plain-query workspace (SLASH_ENOMEM
 * if it cannot grow).  Errors: SLASH_EINVAL (m too small, NULL, or S*L*R too
 * large for one CTA's shared memory), SLASH_ENOMEM, SLASH_ECUDA. */
int slash_query_candidates(slash_index *ix, const uint64_t *d_offs, const uint32_t *d_cols, uint32_t n_queries,
                           uint32_t m, int32_t *d_counts, int32_t *d_ids, void *cuda_stream);

/* This index's count-min cells of the gathered candidates: for process w <
 * world, query q and j < m, d_cells[((w*n_queries + q)*m + j)*d + r] = this
 * index's sketch count in row r (d = cm_rows) at the cell of d_ids[(w*n_queries
 * + q)*m + j], the sketch being the one query q builds from its own buckets;
 * entries with j >= d_counts[w*n_queries + q] are not written (the ranking
 * reads only those below the count).  Here m is the row length of the gathered
 * ids (>= 1; rows may be cut to the largest count, and counts above m are
 * read as m).  d_cells must be 16-byte aligned.  Errors: SLASH_EINVAL (world
 * 1..64, m = 0, NULL, misaligned d_cells), SLASH_ENOMEM, SLASH_ECUDA. */
int slash_query_cells(slash_index *ix, const uint64_t *d_offs, const uint32_t *d_cols, uint32_t n_queries,
                      uint32_t world, uint32_t m, const int32_t *d_counts, const int32_t *d_ids, uint32_t *d_cells,
                      void *cuda_stream);

/* The ranking of Algorithm 2 from gathered candidates and their cells summed
 * over processes: per query, every id j < d_counts[w*n_queries + q] of every
 * process w gets the estimate min over r of its d cells; the top-k by (estimate
 * descending, id ascending) go to d_ids_out int32 [n_queries][topk] and
 * d_scores_out uint32 (padding -1 / 0).  Needs no index.  Errors: SLASH_EINVAL
 * (world 1..64, d 1..SLASH_MAX_CMROWS, topk 1..SLASH_MAX_TOPK, NULL), SLASH_ECUDA. */
int slash_rank_candidates(uint32_t world, uint32_t n_queries, uint32_t m, uint32_t d, const int32_t *d_counts,
                          const int32_t *d_ids, const uint32_t *d_cells, uint32_t topk, int32_t *d_ids_out,
                          uint32_t *d_scores_out, void *cuda_stream);

/* Allocator hook (no counterpart in the paper): the index's workspace -- the
 * insert buffers (addresses, staged ids, merge lists), the plain-query
 * addresses and the host-fed insert's device staging -- comes from
 * alloc(bytes, ctx), which returns device memory on the index's device (at
 * least 256-byte aligned) or NULL when it has none, and goes back through
 * release(ptr, ctx).  Lets a host's caching allocator (for example PyTorch's)
 * supply and account that memory.  The index's own arrays (buckets, fills,
 * counters) stay where slash_build_index put them.  Workspace is taken when a
 * call first needs it or needs more, and released when it grows, when the
 * allocator changes and at slash_free; before each release the library waits
 * for the device, so released memory is idle.  alloc = release = NULL restores
 * cudaMalloc/cudaFree.  A NULL from alloc makes the call that needed the
 * memory return SLASH_ENOMEM with the index unchanged.  Setting it releases
 * the current workspace with the allocator that made it.  Synchronises the
 * device.  Errors: SLASH_EINVAL (NULL index, or only one of alloc / release),
 * SLASH_ECUDA. */
typedef void *(*slash_alloc_fn)(size_t bytes, void *ctx);
typedef void (*slash_free_fn)(void *ptr, void *ctx);
int slash_set_allocator(slash_index *ix, slash_alloc_fn alloc, slash_free_fn release, void *ctx);

/* Checkpoint (no counterpart in the paper, whose index lives only for one run):
 * write the whole index state -- parameters, the next id, fill counts and
 * bucket slots -- to the file `path` (created or truncated), after a header
 * with a 64-bit checksum of the arrays.  Synchronises the device.
 * Errors: SLASH_EINVAL (NULL), SLASH_EIO (file), SLASH_ECUDA, SLASH_ENOMEM
 * (the 64 MiB page-locked staging buffer). */
int slash_save(slash_index *ix, const char *path);

/* Build an index on the current device from a slash_save file; inserts and
 * queries then continue exactly as on the saved index (same ids, buckets and
 * results).  Synchronises.  Errors: SLASH_EIO (cannot open), SLASH_EINVAL (not
 * such a checkpoint, parameters outside the limits, truncated, trailing bytes
 * or checksum mismatch; nothing is returned), SLASH_ENOMEM, SLASH_ECUDA. */
int slash_load(const char *path, void *cuda_stream, slash_index **out);

/* The parameters the index was built (or loaded) with.  Errors: SLASH_EINVAL. */
int slash_get_params(const slash_index *ix, slash_params *out);

/* Release the index and its workspace (synchronises the device first).
 * NULL is accepted.  Always SLASH_OK unless a CUDA call fails. */
int slash_free(slash_index *ix);

/* Human-readable name of a return code (static storage). */
const char *slash_strerror(int code);

/* Wait for `cuda_stream`, then report and clear the sticky device error word:
 * SLASH_EDATA if invalid input data was seen since the last call, SLASH_ECUDA
 * on an asynchronous CUDA error, else SLASH_OK. */
int slash_sync(slash_index *ix, void *cuda_stream);

/* Empty every bucket and restart ids at 0 (same state as a fresh build). */
int slash_reset(slash_index *ix, void *cuda_stream);

/* Number of ids inserted so far. */
uint64_t slash_size(const slash_index *ix);

/* Profiling support -- when enabled (enable != 0), every kernel the index
 * launches is bracketed by CUDA events recorded on its launch stream.  Each
 * call synchronises the device and discards the previous record. */
int slash_profile(slash_index *ix, int enable);

/* Profiling support -- per kernel name (at most max_kernels of them, in first
 * launch order): h_names char [max_kernels][32] (NUL-terminated), h_ms summed
 * event time in milliseconds, h_launches launch count; *n_kernels_out = the
 * number of distinct kernels recorded; *total_launches_out (may be NULL) =
 * kernel launches issued by this index since it was built, profiled or not.
 * Synchronises.  Any output array may be NULL.  Errors: SLASH_EINVAL, SLASH_ECUDA. */
int slash_profile_read(slash_index *ix, uint32_t max_kernels, char *h_names, float *h_ms,
                       uint32_t *h_launches, uint32_t *n_kernels_out, uint64_t *total_launches_out);

/* Test support -- the DOPH codes (Sec. 2.2, after densification) d_codes
 * uint32 [n][K*L] (may be NULL) and table addresses d_buckets uint32 [L][n]
 * (table-major) of n CSR rows, computed by the same kernel that insert and
 * query use.  Errors: SLASH_EINVAL, SLASH_ECUDA. */
int slash_debug_hash(slash_index *ix, const uint64_t *d_offs, const uint32_t *d_cols, uint32_t n,
                     uint32_t *d_codes, uint32_t *d_buckets, void *cuda_stream);

/* Measurement support (no counterpart in the paper) -- a shared-memory
 * microbenchmark on the current device that gives the count-min update its
 * ceiling: `ctas_per_sm` CTAs of `threads` threads per SM (256, 512 or 1024;
 * 1..8) each run `iters` operations per thread on a shared table of `words`
 * 32-bit words (a power of two, 32..65536) at pseudo-random addresses.  mode 0:
 * atomicAdd at a random word (the sketch update); 1: plain load at a random word;
 * 2: atomicAdd at a random word of the lane's own bank (no bank conflicts);
 * 3: atomicAdd with every lane of a warp on one word.  *ms_out = the fastest of
 * three timed launches (after a warm-up), *ops_out = operations per launch.
 * Synchronises the device.  Errors: SLASH_EINVAL, SLASH_ENOMEM, SLASH_ECUDA. */
int slash_probe_smem(uint32_t mode, uint32_t words, uint32_t iters, uint32_t threads, uint32_t ctas_per_sm,
                     float *ms_out, uint64_t *ops_out);

/* Test support -- resident CTAs per SM that the occupancy calculator allows
 * the query kernel of schedule (mode, threads) at this index's shape, before any
 * cap the launch applies.  Errors: SLASH_EINVAL, SLASH_ECUDA. */
int slash_debug_occupancy(slash_index *ix, uint32_t mode, uint32_t threads, int *ctas_per_sm_out);

/* Test support -- the next `count` device allocations this index makes for its
 * workspace (insert, plain-query and host-staging buffers) fail as if the device
 * were out of memory: the call that needed them returns SLASH_ENOMEM before any
 * work is enqueued, and the index (its buckets, fills and next id) is unchanged.
 * count = 0 cancels.  Errors: SLASH_EINVAL (NULL). */
int slash_debug_fail_alloc(slash_index *ix, uint32_t count);

/* Test support -- while enabled, the shared-memory copy wait of the staged
 * query engine (the one serving topk <= 10 when R is a multiple of 4 and S*L <=
 * 128) waits for
 * 16 bytes that no copy delivers, so every such wait gives up after its 1 s
 * limit: the kernel sets the sticky error word and returns, the next
 * slash_sync() reports SLASH_ETIMEOUT, and the device stays usable.  Query
 * outputs of such a call are undefined.  Errors: SLASH_EINVAL (NULL, or an
 * index the staged engine does not serve). */
int slash_debug_stall_copies(slash_index *ix, int enable);

/* Test support -- checked builds.  The library built with -DSLASH_CHECKS
 * (libslash_checked.so, the same entry points) tests every bucket key and
 * staging offset its kernels derive from the data before using it; one out of
 * range raises a device-wide flag and the access is skipped.  This call reports
 * *checked_out = 1 in such a build (0 otherwise) and *errors_out = the flag
 * (nonzero: some kernel found an index out of range since the last call),
 * then clears it.  Synchronises the device in a checked build.
 * Errors: SLASH_EINVAL (NULL), SLASH_ECUDA. */
int slash_debug_bounds(uint32_t *checked_out, uint32_t *errors_out);

/* Test support -- copy the whole index to host memory: h_slots uint32
 * [S][L][2^B][R], h_fill uint32 [S][L][2^B].  Synchronises.  Either pointer
 * may be NULL.  Errors: SLASH_ECUDA. */
int slash_debug_export(slash_index *ix, uint32_t *h_slots, uint32_t *h_fill);

/* Test support -- copy selected buckets to host memory: for i < n,
 * bucket (h_shard[i], h_table[i], h_bucket[i]) -> h_slots[i][R], h_fill[i].
 * Synchronises.  Errors: SLASH_EINVAL (index out of range), SLASH_ECUDA. */
int slash_debug_buckets(slash_index *ix, const uint32_t *h_shard, const uint32_t *h_table,
                        const uint32_t *h_bucket, uint32_t n, uint32_t *h_slots, uint32_t *h_fill);

#ifdef __cplusplus
}
#endif
#endif /* SLASH_H */
