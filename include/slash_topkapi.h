/*
 * slash_topkapi.h -- C ABI of SLASH with TopKAPI sketch buckets on one B300 GPU.
 *
 * The paper's own bucket (Sec. 3.1 "Our Solution: Topkapi Sketches instead of
 * Buckets"; Appendix 2): every bucket address of every table holds a small
 * fixed-size TopKAPI sketch of W rows x C cells, each cell a (heavy hitter,
 * count) pair, instead of a list of ids.  Insertion (Algorithm 1) updates one
 * cell per sketch row; a query (Algorithm 2) merges the query's S*L sketches
 * cell by cell into one sketch and reports its heavy hitters -- no distance is
 * computed and no id list is gathered.  Hashing (DOPH codes, table addresses)
 * is the one of slash.h; the conventions of slash.h (return codes, d_ and h_
 * pointers, streams, CSR input, sticky data-error word) hold here too.
 *
 * Readings fixed by this library:
 *   - Cell of id in sketch row r: mix32(id ^ tk[r]) & (C - 1), with tk the W
 *     row seeds drawn after the table and priority seeds (slash.h's seed order,
 *     W in place of the count-min rows).
 *   - Insert (Appendix 2, "Insertion"): the cell's count goes up when it holds
 *     the id, else down, and a cell left at count 0 (or empty) takes (id, 1).
 *     Ids are unique, so an arriving id never matches: every non-empty cell of
 *     a bucket holds count 1 and the LAST id that reached it, and ids arrive in
 *     ascending order -- so a cell holds the largest id hashed to it.  The
 *     library stores that id + 1 (0 = empty) and takes, per cell, the maximum
 *     over the ids hashed to it -- order-free, so any parallel schedule gives
 *     the sequential rule's state exactly.
 *   - Merge (Appendix 2, "Merging"): same heavy hitter -> counts add; else the
 *     larger count wins with the difference; equal counts leave an empty cell.
 *     The merge depends on order: a query folds shard-major, then table order.
 *   - Query (Appendix 2, "Querying"): a heavy hitter's score is its largest
 *     count over the merged cells; those with score > threshold are ranked by
 *     (score descending, id ascending), top-k, padded with (-1, 0).
 */
#ifndef SLASH_TOPKAPI_H
#define SLASH_TOPKAPI_H

#include <stdint.h>

#include "slash.h"

#ifdef __cplusplus
extern "C" {
#endif

#define SLASH_TK_MAX_ROWS  8u     /* W: sketch rows                       */
#define SLASH_TK_MAX_CELLS 1024u  /* W * C: cells per sketch              */

typedef struct slash_tk_index slash_tk_index; /* opaque; owned by the library */

typedef struct {
  uint32_t dim;           /* D: feature ids must be < dim                              */
  uint32_t K;             /* codes concatenated per table address (>= 1)               */
  uint32_t L;             /* tables (1..SLASH_MAX_L); K*L <= SLASH_MAX_NB              */
  uint32_t log2_buckets;  /* B: 2^B sketches per table (1..30)                         */
  uint32_t rows;          /* W: sketch rows (1..SLASH_TK_MAX_ROWS)                     */
  uint32_t cells;         /* C: cells per row, a power of two; W*C <= SLASH_TK_MAX_CELLS */
  uint32_t shards;        /* S: on-device partitions (1 = single index)                */
  uint32_t densify;       /* SLASH_DENSIFY_SIDE or SLASH_DENSIFY_OPTIMAL (slash.h)     */
  uint64_t seed;          /* the shared random seed                                    */
  uint64_t capacity;      /* max ids ever inserted (1..2^31-1; ids are int32)          */
} slash_tk_params;

/* Allocate and clear the sketches on the current CUDA device: uint32
 * [S][L][2^B][W][C] cell words, all 0 (empty).  Sec. 4 "Initialization".
 * Synchronises `cuda_stream`.  Errors: SLASH_EINVAL (limits above, S*L*2^B*W*C
 * >= 2^40), SLASH_ENOMEM, SLASH_ECUDA. */
int slash_tk_build(const slash_tk_params *p, void *cuda_stream, slash_tk_index **out);

/* Pre-processing (Algorithm 1): rows get ids [*first_id_out, +n_rows) in order;
 * each id is inserted into one sketch per table of shard floor(id*S/capacity).
 * Results do not depend on how rows are split into calls.  Uses per-index
 * workspace grown on demand (addresses and staged ids, 8*L bytes per row of a
 * chunk of up to (2^32-1)/L rows), so one insert at a time per index.
 * n_rows = 0 is a no-op.  Errors: SLASH_EINVAL (NULL pointers with n_rows > 0),
 * SLASH_EFULL, SLASH_ENOMEM (workspace growth), SLASH_ECUDA. */
int slash_tk_insert(slash_tk_index *ix, const uint64_t *d_offs, const uint32_t *d_cols, uint32_t n_rows,
                    uint64_t *first_id_out, void *cuda_stream);

/* Querying (Algorithm 2): for each query, merge the S*L sketches at its table
 * addresses into one and write its top-k heavy hitters with score > threshold,
 * row-major [n_queries][topk]: d_ids_out int32 (-1 padding), d_scores_out uint32
 * (merged counts, 0 padding).  1 <= topk <= SLASH_MAX_TOPK; n_queries = 0 is a
 * no-op.  Errors: SLASH_EINVAL, SLASH_ECUDA. */
int slash_tk_query(slash_tk_index *ix, const uint64_t *d_offs, const uint32_t *d_cols, uint32_t n_queries,
                   uint32_t topk, uint32_t threshold, int32_t *d_ids_out, uint32_t *d_scores_out,
                   void *cuda_stream);

/* Test support -- copy every cell word to host memory, h_cells uint32
 * [S][L][2^B][W][C]: 0 = empty, else (heavy hitter id + 1) with count 1.
 * Synchronises.  Errors: SLASH_EINVAL, SLASH_ECUDA. */
int slash_tk_export(slash_tk_index *ix, uint32_t *h_cells);

/* Test support -- copy selected sketches to host memory: for i < n, sketch
 * (h_shard[i], h_table[i], h_bucket[i]) -> h_cells[i][W][C] (cell words as in
 * slash_tk_export).  Synchronises.  Errors: SLASH_EINVAL (index out of range),
 * SLASH_ECUDA. */
int slash_tk_debug_buckets(slash_tk_index *ix, const uint32_t *h_shard, const uint32_t *h_table,
                           const uint32_t *h_bucket, uint32_t n, uint32_t *h_cells);

/* Wait for `cuda_stream`, then report and clear the sticky device error word
 * (as slash_sync). */
int slash_tk_sync(slash_tk_index *ix, void *cuda_stream);

/* Empty every sketch and restart ids at 0. */
int slash_tk_reset(slash_tk_index *ix, void *cuda_stream);

/* Number of ids inserted so far. */
uint64_t slash_tk_size(const slash_tk_index *ix);

/* Kernel launches issued by this index since it was built. */
uint64_t slash_tk_launches(const slash_tk_index *ix);

/* Checkpoint of a sketch index (as slash_save / slash_load: parameters, next
 * id and every cell word, with a checksum).  Same errors. */
int slash_tk_save(slash_tk_index *ix, const char *path);
int slash_tk_load(const char *path, void *cuda_stream, slash_tk_index **out);

/* The parameters the index was built (or loaded) with.  Errors: SLASH_EINVAL. */
int slash_tk_get_params(const slash_tk_index *ix, slash_tk_params *out);

/* Release the index (synchronises the device first).  NULL is accepted. */
int slash_tk_free(slash_tk_index *ix);

#ifdef __cplusplus
}
#endif
#endif /* SLASH_TOPKAPI_H */
