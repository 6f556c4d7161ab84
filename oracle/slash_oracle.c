/*
 * SLASH oracle: plain, slow, obviously-correct CPU definition of the hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file's library.  The product path
 * (the CUDA library) neither links nor calls it, and this file includes no
 * header of the product path: every primitive below is written out here.
 *
 * What it computes, in the paper's order (arXiv 2008.03260):
 *   1. MinHash on a binary vector with a seeded hash in place of the random
 *      permutation pi (Sec. 2.2, "MinHash and Densified MinHash").
 *   2. Densified one-permutation hashing (DOPH): the hash range is split into
 *      nb = K*L bins; each bin keeps the minimum hash that falls in it; an
 *      empty bin copies the value of the nearest non-empty bin to its left or
 *      right, the side chosen at random (Sec. 2.2).
 *   3. (K, L) LSH: table i's address is built from the K codes
 *      h_{i_1..i_K} of that table (Sec. 2.3; Sec. 4 "Initialization").
 *   4. Pre-processing (Algorithm 1): each vector is inserted into one bucket
 *      per table.  Buckets are fixed-size reservoirs (Sec. 3, "Avoid Skewed
 *      buckets"), read here as: bucket keeps the R inserted ids of smallest
 *      seeded priority, stored in ascending priority.
 *   5. Querying (Algorithm 2, the local merge and the cross-partition merge):
 *      the ids in the query's L buckets are counted in a count-min sketch
 *      (Sec. 3.1 names count-min as TopKAPI's parent; Appendix 2 gives the
 *      row-per-hash layout), the sketches of the partitions are summed, and
 *      candidates are ranked by estimated frequency (Sec. 2.3, "Cheap
 *      Frequency based Filtering and K-NN"), ties broken by smaller id.
 *
 * Fixed readings where the paper leaves a free choice (all integer):
 *   mix32(x)      MurmurHash3 32-bit finaliser (Appleby, public domain)
 *   sub-seeds     SplitMix64 (Steele, Lea & Flood 2014) from `seed`, upper 32
 *                 bits of each output, drawn in the order a, dirseed,
 *                 st[0..L), sp[0..L), sc[0..d)
 *   h(f)          mix32(f ^ a)                           (stands in for pi)
 *   bin(f)        (h(f) * nb) >> 32                      (range partition)
 *   dir(j)        mix32(j ^ dirseed) & 1, 1 = right       (per-bin, not per-row)
 *   address_t     acc = st[t]; acc = (acc ^ code[tK+j]) * 0x9E3779B1 for j < K;
 *                 bucket = mix32(acc) >> (32 - B)
 *   pri(id, t)    mix31((id ^ sp[t]) & 0x7FFFFFFF), mix31 = the same finaliser
 *                 steps with every product reduced mod 2^31: a bijection of the
 *                 id space [0, 2^31), so priorities never tie and never reach
 *                 0xFFFFFFFF
 *   cell_r(id)    mix32(id ^ sc[r]) & (w - 1)
 *   shard(id)     floor(id * S / capacity)               (partitions D_i, Sec. 3)
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_EMPTY 0xFFFFFFFFu

/* ------------------------------------------------------------------ primitives */

uint32_t or_mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x85EBCA6Bu;
  x ^= x >> 13;
  x *= 0xC2B2AE35u;
  x ^= x >> 16;
  return x;
}

uint64_t or_splitmix64_next(uint64_t *state) {
  *state += 0x9E3779B97F4A7C15ull;
  uint64_t z = *state;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* out = [a, dirseed, st[0..L), sp[0..L), sc[0..d)] (2 + 2L + d words).
 * Sec. 4 "Initialization": every partition shares these seeds, so all
 * partitions use the same hash functions. */
void or_derive_seeds(uint64_t seed, uint32_t L, uint32_t d, uint32_t *out) {
  uint64_t s = seed;
  uint32_t n = 2 + 2 * L + d;
  for (uint32_t i = 0; i < n; ++i) out[i] = (uint32_t)(or_splitmix64_next(&s) >> 32);
}

/* out = the or_derive_seeds words, then od (the next SplitMix64 word: the
 * probe seed of optimal densification) and the densification mode:
 * 2 + 2L + d + 2 words in all. */
void or_seeds_init(uint64_t seed, uint32_t L, uint32_t d, uint32_t densify, uint32_t *out) {
  uint64_t s = seed;
  uint32_t n = 2 + 2 * L + d;
  for (uint32_t i = 0; i <= n; ++i) out[i] = (uint32_t)(or_splitmix64_next(&s) >> 32);
  out[n + 1] = densify;
}

/* MinHash of a binary vector under the seeded hash: min over its features (Sec. 2.2).
 * Returns OR_EMPTY for an empty vector. */
uint32_t or_minhash(const uint32_t *cols, uint64_t nnz, uint32_t a) {
  uint32_t m = OR_EMPTY;
  for (uint64_t i = 0; i < nnz; ++i) {
    uint32_t h = or_mix32(cols[i] ^ a);
    if (h < m) m = h;
  }
  return m;
}

/* DOPH with densification (Sec. 2.2).  codes[nb]; nonempty[nb] (optional) gets
 * 1 where the bin held a feature before densification. */
void or_doph(const uint32_t *cols, uint64_t nnz, uint32_t nb, uint32_t a, uint32_t dirseed,
             uint32_t *codes, uint8_t *nonempty) {
  uint32_t *m = (uint32_t *)malloc(sizeof(uint32_t) * nb);
  uint8_t *full = (uint8_t *)calloc(nb, 1);
  for (uint32_t j = 0; j < nb; ++j) m[j] = OR_EMPTY;
  /* one pass over the features: each lands in the bin its hash falls in */
  for (uint64_t i = 0; i < nnz; ++i) {
    uint32_t h = or_mix32(cols[i] ^ a);
    uint32_t j = (uint32_t)(((uint64_t)h * nb) >> 32);
    if (!full[j] || h < m[j]) m[j] = h;
    full[j] = 1;
  }
  int any = 0;
  for (uint32_t j = 0; j < nb; ++j) any |= full[j];
  /* densification: an empty bin takes the nearest non-empty bin on its side */
  for (uint32_t j = 0; j < nb; ++j) {
    if (full[j] || !any) { codes[j] = m[j]; continue; }
    int right = (int)(or_mix32(j ^ dirseed) & 1u);
    uint32_t k = j;
    for (;;) {
      k = right ? (k + 1) % nb : (k + nb - 1) % nb;
      if (full[k]) break;
    }
    codes[j] = m[k];
  }
  if (nonempty) memcpy(nonempty, full, nb);
  free(m);
  free(full);
}

/* Densified one-permutation hashing with optimal densification (Shrivastava,
 * ICML 2017 -- the densified variant Sec. 6 says SLASH implements): the bins
 * are filled as in or_doph; an empty bin j then probes the bins
 *   p_a(j) = (mix32(mix32(j ^ od) + a) * nb) >> 32,  a = 1, 2, ...
 * and copies the value of the first non-empty one.  The probe sequence depends
 * on j and the seed only, never on the row.  After OR_OPT_PROBES(nb) probes
 * without success the bin takes the side rule of or_doph instead (dirseed). */
#define OR_OPT_PROBES(nb) (32u * (nb))

void or_doph_opt(const uint32_t *cols, uint64_t nnz, uint32_t nb, uint32_t a, uint32_t od, uint32_t dirseed,
                 uint32_t *codes, uint8_t *nonempty) {
  uint8_t *full = (uint8_t *)malloc(nb);
  uint32_t *side = (uint32_t *)malloc(sizeof(uint32_t) * nb);
  or_doph(cols, nnz, nb, a, dirseed, side, full);  /* bins + the side rule's codes */
  int any = 0;
  for (uint32_t j = 0; j < nb; ++j) any |= full[j];
  for (uint32_t j = 0; j < nb; ++j) {
    if (full[j] || !any) { codes[j] = side[j]; continue; }
    uint32_t base = or_mix32(j ^ od), found = 0;
    for (uint32_t t = 1; t <= OR_OPT_PROBES(nb) && !found; ++t) {
      uint32_t p = (uint32_t)(((uint64_t)or_mix32(base + t) * nb) >> 32);
      if (full[p]) { codes[j] = side[p]; found = 1; }  /* a non-empty bin keeps its own value */
    }
    if (!found) codes[j] = side[j];
  }
  if (nonempty) memcpy(nonempty, full, nb);
  free(full);
  free(side);
}

/* The index's DOPH: seeds as written by or_seeds_init for L tables, d rows. */
static void or_doph_seeded(const uint32_t *cols, uint64_t nnz, uint32_t nb, const uint32_t *seeds, uint32_t L,
                           uint32_t d, uint32_t *codes) {
  uint32_t od = seeds[2 + 2 * L + d], densify = seeds[2 + 2 * L + d + 1];
  if (densify) or_doph_opt(cols, nnz, nb, seeds[0], od, seeds[1], codes, NULL);
  else or_doph(cols, nnz, nb, seeds[0], seeds[1], codes, NULL);
}

/* H_t: the K codes of table t -> one of 2^B addresses (Sec. 2.3). */
uint32_t or_table_address(const uint32_t *codes, uint32_t t, uint32_t K, uint32_t B, uint32_t st_t) {
  uint32_t acc = st_t;
  for (uint32_t j = 0; j < K; ++j) acc = (acc ^ codes[t * K + j]) * 0x9E3779B1u;
  return or_mix32(acc) >> (32 - B);
}

/* 31-bit bijection: each step (xor-shift, odd multiply mod 2^31) is invertible */
uint32_t or_mix31(uint32_t x) {
  const uint32_t M = 0x7FFFFFFFu;
  x &= M;
  x ^= x >> 16;
  x = (x * 0x85EBCA6Bu) & M;
  x ^= x >> 13;
  x = (x * 0xC2B2AE35u) & M;
  x ^= x >> 16;
  return x;
}

uint32_t or_priority(uint32_t id, uint32_t sp_t) { return or_mix31(id ^ sp_t); }

uint32_t or_cm_cell(uint32_t id, uint32_t sc_r, uint32_t w) { return or_mix32(id ^ sc_r) & (w - 1); }

/* per-row DOPH codes (optional, [n][K*L]) and table addresses ([n][L]) */
void or_hash_rows(uint32_t K, uint32_t L, uint32_t B, uint32_t d, const uint32_t *seeds, const uint64_t *offs,
                  const uint32_t *cols, uint64_t n, uint32_t *codes_out, uint32_t *buckets_out) {
  uint32_t nb = K * L;
  const uint32_t *st = seeds + 2;
  uint32_t *codes = (uint32_t *)malloc(sizeof(uint32_t) * nb);
  for (uint64_t i = 0; i < n; ++i) {
    or_doph_seeded(cols + (offs[i] - offs[0]), offs[i + 1] - offs[i], nb, seeds, L, d, codes);
    if (codes_out) memcpy(codes_out + i * nb, codes, sizeof(uint32_t) * nb);
    for (uint32_t t = 0; t < L; ++t) buckets_out[i * L + t] = or_table_address(codes, t, K, B, st[t]);
  }
  free(codes);
}

/* ------------------------------------------------------------------ index */

typedef struct {
  uint32_t K, L, B, R, d, w, S;
  uint64_t capacity, next_id;
  uint32_t *seeds;      /* or_seeds_init: 2 + 2L + d + 2 */
  /* per shard s: bucket (t, b) lives at storage row map[t*2^B + b] (dense: identity) */
  int64_t *map;         /* NULL = dense */
  uint64_t nstore;      /* materialised buckets per shard */
  uint32_t *slots;      /* [S][nstore][R] */
  uint32_t *fill;       /* [S][nstore]    */
} or_index;

static uint64_t or_loc(const or_index *ix, uint32_t t, uint32_t b) {
  uint64_t key = ((uint64_t)t << ix->B) + b;
  return ix->map ? (uint64_t)ix->map[key] : key;
}

/* dense index (all L * 2^B buckets per shard; calloc keeps untouched pages free) */
void *or_new(uint32_t K, uint32_t L, uint32_t B, uint32_t R, uint32_t d, uint32_t w, uint32_t S,
             uint64_t seed, uint64_t capacity, uint32_t densify) {
  or_index *ix = (or_index *)calloc(1, sizeof(or_index));
  ix->K = K; ix->L = L; ix->B = B; ix->R = R; ix->d = d; ix->w = w; ix->S = S;
  ix->capacity = capacity;
  ix->seeds = (uint32_t *)malloc(sizeof(uint32_t) * (2 + 2 * L + d + 2));
  or_seeds_init(seed, L, d, densify, ix->seeds);
  ix->nstore = (uint64_t)L << B;
  ix->slots = (uint32_t *)calloc(ix->nstore * S * R, sizeof(uint32_t));
  ix->fill = (uint32_t *)calloc(ix->nstore * S, sizeof(uint32_t));
  if (!ix->slots || !ix->fill) { free(ix->slots); free(ix->fill); free(ix->seeds); free(ix); return NULL; }
  return ix;
}

/* partial index: only the listed (t, b) buckets are kept; inserts into other
 * buckets are dropped and queries must only touch listed buckets */
void *or_new_partial(uint32_t K, uint32_t L, uint32_t B, uint32_t R, uint32_t d, uint32_t w, uint32_t S,
                     uint64_t seed, uint64_t capacity, const uint32_t *req_t, const uint32_t *req_b,
                     uint64_t nreq, uint32_t densify) {
  or_index *ix = (or_index *)calloc(1, sizeof(or_index));
  ix->K = K; ix->L = L; ix->B = B; ix->R = R; ix->d = d; ix->w = w; ix->S = S;
  ix->capacity = capacity;
  ix->seeds = (uint32_t *)malloc(sizeof(uint32_t) * (2 + 2 * L + d + 2));
  or_seeds_init(seed, L, d, densify, ix->seeds);
  uint64_t nkeys = (uint64_t)L << B;
  ix->map = (int64_t *)malloc(sizeof(int64_t) * nkeys);
  for (uint64_t k = 0; k < nkeys; ++k) ix->map[k] = -1;
  uint64_t n = 0;
  for (uint64_t i = 0; i < nreq; ++i) {
    uint64_t key = ((uint64_t)req_t[i] << B) + req_b[i];
    if (ix->map[key] < 0) ix->map[key] = (int64_t)n++;
  }
  ix->nstore = n;
  ix->slots = (uint32_t *)calloc(n * S * R + 1, sizeof(uint32_t));
  ix->fill = (uint32_t *)calloc(n * S + 1, sizeof(uint32_t));
  return ix;
}

void or_free(void *p) {
  or_index *ix = (or_index *)p;
  if (!ix) return;
  free(ix->seeds); free(ix->map); free(ix->slots); free(ix->fill); free(ix);
}

const uint32_t *or_seeds(const void *p) { return ((const or_index *)p)->seeds; }

/* Reservoir insert into one bucket: keep the R ids of smallest priority,
 * ascending.  (Sec. 3 "Avoid Skewed buckets": fixed-size sub-sampled buckets.) */
static void or_bucket_insert(uint32_t *slots, uint32_t *fill, uint32_t R, uint32_t id, uint32_t sp_t) {
  uint32_t p = or_priority(id, sp_t);
  uint32_t f = *fill, pos = 0;
  while (pos < f && or_priority(slots[pos], sp_t) < p) ++pos;
  if (pos >= R) return;                       /* R smaller priorities already kept */
  uint32_t last = f < R ? f : R - 1;          /* the element at R-1 falls off when full */
  for (uint32_t k = last; k > pos; --k) slots[k] = slots[k - 1];
  slots[pos] = id;
  if (f < R) *fill = f + 1;
}

static uint32_t or_shard_of(const or_index *ix, uint64_t id) {
  return (uint32_t)(((unsigned __int128)id * ix->S) / ix->capacity);
}

/* Algorithm 1: each row gets the next id and goes into one bucket per table. */
int or_insert(void *p, const uint64_t *offs, const uint32_t *cols, uint64_t n, uint64_t *first_id) {
  or_index *ix = (or_index *)p;
  if (ix->next_id + n > ix->capacity) return -1;
  uint32_t nb = ix->K * ix->L;
  uint32_t *codes = (uint32_t *)malloc(sizeof(uint32_t) * nb);
  const uint32_t *st = ix->seeds + 2, *sp = ix->seeds + 2 + ix->L;
  *first_id = ix->next_id;
  for (uint64_t i = 0; i < n; ++i) {
    uint64_t id = ix->next_id++;
    uint32_t s = or_shard_of(ix, id);
    or_doph_seeded(cols + (offs[i] - offs[0]), offs[i + 1] - offs[i], nb, ix->seeds, ix->L, ix->d, codes);
    for (uint32_t t = 0; t < ix->L; ++t) {
      uint32_t b = or_table_address(codes, t, ix->K, ix->B, st[t]);
      if (ix->map && ix->map[((uint64_t)t << ix->B) + b] < 0) continue;
      uint64_t loc = (uint64_t)s * ix->nstore + or_loc(ix, t, b);
      or_bucket_insert(ix->slots + loc * ix->R, ix->fill + loc, ix->R, (uint32_t)id, sp[t]);
    }
  }
  free(codes);
  return 0;
}

/* Same result as or_insert for rows with ids [id0, id0+n), computed with
 * `threads` workers that each fill a private copy of the listed buckets; the
 * copies are then combined by inserting every kept id of one copy into the
 * other (a bottom-R reservoir of a union is the bottom-R of the two bottom-R
 * reservoirs).  Only for partial indexes (bounded memory). */
typedef struct {
  or_index *ix; const uint64_t *offs; const uint32_t *cols; uint64_t id0, b, e;
  uint32_t *slots, *fill;
} or_pjob;

static void *or_pinsert_run(void *a) {
  or_pjob *j = (or_pjob *)a;
  or_index *ix = j->ix;
  uint32_t nb = ix->K * ix->L;
  uint32_t *codes = (uint32_t *)malloc(sizeof(uint32_t) * nb);
  const uint32_t *st = ix->seeds + 2, *sp = ix->seeds + 2 + ix->L;
  for (uint64_t i = j->b; i < j->e; ++i) {
    uint64_t id = j->id0 + i;
    uint32_t s = or_shard_of(ix, id);
    or_doph_seeded(j->cols + (j->offs[i] - j->offs[0]), j->offs[i + 1] - j->offs[i], nb, ix->seeds, ix->L,
                   ix->d, codes);
    for (uint32_t t = 0; t < ix->L; ++t) {
      uint32_t b = or_table_address(codes, t, ix->K, ix->B, st[t]);
      if (ix->map[((uint64_t)t << ix->B) + b] < 0) continue;
      uint64_t loc = (uint64_t)s * ix->nstore + or_loc(ix, t, b);
      or_bucket_insert(j->slots + loc * ix->R, j->fill + loc, ix->R, (uint32_t)id, sp[t]);
    }
  }
  free(codes);
  return NULL;
}

int or_insert_parallel(void *p, const uint64_t *offs, const uint32_t *cols, uint64_t n,
                       uint64_t *first_id, int threads) {
  or_index *ix = (or_index *)p;
  if (!ix->map) return -2;
  if (ix->next_id + n > ix->capacity) return -1;
  if (threads < 1) threads = 1;
  uint64_t nloc = ix->nstore * ix->S;
  or_pjob *job = (or_pjob *)calloc(threads, sizeof(or_pjob));
  pthread_t *tid = (pthread_t *)calloc(threads, sizeof(pthread_t));
  for (int t = 0; t < threads; ++t) {
    job[t].ix = ix; job[t].offs = offs; job[t].cols = cols; job[t].id0 = ix->next_id;
    job[t].b = n * (uint64_t)t / threads; job[t].e = n * (uint64_t)(t + 1) / threads;
    job[t].slots = (uint32_t *)calloc(nloc * ix->R + 1, sizeof(uint32_t));
    job[t].fill = (uint32_t *)calloc(nloc + 1, sizeof(uint32_t));
    pthread_create(&tid[t], NULL, or_pinsert_run, &job[t]);
  }
  for (int t = 0; t < threads; ++t) pthread_join(tid[t], NULL);
  /* combine: start from the index's current contents, insert every kept id */
  uint32_t L = ix->L;
  const uint32_t *sp = ix->seeds + 2 + L;
  for (uint64_t key = 0; key < ((uint64_t)L << ix->B); ++key) {
    if (ix->map[key] < 0) continue;
    uint32_t t = (uint32_t)(key >> ix->B);
    for (uint32_t s = 0; s < ix->S; ++s) {
      uint64_t loc = (uint64_t)s * ix->nstore + (uint64_t)ix->map[key];
      for (int w = 0; w < threads; ++w)
        for (uint32_t k = 0; k < job[w].fill[loc]; ++k)
          or_bucket_insert(ix->slots + loc * ix->R, ix->fill + loc, ix->R,
                           job[w].slots[loc * ix->R + k], sp[t]);
    }
  }
  for (int t = 0; t < threads; ++t) { free(job[t].slots); free(job[t].fill); }
  free(job); free(tid);
  *first_id = ix->next_id;
  ix->next_id += n;
  return 0;
}

/* Exported contents of bucket (s, t, b): slots (OR_EMPTY past fill) and fill. */
int or_bucket(const void *p, uint32_t s, uint32_t t, uint32_t b, uint32_t *slots_out, uint32_t *fill_out) {
  const or_index *ix = (const or_index *)p;
  if (ix->map && ix->map[((uint64_t)t << ix->B) + b] < 0) return -1;
  uint64_t loc = (uint64_t)s * ix->nstore + or_loc(ix, t, b);
  uint32_t f = ix->fill[loc];
  for (uint32_t k = 0; k < ix->R; ++k) slots_out[k] = k < f ? ix->slots[loc * ix->R + k] : OR_EMPTY;
  *fill_out = f;
  return 0;
}

/* Dense export: slots [S][L][2^B][R], fill [S][L][2^B]. */
int or_export(const void *p, uint32_t *slots_out, uint32_t *fill_out) {
  const or_index *ix = (const or_index *)p;
  if (ix->map) return -2;
  uint64_t nb = ix->nstore * ix->S;
  for (uint64_t loc = 0; loc < nb; ++loc) {
    uint32_t f = ix->fill[loc];
    fill_out[loc] = f;
    for (uint32_t k = 0; k < ix->R; ++k)
      slots_out[loc * ix->R + k] = k < f ? ix->slots[loc * ix->R + k] : OR_EMPTY;
  }
  return 0;
}

/* ------------------------------------------------------------------ query */

static int cmp_u32(const void *a, const void *b) {
  uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
  return (x > y) - (x < y);
}

typedef struct { uint32_t est, id; } or_cand;

/* rank: larger estimate first, then smaller id */
static int cmp_cand(const void *a, const void *b) {
  const or_cand *x = (const or_cand *)a, *y = (const or_cand *)b;
  if (x->est != y->est) return x->est > y->est ? -1 : 1;
  return (x->id > y->id) - (x->id < y->id);
}

/* One query (Algorithm 2, local merge then cross-partition merge).
 * Outputs: ids[k] (-1 pad), scores[k] (0 pad).  Optional detail outputs:
 *   m_out/m_len:   the candidate multiset M (concatenated filled slots)
 *   u_out/u_len:   distinct candidates, ascending id
 *   est_out:       count-min estimate per distinct candidate
 *   cnt_out:       exact occurrence count per distinct candidate
 *   cm_out:        the summed d x w sketch
 * Returns 0, or -1 when a partial index lacks one of the query's buckets. */
int or_query_one(const void *p, const uint32_t *cols, uint64_t nnz, uint32_t k, int32_t *ids,
                 uint32_t *scores, uint32_t *m_out, uint64_t *m_len, uint32_t *u_out,
                 uint64_t *u_len, uint32_t *est_out, uint32_t *cnt_out, uint32_t *cm_out) {
  const or_index *ix = (const or_index *)p;
  uint32_t K = ix->K, L = ix->L, R = ix->R, d = ix->d, w = ix->w, S = ix->S;
  uint32_t nb = K * L;
  const uint32_t *st = ix->seeds + 2, *sc = ix->seeds + 2 + 2 * L;
  uint32_t *codes = (uint32_t *)malloc(sizeof(uint32_t) * nb);
  uint32_t *addr = (uint32_t *)malloc(sizeof(uint32_t) * L);
  /* Algorithm 2, hashing: the query's address in every table */
  or_doph_seeded(cols, nnz, nb, ix->seeds, ix->L, ix->d, codes);
  for (uint32_t t = 0; t < L; ++t) {
    addr[t] = or_table_address(codes, t, K, ix->B, st[t]);
    if (ix->map && ix->map[((uint64_t)t << ix->B) + addr[t]] < 0) { free(codes); free(addr); return -1; }
  }
  /* M: ids of the L buckets of every partition */
  uint64_t cap = (uint64_t)S * L * R, n = 0;
  uint32_t *M = (uint32_t *)malloc(sizeof(uint32_t) * (cap + 1));
  uint32_t *CM = (uint32_t *)calloc((uint64_t)d * w, sizeof(uint32_t));
  uint32_t *CMs = (uint32_t *)malloc(sizeof(uint32_t) * (uint64_t)d * w);
  for (uint32_t s = 0; s < S; ++s) {
    /* local merge on partition s: count its L buckets into its own sketch */
    memset(CMs, 0, sizeof(uint32_t) * (uint64_t)d * w);
    for (uint32_t t = 0; t < L; ++t) {
      uint64_t loc = (uint64_t)s * ix->nstore + or_loc(ix, t, addr[t]);
      for (uint32_t j = 0; j < ix->fill[loc]; ++j) {
        uint32_t id = ix->slots[loc * R + j];
        M[n++] = id;
        for (uint32_t r = 0; r < d; ++r) CMs[(uint64_t)r * w + or_cm_cell(id, sc[r], w)] += 1;
      }
    }
    /* cross-partition merge: count-min sketches add cell by cell */
    for (uint64_t c = 0; c < (uint64_t)d * w; ++c) CM[c] += CMs[c];
  }
  /* distinct candidates */
  uint32_t *U = (uint32_t *)malloc(sizeof(uint32_t) * (n + 1));
  memcpy(U, M, sizeof(uint32_t) * n);
  qsort(U, n, sizeof(uint32_t), cmp_u32);
  uint64_t u = 0;
  for (uint64_t i = 0; i < n; ++i)
    if (u == 0 || U[u - 1] != U[i]) U[u++] = U[i];
  /* estimate = min over sketch rows; rank by (estimate desc, id asc) */
  or_cand *C = (or_cand *)malloc(sizeof(or_cand) * (u + 1));
  for (uint64_t i = 0; i < u; ++i) {
    uint32_t e = UINT32_MAX;
    for (uint32_t r = 0; r < d; ++r) {
      uint32_t v = CM[(uint64_t)r * w + or_cm_cell(U[i], sc[r], w)];
      if (v < e) e = v;
    }
    C[i].est = e;
    C[i].id = U[i];
    if (est_out) est_out[i] = e;
    if (cnt_out) {
      uint32_t c = 0;
      for (uint64_t j = 0; j < n; ++j) c += M[j] == U[i];
      cnt_out[i] = c;
    }
  }
  if (m_out) memcpy(m_out, M, sizeof(uint32_t) * n);
  if (m_len) *m_len = n;
  if (u_out) memcpy(u_out, U, sizeof(uint32_t) * u);
  if (u_len) *u_len = u;
  if (cm_out) memcpy(cm_out, CM, sizeof(uint32_t) * (uint64_t)d * w);
  qsort(C, u, sizeof(or_cand), cmp_cand);
  for (uint32_t i = 0; i < k; ++i) {
    ids[i] = i < u ? (int32_t)C[i].id : -1;
    scores[i] = i < u ? C[i].est : 0;
  }
  free(codes); free(addr); free(M); free(CM); free(CMs); free(U); free(C);
  return 0;
}

/* batch of queries (CSR), ids [nq][k], scores [nq][k] */
int or_query(const void *p, const uint64_t *offs, const uint32_t *cols, uint64_t nq, uint32_t k,
             int32_t *ids, uint32_t *scores) {
  for (uint64_t q = 0; q < nq; ++q) {
    int rc = or_query_one(p, cols + (offs[q] - offs[0]), offs[q + 1] - offs[q], k, ids + q * k,
                          scores + q * k, NULL, NULL, NULL, NULL, NULL, NULL, NULL);
    if (rc) return rc;
  }
  return 0;
}

uint64_t or_next_id(const void *p) { return ((const or_index *)p)->next_id; }

/* Rows inserted next take ids from `id` on: a partition D_i of Sec. 3 built on
 * its own starts at its first global id.  Only forward; -1 if id < next id or
 * id > capacity. */
int or_set_next_id(void *p, uint64_t id) {
  or_index *ix = (or_index *)p;
  if (id < ix->next_id || id > ix->capacity) return -1;
  ix->next_id = id;
  return 0;
}

/* ------------------------------------------------------------------ TopKAPI buckets
 * SLASH's own bucket (Sec. 3.1 and Appendix 2): every bucket address holds a
 * TopKAPI sketch of W rows x Bc cells, each cell a (heavy hitter, count) pair,
 * instead of an id list.  Fixed readings:
 *   cell_i(id)   mix32(id ^ tk[i]) & (Bc - 1); tk = the d = W row seeds drawn
 *                after st and sp (same order as the count-min seeds)
 *   insert x     Appendix 2, read in the order written: if the cell holds x,
 *                count + 1; otherwise count - 1, and when the count is then 0
 *                (or the cell was empty) the cell becomes (x, 1).  A cell is
 *                empty exactly when its count is 0.
 *   order        a bucket takes its ids in ascending id (= data) order
 *   merge        same heavy hitter: counts add; different: the larger count
 *                wins with the difference; equal counts cancel to an empty cell
 *   query        fold the query's buckets, shard-major then table order, into
 *                an empty sketch; each heavy hitter's score is its largest
 *                count over the cells; those with a score above the threshold
 *                (Appendix 2, "Querying") rank by (score desc, id asc); pad (-1,0)
 */
typedef struct {
  uint32_t K, L, B, W, C, S;
  uint64_t capacity, next_id;
  uint32_t *seeds;       /* or_seeds_init: 2 + 2L + W + 2 */
  /* per shard s: sketch (t, b) lives at storage row map[t*2^B + b] (dense: identity) */
  int64_t *map;          /* NULL = dense */
  uint64_t nstore;       /* materialised sketches per shard */
  uint32_t *hh, *cnt;    /* [S][nstore][W][C] */
} or_tk;

/* storage row of sketch (s, t, b), or -1 when a partial index does not keep it */
static int64_t or_tk_loc(const or_tk *ix, uint32_t s, uint32_t t, uint32_t b) {
  uint64_t key = ((uint64_t)t << ix->B) + b;
  int64_t r = ix->map ? ix->map[key] : (int64_t)key;
  return r < 0 ? -1 : (int64_t)((uint64_t)s * ix->nstore + (uint64_t)r);
}

void or_tk_update(uint32_t *hh, uint32_t *cnt, uint32_t x) {
  if (*cnt > 0 && *hh == x) { *cnt += 1; return; }
  if (*cnt > 0) *cnt -= 1;
  if (*cnt == 0) { *hh = x; *cnt = 1; }
}

void or_tk_merge_cell(uint32_t *hh, uint32_t *cnt, uint32_t bh, uint32_t bc) {
  if (bc == 0) return;
  if (*cnt == 0) { *hh = bh; *cnt = bc; return; }
  if (*hh == bh) { *cnt += bc; return; }
  if (bc > *cnt) { *hh = bh; *cnt = bc - *cnt; return; }
  *cnt -= bc;   /* equal counts leave an empty cell */
}

void *or_tk_new(uint32_t K, uint32_t L, uint32_t B, uint32_t W, uint32_t C, uint32_t S, uint64_t seed,
                uint64_t capacity, uint32_t densify) {
  or_tk *ix = (or_tk *)calloc(1, sizeof(or_tk));
  ix->K = K; ix->L = L; ix->B = B; ix->W = W; ix->C = C; ix->S = S; ix->capacity = capacity;
  ix->seeds = (uint32_t *)malloc(sizeof(uint32_t) * (2 + 2 * L + W + 2));
  or_seeds_init(seed, L, W, densify, ix->seeds);
  ix->nstore = (uint64_t)L << B;
  uint64_t n = (uint64_t)S * ix->nstore * W * C;
  ix->hh = (uint32_t *)calloc(n, sizeof(uint32_t));
  ix->cnt = (uint32_t *)calloc(n, sizeof(uint32_t));
  if (!ix->hh || !ix->cnt) { free(ix->hh); free(ix->cnt); free(ix->seeds); free(ix); return NULL; }
  return ix;
}

/* partial sketch index: only the listed (t, b) sketches (of every shard) are kept */
void *or_tk_new_partial(uint32_t K, uint32_t L, uint32_t B, uint32_t W, uint32_t C, uint32_t S, uint64_t seed,
                        uint64_t capacity, uint32_t densify, const uint32_t *req_t, const uint32_t *req_b,
                        uint64_t nreq) {
  or_tk *ix = (or_tk *)calloc(1, sizeof(or_tk));
  ix->K = K; ix->L = L; ix->B = B; ix->W = W; ix->C = C; ix->S = S; ix->capacity = capacity;
  ix->seeds = (uint32_t *)malloc(sizeof(uint32_t) * (2 + 2 * L + W + 2));
  or_seeds_init(seed, L, W, densify, ix->seeds);
  uint64_t nkeys = (uint64_t)L << B;
  ix->map = (int64_t *)malloc(sizeof(int64_t) * nkeys);
  for (uint64_t k = 0; k < nkeys; ++k) ix->map[k] = -1;
  uint64_t n = 0;
  for (uint64_t i = 0; i < nreq; ++i) {
    uint64_t key = ((uint64_t)req_t[i] << B) + req_b[i];
    if (ix->map[key] < 0) ix->map[key] = (int64_t)n++;
  }
  ix->nstore = n;
  ix->hh = (uint32_t *)calloc((uint64_t)S * n * W * C + 1, sizeof(uint32_t));
  ix->cnt = (uint32_t *)calloc((uint64_t)S * n * W * C + 1, sizeof(uint32_t));
  return ix;
}

void or_tk_free(void *p) {
  or_tk *ix = (or_tk *)p;
  if (!ix) return;
  free(ix->seeds); free(ix->map); free(ix->hh); free(ix->cnt); free(ix);
}

/* Algorithm 1 with sketches: each row's id goes into one sketch per table. */
int or_tk_insert(void *p, const uint64_t *offs, const uint32_t *cols, uint64_t n, uint64_t *first_id) {
  or_tk *ix = (or_tk *)p;
  if (ix->next_id + n > ix->capacity) return -1;
  uint32_t nb = ix->K * ix->L;
  uint32_t *codes = (uint32_t *)malloc(sizeof(uint32_t) * nb);
  const uint32_t *st = ix->seeds + 2, *tk = ix->seeds + 2 + 2 * ix->L;
  *first_id = ix->next_id;
  for (uint64_t i = 0; i < n; ++i) {
    uint64_t id = ix->next_id++;
    uint32_t s = (uint32_t)(((unsigned __int128)id * ix->S) / ix->capacity);
    or_doph_seeded(cols + (offs[i] - offs[0]), offs[i + 1] - offs[i], nb, ix->seeds, ix->L, ix->W, codes);
    for (uint32_t t = 0; t < ix->L; ++t) {
      uint32_t b = or_table_address(codes, t, ix->K, ix->B, st[t]);
      int64_t loc = or_tk_loc(ix, s, t, b);
      if (loc < 0) continue;  /* a partial index does not keep this sketch */
      uint64_t base = (uint64_t)loc * ix->W * ix->C;
      for (uint32_t r = 0; r < ix->W; ++r) {
        uint64_t c = base + (uint64_t)r * ix->C + (or_mix32((uint32_t)id ^ tk[r]) & (ix->C - 1));
        or_tk_update(ix->hh + c, ix->cnt + c, (uint32_t)id);
      }
    }
  }
  free(codes);
  return 0;
}

/* or_tk_insert with the rows' table addresses computed by `threads` threads
 * (a row's hash depends on that row alone); the cell updates then run on one
 * thread in ascending id order, exactly as in or_tk_insert. */
typedef struct {
  const or_tk *ix; const uint64_t *offs; const uint32_t *cols; uint64_t b, e; uint32_t *addr;
} or_tk_hjob;

static void *or_tk_hash_run(void *a) {
  or_tk_hjob *j = (or_tk_hjob *)a;
  const or_tk *ix = j->ix;
  uint32_t nb = ix->K * ix->L;
  uint32_t *codes = (uint32_t *)malloc(sizeof(uint32_t) * nb);
  for (uint64_t i = j->b; i < j->e; ++i) {
    or_doph_seeded(j->cols + (j->offs[i] - j->offs[0]), j->offs[i + 1] - j->offs[i], nb, ix->seeds, ix->L, ix->W,
                   codes);
    for (uint32_t t = 0; t < ix->L; ++t)
      j->addr[(i - j->b) * ix->L + t] = or_table_address(codes, t, ix->K, ix->B, ix->seeds[2 + t]);
  }
  free(codes);
  return NULL;
}

int or_tk_insert_parallel(void *p, const uint64_t *offs, const uint32_t *cols, uint64_t n, uint64_t *first_id,
                          int threads) {
  or_tk *ix = (or_tk *)p;
  if (ix->next_id + n > ix->capacity) return -1;
  if (threads < 1) threads = 1;
  const uint32_t *tk = ix->seeds + 2 + 2 * ix->L;
  const uint64_t block = 1u << 20;
  uint32_t *addr = (uint32_t *)malloc(sizeof(uint32_t) * block * ix->L);
  or_tk_hjob *job = (or_tk_hjob *)calloc(threads, sizeof(or_tk_hjob));
  pthread_t *tid = (pthread_t *)calloc(threads, sizeof(pthread_t));
  *first_id = ix->next_id;
  for (uint64_t r0 = 0; r0 < n; r0 += block) {
    uint64_t m = n - r0 < block ? n - r0 : block;
    for (int t = 0; t < threads; ++t) {
      job[t].ix = ix; job[t].offs = offs; job[t].cols = cols;
      job[t].b = r0 + m * (uint64_t)t / threads; job[t].e = r0 + m * (uint64_t)(t + 1) / threads;
      job[t].addr = addr + (job[t].b - r0) * ix->L;
      pthread_create(&tid[t], NULL, or_tk_hash_run, &job[t]);
    }
    for (int t = 0; t < threads; ++t) pthread_join(tid[t], NULL);
    for (uint64_t i = 0; i < m; ++i) {
      uint64_t id = ix->next_id + r0 + i;
      uint32_t s = (uint32_t)(((unsigned __int128)id * ix->S) / ix->capacity);
      for (uint32_t t = 0; t < ix->L; ++t) {
        int64_t loc = or_tk_loc(ix, s, t, addr[i * ix->L + t]);
        if (loc < 0) continue;
        uint64_t base = (uint64_t)loc * ix->W * ix->C;
        for (uint32_t r = 0; r < ix->W; ++r) {
          uint64_t c = base + (uint64_t)r * ix->C + (or_mix32((uint32_t)id ^ tk[r]) & (ix->C - 1));
          or_tk_update(ix->hh + c, ix->cnt + c, (uint32_t)id);
        }
      }
    }
  }
  ix->next_id += n;
  free(addr); free(job); free(tid);
  return 0;
}

/* cells of sketch (s, t, b): out[W*C][2] = (heavy hitter or 0xFFFFFFFF, count); -1 if not kept */
int or_tk_bucket(const void *p, uint32_t s, uint32_t t, uint32_t b, uint32_t *out) {
  const or_tk *ix = (const or_tk *)p;
  int64_t loc = or_tk_loc(ix, s, t, b);
  if (loc < 0) return -1;
  uint64_t base = (uint64_t)loc * ix->W * ix->C;
  for (uint32_t c = 0; c < ix->W * ix->C; ++c) {
    out[2 * c] = ix->cnt[base + c] ? ix->hh[base + c] : OR_EMPTY;
    out[2 * c + 1] = ix->cnt[base + c];
  }
  return 0;
}

/* cells [S][L][2^B][W][C][2] = (heavy hitter or 0xFFFFFFFF when empty, count) */
void or_tk_export(const void *p, uint32_t *out) {
  const or_tk *ix = (const or_tk *)p;
  uint64_t n = (uint64_t)ix->S * ix->nstore * ix->W * ix->C;  /* dense: nstore = L * 2^B */
  for (uint64_t c = 0; c < n; ++c) {
    out[2 * c] = ix->cnt[c] ? ix->hh[c] : OR_EMPTY;
    out[2 * c + 1] = ix->cnt[c];
  }
}

/* Appendix 2 "Merging": fold n sketches of WC cells each, in the order given
 * (sketch i's cells at hh[i*WC ..], cnt[i*WC ..]), into an empty sketch mh/mc. */
void or_tk_fold(const uint32_t *hh, const uint32_t *cnt, uint64_t n, uint32_t WC, uint32_t *mh, uint32_t *mc) {
  for (uint32_t c = 0; c < WC; ++c) { mh[c] = OR_EMPTY; mc[c] = 0; }
  for (uint64_t i = 0; i < n; ++i)
    for (uint32_t c = 0; c < WC; ++c) or_tk_merge_cell(mh + c, mc + c, hh[i * WC + c], cnt[i * WC + c]);
}

/* Appendix 2 "Querying" on a merged sketch: the distinct heavy hitters, each
 * scored by its largest count over the cells; those whose score exceeds the
 * threshold are ranked (score desc, id asc); the first k are written, padded
 * with (-1, 0). */
void or_tk_rank(const uint32_t *mh, const uint32_t *mc, uint32_t WC, uint32_t k, uint32_t threshold,
                int32_t *ids, uint32_t *scores) {
  or_cand *cand = (or_cand *)malloc(sizeof(or_cand) * (WC + 1));
  uint32_t nc = 0;
  for (uint32_t c = 0; c < WC; ++c) {
    if (mc[c] == 0 || mc[c] <= threshold) continue;
    uint32_t j = 0;
    while (j < nc && cand[j].id != mh[c]) ++j;
    if (j == nc) { cand[nc].id = mh[c]; cand[nc].est = mc[c]; ++nc; }
    else if (mc[c] > cand[j].est) cand[j].est = mc[c];
  }
  qsort(cand, nc, sizeof(or_cand), cmp_cand);
  for (uint32_t i = 0; i < k; ++i) {
    ids[i] = i < nc ? (int32_t)cand[i].id : -1;
    scores[i] = i < nc ? cand[i].est : 0;
  }
  free(cand);
}

/* Algorithm 2 with sketches: the query's S*L sketches, shard-major then in
 * table order, are folded into one (or_tk_fold) and ranked (or_tk_rank). */
int or_tk_query(const void *p, const uint64_t *offs, const uint32_t *cols, uint64_t nq, uint32_t k,
                uint32_t threshold, int32_t *ids, uint32_t *scores) {
  const or_tk *ix = (const or_tk *)p;
  uint32_t nb = ix->K * ix->L, WC = ix->W * ix->C;
  uint64_t n = (uint64_t)ix->S * ix->L;
  const uint32_t *st = ix->seeds + 2;
  uint32_t *codes = (uint32_t *)malloc(sizeof(uint32_t) * nb);
  uint32_t *mh = (uint32_t *)malloc(sizeof(uint32_t) * WC), *mc = (uint32_t *)malloc(sizeof(uint32_t) * WC);
  uint32_t *sh = (uint32_t *)malloc(sizeof(uint32_t) * n * WC), *sn = (uint32_t *)malloc(sizeof(uint32_t) * n * WC);
  int rc = 0;
  for (uint64_t q = 0; q < nq && rc == 0; ++q) {
    or_doph_seeded(cols + (offs[q] - offs[0]), offs[q + 1] - offs[q], nb, ix->seeds, ix->L, ix->W, codes);
    uint64_t i = 0;
    for (uint32_t s = 0; s < ix->S && rc == 0; ++s)
      for (uint32_t t = 0; t < ix->L; ++t, ++i) {
        uint32_t b = or_table_address(codes, t, ix->K, ix->B, st[t]);
        int64_t loc = or_tk_loc(ix, s, t, b);
        if (loc < 0) { rc = -1; break; }
        memcpy(sh + i * WC, ix->hh + (uint64_t)loc * WC, sizeof(uint32_t) * WC);
        memcpy(sn + i * WC, ix->cnt + (uint64_t)loc * WC, sizeof(uint32_t) * WC);
      }
    if (rc) break;
    or_tk_fold(sh, sn, n, WC, mh, mc);
    or_tk_rank(mh, mc, WC, k, threshold, ids + q * k, scores + q * k);
  }
  free(codes); free(mh); free(mc); free(sh); free(sn);
  return rc;
}

/* ------------------------------------------------------------------ exact neighbours (ground truth)
 * The quality the index approximates (Sec. 2.2: MinHash collides with
 * probability equal to the Jaccard similarity): for each query, the k rows of
 * the collection with the largest Jaccard similarity |q & x| / |q | x|,
 * ranked (similarity desc, id asc), by brute force.  Rows and queries are sets
 * of feature ids < dim (no duplicates); an empty union counts as similarity 0.
 * ids[q*k + i] (-1 pad), inter/uni[q*k + i] the similarity's numerator and
 * denominator.  `threads` workers take disjoint query ranges. */
typedef struct {
  const uint64_t *offs; const uint32_t *cols; uint64_t n; uint32_t dim;
  const uint64_t *qoffs; const uint32_t *qcols; uint64_t q0, q1; uint32_t k;
  int32_t *ids; uint32_t *inter, *uni;
} or_jac_job;

/* a/b > c/d for similarities (b, d > 0; a similarity with b == 0 is 0) */
static int or_jac_better(uint32_t a, uint32_t b, uint64_t ia, uint32_t c, uint32_t d, uint64_t ic) {
  uint64_t l = b ? (uint64_t)a * (d ? d : 1) : 0, r = d ? (uint64_t)c * (b ? b : 1) : 0;
  if (b == 0) l = 0;
  if (d == 0) r = 0;
  if (l != r) return l > r;
  return ia < ic;
}

static void *or_jac_run(void *arg) {
  or_jac_job *j = (or_jac_job *)arg;
  uint64_t words = ((uint64_t)j->dim + 63) / 64;
  uint64_t *bits = (uint64_t *)calloc(words, sizeof(uint64_t));
  for (uint64_t q = j->q0; q < j->q1; ++q) {
    const uint32_t *qc = j->qcols + (j->qoffs[q] - j->qoffs[0]);
    uint32_t qn = (uint32_t)(j->qoffs[q + 1] - j->qoffs[q]);
    for (uint32_t i = 0; i < qn; ++i) bits[qc[i] >> 6] |= 1ull << (qc[i] & 63);
    int32_t *bi = j->ids + q * j->k;
    uint32_t *bn = j->inter + q * j->k, *bu = j->uni + q * j->k;
    uint32_t have = 0;
    for (uint64_t x = 0; x < j->n; ++x) {
      const uint32_t *xc = j->cols + (j->offs[x] - j->offs[0]);
      uint32_t xn = (uint32_t)(j->offs[x + 1] - j->offs[x]), in = 0;
      for (uint32_t i = 0; i < xn; ++i) in += (uint32_t)((bits[xc[i] >> 6] >> (xc[i] & 63)) & 1u);
      uint32_t un = qn + xn - in;
      if (have == j->k && !or_jac_better(in, un, x, bn[have - 1], bu[have - 1], (uint64_t)bi[have - 1])) continue;
      uint32_t pos = have < j->k ? have++ : j->k - 1;
      while (pos > 0 && or_jac_better(in, un, x, bn[pos - 1], bu[pos - 1], (uint64_t)bi[pos - 1])) {
        bi[pos] = bi[pos - 1]; bn[pos] = bn[pos - 1]; bu[pos] = bu[pos - 1];
        --pos;
      }
      bi[pos] = (int32_t)x; bn[pos] = in; bu[pos] = un;
    }
    for (uint32_t i = have; i < j->k; ++i) { bi[i] = -1; bn[i] = 0; bu[i] = 0; }
    for (uint32_t i = 0; i < qn; ++i) bits[qc[i] >> 6] = 0;
  }
  free(bits);
  return NULL;
}

int or_jaccard_topk(const uint64_t *offs, const uint32_t *cols, uint64_t n, uint32_t dim, const uint64_t *qoffs,
                    const uint32_t *qcols, uint64_t nq, uint32_t k, int threads, int32_t *ids, uint32_t *inter,
                    uint32_t *uni) {
  if (threads < 1) threads = 1;
  if ((uint64_t)threads > nq) threads = nq ? (int)nq : 1;
  or_jac_job *job = (or_jac_job *)calloc(threads, sizeof(or_jac_job));
  pthread_t *tid = (pthread_t *)calloc(threads, sizeof(pthread_t));
  for (int t = 0; t < threads; ++t) {
    or_jac_job *j = &job[t];
    j->offs = offs; j->cols = cols; j->n = n; j->dim = dim; j->qoffs = qoffs; j->qcols = qcols;
    j->q0 = nq * (uint64_t)t / threads; j->q1 = nq * (uint64_t)(t + 1) / threads; j->k = k;
    j->ids = ids; j->inter = inter; j->uni = uni;
    pthread_create(&tid[t], NULL, or_jac_run, j);
  }
  for (int t = 0; t < threads; ++t) pthread_join(tid[t], NULL);
  free(job); free(tid);
  return 0;
}
