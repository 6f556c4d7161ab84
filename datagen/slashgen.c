/*
 * Seeded synthetic input generator for the SLASH similarity-search hot path.
 *
 * This module produces INPUTS only (sparse binary rows and queries in CSR
 * form).  It holds none of the method's arithmetic: no MinHash, no
 * densification, no table addressing, no reservoir and no sketch.  Both the
 * CPU oracle and the CUDA path consume what it writes.
 *
 * Workload shape (stand-in for the Criteo click logs of the paper's
 * evaluation, Sec. 6: about 40 non-zeros per row over 2^20 hashed features
 * with power-law feature frequencies):
 *   - row nnz ~ Poisson(lambda) clamped to [lo, hi]        (clamp, not resample)
 *   - random-query nnz ~ round(LogNormal(mu, sigma)) clamped to [rlo, rhi]
 *   - features: rank ~ Zipf(s) over [1, D], feature = perm(rank - 1) where perm
 *     is a seeded 4-round Feistel bijection on [0, D); duplicates in a row are
 *     redrawn; columns are stored ascending
 *   - planted queries: a dataset row chosen uniformly, each feature replaced
 *     independently with probability p by a fresh Zipf draw that is neither in
 *     the source row nor already drawn, so nnz is kept and J = (n-r)/(n+r)
 *
 * Randomness is counter based: every uniform is the SplitMix64 output function
 * (Steele, Lea & Flood, OOPSLA 2014) applied to a key derived from
 * (seed, stream) plus a golden-ratio stride of the counter (row, draw).  All
 * sampling is integer inverse-CDF lookup in uint64 fixed-point tables built
 * once on the host, so any other implementation that receives the same tables
 * reproduces the same bytes.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SG_GOLDEN 0x9E3779B97F4A7C15ull
#define SG_MAX_DRAWS 65535u /* per row / per query, then deterministic padding */

enum { ST_ROW_NNZ = 0, ST_ROW_FEAT = 1, ST_Q_SRC = 2, ST_Q_COIN = 3,
       ST_Q_NNZ = 4, ST_Q_FEAT = 5, ST_Q_KIND = 6, ST_PERM = 7 };

static inline uint64_t sg_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* uniform 64-bit word number j of `row` in `stream` */
static inline uint64_t sg_u64(uint64_t seed, uint32_t stream, uint64_t row, uint32_t j) {
  uint64_t key = sg_mix64(seed + (uint64_t)(stream + 1) * SG_GOLDEN);
  return sg_mix64(key + ((row << 16) + (uint64_t)j + 1) * SG_GOLDEN);
}

/* ---------------- inverse-CDF tables ---------------- */
typedef struct {
  uint64_t *cdf;  /* cdf[i] = floor(P(X <= value_i) * 2^64), last = UINT64_MAX */
  uint32_t n;
  uint32_t *guide; /* 65537 entries: guide[g] = first i with cdf[i] > g<<48 */
} sg_icdf;

static void icdf_finish(sg_icdf *t) {
  t->cdf[t->n - 1] = UINT64_MAX;
  t->guide = (uint32_t *)malloc(sizeof(uint32_t) * 65537);
  uint32_t i = 0;
  for (uint32_t g = 0; g < 65536; ++g) {
    uint64_t lim = (uint64_t)g << 48;
    while (i < t->n - 1 && t->cdf[i] <= lim) ++i;
    t->guide[g] = i;
  }
  t->guide[65536] = t->n - 1;
}

static uint64_t to_fixed(long double p) {
  if (p <= 0.0L) return 0;
  if (p >= 1.0L) return UINT64_MAX;
  long double v = p * 18446744073709551616.0L;
  if (v >= 18446744073709551615.0L) return UINT64_MAX;
  return (uint64_t)v;
}

/* smallest i with u < cdf[i] (last index if none) */
static inline uint32_t icdf_sample(const sg_icdf *t, uint64_t u) {
  uint32_t g = (uint32_t)(u >> 48);
  uint32_t lo = t->guide[g], hi = t->guide[g + 1];
  while (lo < hi) {
    uint32_t mid = lo + ((hi - lo) >> 1);
    if (u < t->cdf[mid]) hi = mid; else lo = mid + 1;
  }
  return lo;
}

typedef struct {
  uint32_t dim_bits, dim;
  sg_icdf zipf;    /* value = rank-1 in [0, dim) */
  sg_icdf pois;    /* value = k in [0, n) */
  sg_icdf lnorm;   /* value = n-1, n in [1, ln_max] */
} sg_gen;

void *sg_new(uint32_t dim_bits, double zipf_s, double pois_lambda, double ln_mu,
             double ln_sigma, uint32_t ln_max) {
  if (dim_bits < 2 || dim_bits > 30 || (dim_bits & 1u) || ln_max < 1) return NULL;
  sg_gen *g = (sg_gen *)calloc(1, sizeof(sg_gen));
  g->dim_bits = dim_bits;
  g->dim = 1u << dim_bits;
  /* Zipf(s) over ranks 1..dim */
  g->zipf.n = g->dim;
  g->zipf.cdf = (uint64_t *)malloc(sizeof(uint64_t) * g->dim);
  long double h = 0.0L;
  for (uint32_t k = g->dim; k >= 1; --k) h += powl((long double)k, -(long double)zipf_s);
  long double c = 0.0L;
  for (uint32_t k = 1; k <= g->dim; ++k) {
    c += powl((long double)k, -(long double)zipf_s);
    g->zipf.cdf[k - 1] = to_fixed(c / h);
  }
  icdf_finish(&g->zipf);
  /* Poisson(lambda) over k = 0..n-1 */
  uint32_t pn = (uint32_t)(4.0 * pois_lambda + 64.0);
  g->pois.n = pn;
  g->pois.cdf = (uint64_t *)malloc(sizeof(uint64_t) * pn);
  c = 0.0L;
  for (uint32_t k = 0; k < pn; ++k) {
    long double lp = -(long double)pois_lambda + (long double)k * logl((long double)pois_lambda) -
                     lgammal((long double)k + 1.0L);
    c += expl(lp);
    g->pois.cdf[k] = to_fixed(c);
  }
  icdf_finish(&g->pois);
  /* round(LogNormal(mu, sigma)) clamped to [1, ln_max]: P(round(X) <= n) = Phi((ln(n+.5)-mu)/sigma) */
  g->lnorm.n = ln_max;
  g->lnorm.cdf = (uint64_t *)malloc(sizeof(uint64_t) * ln_max);
  for (uint32_t n = 1; n <= ln_max; ++n) {
    double z = (log((double)n + 0.5) - ln_mu) / ln_sigma;
    g->lnorm.cdf[n - 1] = to_fixed((long double)(0.5 * erfc(-z / sqrt(2.0))));
  }
  icdf_finish(&g->lnorm);
  return g;
}

void sg_free(void *p) {
  sg_gen *g = (sg_gen *)p;
  if (!g) return;
  free(g->zipf.cdf); free(g->zipf.guide);
  free(g->pois.cdf); free(g->pois.guide);
  free(g->lnorm.cdf); free(g->lnorm.guide);
  free(g);
}

/* expose the Zipf and Poisson tables so that other generators (and tests) can use them */
const uint64_t *sg_zipf_cdf(const void *p) { return ((const sg_gen *)p)->zipf.cdf; }
const uint64_t *sg_pois_cdf(const void *p, uint32_t *n) { *n = ((const sg_gen *)p)->pois.n; return ((const sg_gen *)p)->pois.cdf; }
const uint64_t *sg_lnorm_cdf(const void *p, uint32_t *n) { *n = ((const sg_gen *)p)->lnorm.n; return ((const sg_gen *)p)->lnorm.cdf; }
const uint32_t *sg_zipf_guide(const void *p) { return ((const sg_gen *)p)->zipf.guide; }
const uint32_t *sg_pois_guide(const void *p) { return ((const sg_gen *)p)->pois.guide; }
uint32_t sg_dim_bits(const void *p) { return ((const sg_gen *)p)->dim_bits; }

/* 4-round Feistel bijection on [0, 2^dim_bits) keyed by the dataset seed */
static inline uint32_t sg_perm(const sg_gen *g, uint64_t seed, uint32_t x) {
  uint32_t hb = g->dim_bits >> 1, mask = (1u << hb) - 1u;
  uint32_t l = x >> hb, r = x & mask;
  for (uint32_t i = 0; i < 4; ++i) {
    uint32_t k = (uint32_t)(sg_u64(seed, ST_PERM, 0, i) >> 32);
    uint32_t f = (uint32_t)sg_mix64(((uint64_t)k << 32) | r) & mask;
    uint32_t nl = r, nr = l ^ f;
    l = nl; r = nr;
  }
  return (l << hb) | r;
}

uint32_t sg_feature(const void *p, uint64_t seed, uint64_t u) {
  const sg_gen *g = (const sg_gen *)p;
  return sg_perm(g, seed, icdf_sample(&g->zipf, u));
}

/* ---------------- small per-row set (open addressing, key+1, 0 = empty) ---------------- */
typedef struct { uint32_t *slot; uint32_t cap; } sg_set;

static void set_reset(sg_set *s, uint32_t need) {
  uint32_t cap = 16;
  while (cap < 2 * need + 2) cap <<= 1;
  if (cap > s->cap) { free(s->slot); s->slot = (uint32_t *)malloc(sizeof(uint32_t) * cap); s->cap = cap; }
  memset(s->slot, 0, sizeof(uint32_t) * cap);
  s->cap = cap;
}
/* returns 1 if inserted, 0 if present */
static int set_add(sg_set *s, uint32_t key) {
  uint32_t m = s->cap - 1, i = (uint32_t)(sg_mix64(key) & m);
  for (;;) {
    if (s->slot[i] == 0) { s->slot[i] = key + 1; return 1; }
    if (s->slot[i] == key + 1) return 0;
    i = (i + 1) & m;
  }
}
static int set_has(const sg_set *s, uint32_t key) {
  uint32_t m = s->cap - 1, i = (uint32_t)(sg_mix64(key) & m);
  for (;;) {
    if (s->slot[i] == 0) return 0;
    if (s->slot[i] == key + 1) return 1;
    i = (i + 1) & m;
  }
}

static int cmp_u32(const void *a, const void *b) {
  uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
  return (x > y) - (x < y);
}

static inline uint32_t clampu(uint32_t v, uint32_t lo, uint32_t hi) { return v < lo ? lo : (v > hi ? hi : v); }

static uint32_t row_nnz(const sg_gen *g, uint64_t seed, uint64_t row, uint32_t lo, uint32_t hi) {
  uint32_t n = clampu(icdf_sample(&g->pois, sg_u64(seed, ST_ROW_NNZ, row, 0)), lo, hi);
  return n > g->dim ? g->dim : n;
}

/* dataset row `row` -> out[0..n) ascending */
static void row_cols(const sg_gen *g, uint64_t seed, uint64_t row, uint32_t n, uint32_t *out, sg_set *s) {
  set_reset(s, n);
  uint32_t c = 0;
  for (uint32_t j = 0; c < n && j < SG_MAX_DRAWS; ++j) {
    uint32_t f = sg_perm(g, seed, icdf_sample(&g->zipf, sg_u64(seed, ST_ROW_FEAT, row, j)));
    if (set_add(s, f)) out[c++] = f;
  }
  for (uint32_t f = 0; c < n; ++f) /* deterministic padding, practically never reached */
    if (set_add(s, f)) out[c++] = f;
  qsort(out, n, sizeof(uint32_t), cmp_u32);
}

/* ---------------- tiny pthread parallel-for ---------------- */
typedef void (*sg_body)(void *ctx, uint64_t b, uint64_t e);
typedef struct { sg_body fn; void *ctx; uint64_t b, e; } sg_job;
static void *sg_run(void *a) { sg_job *j = (sg_job *)a; j->fn(j->ctx, j->b, j->e); return NULL; }
static void sg_parallel(uint64_t n, int threads, sg_body fn, void *ctx) {
  if (threads < 1) threads = 1;
  if ((uint64_t)threads > n) threads = n ? (int)n : 1;
  if (threads == 1) { fn(ctx, 0, n); return; }
  pthread_t *tid = (pthread_t *)malloc(sizeof(pthread_t) * threads);
  sg_job *job = (sg_job *)malloc(sizeof(sg_job) * threads);
  for (int t = 0; t < threads; ++t) {
    job[t].fn = fn; job[t].ctx = ctx;
    job[t].b = n * (uint64_t)t / threads; job[t].e = n * (uint64_t)(t + 1) / threads;
    pthread_create(&tid[t], NULL, sg_run, &job[t]);
  }
  for (int t = 0; t < threads; ++t) pthread_join(tid[t], NULL);
  free(tid); free(job);
}

/* ---------------- dataset rows ---------------- */
typedef struct {
  const sg_gen *g; uint64_t seed, row0; uint32_t lo, hi;
  uint32_t *nnz; const uint64_t *offs; uint32_t *cols;
} rows_ctx;

static void rows_nnz_body(void *c, uint64_t b, uint64_t e) {
  rows_ctx *x = (rows_ctx *)c;
  for (uint64_t i = b; i < e; ++i) x->nnz[i] = row_nnz(x->g, x->seed, x->row0 + i, x->lo, x->hi);
}
static void rows_cols_body(void *c, uint64_t b, uint64_t e) {
  rows_ctx *x = (rows_ctx *)c;
  sg_set s = {NULL, 0};
  for (uint64_t i = b; i < e; ++i) {
    uint32_t n = (uint32_t)(x->offs[i + 1] - x->offs[i]);
    row_cols(x->g, x->seed, x->row0 + i, n, x->cols + (x->offs[i] - x->offs[0]), &s);
  }
  free(s.slot);
}

/* nnz of rows [row0, row0+n) */
void sg_rows_nnz(const void *g, uint64_t seed, uint64_t row0, uint64_t n, uint32_t lo, uint32_t hi,
                 uint32_t *nnz, int threads) {
  rows_ctx c = {(const sg_gen *)g, seed, row0, lo, hi, nnz, NULL, NULL};
  sg_parallel(n, threads, rows_nnz_body, &c);
}

/* cols of rows [row0, row0+n); offs[0..n] from sg_rows_nnz's prefix sum; cols[offs[i]-offs[0]...] */
void sg_rows_cols(const void *g, uint64_t seed, uint64_t row0, uint64_t n, const uint64_t *offs,
                  uint32_t *cols, int threads) {
  rows_ctx c = {(const sg_gen *)g, seed, row0, 0, 0, NULL, offs, cols};
  sg_parallel(n, threads, rows_cols_body, &c);
}

/* ---------------- queries ---------------- */
typedef struct {
  const sg_gen *g; uint64_t seed, qseed, q0, n_rows;
  uint32_t lo, hi, rlo, rhi;
  uint64_t planted_thr; int all_planted;
  uint64_t pert_thr; int pert_all;
  int64_t *src; const int64_t *csrc; uint32_t *nnz; const uint64_t *offs; uint32_t *cols;
} q_ctx;

static void q_meta_body(void *c, uint64_t b, uint64_t e) {
  q_ctx *x = (q_ctx *)c;
  for (uint64_t i = b; i < e; ++i) {
    uint64_t q = x->q0 + i;
    int planted = x->all_planted || sg_u64(x->qseed, ST_Q_KIND, q, 0) < x->planted_thr;
    if (planted && x->n_rows > 0) {
      uint64_t u = sg_u64(x->qseed, ST_Q_SRC, q, 0);
      uint64_t r = (uint64_t)(((unsigned __int128)u * x->n_rows) >> 64);
      x->src[i] = (int64_t)r;
      x->nnz[i] = row_nnz(x->g, x->seed, r, x->lo, x->hi);
    } else {
      x->src[i] = -1;
      uint32_t n = clampu(icdf_sample(&x->g->lnorm, sg_u64(x->qseed, ST_Q_NNZ, q, 0)) + 1, x->rlo, x->rhi);
      x->nnz[i] = n > x->g->dim ? x->g->dim : n;
    }
  }
}

static void q_cols_body(void *c, uint64_t b, uint64_t e) {
  q_ctx *x = (q_ctx *)c;
  sg_set s = {NULL, 0}, s2 = {NULL, 0};
  uint32_t *tmp = NULL; uint32_t tcap = 0;
  for (uint64_t i = b; i < e; ++i) {
    uint64_t q = x->q0 + i;
    uint32_t n = (uint32_t)(x->offs[i + 1] - x->offs[i]);
    uint32_t *out = x->cols + (x->offs[i] - x->offs[0]);
    if (x->csrc[i] < 0) {          /* random Zipf row, keyed by the query seed */
      set_reset(&s, n);
      uint32_t cnt = 0;
      for (uint32_t j = 0; cnt < n && j < SG_MAX_DRAWS; ++j) {
        uint32_t f = sg_perm(x->g, x->seed, icdf_sample(&x->g->zipf, sg_u64(x->qseed, ST_Q_FEAT, q, j)));
        if (set_add(&s, f)) out[cnt++] = f;
      }
      for (uint32_t f = 0; cnt < n; ++f) if (set_add(&s, f)) out[cnt++] = f;
      qsort(out, n, sizeof(uint32_t), cmp_u32);
      continue;
    }
    /* planted: regenerate the source row, then perturb */
    if (tcap < n) { free(tmp); tmp = (uint32_t *)malloc(sizeof(uint32_t) * n); tcap = n; }
    row_cols(x->g, x->seed, (uint64_t)x->csrc[i], n, tmp, &s);   /* s = set of source features */
    set_reset(&s2, n);                                            /* s2 = replacements drawn */
    uint32_t cnt = 0, rep = 0;
    for (uint32_t p = 0; p < n; ++p) {
      int replace = x->pert_all || sg_u64(x->qseed, ST_Q_COIN, q, p) < x->pert_thr;
      if (replace) ++rep; else out[cnt++] = tmp[p];
    }
    uint32_t got = 0;
    for (uint32_t j = 0; got < rep && j < SG_MAX_DRAWS; ++j) {
      uint32_t f = sg_perm(x->g, x->seed, icdf_sample(&x->g->zipf, sg_u64(x->qseed, ST_Q_FEAT, q, j)));
      if (set_has(&s, f)) continue;
      if (set_add(&s2, f)) { out[cnt++] = f; ++got; }
    }
    for (uint32_t f = 0; got < rep; ++f)
      if (!set_has(&s, f) && set_add(&s2, f)) { out[cnt++] = f; ++got; }
    qsort(out, n, sizeof(uint32_t), cmp_u32);
  }
  free(s.slot); free(s2.slot); free(tmp);
}

static uint64_t frac_thr(double f, int *all) {
  *all = f >= 1.0;
  if (f <= 0.0) return 0;
  if (f >= 1.0) return UINT64_MAX;
  return (uint64_t)ldexp(f, 64);
}

/* query plan: source row (or -1 for a random row) and nnz of queries [q0, q0+nq) */
void sg_queries_meta(const void *g, uint64_t seed, uint64_t qseed, uint64_t q0, uint64_t nq,
                     uint64_t n_rows, uint32_t lo, uint32_t hi, double planted_frac,
                     uint32_t rlo, uint32_t rhi, int64_t *src, uint32_t *nnz, int threads) {
  q_ctx c; memset(&c, 0, sizeof c);
  c.g = (const sg_gen *)g; c.seed = seed; c.qseed = qseed; c.q0 = q0; c.n_rows = n_rows;
  c.lo = lo; c.hi = hi; c.rlo = rlo; c.rhi = rhi;
  c.planted_thr = frac_thr(planted_frac, &c.all_planted);
  c.src = src; c.nnz = nnz;
  sg_parallel(nq, threads, q_meta_body, &c);
}

void sg_queries_cols(const void *g, uint64_t seed, uint64_t qseed, uint64_t q0, uint64_t nq,
                     double p_perturb, const int64_t *src, const uint64_t *offs, uint32_t *cols,
                     int threads) {
  q_ctx c; memset(&c, 0, sizeof c);
  c.g = (const sg_gen *)g; c.seed = seed; c.qseed = qseed; c.q0 = q0;
  c.pert_thr = frac_thr(p_perturb, &c.pert_all);
  if (p_perturb <= 0.0) c.pert_all = 0;
  c.csrc = src; c.offs = offs; c.cols = cols;
  sg_parallel(nq, threads, q_cols_body, &c);
}

uint64_t sg_u64_public(uint64_t seed, uint32_t stream, uint64_t row, uint32_t j) { return sg_u64(seed, stream, row, j); }
