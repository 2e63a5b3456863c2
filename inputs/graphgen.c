/*
 * graphgen.c -- seeded synthetic graph generators.
 *
 * This module is INPUT SIDE ONLY: it draws random graphs and lays them out as
 * symmetric CSR (int64 row offsets, int32 column indices, rows sorted
 * ascending, no duplicates, no self-loops).  It contains none of the label
 * propagation, splitting or modularity arithmetic; the CPU oracle and the CUDA
 * library both consume the arrays written here and neither is linked into it.
 *
 * Randomness is counter based so that any thread count gives the same graph:
 * every draw is the ctr-th output of a SplitMix64 stream (Steele, Lea and
 * Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014),
 * keyed by (seed, stream).  Floating point is limited to +,-,*,/ and
 * frexp, and the file is compiled with -ffp-contract=off, so x86-64 and
 * aarch64 builds produce bit-identical graphs.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include <math.h>

#define GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
/* ctr-th output of the SplitMix64 sequence whose state starts at `key`. */
static inline uint64_t rng_at(uint64_t key, uint64_t ctr) { return mix64(key + (ctr + 1) * GAMMA); }
static inline uint64_t stream_key(uint64_t seed, uint64_t stream) {
  return mix64(mix64(seed + GAMMA) ^ mix64(stream * 0xD1B54A32D192ED03ULL + 0x632BE59BD9B4E019ULL));
}
/* uniform double in [0,1) from the top 53 bits */
static inline double u01(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }
/* uniform integer in [0, range) by multiply-high (Lemire); bias < range/2^64 */
static inline uint64_t below(uint64_t x, uint64_t range) {
  return (uint64_t)(((unsigned __int128)x * range) >> 64);
}

/* Natural log from +,-,*,/ only: x = m 2^e with m in [sqrt(1/2), sqrt(2)),
 * ln m = 2 atanh(s), s = (m-1)/(m+1), |s| < 0.1716, series to s^41. */
static double det_log(double x) {
  int e;
  double m = frexp(x, &e);
  if (m < 0.70710678118654752440) { m *= 2.0; e -= 1; }
  double s = (m - 1.0) / (m + 1.0), s2 = s * s, term = s, sum = 0.0;
  for (int k = 1; k <= 41; k += 2) { sum += term / (double)k; term *= s2; }
  return 2.0 * sum + (double)e * 0.69314718055994530942;
}
/* exp from +,-,*,/ only: e^x = 2^k e^r, |r| <= ln2/2, Taylor to r^24. */
static double det_exp(double x) {
  double kf = x / 0.69314718055994530942;
  long k = (long)(kf < 0 ? kf - 0.5 : kf + 0.5);
  double r = x - (double)k * 0.69314718055994530942;
  double term = 1.0, sum = 1.0;
  for (int i = 1; i <= 24; ++i) { term *= r / (double)i; sum += term; }
  return ldexp(sum, (int)k);
}

/* ------------------------------------------------------------------ */
/* tiny parallel-for                                                   */
typedef void (*pf_fn)(int tid, int nt, void* arg);
typedef struct { pf_fn fn; int tid, nt; void* arg; } pf_job;
static void* pf_tramp(void* p) { pf_job* j = (pf_job*)p; j->fn(j->tid, j->nt, j->arg); return NULL; }
static void parallel_for(int nt, pf_fn fn, void* arg) {
  if (nt < 1) nt = 1;
  if (nt > 256) nt = 256;
  pthread_t th[256];
  pf_job jobs[256];
  for (int t = 0; t < nt; ++t) { jobs[t].fn = fn; jobs[t].tid = t; jobs[t].nt = nt; jobs[t].arg = arg; }
  for (int t = 1; t < nt; ++t) pthread_create(&th[t], NULL, pf_tramp, &jobs[t]);
  pf_tramp(&jobs[0]);
  for (int t = 1; t < nt; ++t) pthread_join(th[t], NULL);
}
static inline void slice(int64_t n, int tid, int nt, int64_t* lo, int64_t* hi) {
  *lo = n * tid / nt;
  *hi = n * (tid + 1) / nt;
}
static int ceil_log2(uint64_t x) { int b = 0; while ((1ULL << b) < x) ++b; return b; }

/* ------------------------------------------------------------------ */
/* parallel sort of u64 keys holding `nbits` significant bits:          */
/* one MSD partition on the top bits, then LSD radix inside each bucket */
typedef struct {
  uint64_t* keys; uint64_t* tmp; int64_t n; int nbits, bd, nb;
  int64_t* hist;      /* nt x nb */
  int64_t* bstart;    /* nb + 1 */
  int64_t next_bucket; /* atomic work counter */
  int nt;
} psort_t;

static void psort_count(int tid, int nt, void* a) {
  psort_t* p = (psort_t*)a;
  int64_t lo, hi; slice(p->n, tid, nt, &lo, &hi);
  int64_t* h = p->hist + (int64_t)tid * p->nb;
  memset(h, 0, sizeof(int64_t) * p->nb);
  int sh = p->nbits - p->bd;
  for (int64_t i = lo; i < hi; ++i) h[p->keys[i] >> sh]++;
}
static void psort_scatter(int tid, int nt, void* a) {
  psort_t* p = (psort_t*)a;
  int64_t lo, hi; slice(p->n, tid, nt, &lo, &hi);
  int64_t* h = p->hist + (int64_t)tid * p->nb;  /* holds write cursors */
  int sh = p->nbits - p->bd;
  for (int64_t i = lo; i < hi; ++i) { uint64_t k = p->keys[i]; p->tmp[h[k >> sh]++] = k; }
}
static void lsd_sort(uint64_t* a, uint64_t* s, int64_t n, int bits) {
  /* sorts a[0..n) on its low `bits` bits; s is scratch of n; result in a */
  if (n < 2 || bits <= 0) return;
  if (n <= 48) {
    for (int64_t i = 1; i < n; ++i) {
      uint64_t k = a[i]; int64_t j = i - 1;
      while (j >= 0 && a[j] > k) { a[j + 1] = a[j]; --j; }
      a[j + 1] = k;
    }
    return;
  }
  const int D = 11; const int R = 1 << D;
  int64_t cnt[1 << 11];
  uint64_t* src = a; uint64_t* dst = s;
  int passes = 0;
  for (int sh = 0; sh < bits; sh += D) {
    memset(cnt, 0, sizeof(cnt));
    for (int64_t i = 0; i < n; ++i) cnt[(src[i] >> sh) & (R - 1)]++;
    int64_t run = 0;
    for (int d = 0; d < R; ++d) { int64_t c = cnt[d]; cnt[d] = run; run += c; }
    for (int64_t i = 0; i < n; ++i) { uint64_t k = src[i]; dst[cnt[(k >> sh) & (R - 1)]++] = k; }
    uint64_t* t = src; src = dst; dst = t; ++passes;
  }
  if (src != a) memcpy(a, src, sizeof(uint64_t) * n);
}
static void psort_buckets(int tid, int nt, void* a) {
  psort_t* p = (psort_t*)a;
  (void)tid; (void)nt;
  int64_t maxb = 0;
  for (int b = 0; b < p->nb; ++b) { int64_t s = p->bstart[b + 1] - p->bstart[b]; if (s > maxb) maxb = s; }
  uint64_t* scratch = (uint64_t*)malloc(sizeof(uint64_t) * (maxb > 0 ? maxb : 1));
  for (;;) {
    int64_t b = __atomic_fetch_add(&p->next_bucket, 1, __ATOMIC_RELAXED);
    if (b >= p->nb) break;
    int64_t s = p->bstart[b], e = p->bstart[b + 1];
    lsd_sort(p->tmp + s, scratch, e - s, p->nbits - p->bd);
  }
  free(scratch);
}
/* Sorts keys[0..n) ascending; the result is left in tmp (n entries). */
static int psort_u64(uint64_t* keys, uint64_t* tmp, int64_t n, int nbits, int nt) {
  psort_t p;
  memset(&p, 0, sizeof(p));
  p.keys = keys; p.tmp = tmp; p.n = n; p.nbits = nbits < 1 ? 1 : nbits; p.nt = nt;
  p.bd = p.nbits < 12 ? p.nbits : 12;
  p.nb = 1 << p.bd;
  p.hist = (int64_t*)malloc(sizeof(int64_t) * (int64_t)nt * p.nb);
  p.bstart = (int64_t*)malloc(sizeof(int64_t) * (p.nb + 1));
  if (!p.hist || !p.bstart) { free(p.hist); free(p.bstart); return -1; }
  parallel_for(nt, psort_count, &p);
  int64_t run = 0;
  for (int b = 0; b < p.nb; ++b) {
    p.bstart[b] = run;
    for (int t = 0; t < nt; ++t) { int64_t c = p.hist[(int64_t)t * p.nb + b]; p.hist[(int64_t)t * p.nb + b] = run; run += c; }
  }
  p.bstart[p.nb] = run;
  parallel_for(nt, psort_scatter, &p);
  p.next_bucket = 0;
  parallel_for(nt, psort_buckets, &p);
  free(p.hist); free(p.bstart);
  return 0;
}

/* ------------------------------------------------------------------ */
/* CSR from undirected pairs                                           */
typedef struct {
  int64_t n, m; const int32_t* u; const int32_t* v; const int32_t* perm;
  uint64_t* keys; int64_t* kcount; int bits_d;
  const uint64_t* sorted; int64_t nkeys; int64_t* uniq_start; int64_t* uniq_cnt;
  int64_t* deg; int32_t* cols;
} csrb_t;

static void csrb_count(int tid, int nt, void* a) {
  csrb_t* c = (csrb_t*)a;
  int64_t lo, hi; slice(c->m, tid, nt, &lo, &hi);
  int64_t k = 0;
  for (int64_t i = lo; i < hi; ++i) if (c->u[i] != c->v[i]) k += 2;
  c->kcount[tid] = k;
}
static void csrb_keys(int tid, int nt, void* a) {
  csrb_t* c = (csrb_t*)a;
  int64_t lo, hi; slice(c->m, tid, nt, &lo, &hi);
  int64_t w = c->kcount[tid];
  for (int64_t i = lo; i < hi; ++i) {
    int64_t x = c->u[i], y = c->v[i];
    if (x == y) continue;
    if (c->perm) { x = c->perm[x]; y = c->perm[y]; }
    c->keys[w++] = ((uint64_t)x << c->bits_d) | (uint64_t)y;
    c->keys[w++] = ((uint64_t)y << c->bits_d) | (uint64_t)x;
  }
}
/* per-thread slice of the sorted key array, aligned so that equal keys and
 * equal sources never straddle two slices */
static void aligned_slice(const uint64_t* s, int64_t n, int bits_d, int tid, int nt, int64_t* lo, int64_t* hi) {
  int64_t a, b; slice(n, tid, nt, &a, &b);
  while (a > 0 && a < n && (s[a] >> bits_d) == (s[a - 1] >> bits_d)) ++a;
  while (b > 0 && b < n && (s[b] >> bits_d) == (s[b - 1] >> bits_d)) ++b;
  *lo = a; *hi = b;
}
static void csrb_uniq(int tid, int nt, void* a) {
  csrb_t* c = (csrb_t*)a;
  int64_t lo, hi; aligned_slice(c->sorted, c->nkeys, c->bits_d, tid, nt, &lo, &hi);
  int64_t k = 0;
  for (int64_t i = lo; i < hi; ++i) if (i == lo || c->sorted[i] != c->sorted[i - 1]) ++k;
  c->uniq_cnt[tid] = k;
}
static void csrb_emit(int tid, int nt, void* a) {
  csrb_t* c = (csrb_t*)a;
  int64_t lo, hi; aligned_slice(c->sorted, c->nkeys, c->bits_d, tid, nt, &lo, &hi);
  int64_t w = c->uniq_start[tid];
  uint64_t dmask = (c->bits_d >= 64) ? ~0ULL : ((1ULL << c->bits_d) - 1);
  for (int64_t i = lo; i < hi; ++i) {
    if (i != lo && c->sorted[i] == c->sorted[i - 1]) continue;
    uint64_t k = c->sorted[i];
    c->deg[k >> c->bits_d]++;   /* rows never straddle slices */
    c->cols[w++] = (int32_t)(k & dmask);
  }
}

/* Builds the symmetric CSR of the undirected multigraph {(u[i], v[i])}:
 * self-loops dropped, both directions added, duplicates merged, every row
 * sorted ascending.  If perm is given, vertex x is renamed perm[x] first.
 * offsets has n+1 entries; cols has room for cols_cap entries.
 * Returns nnz, or -1 (cols_cap too small / out of memory / bad sizes). */
int64_t gg_csr_from_pairs(int64_t n, int64_t m, const int32_t* u, const int32_t* v,
                          const int32_t* perm, int threads,
                          int64_t* offsets, int32_t* cols, int64_t cols_cap) {
  if (n < 0 || m < 0 || n > 2147483647LL) return -1;
  int nt = threads < 1 ? 1 : threads;
  csrb_t c;
  memset(&c, 0, sizeof(c));
  c.n = n; c.m = m; c.u = u; c.v = v; c.perm = perm;
  c.bits_d = ceil_log2((uint64_t)(n > 1 ? n : 2));
  int64_t kc[256];
  c.kcount = kc;
  if (nt > 256) nt = 256;
  parallel_for(nt, csrb_count, &c);
  int64_t total = 0;
  for (int t = 0; t < nt; ++t) { int64_t k = kc[t]; kc[t] = total; total += k; }
  uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (total > 0 ? total : 1));
  uint64_t* tmp = (uint64_t*)malloc(sizeof(uint64_t) * (total > 0 ? total : 1));
  int64_t* deg = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!keys || !tmp || !deg) { free(keys); free(tmp); free(deg); return -1; }
  c.keys = keys;
  parallel_for(nt, csrb_keys, &c);
  if (psort_u64(keys, tmp, total, 2 * c.bits_d, nt) != 0) { free(keys); free(tmp); free(deg); return -1; }
  free(keys);
  c.sorted = tmp; c.nkeys = total;
  int64_t ucnt[256], ustart[256];
  c.uniq_cnt = ucnt; c.uniq_start = ustart;
  parallel_for(nt, csrb_uniq, &c);
  int64_t nnz = 0;
  for (int t = 0; t < nt; ++t) { ustart[t] = nnz; nnz += ucnt[t]; }
  if (nnz > cols_cap) { free(tmp); free(deg); return -1; }
  c.deg = deg; c.cols = cols;
  parallel_for(nt, csrb_emit, &c);
  int64_t run = 0;
  for (int64_t x = 0; x < n; ++x) { offsets[x] = run; run += deg[x]; }
  offsets[n] = run;
  free(tmp); free(deg);
  return nnz;
}

/* ------------------------------------------------------------------ */
/* random permutation: new id of x = rank of x in ascending order of    */
/* (top bits of rng(seed, x), x)                                        */
typedef struct { int64_t n; uint64_t key; int bits; uint64_t* keys; } perm_t;
static void perm_keys(int tid, int nt, void* a) {
  perm_t* p = (perm_t*)a;
  int64_t lo, hi; slice(p->n, tid, nt, &lo, &hi);
  uint64_t lowmask = (1ULL << p->bits) - 1;
  for (int64_t x = lo; x < hi; ++x) p->keys[x] = (rng_at(p->key, (uint64_t)x) & ~lowmask) | (uint64_t)x;
}
int gg_permutation(int64_t n, uint64_t seed, int threads, int32_t* perm) {
  if (n <= 0) return 0;
  perm_t p;
  p.n = n; p.key = stream_key(seed, 0x5045524DULL); p.bits = ceil_log2((uint64_t)n);
  if (p.bits < 1) p.bits = 1;
  p.keys = (uint64_t*)malloc(sizeof(uint64_t) * n);
  uint64_t* tmp = (uint64_t*)malloc(sizeof(uint64_t) * n);
  if (!p.keys || !tmp) { free(p.keys); free(tmp); return -1; }
  parallel_for(threads, perm_keys, &p);
  psort_u64(p.keys, tmp, n, 64, threads);
  uint64_t lowmask = (1ULL << p.bits) - 1;
  for (int64_t r = 0; r < n; ++r) perm[tmp[r] & lowmask] = (int32_t)r;
  free(p.keys); free(tmp);
  return 0;
}

/* ------------------------------------------------------------------ */
/* R-MAT edge samples (Chakrabarti, Zhan, Faloutsos, SDM 2004)          */
typedef struct { int scale; int64_t m; uint32_t ta, tab, tabc; uint64_t key; int32_t* u; int32_t* v; } rmat_t;
static void rmat_body(int tid, int nt, void* a) {
  rmat_t* r = (rmat_t*)a;
  int64_t lo, hi; slice(r->m, tid, nt, &lo, &hi);
  int draws = (r->scale + 1) / 2;
  for (int64_t k = lo; k < hi; ++k) {
    uint32_t x = 0, y = 0;
    for (int l = 0; l < r->scale; ++l) {
      uint64_t d = rng_at(r->key, (uint64_t)k * draws + (uint64_t)(l >> 1));
      uint32_t q = (l & 1) ? (uint32_t)d : (uint32_t)(d >> 32);
      uint32_t bx, by;
      if (q < r->ta) { bx = 0; by = 0; }
      else if (q < r->tab) { bx = 0; by = 1; }
      else if (q < r->tabc) { bx = 1; by = 0; }
      else { bx = 1; by = 1; }
      x = (x << 1) | bx; y = (y << 1) | by;
    }
    r->u[k] = (int32_t)x; r->v[k] = (int32_t)y;
  }
}
static uint32_t prob32(double p) {
  if (p <= 0.0) return 0;
  if (p >= 1.0) return 0xFFFFFFFFu;
  return (uint32_t)(p * 4294967296.0);
}
/* m samples on 2^scale vertices; quadrant probabilities a, b, c, d=1-a-b-c. */
int gg_rmat_samples(int scale, int64_t m, double a, double b, double c, uint64_t seed,
                    int threads, int32_t* u, int32_t* v) {
  if (scale < 1 || scale > 30 || m < 0) return -1;
  rmat_t r;
  r.scale = scale; r.m = m; r.u = u; r.v = v;
  r.ta = prob32(a); r.tab = prob32(a + b); r.tabc = prob32(a + b + c);
  r.key = stream_key(seed, 0x524D4154ULL);
  parallel_for(threads, rmat_body, &r);
  return 0;
}

/* ------------------------------------------------------------------ */
/* planted partition (SBM) with contiguous blocks                       */
/* Pairs u<v are independent Bernoulli draws: p_in inside a block,      */
/* p_out across blocks.  Drawn with geometric skips (one draw per kept  */
/* pair), each vertex u on its own counter stream.                      */
typedef struct {
  int64_t n; const int64_t* bstart; int64_t nblocks;   /* block b = [bstart[b], bstart[b+1]) */
  double p_in, p_out, lq_in, lq_out; uint64_t key;
  int64_t* cnt;       /* per-vertex pair counts (pass 1) */
  int64_t* pos;       /* per-vertex write offsets (pass 2) */
  int32_t* u; int32_t* v; int pass;
} sbm_t;

static inline int64_t geo_skip(uint64_t r, double p, double lq) {
  /* failures before the next success of a Bernoulli(p) sequence */
  if (p >= 1.0) return 0;
  double U = 1.0 - u01(r);          /* (0,1] */
  double g = det_log(U) / lq;       /* lq = ln(1-p) < 0 */
  if (g >= 9.0e18) return INT64_MAX / 4;
  return (int64_t)g;
}
static int64_t block_of(const sbm_t* s, int64_t x) {
  int64_t lo = 0, hi = s->nblocks;  /* bstart[lo] <= x < bstart[hi] */
  while (hi - lo > 1) { int64_t mid = (lo + hi) / 2; if (s->bstart[mid] <= x) lo = mid; else hi = mid; }
  return lo;
}
static void sbm_body(int tid, int nt, void* a) {
  sbm_t* s = (sbm_t*)a;
  int64_t lo, hi; slice(s->n, tid, nt, &lo, &hi);
  for (int64_t x = lo; x < hi; ++x) {
    uint64_t key = mix64(s->key ^ mix64((uint64_t)x + 0x9E37ULL));
    uint64_t ctr = 0;
    int64_t bend = s->bstart[block_of(s, x) + 1];
    int64_t k = 0, w = (s->pass == 2) ? s->pos[x] : 0;
    if (s->p_in > 0.0) {
      int64_t y = x + 1 + geo_skip(rng_at(key, ctr++), s->p_in, s->lq_in);
      while (y < bend) {
        if (s->pass == 2) { s->u[w] = (int32_t)x; s->v[w] = (int32_t)y; ++w; }
        ++k;
        y += 1 + geo_skip(rng_at(key, ctr++), s->p_in, s->lq_in);
      }
    }
    ctr = 1ULL << 40;
    if (s->p_out > 0.0) {
      int64_t y = bend + geo_skip(rng_at(key, ctr++), s->p_out, s->lq_out);
      while (y < s->n) {
        if (s->pass == 2) { s->u[w] = (int32_t)x; s->v[w] = (int32_t)y; ++w; }
        ++k;
        y += 1 + geo_skip(rng_at(key, ctr++), s->p_out, s->lq_out);
      }
    }
    if (s->pass == 1) s->cnt[x] = k;
  }
}
static double clamp01(double p) { return p < 0.0 ? 0.0 : (p > 1.0 ? 1.0 : p); }
/* Pass 1: returns the number of undirected pairs (u<v) the SBM draws. */
static void sbm_setup(sbm_t* s, int64_t n, const int64_t* bstart, int64_t nblocks, double p_in, double p_out, uint64_t seed) {
  memset(s, 0, sizeof(*s));
  s->n = n; s->bstart = bstart; s->nblocks = nblocks;
  s->p_in = clamp01(p_in); s->p_out = clamp01(p_out);
  s->lq_in = s->p_in < 1.0 ? det_log(1.0 - s->p_in) : -1.0;
  s->lq_out = s->p_out < 1.0 ? det_log(1.0 - s->p_out) : -1.0;
  s->key = stream_key(seed, 0x53424DULL);
}
int64_t gg_sbm_count(int64_t n, const int64_t* bstart, int64_t nblocks, double p_in, double p_out,
                     uint64_t seed, int threads, int64_t* per_vertex) {
  sbm_t s;
  sbm_setup(&s, n, bstart, nblocks, p_in, p_out, seed);
  s.cnt = per_vertex; s.pass = 1;
  parallel_for(threads, sbm_body, &s);
  int64_t total = 0;
  for (int64_t x = 0; x < n; ++x) total += per_vertex[x];
  return total;
}
/* Pass 2: writes the pairs; per_vertex holds the counts from pass 1 and is
 * turned into exclusive offsets here. */
int gg_sbm_pairs(int64_t n, const int64_t* bstart, int64_t nblocks, double p_in, double p_out,
                 uint64_t seed, int threads, int64_t* per_vertex, int32_t* u, int32_t* v) {
  sbm_t s;
  sbm_setup(&s, n, bstart, nblocks, p_in, p_out, seed);
  int64_t run = 0;
  for (int64_t x = 0; x < n; ++x) { int64_t c = per_vertex[x]; per_vertex[x] = run; run += c; }
  s.pos = per_vertex; s.u = u; s.v = v; s.pass = 2;
  parallel_for(threads, sbm_body, &s);
  return 0;
}

/* ------------------------------------------------------------------ */
/* road / k-mer-like: R x C 4-neighbour lattice with each edge deleted   */
/* with probability p_del, plus `shortcuts` uniform random pairs, plus   */
/* n_chains disjoint paths whose vertex counts are uniform in [lo, hi]   */
typedef struct {
  int64_t R, C; uint32_t tdel; uint64_t kdel, ksc, kch;
  int64_t nh, ne; /* horizontal edge count, total lattice edges */
  int64_t* tcount; int32_t* u; int32_t* v; int pass;
} lat_t;
static inline void lat_edge(const lat_t* L, int64_t e, int64_t* a, int64_t* b) {
  if (e < L->nh) { int64_t r = e / (L->C - 1), c = e % (L->C - 1); *a = r * L->C + c; *b = *a + 1; }
  else { int64_t f = e - L->nh; *a = f; *b = f + L->C; }
}
static void lat_body(int tid, int nt, void* a) {
  lat_t* L = (lat_t*)a;
  int64_t lo, hi; slice(L->ne, tid, nt, &lo, &hi);
  int64_t k = 0, w = (L->pass == 2) ? L->tcount[tid] : 0;
  for (int64_t e = lo; e < hi; ++e) {
    if ((uint32_t)(rng_at(L->kdel, (uint64_t)e) >> 32) < L->tdel) continue;  /* deleted */
    if (L->pass == 2) { int64_t x, y; lat_edge(L, e, &x, &y); L->u[w] = (int32_t)x; L->v[w] = (int32_t)y; ++w; }
    ++k;
  }
  if (L->pass == 1) L->tcount[tid] = k;
}
/* Returns the number of kept lattice edges (pass 1). */
int64_t gg_lattice_kept(int64_t R, int64_t C, double p_del, uint64_t seed, int threads) {
  lat_t L;
  memset(&L, 0, sizeof(L));
  L.R = R; L.C = C; L.tdel = prob32(p_del); L.kdel = stream_key(seed, 0x4C415444ULL);
  L.nh = R * (C - 1); L.ne = L.nh + (R - 1) * C;
  int64_t tc[256]; int nt = threads < 1 ? 1 : (threads > 256 ? 256 : threads);
  L.tcount = tc; L.pass = 1;
  parallel_for(nt, lat_body, &L);
  int64_t total = 0;
  for (int t = 0; t < nt; ++t) total += tc[t];
  return total;
}
/* Chain vertex counts (uniform in [lo, hi]) for chain i. */
int gg_chain_lengths(int64_t n_chains, int64_t lo, int64_t hi, uint64_t seed, int32_t* len) {
  uint64_t k = stream_key(seed, 0x4348414EULL);
  for (int64_t i = 0; i < n_chains; ++i) len[i] = (int32_t)(lo + (int64_t)below(rng_at(k, (uint64_t)i), (uint64_t)(hi - lo + 1)));
  return 0;
}
/* Writes all undirected pairs of the lattice+shortcuts+chains graph.
 * Layout: kept lattice edges (lattice ids r*C+c), then `shortcuts` random
 * lattice pairs, then the chains (ids R*C + prefix of chain lengths).
 * u, v must hold kept + shortcuts + sum(len_i - 1) entries. */
int gg_lattice_pairs(int64_t R, int64_t C, double p_del, int64_t shortcuts,
                     int64_t n_chains, const int32_t* chain_len, uint64_t seed, int threads,
                     int32_t* u, int32_t* v) {
  lat_t L;
  memset(&L, 0, sizeof(L));
  L.R = R; L.C = C; L.tdel = prob32(p_del); L.kdel = stream_key(seed, 0x4C415444ULL);
  L.nh = R * (C - 1); L.ne = L.nh + (R - 1) * C;
  int64_t tc[256]; int nt = threads < 1 ? 1 : (threads > 256 ? 256 : threads);
  L.tcount = tc; L.pass = 1;
  parallel_for(nt, lat_body, &L);
  int64_t run = 0;
  for (int t = 0; t < nt; ++t) { int64_t c = tc[t]; tc[t] = run; run += c; }
  L.pass = 2; L.u = u; L.v = v;
  parallel_for(nt, lat_body, &L);
  int64_t w = run, RC = R * C;
  uint64_t ks = stream_key(seed, 0x53484F52ULL);
  for (int64_t i = 0; i < shortcuts; ++i) {
    u[w] = (int32_t)below(rng_at(ks, 2 * (uint64_t)i), (uint64_t)RC);
    v[w] = (int32_t)below(rng_at(ks, 2 * (uint64_t)i + 1), (uint64_t)RC);
    ++w;
  }
  int64_t base = RC;
  for (int64_t c = 0; c < n_chains; ++c) {
    for (int32_t j = 0; j + 1 < chain_len[c]; ++j) { u[w] = (int32_t)(base + j); v[w] = (int32_t)(base + j + 1); ++w; }
    base += chain_len[c];
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* scalar helpers exposed for parameter laws (log-uniform sizes etc.)   */
double gg_det_log(double x) { return det_log(x); }
double gg_det_exp(double x) { return det_exp(x); }
uint64_t gg_rng(uint64_t seed, uint64_t stream, uint64_t ctr) { return rng_at(stream_key(seed, stream), ctr); }
double gg_u01(uint64_t seed, uint64_t stream, uint64_t ctr) { return u01(rng_at(stream_key(seed, stream), ctr)); }
uint64_t gg_below(uint64_t seed, uint64_t stream, uint64_t ctr, uint64_t range) {
  return below(rng_at(stream_key(seed, stream), ctr), range);
}
