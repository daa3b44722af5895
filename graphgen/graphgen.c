/*
 * graphgen.c -- seeded, platform-independent synthetic graph generators.
 *
 * This module is shared by the CPU oracle and by the GPU benchmarks/tests.
 * It holds none of the graphlet-counting arithmetic: it only draws graphs
 * and writes them as CSR (int32 row pointers, int32 column indices sorted
 * ascending within each row, symmetric, no self-loops, no duplicates).
 *
 * Randomness: one counter-based generator, SplitMix64 (Steele, Lea and
 * Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
 * value(key, i) = mix64(key + (i + 1) * 0x9E3779B97F4A7C15), where mix64 is
 * the SplitMix64 output function and key = mix64(mix64(seed + gamma) ^
 * stream * 0xD1B54A32D192ED03).  Uniform doubles take the top 53 bits.
 * Everything is integer or IEEE double arithmetic with no contraction, so
 * x86_64 and aarch64 builds draw bit-identical graphs.
 *
 * Workload shapes (the paper's graphs are power-law, skewed per-edge work,
 * Fig. 1; its synthetic comparison graphs are ER/BA/GEO, Sec. 5):
 *   gg_er        G(n, p): Bernoulli per pair i < j in lexicographic order.
 *   gg_chung_lu  weights (i+1)^(-1/(gamma-1)) scaled to sum_w, capped at
 *                w_cap; endpoint pairs drawn from an alias table; drawn
 *                until m_target distinct non-loop pairs exist.
 *   gg_rmat      2^scale vertices, edge_factor * 2^scale directed draws with
 *                quadrant probabilities (a, b, c, 1-a-b-c), no noise, no
 *                permutation; symmetrised, deduplicated, loops dropped;
 *                isolated vertices are kept in n.
 *   gg_batch     mixed batch of small graphs (even ids ER, odd Chung-Lu).
 *   gg_serving_sizes  per-request (m, n, gamma) of the serving stream.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <pthread.h>
#include <unistd.h>

#define GG_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t gg_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static inline uint64_t gg_key(uint64_t seed, uint64_t stream) {
  return gg_mix64(gg_mix64(seed + GG_GAMMA) ^ (stream * 0xD1B54A32D192ED03ULL));
}
static inline uint64_t gg_at(uint64_t key, uint64_t i) {
  return gg_mix64(key + (i + 1) * GG_GAMMA);
}
static inline double gg_u01(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

/* exported for tests of the generator itself */
uint64_t gg_splitmix_at(uint64_t seed, uint64_t stream, uint64_t i) {
  return gg_at(gg_key(seed, stream), i);
}

void gg_free(void* p) { free(p); }

/* ---------- parallel LSD radix sort of uint64 keys (16-bit digits) ---------- */
static int gg_threads(void) {
  long p = sysconf(_SC_NPROCESSORS_ONLN);
  if (p < 1) p = 1;
  if (p > 32) p = 32;
  return (int)p;
}

typedef struct {
  const uint64_t* src; uint64_t* dst; int64_t lo, hi; int shift; int64_t* cnt;
} gg_rs_job_t;

static void* gg_rs_hist(void* a) {
  gg_rs_job_t* j = (gg_rs_job_t*)a;
  memset(j->cnt, 0, 65536 * sizeof(int64_t));
  for (int64_t i = j->lo; i < j->hi; ++i) j->cnt[(j->src[i] >> j->shift) & 0xFFFF]++;
  return NULL;
}
static void* gg_rs_scatter(void* a) {
  gg_rs_job_t* j = (gg_rs_job_t*)a;
  for (int64_t i = j->lo; i < j->hi; ++i) {
    uint64_t x = j->src[i];
    j->dst[j->cnt[(x >> j->shift) & 0xFFFF]++] = x;
  }
  return NULL;
}

/* Small arrays (the graphs of a batch): 8-bit digits with the histogram on
 * the stack, so that many threads sorting small arrays at once do not
 * allocate and clear large histograms. Same sorted output. */
static int gg_radix_sort_small(uint64_t* a, int64_t n, int key_bits) {
  uint64_t* tmp = (uint64_t*)malloc((size_t)n * sizeof(uint64_t));
  if (!tmp) return -1;
  uint64_t* src = a; uint64_t* dst = tmp;
  int64_t cnt[256];
  for (int shift = 0; shift < key_bits; shift += 8) {
    memset(cnt, 0, sizeof(cnt));
    for (int64_t i = 0; i < n; ++i) cnt[(src[i] >> shift) & 0xFF]++;
    if (cnt[(src[0] >> shift) & 0xFF] == n) continue;  /* one digit value: order unchanged */
    int64_t s = 0;
    for (int d = 0; d < 256; ++d) { int64_t c = cnt[d]; cnt[d] = s; s += c; }
    for (int64_t i = 0; i < n; ++i) dst[cnt[(src[i] >> shift) & 0xFF]++] = src[i];
    uint64_t* x = src; src = dst; dst = x;
  }
  if (src != a) memcpy(a, src, (size_t)n * sizeof(uint64_t));
  free(tmp);
  return 0;
}

static int gg_radix_sort_u64(uint64_t* a, int64_t n, int key_bits) {
  if (n <= 1) return 0;
  if (n < (1 << 16)) return gg_radix_sort_small(a, n, key_bits);
  int T = gg_threads();
  if (n < (1 << 20)) T = 1;
  uint64_t* tmp = (uint64_t*)malloc((size_t)n * sizeof(uint64_t));
  int64_t* cnt = (int64_t*)malloc((size_t)T * 65536 * sizeof(int64_t));
  gg_rs_job_t* jobs = (gg_rs_job_t*)malloc((size_t)T * sizeof(gg_rs_job_t));
  pthread_t* th = (pthread_t*)malloc((size_t)T * sizeof(pthread_t));
  if (!tmp || !cnt || !jobs || !th) { free(tmp); free(cnt); free(jobs); free(th); return -1; }
  uint64_t* src = a; uint64_t* dst = tmp;
  for (int shift = 0; shift < key_bits; shift += 16) {
    for (int t = 0; t < T; ++t) {
      jobs[t].src = src; jobs[t].dst = dst; jobs[t].shift = shift;
      jobs[t].lo = n * t / T; jobs[t].hi = n * (t + 1) / T; jobs[t].cnt = cnt + (size_t)t * 65536;
    }
    for (int t = 1; t < T; ++t) pthread_create(&th[t], NULL, gg_rs_hist, &jobs[t]);
    gg_rs_hist(&jobs[0]);
    for (int t = 1; t < T; ++t) pthread_join(th[t], NULL);
    int64_t s = 0;
    for (int d = 0; d < 65536; ++d)
      for (int t = 0; t < T; ++t) { int64_t c = cnt[(size_t)t * 65536 + d]; cnt[(size_t)t * 65536 + d] = s; s += c; }
    for (int t = 1; t < T; ++t) pthread_create(&th[t], NULL, gg_rs_scatter, &jobs[t]);
    gg_rs_scatter(&jobs[0]);
    for (int t = 1; t < T; ++t) pthread_join(th[t], NULL);
    uint64_t* x = src; src = dst; dst = x;
  }
  if (src != a) memcpy(a, src, (size_t)n * sizeof(uint64_t));
  free(tmp); free(cnt); free(jobs); free(th);
  return 0;
}

static int64_t gg_unique_sorted(uint64_t* a, int64_t n) {
  if (n == 0) return 0;
  int64_t w = 1;
  for (int64_t i = 1; i < n; ++i) if (a[i] != a[w - 1]) a[w++] = a[i];
  return w;
}

/* Build a symmetric CSR from sorted unique pair keys (u << 32 | v), u < v.
 * Row r receives first its smaller neighbours (from pairs (u, r)) in
 * ascending u, then its larger neighbours (from pairs (r, v)) in ascending
 * v, so every row comes out sorted. Returns -2 if 2m does not fit int32. */
static int gg_csr_from_pairs(int32_t n, const uint64_t* keys, int64_t m,
                             int32_t** rp_out, int32_t** ci_out) {
  if (2 * m > 2147483647LL) return -2;
  int32_t* rp = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t));
  int32_t* ci = (int32_t*)malloc((size_t)(2 * m > 0 ? 2 * m : 1) * sizeof(int32_t));
  int32_t* pos = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t));
  if (!rp || !ci || !pos) { free(rp); free(ci); free(pos); return -1; }
  memset(rp, 0, ((size_t)n + 1) * sizeof(int32_t));
  for (int64_t i = 0; i < m; ++i) {
    uint32_t u = (uint32_t)(keys[i] >> 32), v = (uint32_t)(keys[i] & 0xFFFFFFFFu);
    rp[u + 1]++; rp[v + 1]++;
  }
  for (int32_t i = 0; i < n; ++i) rp[i + 1] += rp[i];
  memcpy(pos, rp, ((size_t)n + 1) * sizeof(int32_t));
  for (int64_t i = 0; i < m; ++i) {          /* row v gets u (u < v) */
    uint32_t u = (uint32_t)(keys[i] >> 32), v = (uint32_t)(keys[i] & 0xFFFFFFFFu);
    ci[pos[v]++] = (int32_t)u;
  }
  for (int64_t i = 0; i < m; ++i) {          /* row u gets v (v > u) */
    uint32_t u = (uint32_t)(keys[i] >> 32), v = (uint32_t)(keys[i] & 0xFFFFFFFFu);
    ci[pos[u]++] = (int32_t)v;
  }
  free(pos);
  *rp_out = rp; *ci_out = ci;
  return 0;
}

static int gg_bits(uint64_t x) { int b = 0; while (x) { ++b; x >>= 1; } return b; }

/* keys: canonical (min << 32 | max); sort + unique + CSR. sorted: the keys
 * are already strictly ascending (Erdos-Renyi draws pairs in lexicographic
 * order), so the sort is skipped -- the same result. */
static int gg_finish_keys(int32_t n, uint64_t* keys, int64_t k, int sorted, int64_t* m_out,
                          int32_t** rp, int32_t** ci) {
  int bits = 32 + gg_bits((uint64_t)(n > 0 ? n - 1 : 0));
  if (!sorted && gg_radix_sort_u64(keys, k, bits) != 0) return -1;
  int64_t m = gg_unique_sorted(keys, k);
  while (m > 0 && keys[m - 1] == 0xFFFFFFFFFFFFFFFFULL) --m;  /* dropped self-loops sort last */
  int rc = gg_csr_from_pairs(n, keys, m, rp, ci);
  if (rc == 0) *m_out = m;
  return rc;
}
static int gg_finish(int32_t n, uint64_t* keys, int64_t k, int64_t* m_out, int32_t** rp, int32_t** ci) {
  return gg_finish_keys(n, keys, k, 0, m_out, rp, ci);
}

/* ---------------- Erdos-Renyi G(n, p) ---------------- */
static int64_t gg_er_keys(int32_t n, double p, uint64_t key, uint64_t* keys) {
  int64_t k = 0, rank = 0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = i + 1; j < n; ++j, ++rank)
      if (gg_u01(gg_at(key, (uint64_t)rank)) < p) keys[k++] = ((uint64_t)i << 32) | (uint64_t)j;
  return k;
}

int gg_er(int32_t n, double p, uint64_t seed, int64_t* m_out, int32_t** rp, int32_t** ci) {
  if (n < 0 || n > 200000 || !(p >= 0.0 && p <= 1.0)) return -3;
  int64_t pairs = (int64_t)n * (n - 1) / 2;
  /* at most all pairs; allocate a bound with slack above the mean */
  double mean = p * (double)pairs;
  int64_t cap = (int64_t)(mean + 10.0 * sqrt(mean + 1.0) + 64.0);
  if (cap > pairs) cap = pairs;
  uint64_t* keys = (uint64_t*)malloc((size_t)(cap > 0 ? cap : 1) * sizeof(uint64_t));
  if (!keys) return -1;
  uint64_t key = gg_key(seed, 1);
  /* count first so the bound can never overflow */
  int64_t cnt = 0, rank = 0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = i + 1; j < n; ++j, ++rank)
      if (gg_u01(gg_at(key, (uint64_t)rank)) < p) ++cnt;
  if (cnt > cap) {
    free(keys);
    keys = (uint64_t*)malloc((size_t)(cnt > 0 ? cnt : 1) * sizeof(uint64_t));
    if (!keys) return -1;
  }
  int64_t k = gg_er_keys(n, p, key, keys);
  int rc = gg_finish(n, keys, k, m_out, rp, ci);
  free(keys);
  return rc;
}

/* ---------------- Chung-Lu ---------------- */
typedef struct { double* prob; int32_t* alias; int32_t n; } gg_alias_t;

/* Vose's alias method (Vose, IEEE TSE 1991). */
static int gg_alias_build(const double* w, int32_t n, gg_alias_t* t) {
  t->n = n;
  t->prob = (double*)malloc((size_t)n * sizeof(double));
  t->alias = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  int32_t* small = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  int32_t* large = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  double* q = (double*)malloc((size_t)n * sizeof(double));
  if (!t->prob || !t->alias || !small || !large || !q) {
    free(t->prob); free(t->alias); free(small); free(large); free(q); return -1;
  }
  double s = 0.0;
  for (int32_t i = 0; i < n; ++i) s += w[i];
  int32_t ns = 0, nl = 0;
  for (int32_t i = 0; i < n; ++i) {
    q[i] = w[i] * (double)n / s;
    if (q[i] < 1.0) small[ns++] = i; else large[nl++] = i;
  }
  while (ns > 0 && nl > 0) {
    int32_t l = small[--ns], g = large[--nl];
    t->prob[l] = q[l]; t->alias[l] = g;
    q[g] = (q[g] + q[l]) - 1.0;
    if (q[g] < 1.0) small[ns++] = g; else large[nl++] = g;
  }
  while (nl > 0) { int32_t g = large[--nl]; t->prob[g] = 1.0; t->alias[g] = g; }
  while (ns > 0) { int32_t l = small[--ns]; t->prob[l] = 1.0; t->alias[l] = l; }
  free(small); free(large); free(q);
  return 0;
}
static void gg_alias_free(gg_alias_t* t) { free(t->prob); free(t->alias); }

static inline int32_t gg_alias_draw(const gg_alias_t* t, uint64_t x) {
  uint32_t i = (uint32_t)(((x >> 32) * (uint64_t)(uint32_t)t->n) >> 32);
  double c = (double)(x & 0xFFFFFFFFu) * (1.0 / 4294967296.0);
  return c < t->prob[i] ? (int32_t)i : t->alias[i];
}

/* open-addressing set of nonzero uint64 keys */
typedef struct { uint64_t* slot; uint64_t mask; int64_t size; } gg_set_t;
static int gg_set_init(gg_set_t* s, int64_t want) {
  uint64_t cap = 16; while (cap < (uint64_t)(want * 2)) cap <<= 1;
  s->slot = (uint64_t*)calloc(cap, sizeof(uint64_t));
  s->mask = cap - 1; s->size = 0;
  return s->slot ? 0 : -1;
}
/* returns 1 if inserted, 0 if present */
static inline int gg_set_insert(gg_set_t* s, uint64_t k) {
  uint64_t h = gg_mix64(k) & s->mask;
  for (;;) {
    uint64_t c = s->slot[h];
    if (c == 0) { s->slot[h] = k; s->size++; return 1; }
    if (c == k) return 0;
    h = (h + 1) & s->mask;
  }
}

/* Keys stored as ((u << 32) | v) + 1 so that 0 marks an empty slot. */
static int gg_chung_lu_keys(int32_t n, int64_t m_target, double gamma, double sum_w,
                            double w_cap, uint64_t key, uint64_t** keys_out, int64_t* k_out) {
  double* w = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
  if (!w) return -1;
  double ex = -1.0 / (gamma - 1.0), s = 0.0;
  for (int32_t i = 0; i < n; ++i) { w[i] = pow((double)(i + 1), ex); s += w[i]; }
  for (int32_t i = 0; i < n; ++i) { w[i] = w[i] * (sum_w / s); if (w[i] > w_cap) w[i] = w_cap; }
  gg_alias_t t;
  if (gg_alias_build(w, n, &t) != 0) { free(w); return -1; }
  free(w);
  int64_t maxpairs = (int64_t)n * (n - 1) / 2;
  if (m_target > maxpairs) m_target = maxpairs;
  gg_set_t set;
  if (gg_set_init(&set, m_target + 1) != 0) { gg_alias_free(&t); return -1; }
  uint64_t* keys = (uint64_t*)malloc((size_t)(m_target > 0 ? m_target : 1) * sizeof(uint64_t));
  if (!keys) { free(set.slot); gg_alias_free(&t); return -1; }
  int64_t k = 0;
  uint64_t max_draws = (uint64_t)(m_target > 0 ? m_target : 1) * 64ULL + 1024ULL;
  for (uint64_t j = 0; k < m_target && j < max_draws; ++j) {
    int32_t a = gg_alias_draw(&t, gg_at(key, 2 * j));
    int32_t b = gg_alias_draw(&t, gg_at(key, 2 * j + 1));
    if (a == b) continue;
    uint64_t lo = (uint64_t)(a < b ? a : b), hi = (uint64_t)(a < b ? b : a);
    uint64_t kk = (lo << 32) | hi;
    if (gg_set_insert(&set, kk + 1)) keys[k++] = kk;
  }
  free(set.slot); gg_alias_free(&t);
  *keys_out = keys; *k_out = k;
  return 0;
}

int gg_chung_lu(int32_t n, int64_t m_target, double gamma, double sum_w, double w_cap,
                uint64_t seed, int64_t* m_out, int32_t** rp, int32_t** ci) {
  if (n < 2 || !(gamma > 1.0) || m_target < 0) return -3;
  uint64_t* keys; int64_t k;
  int rc = gg_chung_lu_keys(n, m_target, gamma, sum_w, w_cap, gg_key(seed, 2), &keys, &k);
  if (rc) return rc;
  rc = gg_finish(n, keys, k, m_out, rp, ci);
  free(keys);
  return rc;
}

/* ---------------- R-MAT ---------------- */
typedef struct {
  uint64_t key; int scale; double a, ab, abc; int64_t lo, hi; uint64_t* keys;
} gg_rmat_job_t;

#define GG_NONE 0xFFFFFFFFFFFFFFFFULL  /* self-loop marker: sorts after every pair */

static void* gg_rmat_draw(void* p) {
  gg_rmat_job_t* j = (gg_rmat_job_t*)p;
  for (int64_t i = j->lo; i < j->hi; ++i) {
    uint64_t u = 0, v = 0;
    for (int l = 0; l < j->scale; ++l) {
      double r = gg_u01(gg_at(j->key, (uint64_t)i * (uint64_t)j->scale + (uint64_t)l));
      uint64_t rb, cb;
      if (r < j->a) { rb = 0; cb = 0; }
      else if (r < j->ab) { rb = 0; cb = 1; }
      else if (r < j->abc) { rb = 1; cb = 0; }
      else { rb = 1; cb = 1; }
      u = (u << 1) | rb; v = (v << 1) | cb;
    }
    j->keys[i] = u == v ? GG_NONE : (u < v ? ((u << 32) | v) : ((v << 32) | u));
  }
  return NULL;
}

int gg_rmat(int scale, int64_t edge_factor, double a, double b, double c, uint64_t seed,
            int32_t* n_out, int64_t* m_out, int32_t** rp, int32_t** ci) {
  if (scale < 1 || scale > 30 || edge_factor < 0) return -3;
  int64_t draws = edge_factor << scale;
  uint64_t* keys = (uint64_t*)malloc((size_t)(draws > 0 ? draws : 1) * sizeof(uint64_t));
  if (!keys) return -1;
  int T = gg_threads();
  if (draws < (1 << 18)) T = 1;
  gg_rmat_job_t jobs[32];
  pthread_t th[32];
  for (int t = 0; t < T; ++t) {
    jobs[t].key = gg_key(seed, 3); jobs[t].scale = scale;
    jobs[t].a = a; jobs[t].ab = a + b; jobs[t].abc = a + b + c;
    jobs[t].lo = draws * t / T; jobs[t].hi = draws * (t + 1) / T; jobs[t].keys = keys;
  }
  for (int t = 1; t < T; ++t) pthread_create(&th[t], NULL, gg_rmat_draw, &jobs[t]);
  gg_rmat_draw(&jobs[0]);
  for (int t = 1; t < T; ++t) pthread_join(th[t], NULL);
  int32_t n = (int32_t)(1 << scale);
  int rc = gg_finish(n, keys, draws, m_out, rp, ci);
  free(keys);
  if (rc == 0) *n_out = n;
  return rc;
}

/* ---------------- batches of small graphs ----------------
 * Graph g draws its parameters from stream 16 + g of `seed`:
 *   n = n_lo + floor(u0 * (n_hi - n_lo + 1))
 *   even g: ER with p = p_lo + u1 * (p_hi - p_lo), pair stream key(seed', 1)
 *   odd g : Chung-Lu with gamma = g_lo + u1 * (g_hi - g_lo), mean degree
 *           dbar = 2 + u2 * (min(32, (n-1)/4) - 2), m_target = round(n*dbar/2),
 *           sum_w = n * dbar, w_cap = n - 1, pair stream key(seed', 2)
 * where seed' = value(stream 16 + g, 3). Output is concatenated:
 *   nvert[g], voff[g] (int64 offset of graph g's row_ptr, n_g + 1 entries,
 *   local, starting at 0), eoff[g] (int64 offset of its col_idx, local ids).
 */
typedef struct {
  int32_t n; int kind; double p_or_gamma; double dbar; uint64_t seed2;
} gg_bparams_t;

static void gg_batch_params(uint64_t seed, int64_t g, int32_t n_lo, int32_t n_hi,
                            double p_lo, double p_hi, double g_lo, double g_hi,
                            gg_bparams_t* bp) {
  uint64_t key = gg_key(seed, 16 + (uint64_t)g);
  double u0 = gg_u01(gg_at(key, 0)), u1 = gg_u01(gg_at(key, 1)), u2 = gg_u01(gg_at(key, 2));
  int32_t n = n_lo + (int32_t)(u0 * (double)(n_hi - n_lo + 1));
  if (n > n_hi) n = n_hi;
  bp->n = n;
  bp->seed2 = gg_at(key, 3);
  if ((g & 1) == 0) {
    bp->kind = 0; bp->p_or_gamma = p_lo + u1 * (p_hi - p_lo); bp->dbar = 0.0;
  } else {
    double dmax = (double)(n - 1) / 4.0; if (dmax > 32.0) dmax = 32.0;
    if (dmax < 2.0) dmax = 2.0;
    bp->kind = 1; bp->p_or_gamma = g_lo + u1 * (g_hi - g_lo);
    bp->dbar = 2.0 + u2 * (dmax - 2.0);
  }
}

typedef struct {
  int64_t G, t, T; int32_t n_lo, n_hi; double p_lo, p_hi, g_lo, g_hi; uint64_t seed;
  int32_t* nvert; int64_t* m; int32_t** rps; int32_t** cis; int rc;
} gg_batch_job_t;

static void* gg_batch_worker(void* arg) {
  gg_batch_job_t* j = (gg_batch_job_t*)arg;
  for (int64_t g = j->t; g < j->G && j->rc == 0; g += j->T) {
    gg_bparams_t bp;
    gg_batch_params(j->seed, g, j->n_lo, j->n_hi, j->p_lo, j->p_hi, j->g_lo, j->g_hi, &bp);
    int64_t m = 0;
    int rc;
    if (bp.kind == 0) {
      uint64_t pairs = (uint64_t)bp.n * (uint64_t)(bp.n - 1) / 2;
      uint64_t* keys = (uint64_t*)malloc((size_t)(pairs > 0 ? pairs : 1) * sizeof(uint64_t));
      if (!keys) { j->rc = -1; break; }
      int64_t k = gg_er_keys(bp.n, bp.p_or_gamma, gg_key(bp.seed2, 1), keys);
      rc = gg_finish_keys(bp.n, keys, k, 1, &m, &j->rps[g], &j->cis[g]);
      free(keys);
    } else {
      int64_t mt = (int64_t)((double)bp.n * bp.dbar / 2.0 + 0.5);
      uint64_t* keys; int64_t k;
      rc = gg_chung_lu_keys(bp.n, mt, bp.p_or_gamma, (double)bp.n * bp.dbar, (double)(bp.n - 1),
                            gg_key(bp.seed2, 2), &keys, &k);
      if (rc == 0) { rc = gg_finish(bp.n, keys, k, &m, &j->rps[g], &j->cis[g]); free(keys); }
    }
    if (rc) { j->rc = rc; break; }
    j->nvert[g] = bp.n;
    j->m[g] = m;
  }
  return NULL;
}

int gg_batch(int64_t G, int32_t n_lo, int32_t n_hi, double p_lo, double p_hi,
             double g_lo, double g_hi, uint64_t seed,
             int32_t** nvert_out, int64_t** voff_out, int64_t** eoff_out,
             int32_t** rp_out, int32_t** ci_out, int64_t* total_rows_out, int64_t* total_nnz_out) {
  if (G < 0 || n_lo < 2 || n_hi < n_lo || n_hi > 65535) return -3;
  int32_t* nvert = (int32_t*)malloc((size_t)(G > 0 ? G : 1) * sizeof(int32_t));
  int64_t* mm = (int64_t*)malloc((size_t)(G > 0 ? G : 1) * sizeof(int64_t));
  int64_t* voff = (int64_t*)malloc((size_t)(G + 1) * sizeof(int64_t));
  int64_t* eoff = (int64_t*)malloc((size_t)(G + 1) * sizeof(int64_t));
  int32_t** rps = (int32_t**)calloc((size_t)(G > 0 ? G : 1), sizeof(int32_t*));
  int32_t** cis = (int32_t**)calloc((size_t)(G > 0 ? G : 1), sizeof(int32_t*));
  if (!nvert || !mm || !voff || !eoff || !rps || !cis) return -1;
  int T = gg_threads();
  if (G < 64) T = 1;
  gg_batch_job_t jobs[32];
  pthread_t th[32];
  for (int t = 0; t < T; ++t) {
    gg_batch_job_t jb = {G, t, T, n_lo, n_hi, p_lo, p_hi, g_lo, g_hi, seed, nvert, mm, rps, cis, 0};
    jobs[t] = jb;
  }
  for (int t = 1; t < T; ++t) pthread_create(&th[t], NULL, gg_batch_worker, &jobs[t]);
  gg_batch_worker(&jobs[0]);
  for (int t = 1; t < T; ++t) pthread_join(th[t], NULL);
  int rc = 0;
  for (int t = 0; t < T; ++t) if (jobs[t].rc) rc = jobs[t].rc;
  voff[0] = 0; eoff[0] = 0;
  if (rc == 0)
    for (int64_t g = 0; g < G; ++g) { voff[g + 1] = voff[g] + nvert[g] + 1; eoff[g + 1] = eoff[g] + 2 * mm[g]; }
  if (rc == 0) {
    int32_t* rp = (int32_t*)malloc((size_t)(voff[G] > 0 ? voff[G] : 1) * sizeof(int32_t));
    int32_t* ci = (int32_t*)malloc((size_t)(eoff[G] > 0 ? eoff[G] : 1) * sizeof(int32_t));
    if (!rp || !ci) { free(rp); free(ci); rc = -1; }
    else {
      for (int64_t g = 0; g < G; ++g) {
        memcpy(rp + voff[g], rps[g], (size_t)(nvert[g] + 1) * sizeof(int32_t));
        memcpy(ci + eoff[g], cis[g], (size_t)(eoff[g + 1] - eoff[g]) * sizeof(int32_t));
      }
      *rp_out = rp; *ci_out = ci;
      *total_rows_out = voff[G]; *total_nnz_out = eoff[G];
    }
  }
  for (int64_t g = 0; g < G; ++g) { free(rps[g]); free(cis[g]); }
  free(rps); free(cis); free(mm);
  if (rc != 0) { free(nvert); free(voff); free(eoff); return rc; }
  *nvert_out = nvert; *voff_out = voff; *eoff_out = eoff;
  return 0;
}

/* Serving stream: request r draws from stream 1'000'000 + r:
 *   m_r = round(exp(log(m_lo) + u0 * (log(m_hi) - log(m_lo))))
 *   gamma_r = g_lo + u1 * (g_hi - g_lo)
 *   n_r = max(64, m_r / 8); inter-arrival gap = -log(1 - u2) (unit rate)
 *   seed_r = value(., 3)
 * The graph itself is gg_chung_lu(n_r, m_r, gamma_r, 2 m_r, min(50000, n_r-1), seed_r). */
int gg_serving_params(int64_t R, int64_t m_lo, int64_t m_hi, double g_lo, double g_hi,
                      uint64_t seed, int64_t* m_out, int32_t* n_out, double* gamma_out,
                      double* gap_out, uint64_t* seed_out) {
  if (R < 0 || m_lo < 1 || m_hi < m_lo) return -3;
  for (int64_t r = 0; r < R; ++r) {
    uint64_t key = gg_key(seed, 1000000ULL + (uint64_t)r);
    double u0 = gg_u01(gg_at(key, 0)), u1 = gg_u01(gg_at(key, 1)), u2 = gg_u01(gg_at(key, 2));
    double lm = log((double)m_lo) + u0 * (log((double)m_hi) - log((double)m_lo));
    int64_t m = (int64_t)(exp(lm) + 0.5);
    if (m < m_lo) m = m_lo;
    if (m > m_hi) m = m_hi;
    int64_t n = m / 8; if (n < 64) n = 64;
    m_out[r] = m; n_out[r] = (int32_t)n;
    gamma_out[r] = g_lo + u1 * (g_hi - g_lo);
    gap_out[r] = -log(1.0 - u2);
    seed_out[r] = gg_at(key, 3);
  }
  return 0;
}
