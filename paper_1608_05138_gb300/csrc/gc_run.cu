// gc_run.cu -- the sequence of one count, shared by the whole-graph and the
// batched paths.
//
//   pass T  triangle step: |T| per edge, by lowest vertex         (Alg. 1)
//   pass C  4-cycles through every edge, degree-ordered wedges   (Alg. 4/6)
//   pass K  4-cliques and cross terms by lowest vertex           (Alg. 3/5)
//   finish  x10, per-edge columns, unrestricted sums             (Sec. 4.5)
//   derive  X_1..X_17                                            (Sec. 4.6)
//
// Everything is queued on one stream with no host synchronisation: the unit
// lists and their tier boundaries are fixed when the graph is prepared.
#include <cuda_runtime.h>

#include <cstdlib>

#include "gc_internal.h"

namespace gc {

namespace {
// Total bytes the pass-K global tier may hold at once.
constexpr size_t kKbufBudget = size_t(2) << 30;
// Largest list of the edges of all H_a that pass T keeps for pass K.
constexpr long long kTListBudget = 24LL << 30;
// Largest per-CTA list of H_a edges in pass K (units with more edges rescan
// their out-lists instead): 2^19 entries, or the environment's GC_K_LIST_CAP
// (1 .. 2^19), read once per process.
long long k_list_cap() {
  static long long v = [] {
    const char* e = getenv("GC_K_LIST_CAP");
    long long x = e ? atoll(e) : (1LL << 19);
    return x < 1 ? 1LL : (x > (1LL << 19) ? (1LL << 19) : x);
  }();
  return v;
}
// Bound on the entries of pass T's edge lists from the environment's
// GC_T_LIST_CAP (>= 1; units past it scan again in pass K), read once per
// process; 0: not set.
long long t_list_cap_knob() {
  static long long v = [] {
    const char* e = getenv("GC_T_LIST_CAP");
    const long long x = e ? atoll(e) : 0;
    return e ? (x < 1 ? 1LL : x) : 0LL;
  }();
  return v;
}
}  // namespace

void scratch_free(Scratch* sc, cudaStream_t s) {
  for (void* p : {(void*)sc->trio, (void*)sc->P, (void*)sc->xc, (void*)sc->misc,
                  (void*)sc->cbuf, (void*)sc->tables, (void*)sc->kbuf, (void*)sc->hitbuf, (void*)sc->work,
                  (void*)sc->tlist, (void*)sc->tl_off, (void*)sc->tl_cnt, (void*)sc->tl_fill, (void*)sc->dsum,
                  (void*)sc->vsum})
    if (p) cudaFreeAsync(p, s);
  *sc = Scratch();
}

gc_status scratch_init(Scratch* sc, int32_t m, int32_t table_n, int32_t kmax, int32_t cnx_max, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
#define GS_TRY(call)                                \
  do {                                              \
    e = (call);                                     \
    if (e != cudaSuccess) return cuda_fail(e, "scratch alloc"); \
  } while (0)
  const size_t m1 = (size_t)(m > 0 ? m : 1);
  GS_TRY(pool_alloc(&sc->trio, sizeof(int32_t) * m1, s));
  GS_TRY(pool_alloc(&sc->P, sizeof(unsigned long long) * 2 * m1, s));
  GS_TRY(pool_alloc(&sc->xc, sizeof(unsigned long long) * 2 * m1, s));
  GS_TRY(pool_alloc(&sc->misc, sizeof(int32_t) * 32, s));
  GS_TRY(pool_alloc(&sc->work, sizeof(unsigned long long) * kNumWork, s));
  if (table_n > kSmemTableMax) {
    sc->tables_n = (size_t)count_grid_size() * (size_t)table_n;
    GS_TRY(pool_alloc(&sc->tables, sizeof(uint32_t) * sc->tables_n, s));
    GS_TRY(cudaMemsetAsync(sc->tables, 0, sizeof(uint32_t) * sc->tables_n, s));
  }
  if (cnx_max > 0) {
    sc->cbuf_nx = cnx_max;
    GS_TRY(pool_alloc(&sc->cbuf, sizeof(int32_t) * 3 * (size_t)cnx_max * (size_t)(count_grid_size() / kCtasPerSm), s));
  }
  {  // pass K: each CTA records the edges of its current H_a (at most C(kmax, 2))
    const long long full = (long long)kmax * (kmax - 1) / 2;
    const long long cap = k_list_cap();
    sc->hitcap = (int32_t)(full < cap ? (full > 0 ? full : 1) : cap);
    sc->hitbuf_ctas = 4 * (count_grid_size() / kCtasPerSm);  // up to four CTAs per SM in any tier
    GS_TRY(pool_alloc(&sc->hitbuf, sizeof(int32_t) * 2 * (size_t)sc->hitcap * (size_t)sc->hitbuf_ctas, s));
  }
  if (kmax > kTierCap[kTier1024]) {
    sc->kbuf_cap = kmax;
    sc->kbuf_stride = kbuf_bytes(kmax);
    size_t ctas = kKbufBudget / sc->kbuf_stride;
    const size_t sms = (size_t)(count_grid_size() / kCtasPerSm);
    if (ctas > sms) ctas = sms;
    if (ctas < 1) ctas = 1;
    sc->kbuf_ctas = (int32_t)ctas;
    GS_TRY(pool_alloc(&sc->kbuf, sc->kbuf_stride * ctas, s));
  }
#undef GS_TRY
  return GC_OK;
}

void scratch_guess_tlist(Scratch* sc, int64_t m) {
  const long long cap = kTListBudget / (long long)sizeof(int2);
  sc->tlist_want = 32 * m < cap ? 32 * m : cap;
}

static int32_t ku_total(const KUnits& ku) { return ku.tier_off[kNumTiers]; }

gc_status run_count(const DevGraph& g, const int32_t* units, int32_t n_units, const KUnits& ku,
                    uint64_t* per_edge, unsigned long long* csum, unsigned long long* x, Scratch* sc,
                    cudaStream_t s, cudaEvent_t* ev, bool per_edge_host, uint64_t* induced, bool induced_host) {
  cudaError_t e = cudaSuccess;
  gc_status st = GC_OK;
#define GR_TRY(call, what)                  \
  do {                                      \
    e = (call);                             \
    if (e != cudaSuccess) return cuda_fail(e, what); \
  } while (0)
#define GR_EVENT(i) \
  if (ev) GR_TRY(cudaEventRecord(ev[i], s), "event")
  CountArgs a;
  a.units = units;
  a.n_units = n_units;
  a.kunits = ku.units;
  a.cunits = ku.cunits;
  a.n_cheavy = ku.n_cheavy;
  a.cjobs = ku.cjobs;
  a.n_cjobs = ku.n_cjobs;
  a.chash_w = ku.chash_w;
  a.n_chash = ku.n_chash;
  a.n_chash_big = ku.n_chash_big;
  a.n_chash_mid = ku.n_chash_mid;
  a.n_chash2_big = ku.n_chash2_big;
  a.n_chash2 = ku.n_chash2;
  a.cbuf = sc->cbuf;
  a.cbuf_nx = sc->cbuf_nx;
  a.hub_tab = hub_tab_words();
  for (int t = 0; t <= kNumTiers; ++t) a.ktier_off[t] = ku.tier_off[t];
  a.cursor = sc->misc;  // [0] pass C, [2 + tier] pass K, [8] pass C hubs, [9] pass C hashed, [10 + tier] pass T,
                        // [15] pass C packed-key hash, [7] pass C hashed small units,
                        // [16] pass C hashed middle units, [17] pass C packed-key hash, half tables
  a.status = sc->misc + 1;
  a.tables = g.table_n > kSmemTableMax ? sc->tables : nullptr;
  a.trio = sc->trio;
  a.P = sc->P;
  a.xc = sc->xc;
  a.kbuf = sc->kbuf;
  a.kbuf_stride = sc->kbuf_stride;
  a.kbuf_ctas = sc->kbuf_ctas;
  a.kbuf_cap = sc->kbuf_cap;
  a.hitbuf = sc->hitbuf;
  a.hitcap = sc->hitcap;
  a.hitbuf_ctas = sc->hitbuf_ctas;
  // Pass T keeps the edges of the H_a for pass K, in a list sized by the
  // triangles of the previous count of this scratch (or by a first guess);
  // units that do not fit scan their out-lists again in pass K.
  {
    const int32_t nku = ku_total(ku);
    const long long want = sc->tlist_want;
    if (want > 0 && want * (long long)sizeof(int2) <= kTListBudget && nku > 0) {
      long long need = want + want / 16 + 1024;
      if (t_list_cap_knob() && need > t_list_cap_knob()) need = t_list_cap_knob();
      if (need > sc->tlist_cap) {
        if (sc->tlist) cudaFreeAsync(sc->tlist, s);
        sc->tlist = nullptr;
        sc->tlist_cap = 0;
        const long long cap = need;
        if (pool_alloc(&sc->tlist, sizeof(int2) * (size_t)cap, s) == cudaSuccess) sc->tlist_cap = cap;
        else cudaGetLastError();  // no list: pass K scans
      }
      if (nku > sc->tl_units) {
        for (void* p : {(void*)sc->tl_off, (void*)sc->tl_cnt})
          if (p) cudaFreeAsync(p, s);
        GR_TRY(pool_alloc(&sc->tl_off, sizeof(long long) * (size_t)nku, s), "alloc list index");
        GR_TRY(pool_alloc(&sc->tl_cnt, sizeof(int32_t) * (size_t)nku, s), "alloc list index");
        sc->tl_units = nku;
      }
      if (!sc->tl_fill) GR_TRY(pool_alloc(&sc->tl_fill, sizeof(unsigned long long), s), "alloc list fill");
    }
  }
  a.tlist = sc->tlist_cap > 0 ? sc->tlist : nullptr;
  a.tlist_cap = sc->tlist_cap;
  a.tlist_fill = sc->tl_fill;
  a.tl_off = sc->tl_off;
  a.tl_cnt = sc->tl_cnt;
  if (a.tlist) GR_TRY(cudaMemsetAsync(sc->tl_fill, 0, sizeof(unsigned long long), s), "zero list fill");
  a.per_edge = per_edge;
  a.per_edge_host = per_edge != nullptr && per_edge_host;
  a.dsum = nullptr;
  const bool want_induced = induced != nullptr && g.m > 0;
  if (want_induced) {  // scratch of the per-edge induced counts, kept with the graph
    if (!sc->dsum) GR_TRY(pool_alloc(&sc->dsum, sizeof(unsigned long long) * (size_t)g.m, s), "alloc dsum");
    if (!sc->vsum)
      GR_TRY(pool_alloc(&sc->vsum, sizeof(unsigned long long) * 2 * (size_t)(g.n > 0 ? g.n : 1), s),
             "alloc vsum");
    GR_TRY(cudaMemsetAsync(sc->dsum, 0, sizeof(unsigned long long) * (size_t)g.m, s), "zero dsum");
    a.dsum = sc->dsum;
  }
  a.csum = csum;
  a.work = sc->work;
  const size_t m1 = (size_t)(g.m > 0 ? g.m : 1);
  GR_TRY(cudaMemsetAsync(sc->misc, 0, sizeof(int32_t) * 32, s), "memset misc");
  GR_TRY(cudaMemsetAsync(sc->work, 0, sizeof(unsigned long long) * kNumWork, s), "memset work");
  GR_TRY(cudaMemsetAsync(csum, 0, sizeof(unsigned long long) * 26 * (size_t)g.G, s), "memset sums");
  GR_TRY(cudaMemsetAsync(sc->P, 0, sizeof(unsigned long long) * 2 * m1, s), "zero P");
  GR_TRY(cudaMemsetAsync(sc->xc, 0, sizeof(unsigned long long) * 2 * m1, s), "zero x7 and cross");
  GR_TRY(cudaMemsetAsync(sc->trio, 0, sizeof(int32_t) * m1, s), "zero T");
  int launches = 0;
  GR_EVENT(kPhasePassT);
  int t_launches = 0;
  if ((st = run_pass_t(g, a, s, &t_launches)) != GC_OK) return st;
  launches += t_launches;
  GR_EVENT(kPhasePassC);
  const int32_t n_cunits = ku.n_cunits;  // pass C units: hubs, hashed units, the others
  if (n_cunits > 0) {
    if (a.n_cheavy > 0) {
      if ((st = run_pass_c_heavy(g, a, s)) != GC_OK) return st;
      launches += 1;
    }
    if (a.n_chash > 0) {
      if ((st = run_pass_c_hash(g, a, s)) != GC_OK) return st;
      launches += 1;
    }
    if (a.n_chash2 > 0) {
      if ((st = run_pass_c_hash2(g, a, s)) != GC_OK) return st;
      launches += 1;
    }
    const int32_t n_hashed = a.n_cheavy + a.n_chash + a.n_chash2;
    if (n_cunits > n_hashed) {
      CountArgs al = a;  // the remaining units on the vertex-indexed tables
      al.units = a.cunits + n_hashed;
      al.n_units = n_cunits - n_hashed;
      GR_TRY(cudaMemsetAsync(a.cursor, 0, sizeof(int32_t), s), "reset cursor");
      if ((st = run_pass_c(g, al, s)) != GC_OK) return st;
      launches += 1;
    }
  }
  GR_EVENT(kPhasePassK);
  int k_launches = 0;
  if ((st = run_pass_k(g, a, s, &k_launches)) != GC_OK) return st;
  launches += k_launches;
  GR_EVENT(kPhaseFinish);
  if ((st = run_finish(g, a, s)) != GC_OK) return st;
  launches += g.m > 0 ? 1 : 0;
  GR_EVENT(kPhaseInduced);
  if (want_induced) {
    if ((st = run_induced(g, a, sc->vsum, induced, induced_host, s)) != GC_OK) return st;
    launches += 2;
  }
  GR_EVENT(kPhaseDerive);
  if ((st = run_derive(g, csum, x, a.status, s)) != GC_OK) return st;
  sc->launches = launches + 1;
  GR_EVENT(kPhaseCopy);
#undef GR_EVENT
#undef GR_TRY
  return GC_OK;
}

}  // namespace gc
