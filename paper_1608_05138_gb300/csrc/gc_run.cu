// gc_run.cu -- the sequence of one count, shared by the whole-graph and the
// batched paths.
//
//   pass A  triangle step: |T| per edge                          (Alg. 1)
//   pass C  4-cycles through every edge, degree-ordered wedges   (Alg. 4/6)
//   chunks  split v-groups into balanced units (|T| now known)   (Sec. 4.5)
//   pass B  4-cliques, per-edge columns, unrestricted sums       (Alg. 5, Sec. 4.5)
//   big     the edges whose T exceeds a warp buffer, one CTA each
//   derive  X_1..X_17                                            (Sec. 4.6)
//
// Two host synchronisations sit inside: after pass A (largest |T|, to size
// the large-T buffers) folded into the chunking step, which reads back the
// total estimated work.
#include <cuda_runtime.h>

#include "gc_internal.h"

namespace gc {

void scratch_free(Scratch* sc, cudaStream_t s) {
  for (void* p : {(void*)sc->tri, (void*)sc->P, (void*)sc->chunks, (void*)sc->off, (void*)sc->misc,
                  (void*)sc->total, (void*)sc->tables, (void*)sc->tbuf, (void*)sc->deferred, (void*)sc->work})
    if (p) cudaFreeAsync(p, s);
  *sc = Scratch();
}

gc_status scratch_init(Scratch* sc, int32_t m, int32_t n_units, int32_t table_n, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
#define GS_TRY(call)                                \
  do {                                              \
    e = (call);                                     \
    if (e != cudaSuccess) return cuda_fail(e, "scratch alloc"); \
  } while (0)
  GS_TRY(cudaMallocAsync(&sc->tri, sizeof(int32_t) * (size_t)(m > 0 ? m : 1), s));
  GS_TRY(cudaMallocAsync(&sc->P, sizeof(unsigned long long) * (size_t)(m > 0 ? 2 * (size_t)m : 1), s));
  GS_TRY(cudaMallocAsync(&sc->chunks, sizeof(int32_t) * 3 * chunk_capacity(n_units), s));
  GS_TRY(cudaMallocAsync(&sc->off, sizeof(int32_t) * ((size_t)n_units + 1), s));
  GS_TRY(cudaMallocAsync(&sc->misc, sizeof(int32_t) * 8, s));
  GS_TRY(cudaMallocAsync(&sc->total, sizeof(unsigned long long), s));
  GS_TRY(cudaMallocAsync(&sc->work, sizeof(unsigned long long) * kNumWork, s));
  if (table_n > kSmemTableMax) {
    sc->tables_n = (size_t)count_grid_size() * (size_t)table_n;
    GS_TRY(cudaMallocAsync(&sc->tables, sizeof(uint32_t) * sc->tables_n, s));
    GS_TRY(cudaMemsetAsync(sc->tables, 0, sizeof(uint32_t) * sc->tables_n, s));
  }
#undef GS_TRY
  return GC_OK;
}

gc_status run_count(const DevGraph& g, const int32_t* units, int32_t n_units, uint64_t* per_edge,
                    unsigned long long* csum, unsigned long long* x, Scratch* sc, cudaStream_t s,
                    cudaEvent_t* ev) {
  cudaError_t e = cudaSuccess;
  gc_status st = GC_OK;
#define GR_TRY(call, what)                  \
  do {                                      \
    e = (call);                             \
    if (e != cudaSuccess) return cuda_fail(e, what); \
  } while (0)
#define GR_EVENT(i) \
  if (ev) GR_TRY(cudaEventRecord(ev[i], s), "event")
  int32_t* cursor = sc->misc;
  int32_t* status = sc->misc + 1;
  int32_t* tmax_dev = sc->misc + 2;
  int32_t* nbig_dev = sc->misc + 3;
  int32_t* ndef_dev = sc->misc + 4;
  CountArgs a;
  a.units = units;
  a.n_units = n_units;
  a.chunks = sc->chunks;
  a.n_chunks = sc->off + n_units;
  a.cursor = cursor;
  a.tables = g.table_n > kSmemTableMax ? sc->tables : nullptr;
  a.tri = sc->tri;
  a.P = sc->P;
  a.tbuf = nullptr;
  a.tbuf_len = 0;
  a.deferred = nullptr;
  a.deferred_cap = 0;
  a.n_deferred = ndef_dev;
  a.big_t = big_t_threshold();
  a.per_edge = per_edge;
  a.csum = csum;
  a.status = status;
  a.work = sc->work;
  GR_TRY(cudaMemsetAsync(sc->misc, 0, sizeof(int32_t) * 8, s), "memset misc");
  GR_TRY(cudaMemsetAsync(sc->work, 0, sizeof(unsigned long long) * kNumWork, s), "memset work");
  GR_TRY(cudaMemsetAsync(csum, 0, sizeof(unsigned long long) * 26 * (size_t)g.G, s), "memset sums");
  GR_EVENT(kPhasePassA);
  int32_t nbig = 0;
  if (n_units > 0) {
    if ((st = run_pass_a(g, a, s)) != GC_OK) return st;
    if ((st = run_max_tri(sc->tri, g.m, tmax_dev, s)) != GC_OK) return st;
    GR_EVENT(kPhasePassC);
    GR_TRY(cudaMemsetAsync(sc->P, 0, sizeof(unsigned long long) * 2 * (size_t)g.m, s), "zero P");
    GR_TRY(cudaMemsetAsync(cursor, 0, sizeof(int32_t), s), "reset cursor");
    if ((st = run_pass_c(g, a, s)) != GC_OK) return st;
    if ((st = run_make_chunks(g, units, n_units, sc->tri, sc->chunks, sc->off, sc->total, nbig_dev, a.big_t, s)) != GC_OK)
      return st;
    int32_t hm[2] = {0, 0};  // max |T|, number of large-T edges (complete: the chunking synchronised)
    GR_TRY(cudaMemcpyAsync(hm, tmax_dev, sizeof(hm), cudaMemcpyDeviceToHost, s), "copy counts");
    GR_TRY(cudaStreamSynchronize(s), "sync counts");
    nbig = hm[1];
    if (nbig > 0) {
      if (sc->tbuf_len < hm[0]) {
        if (sc->tbuf) cudaFreeAsync(sc->tbuf, s);
        sc->tbuf_len = hm[0];
        GR_TRY(cudaMallocAsync(&sc->tbuf, sizeof(int32_t) * (size_t)big_grid_size() * sc->tbuf_len, s),
               "alloc T buffers");
      }
      if (sc->deferred_cap < nbig) {
        if (sc->deferred) cudaFreeAsync(sc->deferred, s);
        sc->deferred_cap = nbig;
        GR_TRY(cudaMallocAsync(&sc->deferred, sizeof(int32_t) * 2 * (size_t)nbig, s), "alloc deferred");
      }
      a.deferred = sc->deferred;
      a.deferred_cap = sc->deferred_cap;
      a.tbuf = sc->tbuf;
      a.tbuf_len = sc->tbuf_len;
    }
    GR_TRY(cudaMemsetAsync(cursor, 0, sizeof(int32_t), s), "reset cursor");
  } else {
    GR_EVENT(kPhasePassC);
  }
  GR_EVENT(kPhasePassB);
  if (n_units > 0) {
    if ((st = run_pass_b(g, a, s)) != GC_OK) return st;
  }
  GR_EVENT(kPhaseBig);
  if (nbig > 0) {
    GR_TRY(cudaMemsetAsync(cursor, 0, sizeof(int32_t), s), "reset cursor");
    if ((st = run_pass_big(g, a, nbig, s)) != GC_OK) return st;
  }
  GR_EVENT(kPhaseDerive);
  if ((st = run_derive(g, csum, x, status, s)) != GC_OK) return st;
  GR_EVENT(kPhaseCopy);
#undef GR_EVENT
#undef GR_TRY
  return GC_OK;
}

}  // namespace gc
