// gc_api.cu -- C ABI of the plain whole-graph path (see include/gc.h).
//
// Host-side CSR validation (Problem 1's input: simple undirected graph), the
// graph handle with its device-resident data, and the orchestration of one
// count: pass A (triangle step), pass B (clique/cycle steps, per-edge
// columns, unrestricted counts), derive (global counts), copies back.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "gc_internal.h"

namespace gc {

static thread_local std::string t_err;

void set_error(const std::string& msg) { t_err = msg; }

gc_status cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
  if (e == cudaErrorMemoryAllocation) return GC_ERR_NOMEM;
  return GC_ERR_CUDA;
}

// Host checks of a CSR (multi-threaded over rows). Symmetry is checked too:
// for every (x, y) the row of y must contain x.
gc_status validate_csr(int32_t n, const int32_t* rp, const int32_t* ci) {
  if (n < 0) { set_error("n < 0"); return GC_ERR_ARG; }
  if (rp[0] != 0) { set_error("row_ptr[0] != 0"); return GC_ERR_RANGE; }
  for (int32_t x = 0; x < n; ++x)
    if (rp[x + 1] < rp[x]) {
      set_error("row_ptr decreases at row " + std::to_string(x));
      return GC_ERR_UNSORTED;
    }
  if (rp[n] % 2 != 0) { set_error("row_ptr[n] is odd: the graph cannot be symmetric"); return GC_ERR_ASYMMETRIC; }
  unsigned hw = std::thread::hardware_concurrency();
  int nt = (int)std::min<unsigned>(hw ? hw : 1, 16);
  if ((int64_t)rp[n] < 1000000) nt = 1;
  std::vector<gc_status> res(nt, GC_OK);
  std::vector<std::string> msg(nt);
  auto work = [&](int t) {  // symmetry; rows are known sorted here
    int32_t x0 = (int32_t)((int64_t)n * t / nt), x1 = (int32_t)((int64_t)n * (t + 1) / nt);
    for (int32_t x = x0; x < x1; ++x)
      for (int32_t p = rp[x]; p < rp[x + 1]; ++p) {
        int32_t y = ci[p];
        if (!std::binary_search(ci + rp[y], ci + rp[y + 1], x)) {
          res[t] = GC_ERR_ASYMMETRIC;
          msg[t] = "edge (" + std::to_string(x) + "," + std::to_string(y) + ") has no reverse";
          return;
        }
      }
  };
  // Range, loop, duplicate and order checks finish for every row before the
  // symmetry check, whose binary search needs sorted rows.
  {
    std::vector<gc_status> r1(nt, GC_OK);
    std::vector<std::string> m1(nt);
    auto sorted_only = [&](int t) {
      int32_t x0 = (int32_t)((int64_t)n * t / nt), x1 = (int32_t)((int64_t)n * (t + 1) / nt);
      for (int32_t x = x0; x < x1; ++x)
        for (int32_t p = rp[x]; p < rp[x + 1]; ++p) {
          int32_t y = ci[p];
          if (y < 0 || y >= n) { r1[t] = GC_ERR_RANGE; m1[t] = "column " + std::to_string(y) + " out of range in row " + std::to_string(x); return; }
          if (y == x) { r1[t] = GC_ERR_SELF_LOOP; m1[t] = "self-loop at vertex " + std::to_string(x); return; }
          if (p > rp[x] && ci[p - 1] == y) { r1[t] = GC_ERR_DUPLICATE; m1[t] = "duplicate neighbour " + std::to_string(y) + " in row " + std::to_string(x); return; }
          if (p > rp[x] && ci[p - 1] > y) { r1[t] = GC_ERR_UNSORTED; m1[t] = "row " + std::to_string(x) + " not ascending"; return; }
        }
    };
    std::vector<std::thread> th;
    for (int t = 1; t < nt; ++t) th.emplace_back(sorted_only, t);
    sorted_only(0);
    for (auto& x : th) x.join();
    for (int t = 0; t < nt; ++t)
      if (r1[t] != GC_OK) { set_error(m1[t]); return r1[t]; }
  }
  std::vector<std::thread> th;
  for (int t = 1; t < nt; ++t) th.emplace_back(work, t);
  work(0);
  for (auto& x : th) x.join();
  for (int t = 0; t < nt; ++t)
    if (res[t] != GC_OK) { set_error(msg[t]); return res[t]; }
  return GC_OK;
}

}  // namespace gc

using namespace gc;

struct gc_graph_s {
  int32_t n = 0;
  int32_t m = 0;
  cudaStream_t stream = nullptr;
  int32_t* d_rp = nullptr;
  int32_t* d_ci = nullptr;
  PrepBuffers prep;
  // single-graph descriptors (G = 1)
  int32_t* d_gbase = nullptr;  // [1] 0
  int32_t* d_gn = nullptr;     // [1] n
  int64_t* d_gm = nullptr;     // [1] m
  // counting scratch
  int32_t* d_tri = nullptr;
  uint32_t* d_tables = nullptr;
  int32_t* d_spill = nullptr;
  int32_t spill_len = 0;
  unsigned long long* d_csum = nullptr;  // [13][2]
  unsigned long long* d_x = nullptr;     // [17][2]
  int32_t* d_misc = nullptr;             // [0] cursor, [1] status, [2] max |T|
  uint64_t* d_pe_tmp = nullptr;          // device staging for a host per-edge buffer
  cudaEvent_t ev[kNumPhases + 1] = {};
  bool counted = false;
  uint64_t csum_lo[13] = {0}, csum_hi[13] = {0};
};

extern "C" {

const char* gc_last_error(void) { return t_err.c_str(); }

static void graph_release(gc_graph g) {
  if (!g) return;
  if (g->stream) cudaStreamSynchronize(g->stream);
  cudaFree(g->d_rp);
  cudaFree(g->d_ci);
  free_prep(&g->prep, g->stream);
  cudaStreamSynchronize(g->stream);
  cudaFree(g->d_gbase);
  cudaFree(g->d_tri);
  cudaFree(g->d_tables);
  cudaFree(g->d_spill);
  cudaFree(g->d_csum);
  cudaFree(g->d_misc);
  cudaFree(g->d_pe_tmp);
  for (auto& e : g->ev)
    if (e) cudaEventDestroy(e);
  delete g;
}

gc_status gc_graph_upload(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, uint32_t flags,
                          void* stream, gc_graph* out) {
  if (!out) { set_error("out is NULL"); return GC_ERR_ARG; }
  *out = nullptr;
  if (n < 0 || !row_ptr || (!col_idx && n > 0 && row_ptr[n] > 0)) {
    set_error("bad arguments to gc_graph_upload");
    return GC_ERR_ARG;
  }
  if (flags & ~GC_NO_VALIDATE) { set_error("unknown flags"); return GC_ERR_ARG; }
  if (!(flags & GC_NO_VALIDATE)) {
    gc_status st = validate_csr(n, row_ptr, col_idx);
    if (st != GC_OK) return st;
  }
  const int64_t nnz = row_ptr[n];
  if (nnz < 0 || nnz % 2) { set_error("row_ptr[n] must be even and >= 0"); return GC_ERR_ARG; }
  gc_graph g = new (std::nothrow) gc_graph_s();
  if (!g) { set_error("host allocation failed"); return GC_ERR_NOMEM; }
  g->n = n;
  g->m = (int32_t)(nnz / 2);
  g->stream = (cudaStream_t)stream;
  cudaStream_t s = g->stream;
  cudaError_t e;
  gc_status st = GC_OK;
#define GC_CHECK(call, what)            \
  do {                                  \
    e = (call);                         \
    if (e != cudaSuccess) {             \
      st = cuda_fail(e, what);          \
      graph_release(g);                 \
      return st;                        \
    }                                   \
  } while (0)
  GC_CHECK(cudaMalloc(&g->d_rp, sizeof(int32_t) * ((size_t)n + 1)), "alloc row_ptr");
  GC_CHECK(cudaMalloc(&g->d_ci, sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1)), "alloc col_idx");
  GC_CHECK(cudaMemcpyAsync(g->d_rp, row_ptr, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice, s),
           "copy row_ptr");
  if (nnz > 0)
    GC_CHECK(cudaMemcpyAsync(g->d_ci, col_idx, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice, s),
             "copy col_idx");
  st = prepare_graph(n, g->m, g->d_rp, g->d_ci, nullptr, &g->prep, s);
  if (st != GC_OK) { graph_release(g); return st; }
  // single-graph descriptor block: gbase | gn | gm (gm 8-byte aligned)
  GC_CHECK(cudaMalloc(&g->d_gbase, 32), "alloc descriptors");
  {
    int32_t hb[4] = {0, n, 0, 0};
    int64_t hm = g->m;
    GC_CHECK(cudaMemcpyAsync(g->d_gbase, hb, 16, cudaMemcpyHostToDevice, s), "copy descriptors");
    GC_CHECK(cudaMemcpyAsync(reinterpret_cast<char*>(g->d_gbase) + 16, &hm, 8, cudaMemcpyHostToDevice, s),
             "copy descriptors");
    g->d_gn = g->d_gbase + 1;
    g->d_gm = reinterpret_cast<int64_t*>(reinterpret_cast<char*>(g->d_gbase) + 16);
  }
  GC_CHECK(cudaMalloc(&g->d_csum, sizeof(unsigned long long) * (13 * 2 + 17 * 2)), "alloc sums");
  g->d_x = g->d_csum + 13 * 2;
  GC_CHECK(cudaMalloc(&g->d_misc, sizeof(int32_t) * 4), "alloc misc");
  GC_CHECK(cudaMalloc(&g->d_tri, sizeof(int32_t) * (size_t)(g->m > 0 ? g->m : 1)), "alloc tri");
  if (n > kSmemTableMax) {
    size_t words = (size_t)count_grid_size() * (size_t)n;
    GC_CHECK(cudaMalloc(&g->d_tables, sizeof(uint32_t) * words), "alloc Psi tables");
    GC_CHECK(cudaMemsetAsync(g->d_tables, 0, sizeof(uint32_t) * words, s), "zero Psi tables");
  }
  for (auto& ev : g->ev) GC_CHECK(cudaEventCreate(&ev), "event create");
  GC_CHECK(cudaStreamSynchronize(s), "sync upload");
#undef GC_CHECK
  *out = g;
  return GC_OK;
}

gc_status gc_graph_info(gc_graph g, int64_t* n, int64_t* m) {
  if (!g) { set_error("graph is NULL"); return GC_ERR_ARG; }
  if (n) *n = g->n;
  if (m) *m = g->m;
  return GC_OK;
}

gc_status gc_graph_edges(gc_graph g, int32_t* uv) {
  if (!g || !uv) { set_error("NULL argument"); return GC_ERR_ARG; }
  if (g->m == 0) return GC_OK;
  cudaError_t e = cudaMemcpyAsync(uv, g->prep.uv, sizeof(int32_t) * 2 * (size_t)g->m,
                                  cudaMemcpyDeviceToHost, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  return e == cudaSuccess ? GC_OK : cuda_fail(e, "copy edges");
}

static bool is_device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

gc_status gc_count_edge_graphlets(gc_graph g, uint64_t* per_edge_out, uint64_t* global_out,
                                  uint64_t* global_hi) {
  if (!g || !global_out) { set_error("NULL argument"); return GC_ERR_ARG; }
  cudaStream_t s = g->stream;
  cudaError_t e;
  gc_status st;
#define GC_CHECK(call, what)                  \
  do {                                        \
    e = (call);                               \
    if (e != cudaSuccess) return cuda_fail(e, what); \
  } while (0)
  uint64_t* pe_dev = nullptr;
  const bool want_pe = per_edge_out != nullptr && g->m > 0;
  if (want_pe) {
    if (is_device_pointer(per_edge_out)) {
      pe_dev = per_edge_out;
    } else {
      if (!g->d_pe_tmp)
        GC_CHECK(cudaMalloc(&g->d_pe_tmp, sizeof(uint64_t) * 13 * (size_t)g->m), "alloc per-edge staging");
      pe_dev = g->d_pe_tmp;
    }
  }
  DevGraph dg;
  dg.n = g->n;
  dg.m = g->m;
  dg.rp = g->d_rp;
  dg.ci = g->d_ci;
  dg.deg = g->prep.deg;
  dg.eid = g->prep.eid;
  dg.out_ptr = g->prep.out_ptr;
  dg.out_idx = g->prep.out_idx;
  dg.G = 1;
  dg.vgid = nullptr;
  dg.gbase = g->d_gbase;
  dg.gn = g->d_gn;
  dg.gm = g->d_gm;
  dg.table_n = g->n;
  CountArgs a;
  a.units = g->prep.units;
  a.n_units = g->prep.n_units;
  a.cursor = g->d_misc;
  a.tables = g->d_tables;
  a.tri = g->d_tri;
  a.spill = nullptr;
  a.spill_len = 0;
  a.per_edge = pe_dev;
  a.csum = g->d_csum;
  a.status = g->d_misc + 1;
  GC_CHECK(cudaMemsetAsync(g->d_misc, 0, sizeof(int32_t) * 4, s), "memset misc");
  GC_CHECK(cudaMemsetAsync(g->d_csum, 0, sizeof(unsigned long long) * 13 * 2, s), "memset sums");
  GC_CHECK(cudaEventRecord(g->ev[kPhasePassA], s), "event");
  if (a.n_units > 0) {
    if ((st = run_pass_a(dg, a, s)) != GC_OK) return st;
    // |T| beyond the shared-memory buffer needs a per-warp spill area.
    if ((st = run_max_tri(g->d_tri, g->m, g->d_misc + 2, s)) != GC_OK) return st;
    int32_t tmax = 0;
    GC_CHECK(cudaMemcpyAsync(&tmax, g->d_misc + 2, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "copy max T");
    GC_CHECK(cudaStreamSynchronize(s), "sync max T");
    if (tmax > kTcap) {
      if (tmax > g->spill_len) {
        cudaFree(g->d_spill);
        g->d_spill = nullptr;
        g->spill_len = 0;
        size_t len = (size_t)count_grid_size() * kWarps * (size_t)tmax;
        GC_CHECK(cudaMalloc(&g->d_spill, sizeof(int32_t) * len), "alloc T spill");
        g->spill_len = tmax;
      }
      a.spill = g->d_spill;
      a.spill_len = g->spill_len;
    }
    GC_CHECK(cudaMemsetAsync(g->d_misc, 0, sizeof(int32_t), s), "reset cursor");
  }
  GC_CHECK(cudaEventRecord(g->ev[kPhasePassB], s), "event");
  if (a.n_units > 0)
    if ((st = run_pass_b(dg, a, s)) != GC_OK) return st;
  GC_CHECK(cudaEventRecord(g->ev[kPhaseDerive], s), "event");
  if ((st = run_derive(dg, g->d_csum, g->d_x, a.status, s)) != GC_OK) return st;
  GC_CHECK(cudaEventRecord(g->ev[kPhaseCopy], s), "event");
  unsigned long long hx[17 * 2 + 13 * 2];
  int32_t hstatus = 0;
  GC_CHECK(cudaMemcpyAsync(hx, g->d_x, sizeof(unsigned long long) * 17 * 2, cudaMemcpyDeviceToHost, s), "copy X");
  GC_CHECK(cudaMemcpyAsync(hx + 34, g->d_csum, sizeof(unsigned long long) * 13 * 2, cudaMemcpyDeviceToHost, s),
           "copy C");
  GC_CHECK(cudaMemcpyAsync(&hstatus, a.status, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "copy status");
  if (want_pe && pe_dev != per_edge_out)
    GC_CHECK(cudaMemcpyAsync(per_edge_out, pe_dev, sizeof(uint64_t) * 13 * (size_t)g->m, cudaMemcpyDeviceToHost, s),
             "copy per-edge");
  GC_CHECK(cudaEventRecord(g->ev[kNumPhases], s), "event");
  GC_CHECK(cudaStreamSynchronize(s), "sync count");
#undef GC_CHECK
  if (hstatus & kSpillOverflow) {
    set_error("internal: triangle list exceeded its buffer");
    return GC_ERR_CUDA;
  }
  if (hstatus & kInexact) {
    set_error("internal: a global relation had a non-zero remainder");
    return GC_ERR_CUDA;
  }
  bool need_hi = false;
  for (int i = 0; i < 17; ++i) {
    global_out[i] = hx[2 * i];
    if (global_hi) global_hi[i] = hx[2 * i + 1];
    if (hx[2 * i + 1]) need_hi = true;
  }
  for (int k = 0; k < 13; ++k) {
    g->csum_lo[k] = hx[34 + 2 * k];
    g->csum_hi[k] = hx[34 + 2 * k + 1];
  }
  g->counted = true;
  if (need_hi && !global_hi) {
    set_error("a global count exceeds 64 bits and global_hi is NULL");
    return GC_ERR_OVERFLOW;
  }
  return GC_OK;
}

gc_status gc_graph_csums(gc_graph g, uint64_t* lo, uint64_t* hi) {
  if (!g || !lo) { set_error("NULL argument"); return GC_ERR_ARG; }
  if (!g->counted) { set_error("graph not counted yet"); return GC_ERR_ARG; }
  for (int k = 0; k < 13; ++k) {
    lo[k] = g->csum_lo[k];
    if (hi) hi[k] = g->csum_hi[k];
  }
  return GC_OK;
}

int gc_phase_count(void) { return kNumPhases; }

const char* gc_phase_name(int i) {
  static const char* names[kNumPhases] = {"pass_a_triangles", "pass_b_cliques_cycles", "derive",
                                          "copy_out"};
  return (i >= 0 && i < kNumPhases) ? names[i] : "";
}

gc_status gc_graph_phase_ms(gc_graph g, double* ms) {
  if (!g || !ms) { set_error("NULL argument"); return GC_ERR_ARG; }
  if (!g->counted) { set_error("graph not counted yet"); return GC_ERR_ARG; }
  for (int i = 0; i < kNumPhases; ++i) {
    float f = 0.f;
    cudaError_t e = cudaEventElapsedTime(&f, g->ev[i], g->ev[i + 1]);
    if (e != cudaSuccess) return cuda_fail(e, "event elapsed");
    ms[i] = f;
  }
  return GC_OK;
}

gc_status gc_graph_free(gc_graph g) {
  graph_release(g);
  return GC_OK;
}

}  // extern "C"
