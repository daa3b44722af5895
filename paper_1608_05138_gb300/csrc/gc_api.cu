// gc_api.cu -- C ABI of the plain whole-graph path (see include/gc.h).
//
// Host-side CSR validation (Problem 1's input: simple undirected graph) and
// the P1 relabelling, the graph handle with its device-resident data, and one
// count (the sequence of gc_run.cu: passes T, C, K, finish, derive) with the
// copies back.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <functional>
#include <memory>
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

namespace {

int host_threads() {
  const unsigned hw = std::thread::hardware_concurrency();
  return (int)std::min<unsigned>(hw ? hw : 1, 32);
}

// Row ranges [b[t], b[t+1]) holding about equal numbers of entries.
std::vector<int32_t> nnz_chunks(int32_t n, const int32_t* rp, int nt) {
  std::vector<int32_t> b((size_t)nt + 1, n);
  b[0] = 0;
  const int64_t nnz = rp[n];
  for (int t = 1; t < nt; ++t) {
    const int32_t target = (int32_t)(nnz * t / nt);
    int32_t x = (int32_t)(std::upper_bound(rp, rp + n + 1, target) - rp) - 1;  // last row starting at or before
    if (x < b[t - 1]) x = b[t - 1];
    if (x > n) x = n;
    b[t] = x;
  }
  return b;
}

template <class F>
void run_threads(int nt, F f) {
  std::vector<std::thread> th;
  for (int t = 1; t < nt; ++t) th.emplace_back(f, t);
  f(0);
  for (auto& x : th) x.join();
}

// First error of a multi-threaded check, by thread (thread order = row order).
struct Checks {
  std::vector<gc_status> st;
  std::vector<std::string> msg;
  explicit Checks(int nt) : st((size_t)nt, GC_OK), msg((size_t)nt) {}
  gc_status first() {
    for (size_t t = 0; t < st.size(); ++t)
      if (st[t] != GC_OK) {
        set_error(msg[t]);
        return st[t];
      }
    return GC_OK;
  }
};

}  // namespace

// Reverse slots of a CSR and, with check, the checks of Problem 1's input (a
// simple undirected graph): row_ptr from 0 and non-decreasing, columns in
// range, rows strictly ascending (no duplicates), no self-loops, symmetric.
// rev (optional, [row_ptr[n]]): slot of (y, x) for the slot of (x, y).
//
// Symmetry: rows x are walked in order in chunks of about equal entries; the
// k-th row (in order) that names y must name it from the k-th entry of row y,
// so a per-chunk counter per y (started, on first use, at the number of
// entries of row y below the chunk's first row) gives the slot where x must
// stand in row y, and the entry there is compared with x. Every entry is
// checked against a slot of row y, so a missing reverse always fails, and a
// symmetric graph always passes. Without check, an entry whose reverse is not
// found gets rev = its own slot.
gc_status csr_reverse(int32_t n, const int32_t* rp, const int32_t* ci, int32_t* rev, bool check) {
  if (n < 0) { set_error("n < 0"); return GC_ERR_ARG; }
  if (check) {
    if (rp[0] != 0) { set_error("row_ptr[0] != 0"); return GC_ERR_RANGE; }
    for (int32_t x = 0; x < n; ++x)
      if (rp[x + 1] < rp[x]) {
        set_error("row_ptr decreases at row " + std::to_string(x));
        return GC_ERR_UNSORTED;
      }
    if (rp[n] % 2 != 0) { set_error("row_ptr[n] is odd: the graph cannot be symmetric"); return GC_ERR_ASYMMETRIC; }
  }
  const int64_t nnz = rp[n];
  int nt = host_threads();
  if (nnz < (1 << 20)) nt = 1;
  if (check) {  // range, loop, duplicate and order: every row before any symmetry probe
    const std::vector<int32_t> b = nnz_chunks(n, rp, nt);
    Checks c(nt);
    run_threads(nt, [&](int t) {
      for (int32_t x = b[t]; x < b[t + 1]; ++x)
        for (int32_t p = rp[x]; p < rp[x + 1]; ++p) {
          const int32_t y = ci[p];
          if (y < 0 || y >= n) { c.st[t] = GC_ERR_RANGE; c.msg[t] = "column " + std::to_string(y) + " out of range in row " + std::to_string(x); return; }
          if (y == x) { c.st[t] = GC_ERR_SELF_LOOP; c.msg[t] = "self-loop at vertex " + std::to_string(x); return; }
          if (p > rp[x] && ci[p - 1] == y) { c.st[t] = GC_ERR_DUPLICATE; c.msg[t] = "duplicate neighbour " + std::to_string(y) + " in row " + std::to_string(x); return; }
          if (p > rp[x] && ci[p - 1] > y) { c.st[t] = GC_ERR_UNSORTED; c.msg[t] = "row " + std::to_string(x) + " not ascending"; return; }
        }
    });
    const gc_status st = c.first();
    if (st != GC_OK) return st;
  }
  // per-chunk counters: n ints per thread, at most 1 GiB in all
  const int64_t per = 4 * (int64_t)(n > 0 ? n : 1);
  int nts = (int)std::max<int64_t>(1, std::min<int64_t>(nt, (int64_t(1) << 30) / per));
  const std::vector<int32_t> b = nnz_chunks(n, rp, nts);
  Checks c(nts);
  run_threads(nts, [&](int t) {
    std::vector<int32_t> fill((size_t)(n > 0 ? n : 1), -1);
    const int32_t x0 = b[t];
    for (int32_t x = x0; x < b[t + 1]; ++x)
      for (int32_t p = rp[x]; p < rp[x + 1]; ++p) {
        const int32_t y = ci[p];
        const int32_t yb = rp[y], ye = rp[y + 1];
        int32_t f = fill[y];
        if (f < 0) f = (int32_t)(std::lower_bound(ci + yb, ci + ye, x0) - (ci + yb));
        fill[y] = f + 1;
        const int32_t q = yb + f;
        if (q < ye && ci[q] == x) {
          if (rev) rev[p] = q;
        } else if (check) {
          c.st[t] = GC_ERR_ASYMMETRIC;
          c.msg[t] = "edge (" + std::to_string(x) + "," + std::to_string(y) + ") has no reverse";
          return;
        } else if (rev) {
          const int32_t* r = std::lower_bound(ci + yb, ci + ye, x);
          rev[p] = (r < ci + ye && *r == x) ? (int32_t)(r - ci) : p;
        }
      }
  });
  return c.first();
}

gc_status validate_csr(int32_t n, const int32_t* rp, const int32_t* ci) { return csr_reverse(n, rp, ci, nullptr, true); }

// Preprocessing P1 (Sec. 4.3): relabel vertices by ascending degree (ties by
// id), so that internal ids are the (degree, id) ranks used by P3 and by the
// degree-ordered passes. Rows are re-sorted in the new ids. Edge ids stay
// those of the caller's graph: eid[slot] of every internal slot is the
// caller's edge id, and perm maps internal -> caller vertex ids. rev: the
// reverse slots of the caller's CSR (csr_reverse).
// Host arrays left uninitialised on allocation (every element is written
// before use): a value-initialising std::vector would zero a gigabyte on one
// thread for the larger graphs.
struct HostArray {
  std::unique_ptr<int32_t[]> p;
  int32_t* data() { return p.get(); }
  int32_t& operator[](size_t i) { return p[i]; }
  void resize(size_t n) { p.reset(new int32_t[n > 0 ? n : 1]); }
};

struct Relabeled {
  HostArray rp, ci, eid, perm;
};

Relabeled relabel_by_degree(int32_t n, const int32_t* rp, const int32_t* ci, const int32_t* rev) {
  Relabeled R;
  const int64_t nnz = rp[n];
  const int32_t m = (int32_t)(nnz / 2);
  int nt = host_threads();
  if (nnz < (1 << 20)) nt = 1;
  int32_t dmax = 0;
  for (int32_t x = 0; x < n; ++x) dmax = std::max(dmax, rp[x + 1] - rp[x]);
  // stable counting sort by degree
  std::vector<int32_t> cnt((size_t)dmax + 2, 0);
  for (int32_t x = 0; x < n; ++x) cnt[rp[x + 1] - rp[x] + 1]++;
  for (int32_t d = 0; d <= dmax; ++d) cnt[d + 1] += cnt[d];
  R.perm.resize((size_t)n);
  std::vector<int32_t> newid((size_t)n);
  for (int32_t x = 0; x < n; ++x) {
    const int32_t i = cnt[rp[x + 1] - rp[x]]++;
    R.perm[i] = x;
    newid[x] = i;
  }
  // caller's edge ids: row x's entries y > x are edges up[x], up[x] + 1, ...
  std::vector<int32_t> first_up((size_t)n + 1), up((size_t)n + 1, 0);
  const std::vector<int32_t> b = nnz_chunks(n, rp, nt);
  run_threads(nt, [&](int t) {
    for (int32_t x = b[t]; x < b[t + 1]; ++x) {
      first_up[x] = (int32_t)(std::upper_bound(ci + rp[x], ci + rp[x + 1], x) - ci);
      up[x + 1] = rp[x + 1] - first_up[x];
    }
  });
  for (int32_t x = 0; x < n; ++x) up[x + 1] += up[x];
  HostArray eid_in;
  eid_in.resize((size_t)nnz);
  run_threads(nt, [&](int t) {
    for (int32_t x = b[t]; x < b[t + 1]; ++x)
      for (int32_t p = rp[x]; p < rp[x + 1]; ++p) {
        const int32_t y = ci[p];
        int32_t id;
        if (y > x) {
          id = up[x] + (p - first_up[x]);
        } else {
          const int32_t q = rev[p];  // (y, x) in row y, x > y
          id = up[y] + (q - first_up[y]);
        }
        eid_in[p] = (id >= 0 && id < m) ? id : 0;  // out of range only for an input that skipped validation
      }
  });
  R.rp.resize((size_t)n + 1);
  R.rp[0] = 0;
  for (int32_t i = 0; i < n; ++i) R.rp[i + 1] = R.rp[i] + (rp[R.perm[i] + 1] - rp[R.perm[i]]);
  R.ci.resize((size_t)nnz);
  R.eid.resize((size_t)nnz);
  const std::vector<int32_t> bn = nnz_chunks(n, R.rp.data(), nt);
  run_threads(nt, [&](int t) {
    std::vector<uint64_t> tmp;
    for (int32_t i = bn[t]; i < bn[t + 1]; ++i) {
      const int32_t x = R.perm[i];
      tmp.clear();
      for (int32_t p = rp[x]; p < rp[x + 1]; ++p)
        tmp.push_back(((uint64_t)(uint32_t)newid[ci[p]] << 32) | (uint32_t)eid_in[p]);
      std::sort(tmp.begin(), tmp.end());
      int32_t o = R.rp[i];
      for (uint64_t k : tmp) {
        R.ci[o] = (int32_t)(k >> 32);
        R.eid[o] = (int32_t)(k & 0xffffffffu);
        ++o;
      }
    }
  });
  return R;
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
  Scratch sc;
  unsigned long long* d_csum = nullptr;  // [13][2]
  unsigned long long* d_x = nullptr;     // [17][2]
  uint64_t* d_pe_tmp = nullptr;          // device staging for a host per-edge buffer
  cudaEvent_t ev[kNumPhases + 1] = {};
  bool counted = false;
  uint64_t csum_lo[13] = {0}, csum_hi[13] = {0};
  uint64_t work[kNumWork] = {0};
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
  scratch_free(&g->sc, g->stream);
  cudaStreamSynchronize(g->stream);
  cudaFree(g->d_csum);
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
  const int64_t nnz = row_ptr[n];
  HostArray rev;
  try {
    rev.resize((size_t)(nnz > 0 ? nnz : 1));
  } catch (...) {
    set_error("host allocation failed");
    return GC_ERR_NOMEM;
  }
  {
    const gc_status st0 = csr_reverse(n, row_ptr, col_idx, rev.data(), !(flags & GC_NO_VALIDATE));
    if (st0 != GC_OK) return st0;
  }
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
  Relabeled R;
  try {
    R = relabel_by_degree(n, row_ptr, col_idx, rev.data());
  } catch (...) {
    set_error("host allocation failed");
    graph_release(g);
    return GC_ERR_NOMEM;
  }
  rev.p.reset();
  int32_t* d_eid = nullptr;
  int32_t* d_perm = nullptr;
  GC_CHECK(cudaMalloc(&g->d_rp, sizeof(int32_t) * ((size_t)n + 1)), "alloc row_ptr");
  GC_CHECK(cudaMalloc(&g->d_ci, sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1)), "alloc col_idx");
  GC_CHECK(cudaMallocAsync(&d_eid, sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1), s), "alloc eid");
  GC_CHECK(cudaMallocAsync(&d_perm, sizeof(int32_t) * (size_t)(n > 0 ? n : 1), s), "alloc perm");
  GC_CHECK(cudaMemcpyAsync(g->d_rp, R.rp.data(), sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice, s),
           "copy row_ptr");
  if (nnz > 0) {
    GC_CHECK(cudaMemcpyAsync(g->d_ci, R.ci.data(), sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice, s),
             "copy col_idx");
    GC_CHECK(cudaMemcpyAsync(d_eid, R.eid.data(), sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice, s),
             "copy edge ids");
  }
  if (n > 0)
    GC_CHECK(cudaMemcpyAsync(d_perm, R.perm.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s),
             "copy perm");
  st = prepare_graph(n, g->m, g->d_rp, g->d_ci, nullptr, d_eid, d_perm, &g->prep, s);
  cudaFreeAsync(d_perm, s);
  if (st != GC_OK) { graph_release(g); return st; }
  cudaStreamSynchronize(s);  // host copies of R are released on return
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
  {
    gc_status st2 = scratch_init(&g->sc, g->m, n, g->prep.kmax, g->prep.cnx_max, s);
    if (st2 != GC_OK) { graph_release(g); return st2; }
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
  dg.ocsr = g->prep.ocsr;
  dg.rev = g->prep.rev;
  dg.G = 1;
  dg.vgid = nullptr;
  dg.gbase = g->d_gbase;
  dg.gn = g->d_gn;
  dg.gm = g->d_gm;
  dg.table_n = g->n;
  dg.ranked = true;
  KUnits ku;
  ku.units = g->prep.kunits;
  ku.cunits = g->prep.cunits;
  ku.n_cheavy = g->prep.n_cheavy;
  for (int t = 0; t <= kNumTiers; ++t) ku.tier_off[t] = g->prep.ktier_off[t];
  if ((st = run_count(dg, g->prep.units, g->prep.n_units, ku, pe_dev, g->d_csum, g->d_x, &g->sc, s, g->ev)) != GC_OK)
    return st;
  unsigned long long hx[17 * 2 + 13 * 2];
  int32_t hstatus = 0;
  GC_CHECK(cudaMemcpyAsync(hx, g->d_x, sizeof(unsigned long long) * 17 * 2, cudaMemcpyDeviceToHost, s), "copy X");
  GC_CHECK(cudaMemcpyAsync(hx + 34, g->d_csum, sizeof(unsigned long long) * 13 * 2, cudaMemcpyDeviceToHost, s),
           "copy C");
  GC_CHECK(cudaMemcpyAsync(&hstatus, g->sc.misc + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "copy status");
  GC_CHECK(cudaMemcpyAsync(g->work, g->sc.work, sizeof(g->work), cudaMemcpyDeviceToHost, s), "copy work");
  if (want_pe && pe_dev != per_edge_out)
    GC_CHECK(cudaMemcpyAsync(per_edge_out, pe_dev, sizeof(uint64_t) * 13 * (size_t)g->m, cudaMemcpyDeviceToHost, s),
             "copy per-edge");
  GC_CHECK(cudaEventRecord(g->ev[kNumPhases], s), "event");
  GC_CHECK(cudaStreamSynchronize(s), "sync count");
#undef GC_CHECK
  if (hstatus & kSpillOverflow) {
    set_error("internal: a pass-K unit exceeded its tier");
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

gc_status gc_graph_work_counts(gc_graph g, uint64_t* out) {
  if (!g || !out) { set_error("NULL argument"); return GC_ERR_ARG; }
  if (!g->counted) { set_error("graph not counted yet"); return GC_ERR_ARG; }
  static_assert(kNumWork == GC_NUM_WORK, "work counter count");
  for (int i = 0; i < kNumWork; ++i) out[i] = g->work[i];
  out[kWorkLaunches] = (uint64_t)g->sc.launches;
  return GC_OK;
}

int gc_phase_count(void) { return kNumPhases; }

const char* gc_phase_name(int i) {
  static const char* names[kNumPhases] = {"pass_t_triangles", "pass_c_cycles", "pass_k_cliques",
                                          "finish_columns", "derive", "copy_out"};
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
