// gc_api.cu -- C ABI of the plain whole-graph path (see include/gc.h).
//
// Host-side CSR validation (Problem 1's input: simple undirected graph) and
// the P1 relabelling, the graph handle with its device-resident data, and one
// count (the sequence of gc_run.cu: passes T, C, K, finish, derive) with the
// copies back.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <memory>
#include <mutex>
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
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[kMaxDevices] = {};
}  // namespace

cudaMemPool_t lib_pool() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (g_pools[dev]) return g_pools[dev];
  cudaMemPoolProps props;
  std::memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) cudaGetLastError();
  unsigned long long keep = (unsigned long long)total_b / 4;
  if (const char* e = getenv("GC_POOL_KEEP_BYTES")) keep = strtoull(e, nullptr, 10);
  if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) cudaGetLastError();
  g_pools[dev] = pool;
  return pool;
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

// For a graph that passed the linear checks (columns in range, rows
// ascending) and failed a symmetry check: the message naming the first entry
// (x, y) in row order whose reverse (y, x) is absent, found by a binary
// search in row y per entry (rows in chunks over the host threads). A walk's
// first mismatch need not be that entry -- an extra entry x0 in row y makes
// the next (x1, y) mismatch although (y, x1) exists -- so the failure path
// looks it up directly.
std::string first_without_reverse(int32_t n, const int32_t* rp, const int32_t* ci) {
  const int nt = rp[n] < (1 << 20) ? 1 : host_threads();
  const std::vector<int32_t> b = nnz_chunks(n, rp, nt);
  std::vector<std::pair<int32_t, int32_t>> hit((size_t)nt, {-1, -1});
  run_threads(nt, [&](int t) {
    for (int32_t x = b[t]; x < b[t + 1]; ++x)
      for (int32_t p = rp[x]; p < rp[x + 1]; ++p) {
        const int32_t y = ci[p];
        if (!std::binary_search(ci + rp[y], ci + rp[y + 1], x)) {
          hit[(size_t)t] = {x, y};
          return;
        }
      }
  });
  for (const auto& h : hit)
    if (h.first >= 0) return "edge (" + std::to_string(h.first) + "," + std::to_string(h.second) + ") has no reverse";
  return "asymmetric graph";  // not reached after a failed symmetry check
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

// Checks of Problem 1's input (a simple undirected graph), in two parts.
// Linear checks: row_ptr from 0 and non-decreasing, columns in range, rows
// strictly ascending (no duplicates), no self-loops -- one pass over the
// entries in threads over row ranges of equal entries.
// Whether a row passes every linear check (columns in [0, n), no self-loop,
// strictly ascending): no early exit and no branch in the loop, so that the
// compiler vectorises it; a failing row is examined again entry by entry.
static inline bool row_ok(const int32_t* r, int32_t len, int32_t x, int32_t n) {
  if (len <= 0) return true;
  uint32_t bad = ((uint32_t)r[0] >= (uint32_t)n) | (r[0] == x);
  for (int32_t k = 1; k < len; ++k)
    bad |= ((uint32_t)r[k] >= (uint32_t)n) | (r[k] == x) | (r[k] <= r[k - 1]);
  return bad == 0;
}

gc_status csr_linear_checks(int32_t n, const int32_t* rp, const int32_t* ci) {
  if (n < 0) { set_error("n < 0"); return GC_ERR_ARG; }
  if (rp[0] != 0) { set_error("row_ptr[0] != 0"); return GC_ERR_RANGE; }
  {  // row_ptr ascending: vertex chunks in parallel, the first decrease in row order
    const int ntv = n < (1 << 20) ? 1 : host_threads();
    std::vector<int32_t> first((size_t)ntv, -1);
    run_threads(ntv, [&](int t) {
      const int32_t x1 = (int32_t)((int64_t)n * (t + 1) / ntv);
      for (int32_t x = (int32_t)((int64_t)n * t / ntv); x < x1; ++x)
        if (rp[x + 1] < rp[x]) {
          first[(size_t)t] = x;
          return;
        }
    });
    for (int32_t x : first)
      if (x >= 0) {
        set_error("row_ptr decreases at row " + std::to_string(x));
        return GC_ERR_UNSORTED;
      }
  }
  if (rp[n] % 2 != 0) { set_error("row_ptr[n] is odd: the graph cannot be symmetric"); return GC_ERR_ASYMMETRIC; }
  const int64_t nnz = rp[n];
  const int nt = nnz < (1 << 20) ? 1 : host_threads();
  const std::vector<int32_t> b = nnz_chunks(n, rp, nt);
  Checks c(nt);
  run_threads(nt, [&](int t) {
    for (int32_t x = b[t]; x < b[t + 1]; ++x) {
      if (row_ok(ci + rp[x], rp[x + 1] - rp[x], x, n)) continue;
      for (int32_t p = rp[x]; p < rp[x + 1]; ++p) {  // the first failing entry of the first failing row
        const int32_t y = ci[p];
        if (y < 0 || y >= n) { c.st[t] = GC_ERR_RANGE; c.msg[t] = "column " + std::to_string(y) + " out of range in row " + std::to_string(x); return; }
        if (y == x) { c.st[t] = GC_ERR_SELF_LOOP; c.msg[t] = "self-loop at vertex " + std::to_string(x); return; }
        if (p > rp[x] && ci[p - 1] == y) { c.st[t] = GC_ERR_DUPLICATE; c.msg[t] = "duplicate neighbour " + std::to_string(y) + " in row " + std::to_string(x); return; }
        if (p > rp[x] && ci[p - 1] > y) { c.st[t] = GC_ERR_UNSORTED; c.msg[t] = "row " + std::to_string(x) + " not ascending"; return; }
      }
    }
  });
  return c.first();
}

// Symmetry (needs the linear checks passed): rows x are walked in order in
// chunks of about equal entries; the k-th row (in order) that names y must
// name it from the k-th entry of row y, so a per-chunk counter per y (started,
// on first use, at the number of entries of row y below the chunk's first
// row) gives the slot where x must stand in row y, and the entry there is
// compared with x. Every entry is checked against a slot of row y, so a
// missing reverse always fails, and a symmetric graph always passes. The
// message of a failure, naming the first entry in row order without a
// reverse, is returned in *msg (the calling thread sets it).
gc_status csr_symmetry(int32_t n, const int32_t* rp, const int32_t* ci, std::string* msg) {
  const int64_t nnz = rp[n];
  int nt = nnz < (1 << 20) ? 1 : host_threads();
  // per-chunk counters: n ints per thread, at most 1 GiB in all
  const int64_t per = 4 * (int64_t)(n > 0 ? n : 1);
  nt = (int)std::max<int64_t>(1, std::min<int64_t>(nt, (int64_t(1) << 30) / per));
  const std::vector<int32_t> b = nnz_chunks(n, rp, nt);
  std::vector<gc_status> st((size_t)nt, GC_OK);
  run_threads(nt, [&](int t) {
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
        if (q >= ye || ci[q] != x) {
          st[t] = GC_ERR_ASYMMETRIC;
          return;
        }
      }
  });
  for (int t = 0; t < nt; ++t)
    if (st[t] != GC_OK) {
      *msg = first_without_reverse(n, rp, ci);
      return st[t];
    }
  return GC_OK;
}

// The same checks, in the same order and with the same codes, for one small
// graph on the calling thread, with the caller's scratch for the symmetry
// walk (no allocation once the scratch has grown): what a bulk submission of
// many small graphs runs on each of its threads.
gc_status validate_csr_small(int32_t n, const int32_t* rp, const int32_t* ci, std::vector<int32_t>* fill) {
  if (n < 0) { set_error("n < 0"); return GC_ERR_ARG; }
  if (rp[0] != 0) { set_error("row_ptr[0] != 0"); return GC_ERR_RANGE; }
  for (int32_t x = 0; x < n; ++x)
    if (rp[x + 1] < rp[x]) {
      set_error("row_ptr decreases at row " + std::to_string(x));
      return GC_ERR_UNSORTED;
    }
  if (rp[n] % 2 != 0) { set_error("row_ptr[n] is odd: the graph cannot be symmetric"); return GC_ERR_ASYMMETRIC; }
  for (int32_t x = 0; x < n; ++x) {
    if (row_ok(ci + rp[x], rp[x + 1] - rp[x], x, n)) continue;
    for (int32_t p = rp[x]; p < rp[x + 1]; ++p) {
      const int32_t y = ci[p];
      if (y < 0 || y >= n) { set_error("column " + std::to_string(y) + " out of range in row " + std::to_string(x)); return GC_ERR_RANGE; }
      if (y == x) { set_error("self-loop at vertex " + std::to_string(x)); return GC_ERR_SELF_LOOP; }
      if (p > rp[x] && ci[p - 1] == y) { set_error("duplicate neighbour " + std::to_string(y) + " in row " + std::to_string(x)); return GC_ERR_DUPLICATE; }
      if (p > rp[x] && ci[p - 1] > y) { set_error("row " + std::to_string(x) + " not ascending"); return GC_ERR_UNSORTED; }
    }
  }
  // symmetry. The rows are sorted, so the entries of row y below y (its lower
  // part) must be, in order, the rows x < y that name y: each upper entry
  // (x, y), y > x, taken in row order, is matched with the next unmatched
  // entry of row y, which must be x; at the end every lower part must be
  // matched to its end. One random access per edge instead of one per entry;
  // a failure names the first entry in row order without a reverse, as for a
  // large graph.
  if ((int64_t)fill->size() < 2 * (int64_t)n) fill->resize(2 * (size_t)n);
  int32_t* f = fill->data();      // next unmatched entry of row y
  int32_t* lend = f + n;          // end of row x's lower part
  for (int32_t y = 0; y < n; ++y) f[y] = rp[y];
  bool sym = true;
  for (int32_t x = 0; x < n && sym; ++x) {
    int32_t p = rp[x];
    const int32_t e = rp[x + 1];
    while (p < e && ci[p] < x) ++p;
    lend[x] = p;
    for (; p < e; ++p) {
      const int32_t y = ci[p];
      const int32_t q = f[y]++;
      if (q >= rp[y + 1] || ci[q] != x) {
        sym = false;
        break;
      }
    }
  }
  for (int32_t y = 0; y < n && sym; ++y) sym = f[y] == lend[y];
  if (sym) return GC_OK;
  set_error(first_without_reverse(n, rp, ci));
  return GC_ERR_ASYMMETRIC;
}

gc_status validate_csr(int32_t n, const int32_t* rp, const int32_t* ci) {
  gc_status st = csr_linear_checks(n, rp, ci);
  if (st != GC_OK) return st;
  std::string msg;
  st = csr_symmetry(n, rp, ci, &msg);
  if (st != GC_OK) set_error(msg);
  return st;
}

// Host arrays left uninitialised on allocation (every element is written
// before use).
template <class T>
struct HostBuf {
  std::unique_ptr<T[]> p;
  T* data() { return p.get(); }
  T& operator[](size_t i) { return p[i]; }
  void resize(size_t n) { p.reset(new T[n > 0 ? n : 1]); }
};

// The host half of preprocessing P1 (Sec. 4.3): vertices ranked by ascending
// (degree, id) -- a stable counting sort of the degrees -- and what the
// device relabel needs: internal row pointers, and the internal rows of more
// than 32 entries listed by the sort that takes them.
struct RelabelPlan {
  HostBuf<int32_t> perm, newid, rp;
  std::vector<int32_t> mid, longr;  // rows of 33..4096 entries, and longer ones
  std::vector<int64_t> long_off;    // offset of each long row's padded copy
  int64_t tmp_len = 0;
};

RelabelPlan plan_relabel(int32_t n, const int32_t* rp) {
  RelabelPlan R;
  R.perm.resize((size_t)n);
  R.newid.resize((size_t)n);
  R.rp.resize((size_t)n + 1);
  R.rp[0] = 0;
  if (n == 0) return R;
  // vertex chunks, one per thread (fewer threads when the per-thread degree
  // histograms would pass 2^24 counters)
  int nt = n >= (1 << 16) ? host_threads() : 1;
  std::vector<int32_t> dmx((size_t)nt, 0);
  auto chunk = [&](int t, int T) { return (int32_t)((int64_t)n * t / T); };
  run_threads(nt, [&](int t) {
    int32_t d = 0;
    for (int32_t x = chunk(t, nt); x < chunk(t + 1, nt); ++x) d = std::max(d, rp[x + 1] - rp[x]);
    dmx[(size_t)t] = d;
  });
  const int32_t dmax = *std::max_element(dmx.begin(), dmx.end());
  const size_t D = (size_t)dmax + 1;
  const int nt0 = nt;
  while (nt > 1 && (size_t)nt * D > ((size_t)1 << 24)) nt >>= 1;
  if (nt != nt0) dmx.assign((size_t)nt, 0);
  // cnt[t][d]: vertices of degree d in chunk t, then the first rank each
  // chunk gives its degree-d vertices: ranks ascend by degree, then by chunk,
  // then by id within the chunk -- the (degree, id) order
  std::vector<int32_t> cnt((size_t)nt * D, 0);
  run_threads(nt, [&](int t) {
    int32_t* c = cnt.data() + (size_t)t * D;
    for (int32_t x = chunk(t, nt); x < chunk(t + 1, nt); ++x) c[rp[x + 1] - rp[x]]++;
  });
  std::vector<int32_t> base(D + 1);  // first rank of degree d
  std::vector<int64_t> S(D + 1);     // first internal slot of degree d
  {
    int32_t r = 0;
    int64_t sl = 0;
    for (size_t d = 0; d < D; ++d) {
      base[d] = r;
      S[d] = sl;
      int32_t tot = 0;
      for (int t = 0; t < nt; ++t) {
        int32_t& c = cnt[(size_t)t * D + d];
        const int32_t k = c;
        c = r + tot;  // chunk t's first rank of degree d
        tot += k;
      }
      r += tot;
      sl += (int64_t)tot * (int64_t)d;
    }
    base[D] = r;
    S[D] = sl;
  }
  run_threads(nt, [&](int t) {
    int32_t* c = cnt.data() + (size_t)t * D;
    for (int32_t x = chunk(t, nt); x < chunk(t + 1, nt); ++x) {
      const int32_t i = c[rp[x + 1] - rp[x]]++;
      R.perm[(size_t)i] = x;
      R.newid[(size_t)x] = i;
    }
  });
  // internal row pointers: every row of a degree bucket has that degree
  run_threads(nt, [&](int t) {
    for (int32_t i = chunk(t, nt); i < chunk(t + 1, nt); ++i) {
      const int32_t x = R.perm[(size_t)i];
      const int32_t d = rp[x + 1] - rp[x];
      R.rp[(size_t)i + 1] = (int32_t)(S[(size_t)d] + (int64_t)(i + 1 - base[(size_t)d]) * d);
    }
  });
  // rows of 33..4096 entries and longer ones: the last ranks, in two runs
  const int32_t m0 = base[std::min<size_t>(33, D)], l0 = base[std::min<size_t>(4097, D)];
  R.mid.resize((size_t)(l0 - m0));
  for (int32_t i = m0; i < l0; ++i) R.mid[(size_t)(i - m0)] = i;
  for (int32_t i = l0; i < n; ++i) {
    const int32_t d = R.rp[(size_t)i + 1] - R.rp[(size_t)i];
    int64_t P = 4096;
    while (P < d) P <<= 1;
    R.longr.push_back(i);
    R.long_off.push_back(R.tmp_len);
    R.tmp_len += P;
  }
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
  uint64_t* d_ind_tmp = nullptr;         // device staging for a host per-edge induced buffer
  cudaEvent_t ev[kNumPhases + 1] = {};
  bool counted = false;
  uint64_t csum_lo[13] = {0}, csum_hi[13] = {0};
  uint64_t work[kNumWork] = {0};
};

extern "C" {

const char* gc_last_error(void) { return t_err.c_str(); }

gc_status gc_validate_csr(int32_t n, const int32_t* row_ptr, const int32_t* col_idx) {
  if (n < 0 || !row_ptr || (!col_idx && n > 0 && row_ptr[n] > 0)) {
    set_error("bad arguments to gc_validate_csr");
    return GC_ERR_ARG;
  }
  if (row_ptr[n] >= 0 && row_ptr[n] < (1 << 20)) {
    // the single-threaded checks each graph of a bulk submission gets
    std::vector<int32_t> fill;
    return validate_csr_small(n, row_ptr, col_idx, &fill);
  }
  return validate_csr(n, row_ptr, col_idx);
}

static void graph_release(gc_graph g) {
  if (!g) return;
  // stream-ordered frees into the library pool (after the graph's queued
  // work), then one synchronisation
  const cudaStream_t s = g->stream;
  for (void* p : {(void*)g->d_rp, (void*)g->d_ci, (void*)g->d_gbase, (void*)g->d_csum, (void*)g->d_pe_tmp,
                  (void*)g->d_ind_tmp})
    if (p) cudaFreeAsync(p, s);
  free_prep(&g->prep, s);
  scratch_free(&g->sc, s);
  cudaStreamSynchronize(s);
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
  const bool validate = !(flags & GC_NO_VALIDATE);
  if (validate) {
    const gc_status st0 = csr_linear_checks(n, row_ptr, col_idx);
    if (st0 != GC_OK) return st0;
  }
  const int64_t nnz = row_ptr[n];
  if (nnz < 0 || nnz % 2) { set_error("row_ptr[n] must be even and >= 0"); return GC_ERR_ARG; }
  // Symmetry is checked on the device, where the preparation finds the
  // reverse of every slot: the device steps are safe on an asymmetric input
  // (columns in range, rows sorted), and nothing is counted before the check
  // has passed. If a device step fails, the host checks symmetry instead, so
  // that an invalid input is reported as such (also where there is no GPU).
  gc_graph g = new (std::nothrow) gc_graph_s();
  if (!g) { set_error("host allocation failed"); return GC_ERR_NOMEM; }
  g->n = n;
  g->m = (int32_t)(nnz / 2);
  g->stream = (cudaStream_t)stream;
  cudaStream_t s = g->stream;
  cudaError_t e;
  gc_status st = GC_OK;
  RelabelPlan R;
  int32_t *d_eid = nullptr, *d_perm = nullptr, *d_newid = nullptr, *d_rp0 = nullptr, *d_ci0 = nullptr;
  int32_t* d_lists = nullptr;
  long long* d_tmp = nullptr;
  int64_t* d_loff = nullptr;
  auto drop_temps = [&] {
    for (void* p : {(void*)d_newid, (void*)d_rp0, (void*)d_ci0, (void*)d_lists, (void*)d_tmp, (void*)d_loff})
      if (p) cudaFreeAsync(p, s);
    d_newid = d_rp0 = d_ci0 = d_lists = nullptr;
    d_tmp = nullptr;
    d_loff = nullptr;
  };
  // On a failure the symmetry check is awaited first: an invalid input is
  // reported as such even when a device step failed too (a machine without a
  // GPU still gets the validation codes).
  auto fail = [&](gc_status code) -> gc_status {
    const std::string err = gc_last_error();
    drop_temps();
    if (d_eid) cudaFreeAsync(d_eid, s);
    if (d_perm) cudaFreeAsync(d_perm, s);
    graph_release(g);
    if (validate) {
      std::string msg;
      const gc_status sym_st = csr_symmetry(n, row_ptr, col_idx, &msg);
      if (sym_st != GC_OK) {
        set_error(msg);
        return sym_st;
      }
    }
    set_error(err);
    return code;
  };
#define GC_CHECK(call, what)            \
  do {                                  \
    e = (call);                         \
    if (e != cudaSuccess) return fail(cuda_fail(e, what)); \
  } while (0)
  try {
    R = plan_relabel(n, row_ptr);
  } catch (...) {
    set_error("host allocation failed");
    return fail(GC_ERR_NOMEM);
  }
  const size_t nnz1 = (size_t)(nnz > 0 ? nnz : 1), n1 = (size_t)(n > 0 ? n : 1);
  const size_t n_lists = R.mid.size() + R.longr.size();
  GC_CHECK(pool_alloc(&g->d_rp, sizeof(int32_t) * ((size_t)n + 1), s), "alloc row_ptr");
  GC_CHECK(pool_alloc(&g->d_ci, sizeof(int32_t) * nnz1, s), "alloc col_idx");
  GC_CHECK(pool_alloc(&d_eid, sizeof(int32_t) * nnz1, s), "alloc eid");
  GC_CHECK(pool_alloc(&d_perm, sizeof(int32_t) * n1, s), "alloc perm");
  GC_CHECK(pool_alloc(&d_newid, sizeof(int32_t) * n1, s), "alloc newid");
  GC_CHECK(pool_alloc(&d_rp0, sizeof(int32_t) * ((size_t)n + 1), s), "alloc caller row_ptr");
  GC_CHECK(pool_alloc(&d_ci0, sizeof(int32_t) * nnz1, s), "alloc caller col_idx");
  GC_CHECK(pool_alloc(&d_lists, sizeof(int32_t) * (n_lists > 0 ? n_lists : 1), s), "alloc row lists");
  GC_CHECK(pool_alloc(&d_loff, sizeof(int64_t) * (R.long_off.size() > 0 ? R.long_off.size() : 1), s),
           "alloc row lists");
  GC_CHECK(pool_alloc(&d_tmp, sizeof(long long) * (size_t)(R.tmp_len > 0 ? R.tmp_len : 1), s), "alloc sort buffer");
  GC_CHECK(cudaMemcpyAsync(d_rp0, row_ptr, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice, s),
           "copy row_ptr");
  if (nnz > 0)
    GC_CHECK(cudaMemcpyAsync(d_ci0, col_idx, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice, s), "copy col_idx");
  GC_CHECK(cudaMemcpyAsync(g->d_rp, R.rp.data(), sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice, s),
           "copy internal row_ptr");
  if (n > 0) {
    GC_CHECK(cudaMemcpyAsync(d_perm, R.perm.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s), "copy perm");
    GC_CHECK(cudaMemcpyAsync(d_newid, R.newid.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s),
             "copy ranks");
  }
  if (!R.mid.empty())
    GC_CHECK(cudaMemcpyAsync(d_lists, R.mid.data(), sizeof(int32_t) * R.mid.size(), cudaMemcpyHostToDevice, s),
             "copy row lists");
  if (!R.longr.empty()) {
    GC_CHECK(cudaMemcpyAsync(d_lists + R.mid.size(), R.longr.data(), sizeof(int32_t) * R.longr.size(),
                             cudaMemcpyHostToDevice, s), "copy row lists");
    GC_CHECK(cudaMemcpyAsync(d_loff, R.long_off.data(), sizeof(int64_t) * R.long_off.size(), cudaMemcpyHostToDevice, s),
             "copy row lists");
  }
  st = relabel_on_device(n, g->m, d_rp0, d_ci0, d_perm, d_newid, g->d_rp, g->d_ci, d_eid, d_lists,
                         (int32_t)R.mid.size(), d_lists + R.mid.size(), d_loff, (int32_t)R.longr.size(), d_tmp, s);
  drop_temps();
  if (st != GC_OK) return fail(st);
  st = prepare_graph(n, g->m, g->d_rp, g->d_ci, nullptr, d_eid, d_perm, &g->prep, s);
  d_eid = nullptr;  // owned by the preparation buffers from here on
  if (st != GC_OK) return fail(st);
  cudaFreeAsync(d_perm, s);
  d_perm = nullptr;
  if (validate) {
    int32_t bad = -1;
    if ((st = first_unreversed_slot(nnz, g->prep.rev, &bad, s)) != GC_OK) return fail(st);
    if (bad >= 0) {  // name the edge in the caller's labels
      int32_t y = 0;
      GC_CHECK(cudaMemcpy(&y, g->d_ci + bad, sizeof(int32_t), cudaMemcpyDeviceToHost), "copy slot");
      const int32_t x = (int32_t)(std::upper_bound(R.rp.data(), R.rp.data() + n + 1, bad) - R.rp.data()) - 1;
      set_error("edge (" + std::to_string(R.perm[x]) + "," + std::to_string(R.perm[y]) + ") has no reverse");
      graph_release(g);
      return GC_ERR_ASYMMETRIC;
    }
  }
  cudaStreamSynchronize(s);  // the host arrays of the plan are released on return
  // single-graph descriptor block: gbase | gn | gm (gm 8-byte aligned)
  GC_CHECK(pool_alloc(&g->d_gbase, 32, s), "alloc descriptors");
  {
    int32_t hb[4] = {0, n, 0, 0};
    int64_t hm = g->m;
    GC_CHECK(cudaMemcpyAsync(g->d_gbase, hb, 16, cudaMemcpyHostToDevice, s), "copy descriptors");
    GC_CHECK(cudaMemcpyAsync(reinterpret_cast<char*>(g->d_gbase) + 16, &hm, 8, cudaMemcpyHostToDevice, s),
             "copy descriptors");
    g->d_gn = g->d_gbase + 1;
    g->d_gm = reinterpret_cast<int64_t*>(reinterpret_cast<char*>(g->d_gbase) + 16);
  }
  GC_CHECK(pool_alloc(&g->d_csum, sizeof(unsigned long long) * (13 * 2 + 17 * 2), s), "alloc sums");
  g->d_x = g->d_csum + 13 * 2;
  {
    gc_status st2 = scratch_init(&g->sc, g->m, n, g->prep.kmax, g->prep.cnx_max, s);
    if (st2 != GC_OK) return fail(st2);
    scratch_guess_tlist(&g->sc, g->m);
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

// The address by which the device writes the per-edge rows at p: p itself
// for device or managed memory, the mapped address for pinned host memory
// (the finish kernel then writes the rows over the host link, with no staging
// buffer and no copy; *host = true), nullptr for pageable host memory.
static uint64_t* device_view(uint64_t* p, bool* host) {
  *host = false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return p;
  if (a.type == cudaMemoryTypeHost && a.devicePointer) {
    *host = true;
    return static_cast<uint64_t*>(a.devicePointer);
  }
  return nullptr;
}

// The count behind gc_count_edge_graphlets and gc_count_edge_induced.
static gc_status count_graph(gc_graph g, uint64_t* per_edge_out, uint64_t* induced_out, uint64_t* global_out,
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
  bool staged = false, pe_host = false;
  if (want_pe) {
    if ((pe_dev = device_view(per_edge_out, &pe_host)) == nullptr) {
      staged = true;
      if (!g->d_pe_tmp)
        GC_CHECK(pool_alloc(&g->d_pe_tmp, sizeof(uint64_t) * 13 * (size_t)g->m, g->stream), "alloc per-edge staging");
      pe_dev = g->d_pe_tmp;
    }
  }
  uint64_t* ind_dev = nullptr;
  const bool want_ind = induced_out != nullptr && g->m > 0;
  bool ind_staged = false, ind_host = false;
  if (want_ind) {
    if ((ind_dev = device_view(induced_out, &ind_host)) == nullptr) {
      ind_staged = true;
      if (!g->d_ind_tmp)
        GC_CHECK(pool_alloc(&g->d_ind_tmp, sizeof(uint64_t) * GC_INDUCED_COLS * (size_t)g->m, g->stream),
                 "alloc induced staging");
      ind_dev = g->d_ind_tmp;
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
  dg.e2o = g->prep.e2o;
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
  ku.cjobs = g->prep.cjobs;
  ku.n_cjobs = g->prep.n_cjobs;
  ku.chash_w = g->prep.chash_w;
  ku.n_chash = g->prep.n_chash;
  ku.n_chash2 = g->prep.n_chash2;
  ku.n_chash_big = g->prep.n_chash_big;
  ku.n_chash_mid = g->prep.n_chash_mid;
  ku.n_chash2_big = g->prep.n_chash2_big;
  ku.n_cunits = g->prep.n_cunits;
  for (int t = 0; t <= kNumTiers; ++t) ku.tier_off[t] = g->prep.ktier_off[t];
  if ((st = run_count(dg, g->prep.units, g->prep.n_units, ku, pe_dev, g->d_csum, g->d_x, &g->sc, s, g->ev, pe_host,
                      ind_dev, ind_host)) != GC_OK)
    return st;
  unsigned long long hx[17 * 2 + 13 * 2];
  int32_t hstatus = 0;
  GC_CHECK(cudaMemcpyAsync(hx, g->d_x, sizeof(unsigned long long) * 17 * 2, cudaMemcpyDeviceToHost, s), "copy X");
  GC_CHECK(cudaMemcpyAsync(hx + 34, g->d_csum, sizeof(unsigned long long) * 13 * 2, cudaMemcpyDeviceToHost, s),
           "copy C");
  GC_CHECK(cudaMemcpyAsync(&hstatus, g->sc.misc + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "copy status");
  GC_CHECK(cudaMemcpyAsync(g->work, g->sc.work, sizeof(g->work), cudaMemcpyDeviceToHost, s), "copy work");
  if (staged)
    GC_CHECK(cudaMemcpyAsync(per_edge_out, pe_dev, sizeof(uint64_t) * 13 * (size_t)g->m, cudaMemcpyDeviceToHost, s),
             "copy per-edge");
  if (ind_staged)
    GC_CHECK(cudaMemcpyAsync(induced_out, ind_dev, sizeof(uint64_t) * GC_INDUCED_COLS * (size_t)g->m,
                             cudaMemcpyDeviceToHost, s),
             "copy induced");
  GC_CHECK(cudaEventRecord(g->ev[kNumPhases], s), "event");
  GC_CHECK(cudaStreamSynchronize(s), "sync count");
  g->sc.tlist_want = (long long)g->work[kWorkTTriangles];  // the next count keeps pass T's edge lists
#undef GC_CHECK
  if (hstatus & kSpillOverflow) {
    set_error("internal: a unit outgrew its tier, cursor buffer or hash (only for input that skipped validation)");
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

gc_status gc_count_edge_graphlets(gc_graph g, uint64_t* per_edge_out, uint64_t* global_out,
                                  uint64_t* global_hi) {
  return count_graph(g, per_edge_out, nullptr, global_out, global_hi);
}

gc_status gc_count_edge_induced(gc_graph g, uint64_t* induced_out, uint64_t* per_edge_out, uint64_t* global_out,
                                uint64_t* global_hi) {
  if (!induced_out && g && g->m > 0) { set_error("induced_out is NULL"); return GC_ERR_ARG; }
  return count_graph(g, per_edge_out, induced_out, global_out, global_hi);
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
                                          "finish_columns", "induced_columns", "derive", "copy_out"};
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

gc_status gc_release_cached_memory(void) {
  cudaMemPool_t pool = lib_pool();
  if (!pool) {
    set_error("gc_release_cached_memory: no CUDA device or pool");
    return GC_ERR_CUDA;
  }
  cudaError_t e = cudaDeviceSynchronize();  // every stream-ordered free has reached the pool
  if (e == cudaSuccess) e = cudaMemPoolTrimTo(pool, 0);
  return e == cudaSuccess ? GC_OK : cuda_fail(e, "gc_release_cached_memory");
}

}  // extern "C"
