// gc_batch.cu -- batched and served counting of many graphs (see include/gc.h).
//
// A launch counts all graphs taken from the pending queue as one disjoint
// union: graph g keeps its vertices in the global range [gbase[g],
// gbase[g] + n_g). Triangles, 4-cliques and 4-cycles of a disjoint union are
// those of its components, so the per-edge kernels run unchanged over the
// union -- one persistent grid per pass, CTAs stealing v-groups of every graph
// from one difficulty-binned queue -- while the per-edge columns use each
// graph's own n and m and the unrestricted counts are summed per graph.
//
// Continuous batching: submit() admits a graph while the admitted graphs'
// estimated device footprint stays within the budget; a dispatcher thread
// launches whatever is pending whenever fewer than two launches are in
// flight (each launch on its own stream, so a new launch's preparation
// overlaps the previous launch's counting) and retires finished launches,
// which releases their share of the budget.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <memory>
#include <thread>
#include <vector>

#include "gc_internal.h"

namespace gc {
gc_status validate_csr(int32_t n, const int32_t* rp, const int32_t* ci);
gc_status validate_csr_small(int32_t n, const int32_t* rp, const int32_t* ci, std::vector<int32_t>* fill);

namespace {

__global__ void k_globalize(int32_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ vgid,
                            const int32_t* __restrict__ gbase, int32_t* __restrict__ ci) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int32_t x = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n; x += warps) {
    const int32_t base = gbase[vgid[x]];
    for (int32_t p = rp[x] + lane; p < rp[x + 1]; p += 32) ci[p] += base;
  }
}

// Host buffers for the library's copies of bulk submissions, kept for reuse:
// a submission takes the smallest kept buffer that holds it, whose pages are
// already mapped, instead of a fresh allocation that every submission would
// fault in again. Buffers are not initialised (the copy that fills a buffer
// writes every entry it reads). At most kKeep buffers are kept, the smallest
// dropped first; the cache lives until the batch and its last buffer are gone.
struct HostCache {
  static constexpr int kKeep = 4;
  std::mutex mu;
  std::vector<std::pair<size_t, int32_t*>> free;  // (entries, buffer)
  ~HostCache() {
    for (auto& f : free) delete[] f.second;
  }
};

// A buffer of at least `entries` int32 from the cache (or new); it returns to
// the cache when its last reference goes. Throws std::bad_alloc.
std::shared_ptr<int32_t> host_buffer(const std::shared_ptr<HostCache>& cache, size_t entries) {
  if (entries == 0) entries = 1;
  int32_t* p = nullptr;
  size_t cap = 0;
  {
    std::lock_guard<std::mutex> lk(cache->mu);
    int best = -1;
    for (int i = 0; i < (int)cache->free.size(); ++i)
      if (cache->free[i].first >= entries && (best < 0 || cache->free[i].first < cache->free[best].first)) best = i;
    if (best >= 0) {
      cap = cache->free[best].first;
      p = cache->free[best].second;
      cache->free.erase(cache->free.begin() + best);
    }
  }
  if (!p) {
    p = new int32_t[entries];
    cap = entries;
  }
  std::shared_ptr<HostCache> keep = cache;
  return std::shared_ptr<int32_t>(p, [keep, cap](int32_t* q) {
    std::lock_guard<std::mutex> lk(keep->mu);
    keep->free.emplace_back(cap, q);
    if ((int)keep->free.size() > HostCache::kKeep) {
      auto it = std::min_element(keep->free.begin(), keep->free.end(),
                                 [](const std::pair<size_t, int32_t*>& a, const std::pair<size_t, int32_t*>& b) {
                                   return a.first < b.first;
                                 });
      delete[] it->second;
      keep->free.erase(it);
    }
  });
}

// A graph waiting for a launch. Its CSR is the library's own copy: rp (n + 1
// entries starting at 0) and ci (2m entries) point into `owner` -- a copy of
// one graph (gc_batch_submit), or one shared copy of a whole bulk submission
// (gc_batch_submit_many: one buffer from the batch's host cache and one bulk
// copy per graph, made while validating).
struct PendingGraph {
  uint64_t ticket;
  int32_t n;
  int64_t m;
  int64_t bytes;
  const int32_t* rp = nullptr;
  const int32_t* ci = nullptr;
  std::shared_ptr<int32_t> owner;
};

struct Result {
  uint64_t x[34];
  gc_status status;
};

// Timers of one launch (CUDA events on its stream): the size classes of the
// small-graph kernels (eager launches only), the whole small-graph sequence
// (copies in, kernels, derive, copy out) and the larger graphs' passes.
enum { kEvSmall0 = 0, kEvSmallSeq0 = kSmallClasses + 1, kEvSmallSeq1, kEvUnion0, kEvUnion1, kNumLaunchEv };

struct Launch {
  std::vector<uint64_t> tickets;
  std::vector<int32_t> slot;          // ticket k's row in h_x
  int64_t bytes = 0;
  int stream_slot = 0;
  BatchConfig cfg;                    // the batch's parameters when the launch was taken
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  cudaEvent_t ev[kNumLaunchEv] = {};
  bool timed_classes = false, timed_small = false, timed_union = false, replayed = false;
  unsigned long long* h_x = nullptr;  // pinned [G][17][2]
  int32_t* h_status = nullptr;        // pinned
  gc_status launch_status = GC_OK;
  std::string error;
};

// Device buffers and pinned host staging of the small-graph path, one set per
// stream slot, grown as needed and kept: once warm, a launch allocates
// nothing, and its sequence (copies in, kernels, derive, copy out) can be
// captured and replayed as a CUDA graph. `busy` marks the end of the slot's
// last sequence: the host waits on it before it refills or regrows them.
struct SmallBufs {
  size_t cap_rows = 0, cap_nnz = 0, cap_g = 0;
  int32_t *d_rp = nullptr, *d_ci = nullptr, *d_order = nullptr, *d_gn = nullptr, *d_misc = nullptr;
  int64_t *d_voff = nullptr, *d_eoff = nullptr, *d_gm = nullptr;
  unsigned long long *d_csum = nullptr, *d_x = nullptr;
  int32_t *h_rp = nullptr, *h_ci = nullptr, *h_order = nullptr, *h_gn = nullptr;
  int64_t *h_voff = nullptr, *h_eoff = nullptr, *h_gm = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t busy = nullptr;
};

void free_small_bufs(SmallBufs* b) {
  if (b->busy) cudaEventSynchronize(b->busy);
  for (void* p : {(void*)b->d_rp, (void*)b->d_ci, (void*)b->d_order, (void*)b->d_gn, (void*)b->d_misc,
                  (void*)b->d_voff, (void*)b->d_eoff, (void*)b->d_gm, (void*)b->d_csum, (void*)b->d_x})
    if (p) cudaFree(p);
  for (void* p : {(void*)b->h_rp, (void*)b->h_ci, (void*)b->h_order, (void*)b->h_gn, (void*)b->h_voff,
                  (void*)b->h_eoff, (void*)b->h_gm})
    if (p) cudaFreeHost(p);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->busy) cudaEventDestroy(b->busy);
  *b = SmallBufs();
}

int64_t footprint(int32_t n, int64_t m) {
  int64_t b = 44LL * n + 32LL * m + 1024;
  if (n > kSmemTableMax) b += (int64_t)count_grid_size() * n * 4;
  return b;
}

}  // namespace
}  // namespace gc

using namespace gc;

struct gc_batch_s {
  int64_t budget = 0;
  uint32_t flags = 0;
  BatchConfig cfg;
  SmallBufs small[kMaxInflight];        // per stream slot
  double last_stats[GC_BATCH_STATS] = {};  // of the last retired launch
  int64_t in_use = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<PendingGraph> pending;
  std::vector<Launch*> inflight;
  std::unordered_map<uint64_t, Result> done;
  std::unordered_set<uint64_t> live;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread dispatcher;
  cudaStream_t streams[kMaxInflight] = {};
  int next_stream = 0;                  // manual mode: round-robin over the slots
  int device = 0;
  std::shared_ptr<HostCache> host = std::make_shared<HostCache>();  // bulk-submission copies
};

namespace {

// Counts `graphs` as one launch on `s`. Fills L (results land in L->h_x when
// L->done completes). Runs in the dispatcher thread (or the flushing thread
// in manual mode) without holding the batch lock.
// The graphs too large for the bitmatrix kernel, as one disjoint union
// through the general passes. Results go to h_x_dst ([G][17][2], pinned) and
// the launch status word to *h_status_dst.
gc_status run_union(std::vector<PendingGraph*>& graphs, cudaStream_t s, Launch* L, unsigned long long* h_x_dst,
                    int32_t* h_status_dst) {
  const int32_t G = (int32_t)graphs.size();
  int64_t n_total = 0, nnz_total = 0;
  int32_t table_n = 0;
  for (auto* pg : graphs) {
    n_total += pg->n;
    nnz_total += 2 * pg->m;
    if (pg->n > table_n) table_n = pg->n;
  }
  const int32_t n = (int32_t)n_total;
  const int32_t m = (int32_t)(nnz_total / 2);
  std::vector<int32_t> h_rp((size_t)n + 1), h_ci((size_t)(nnz_total > 0 ? nnz_total : 1)), h_vgid((size_t)(n > 0 ? n : 1));
  std::vector<int32_t> h_desc((size_t)2 * G);  // gbase | gn
  std::vector<int64_t> h_gm((size_t)G);
  {
    int64_t vo = 0, eo = 0;
    for (int32_t gi = 0; gi < G; ++gi) {
      PendingGraph& pg = *graphs[gi];
      for (int32_t i = 0; i < pg.n; ++i) {
        h_rp[vo + i] = (int32_t)(eo + pg.rp[i]);
        h_vgid[vo + i] = gi;
      }
      if (pg.m > 0) std::memcpy(h_ci.data() + eo, pg.ci, sizeof(int32_t) * 2 * pg.m);
      h_desc[gi] = (int32_t)vo;
      h_desc[G + gi] = pg.n;
      h_gm[gi] = pg.m;
      vo += pg.n;
      eo += 2 * pg.m;
    }
    h_rp[n] = (int32_t)eo;
  }
  int32_t *d_rp = nullptr, *d_ci = nullptr, *d_vgid = nullptr, *d_desc = nullptr;
  int64_t* d_gm = nullptr;
  unsigned long long *d_csum = nullptr, *d_x = nullptr;
  PrepBuffers prep;
  Scratch sc;
  cudaError_t e = cudaSuccess;
  gc_status st = GC_OK;
  auto fail = [&](cudaError_t err, const char* what) {
    st = cuda_fail(err, what);
    L->error = gc_last_error();
  };
#define GB_TRY(call, what)  \
  do {                      \
    e = (call);             \
    if (e != cudaSuccess) { \
      fail(e, what);        \
      goto out;             \
    }                       \
  } while (0)
  GB_TRY(pool_alloc(&d_rp, sizeof(int32_t) * ((size_t)n + 1), s), "batch alloc");
  GB_TRY(pool_alloc(&d_ci, sizeof(int32_t) * h_ci.size(), s), "batch alloc");
  GB_TRY(pool_alloc(&d_vgid, sizeof(int32_t) * h_vgid.size(), s), "batch alloc");
  GB_TRY(pool_alloc(&d_desc, sizeof(int32_t) * h_desc.size(), s), "batch alloc");
  GB_TRY(pool_alloc(&d_gm, sizeof(int64_t) * G, s), "batch alloc");
  GB_TRY(pool_alloc(&d_csum, sizeof(unsigned long long) * (size_t)G * 26, s), "batch alloc");
  GB_TRY(pool_alloc(&d_x, sizeof(unsigned long long) * (size_t)G * 34, s), "batch alloc");
  GB_TRY(cudaMemcpyAsync(d_rp, h_rp.data(), sizeof(int32_t) * h_rp.size(), cudaMemcpyHostToDevice, s), "batch copy");
  GB_TRY(cudaMemcpyAsync(d_ci, h_ci.data(), sizeof(int32_t) * h_ci.size(), cudaMemcpyHostToDevice, s), "batch copy");
  GB_TRY(cudaMemcpyAsync(d_vgid, h_vgid.data(), sizeof(int32_t) * h_vgid.size(), cudaMemcpyHostToDevice, s), "batch copy");
  GB_TRY(cudaMemcpyAsync(d_desc, h_desc.data(), sizeof(int32_t) * h_desc.size(), cudaMemcpyHostToDevice, s), "batch copy");
  GB_TRY(cudaMemcpyAsync(d_gm, h_gm.data(), sizeof(int64_t) * G, cudaMemcpyHostToDevice, s), "batch copy");
  if (n > 0) {
    int blocks = (int)std::min<int64_t>(((int64_t)n * 32 + 255) / 256, 65535LL * 8);
    k_globalize<<<blocks, 256, 0, s>>>(n, d_rp, d_vgid, d_desc, d_ci);
    GB_TRY(cudaGetLastError(), "k_globalize");
  }
  if ((st = prepare_graph(n, m, d_rp, d_ci, d_vgid, nullptr, nullptr, &prep, s)) != GC_OK) {
    L->error = gc_last_error();
    goto out;
  }
  if ((st = scratch_init(&sc, m, table_n, prep.kmax, prep.cnx_max, s)) != GC_OK) {
    L->error = gc_last_error();
    goto out;
  }
  {
    DevGraph dg;
    dg.n = n;
    dg.m = m;
    dg.rp = d_rp;
    dg.ci = d_ci;
    dg.deg = prep.deg;
    dg.eid = prep.eid;
    dg.out_ptr = prep.out_ptr;
    dg.out_idx = prep.out_idx;
    dg.ocsr = prep.ocsr;
    dg.e2o = prep.e2o;
    dg.rev = prep.rev;
    dg.G = G;
    dg.vgid = d_vgid;
    dg.gbase = d_desc;
    dg.gn = d_desc + G;
    dg.gm = d_gm;
    dg.table_n = table_n;
    dg.ranked = false;
    KUnits ku;
    ku.units = prep.kunits;
    ku.cunits = prep.cunits;
    ku.n_cheavy = prep.n_cheavy;
    ku.cjobs = prep.cjobs;
    ku.n_cjobs = prep.n_cjobs;
    ku.chash_w = prep.chash_w;
    ku.n_chash = prep.n_chash;
    ku.n_chash2 = prep.n_chash2;
    ku.n_chash_big = prep.n_chash_big;
    ku.n_chash_mid = prep.n_chash_mid;
    ku.n_chash2_big = prep.n_chash2_big;
    ku.n_cunits = prep.n_cunits;
    for (int t = 0; t <= kNumTiers; ++t) ku.tier_off[t] = prep.ktier_off[t];
    if ((st = run_count(dg, prep.units, prep.n_units, ku, nullptr, d_csum, d_x, &sc, s, nullptr)) != GC_OK) {
      L->error = gc_last_error();
      goto out;
    }
    GB_TRY(cudaMemcpyAsync(h_x_dst, d_x, sizeof(unsigned long long) * (size_t)G * 34, cudaMemcpyDeviceToHost, s),
           "batch copy out");
    GB_TRY(cudaMemcpyAsync(h_status_dst, sc.misc + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "batch copy out");
  }
out:
#undef GB_TRY
  free_prep(&prep, s);
  scratch_free(&sc, s);
  for (void* p : {(void*)d_rp, (void*)d_ci, (void*)d_vgid, (void*)d_desc, (void*)d_gm, (void*)d_csum, (void*)d_x})
    if (p) cudaFreeAsync(p, s);
  return st;
}

// Grows the device buffer *d and the pinned host buffer *h (either may be
// absent) to hold `need` elements of T.
template <typename T>
cudaError_t grow_pair(T** d, T** h, size_t* cap, size_t need) {
  if (need <= *cap && (d == nullptr || *d) && (h == nullptr || *h)) return cudaSuccess;
  const size_t want = need + need / 4 + 64;
  if (d && *d) cudaFree(*d);
  if (h && *h) cudaFreeHost(*h);
  if (d) *d = nullptr;
  if (h) *h = nullptr;
  *cap = 0;
  cudaError_t e = cudaSuccess;
  if (d) e = cudaMalloc(d, sizeof(T) * want);
  if (e == cudaSuccess && h) e = cudaMallocHost(h, sizeof(T) * want);
  if (e == cudaSuccess) *cap = want;
  return e;
}

// Graphs of at most cfg.small_n_max vertices: packed as they are (local ids)
// into the slot's pinned staging and counted one CTA per graph on a
// shared-memory bitmatrix, binned by size class. The sequence is captured
// into a CUDA graph and replayed (cudaGraphExecUpdate keeps one executable
// per slot while the shape of the launches stays the same), or issued
// eagerly with per-class timers when cfg.use_graph is 0.
gc_status run_small(std::vector<PendingGraph*>& graphs, cudaStream_t s, Launch* L, unsigned long long* h_x_dst,
                    SmallBufs* sb, const BatchConfig& cfg) {
  const int32_t G = (int32_t)graphs.size();
  std::vector<int64_t> voff((size_t)G + 1), eoff((size_t)G + 1);
  voff[0] = eoff[0] = 0;
  for (int32_t gi = 0; gi < G; ++gi) {
    voff[gi + 1] = voff[gi] + graphs[gi]->n + 1;
    eoff[gi + 1] = eoff[gi] + 2 * graphs[gi]->m;
  }
  const size_t rows = (size_t)voff[G], nnz = (size_t)(eoff[G] > 0 ? eoff[G] : 1);
  gc_status st = GC_OK;
  cudaError_t e = cudaSuccess;
#define GS_TRY(call, what)                   \
  do {                                       \
    e = (call);                              \
    if (e != cudaSuccess) {                  \
      st = cuda_fail(e, what);               \
      L->error = gc_last_error();            \
      return st;                             \
    }                                        \
  } while (0)
  if (sb->busy) GS_TRY(cudaEventSynchronize(sb->busy), "small buffers in use");
  else GS_TRY(cudaEventCreateWithFlags(&sb->busy, cudaEventDisableTiming), "small event");
  {
    size_t cr = sb->cap_rows, cn = sb->cap_nnz, cg = sb->cap_g;
    GS_TRY(grow_pair(&sb->d_rp, &sb->h_rp, &cr, rows), "small buffers");
    GS_TRY(grow_pair(&sb->d_ci, &sb->h_ci, &cn, nnz), "small buffers");
    if ((size_t)G + 1 > sb->cap_g || !sb->d_voff) {
      size_t c1 = 0;
      const size_t need = (size_t)G + 1;
      GS_TRY(grow_pair(&sb->d_voff, &sb->h_voff, &c1, need), "small buffers");
      c1 = 0; GS_TRY(grow_pair(&sb->d_eoff, &sb->h_eoff, &c1, need), "small buffers");
      c1 = 0; GS_TRY(grow_pair(&sb->d_gm, &sb->h_gm, &c1, need), "small buffers");
      c1 = 0; GS_TRY(grow_pair(&sb->d_gn, &sb->h_gn, &c1, need), "small buffers");
      c1 = 0; GS_TRY(grow_pair(&sb->d_order, &sb->h_order, &c1, need), "small buffers");
      c1 = 0; GS_TRY(grow_pair<unsigned long long>(&sb->d_csum, nullptr, &c1, 26 * need), "small buffers");
      c1 = 0; GS_TRY(grow_pair<unsigned long long>(&sb->d_x, nullptr, &c1, 34 * need), "small buffers");
      if (!sb->d_misc) GS_TRY(cudaMalloc(&sb->d_misc, sizeof(int32_t) * (kSmallClasses + 1)), "small buffers");
      cg = c1 / 34;
    }
    sb->cap_rows = cr;
    sb->cap_nnz = cn;
    sb->cap_g = cg;
  }
  // order: graphs binned by size class, largest m first within a class
  int32_t class_off[kSmallClasses + 1] = {0};
  {
    std::vector<int32_t> cls((size_t)G);
    for (int32_t gi = 0; gi < G; ++gi) {
      cls[gi] = small_class_of(graphs[gi]->n);
      ++class_off[cls[gi] + 1];
    }
    for (int c = 0; c < kSmallClasses; ++c) class_off[c + 1] += class_off[c];
    std::vector<int32_t> pos(class_off, class_off + kSmallClasses);
    for (int32_t gi = 0; gi < G; ++gi) sb->h_order[pos[cls[gi]]++] = gi;
    for (int c = 0; c < kSmallClasses; ++c)
      std::sort(sb->h_order + class_off[c], sb->h_order + class_off[c + 1],
                [&](int32_t a, int32_t b) { return graphs[a]->m > graphs[b]->m; });
  }
  std::memcpy(sb->h_voff, voff.data(), sizeof(int64_t) * voff.size());
  std::memcpy(sb->h_eoff, eoff.data(), sizeof(int64_t) * eoff.size());
  for (int32_t gi = 0; gi < G; ++gi) {
    sb->h_gn[gi] = graphs[gi]->n;
    sb->h_gm[gi] = graphs[gi]->m;
  }
  {  // CSR packed on the host cores, each thread the graphs whose entries start in its share
    const unsigned hw = std::thread::hardware_concurrency();
    const int nt = eoff[G] < (1 << 22) ? 1 : (int)std::min<unsigned>(hw ? hw : 1, 32);
    auto pack = [&](int t) {
      const int64_t e0 = eoff[G] * t / nt, e1 = eoff[G] * (t + 1) / nt;
      int32_t gi = (int32_t)(std::lower_bound(eoff.begin(), eoff.begin() + G, e0) - eoff.begin());
      for (; gi < G && (eoff[gi] < e1 || t == nt - 1); ++gi) {
        std::memcpy(sb->h_rp + voff[gi], graphs[gi]->rp, sizeof(int32_t) * (graphs[gi]->n + 1));
        if (graphs[gi]->m > 0)
          std::memcpy(sb->h_ci + eoff[gi], graphs[gi]->ci, sizeof(int32_t) * 2 * graphs[gi]->m);
      }
    };
    std::vector<std::thread> th;
    for (int t = 1; t < nt; ++t) th.emplace_back(pack, t);
    pack(0);
    for (auto& x : th) x.join();
  }
  const bool graph_mode = cfg.use_graph != 0;
  // the sequence; returns the first failure (for a capture, the capture is
  // ended by the caller)
  auto issue = [&]() -> cudaError_t {
    cudaError_t r = cudaSuccess;
    const size_t b4 = sizeof(int32_t), b8 = sizeof(int64_t);
    r = cudaMemcpyAsync(sb->d_rp, sb->h_rp, b4 * rows, cudaMemcpyHostToDevice, s);
    if (r == cudaSuccess && eoff[G] > 0) r = cudaMemcpyAsync(sb->d_ci, sb->h_ci, b4 * (size_t)eoff[G], cudaMemcpyHostToDevice, s);
    if (r == cudaSuccess) r = cudaMemcpyAsync(sb->d_voff, sb->h_voff, b8 * (G + 1), cudaMemcpyHostToDevice, s);
    if (r == cudaSuccess) r = cudaMemcpyAsync(sb->d_eoff, sb->h_eoff, b8 * (G + 1), cudaMemcpyHostToDevice, s);
    if (r == cudaSuccess) r = cudaMemcpyAsync(sb->d_gn, sb->h_gn, b4 * G, cudaMemcpyHostToDevice, s);
    if (r == cudaSuccess) r = cudaMemcpyAsync(sb->d_gm, sb->h_gm, b8 * G, cudaMemcpyHostToDevice, s);
    if (r == cudaSuccess) r = cudaMemcpyAsync(sb->d_order, sb->h_order, b4 * G, cudaMemcpyHostToDevice, s);
    if (r == cudaSuccess) r = cudaMemsetAsync(sb->d_misc, 0, b4 * (kSmallClasses + 1), s);
    if (r == cudaSuccess) r = cudaMemsetAsync(sb->d_csum, 0, sizeof(unsigned long long) * 26 * (size_t)G, s);
    if (r != cudaSuccess) return r;
    if (run_small_graphs(sb->d_rp, sb->d_voff, sb->d_ci, sb->d_eoff, sb->d_order, class_off, sb->d_misc,
                         sb->d_misc + kSmallClasses, sb->d_csum, cfg, graph_mode ? nullptr : L->ev + kEvSmall0,
                         s) != GC_OK)
      return cudaErrorLaunchFailure;
    DevGraph dg = DevGraph();
    dg.G = G;
    dg.gn = sb->d_gn;
    dg.gm = sb->d_gm;
    if (run_derive(dg, sb->d_csum, sb->d_x, sb->d_misc + kSmallClasses, s) != GC_OK) return cudaErrorLaunchFailure;
    r = cudaMemcpyAsync(h_x_dst, sb->d_x, sizeof(unsigned long long) * (size_t)G * 34, cudaMemcpyDeviceToHost, s);
    if (r == cudaSuccess) r = cudaMemcpyAsync(L->h_status, sb->d_misc + kSmallClasses, b4, cudaMemcpyDeviceToHost, s);
    return r;
  };
  GS_TRY(cudaEventRecord(L->ev[kEvSmallSeq0], s), "small event");
  if (graph_mode) {
    cudaGraph_t graph = nullptr;
    GS_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "capture small-graph launch");
    const cudaError_t r = issue();
    const cudaError_t r2 = cudaStreamEndCapture(s, &graph);
    if (r != cudaSuccess || r2 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      GS_TRY(r != cudaSuccess ? r : r2, "capture small-graph launch");
    }
    if (sb->exec) {
      cudaGraphExecUpdateResultInfo info;
      if (cudaGraphExecUpdate(sb->exec, graph, &info) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphExecDestroy(sb->exec);
        sb->exec = nullptr;
      }
    }
    if (!sb->exec) {
      e = cudaGraphInstantiate(&sb->exec, graph, 0);
      if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        sb->exec = nullptr;
        GS_TRY(e, "instantiate small-graph launch");
      }
    }
    cudaGraphDestroy(graph);
    GS_TRY(cudaGraphLaunch(sb->exec, s), "replay small-graph launch");
    L->replayed = true;
  } else {
    GS_TRY(issue(), "small-graph launch");
    L->timed_classes = true;
  }
  GS_TRY(cudaEventRecord(L->ev[kEvSmallSeq1], s), "small event");
  GS_TRY(cudaEventRecord(sb->busy, s), "small event");
  L->timed_small = true;
#undef GS_TRY
  return GC_OK;
}

// Counts `graphs` as one launch on `s`: small graphs on the bitmatrix kernels,
// the others as one disjoint union. Results land in L->h_x when L->done
// completes. Runs in the dispatcher thread (or the flushing thread in manual
// mode) without holding the batch lock.
void run_launch(gc_batch b, std::vector<PendingGraph>& graphs, cudaStream_t s, Launch* L) {
  const BatchConfig cfg = L->cfg;
  auto is_small = [&](const PendingGraph& pg) {
    return pg.n <= cfg.small_n_max && small_class_of(pg.n) < kSmallClasses;
  };
  std::vector<PendingGraph*> small, large;
  for (auto& pg : graphs) (is_small(pg) ? small : large).push_back(&pg);
  L->slot.resize(graphs.size());
  {
    int32_t is = 0, il = (int32_t)small.size();
    for (size_t k = 0; k < graphs.size(); ++k) L->slot[k] = is_small(graphs[k]) ? is++ : il++;
  }
  gc_status st = GC_OK;
  L->h_status[0] = 0;
  L->h_status[1] = 0;
  for (auto& ev : L->ev)
    if (cudaEventCreate(&ev) != cudaSuccess) {
      L->launch_status = cuda_fail(cudaGetLastError(), "batch event");
      L->error = gc_last_error();
      return;
    }
  if (!small.empty()) st = run_small(small, s, L, L->h_x, &b->small[L->stream_slot], cfg);
  if (st == GC_OK && !large.empty()) {
    cudaEventRecord(L->ev[kEvUnion0], s);
    st = run_union(large, s, L, L->h_x + 34 * small.size(), L->h_status + 1);
    cudaEventRecord(L->ev[kEvUnion1], s);
    L->timed_union = st == GC_OK;
  }
  L->launch_status = st;
  if (st == GC_OK) {
    cudaError_t e = cudaEventRecord(L->done, s);
    if (e != cudaSuccess) {
      L->launch_status = cuda_fail(e, "batch event");
      L->error = gc_last_error();
    }
  }
}

// Must hold b->mu.
void retire_locked(gc_batch b) {
  for (size_t i = 0; i < b->inflight.size();) {
    Launch* L = b->inflight[i];
    bool finished = L->launch_status != GC_OK;
    if (!finished) {
      cudaError_t q = cudaEventQuery(L->done);
      if (q == cudaErrorNotReady) {
        ++i;
        continue;
      }
      if (q != cudaSuccess) {
        L->launch_status = cuda_fail(q, "batch launch");
        L->error = gc_last_error();
      }
    }
    if (L->launch_status == GC_OK) {  // device times of the launch
      auto ms = [&](int a, int z) {
        float f = 0.f;
        return cudaEventElapsedTime(&f, L->ev[a], L->ev[z]) == cudaSuccess ? (double)f : 0.0;
      };
      for (int c = 0; c < kSmallClasses; ++c)
        b->last_stats[c] = L->timed_classes ? ms(kEvSmall0 + c, kEvSmall0 + c + 1) : 0.0;
      b->last_stats[kSmallClasses] = L->timed_small ? ms(kEvSmallSeq0, kEvSmallSeq1) : 0.0;
      b->last_stats[kSmallClasses + 1] = L->timed_union ? ms(kEvUnion0, kEvUnion1) : 0.0;
      b->last_stats[kSmallClasses + 2] = L->replayed ? 1.0 : 0.0;
      cudaGetLastError();
    }
    for (size_t k = 0; k < L->tickets.size(); ++k) {
      Result r;
      if (L->launch_status == GC_OK) {
        std::memcpy(r.x, L->h_x + 34 * (size_t)L->slot[k], sizeof(r.x));
        const int32_t dst = L->h_status[0] | L->h_status[1];
        r.status = dst == 0 ? GC_OK : GC_ERR_CUDA;
      } else {
        std::memset(r.x, 0, sizeof(r.x));
        r.status = L->launch_status;
      }
      b->done[L->tickets[k]] = r;
    }
    b->in_use -= L->bytes;
    cudaFreeHost(L->h_x);
    cudaFreeHost(L->h_status);
    cudaEventDestroy(L->done);
    for (auto& ev : L->ev)
      if (ev) cudaEventDestroy(ev);
    delete L;
    b->inflight.erase(b->inflight.begin() + i);
    b->cv.notify_all();
  }
}

// Takes every pending graph (up to the int32 edge limit) and launches it.
// Called without the lock; returns false if nothing was pending.
bool launch_pending(gc_batch b) {
  std::vector<PendingGraph> take;
  Launch* L = new Launch();
  {
    std::lock_guard<std::mutex> lk(b->mu);
    if (b->pending.empty()) {
      delete L;
      return false;
    }
    int64_t nnz = 0, nv = 0;
    while (!b->pending.empty()) {
      PendingGraph& pg = b->pending.front();
      if (!take.empty() && (nnz + 2 * pg.m >= (1LL << 31) - 1 || nv + pg.n >= (1LL << 31) - 1)) break;
      nnz += 2 * pg.m;
      nv += pg.n;
      L->tickets.push_back(pg.ticket);
      L->bytes += pg.bytes;
      take.push_back(std::move(pg));
      b->pending.pop_front();
    }
    // a stream slot no launch in flight holds (the dispatcher keeps fewer
    // than max_inflight launches in flight); manual flushes take the slots in
    // turn (a slot's buffers wait for their previous use)
    int slot = -1;
    for (int k = 0; k < b->cfg.max_inflight && slot < 0; ++k) {
      bool used = false;
      for (Launch* o : b->inflight) used |= o->stream_slot == k;
      if (!used) slot = k;
    }
    if (slot < 0) {
      slot = b->next_stream % b->cfg.max_inflight;
      b->next_stream = slot + 1;
    }
    L->stream_slot = slot;
    L->cfg = b->cfg;
    L->stream = b->streams[slot];
  }
  cudaSetDevice(b->device);
  cudaError_t e1 = cudaMallocHost(&L->h_x, sizeof(unsigned long long) * 34 * take.size());
  cudaError_t e2 = cudaMallocHost(&L->h_status, 2 * sizeof(int32_t));  // small graphs, union
  cudaError_t e3 = cudaEventCreateWithFlags(&L->done, cudaEventDisableTiming);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
    L->launch_status = GC_ERR_NOMEM;
  } else {
    run_launch(b, take, L->stream, L);
  }
  {
    std::lock_guard<std::mutex> lk(b->mu);
    b->inflight.push_back(L);
    b->cv.notify_all();
  }
  return true;
}

void dispatcher_main(gc_batch b) {
  cudaSetDevice(b->device);
  std::unique_lock<std::mutex> lk(b->mu);
  while (!b->stop) {
    retire_locked(b);
    if (!b->pending.empty() && (int)b->inflight.size() < b->cfg.max_inflight) {
      lk.unlock();
      launch_pending(b);
      lk.lock();
      continue;
    }
    b->cv.wait_for(lk, std::chrono::microseconds(100));
  }
}

}  // namespace

extern "C" {

gc_status gc_batch_create(int64_t device_mem_budget_bytes, uint32_t flags, gc_batch* out) {
  if (!out) { set_error("out is NULL"); return GC_ERR_ARG; }
  *out = nullptr;
  if (device_mem_budget_bytes <= 0 || (flags & ~GC_BATCH_MANUAL)) {
    set_error("bad budget or flags");
    return GC_ERR_ARG;
  }
  gc_batch b = new (std::nothrow) gc_batch_s();
  if (!b) { set_error("host allocation failed"); return GC_ERR_NOMEM; }
  b->budget = device_mem_budget_bytes;
  b->flags = flags;
  cudaGetDevice(&b->device);
  for (auto& s : b->streams) {
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      gc_status st = cuda_fail(e, "batch stream");
      for (auto& t : b->streams)
        if (t) cudaStreamDestroy(t);
      delete b;
      return st;
    }
  }
  count_grid_size();
  gc_status st = small_graphs_setup();
  if (st != GC_OK) {
    for (auto& t : b->streams) cudaStreamDestroy(t);
    delete b;
    return st;
  }
  load_tuned_config(&b->cfg, nullptr);
  if (!(flags & GC_BATCH_MANUAL)) b->dispatcher = std::thread(dispatcher_main, b);
  *out = b;
  return GC_OK;
}

gc_status gc_batch_set_param(gc_batch b, int32_t param, int32_t value) {
  if (!b) { set_error("batch is NULL"); return GC_ERR_ARG; }
  std::lock_guard<std::mutex> lk(b->mu);
  if (param == GC_PARAM_SMALL_N_MAX) {
    if (value < 0 || value > kSmallClassN[kSmallClasses - 1]) { set_error("small_n_max outside [0, 1024]"); return GC_ERR_ARG; }
    b->cfg.small_n_max = value;
  } else if (param >= GC_PARAM_BLOCK_N64 && param < GC_PARAM_BLOCK_N64 + kSmallClasses) {
    if (value != 64 && value != 128 && value != 256 && value != 512) { set_error("block must be 64, 128, 256 or 512"); return GC_ERR_ARG; }
    b->cfg.class_block[param - GC_PARAM_BLOCK_N64] = value;
  } else if (param == GC_PARAM_USE_GRAPH) {
    if (value != 0 && value != 1) { set_error("use_graph must be 0 or 1"); return GC_ERR_ARG; }
    b->cfg.use_graph = value;
  } else if (param == GC_PARAM_MAX_INFLIGHT) {
    if (value < 1 || value > kMaxInflight) { set_error("max_inflight must be 1 .. 4"); return GC_ERR_ARG; }
    b->cfg.max_inflight = value;
  } else {
    set_error("unknown parameter");
    return GC_ERR_ARG;
  }
  return GC_OK;
}

gc_status gc_batch_get_param(gc_batch b, int32_t param, int32_t* value) {
  if (!b || !value) { set_error("NULL argument"); return GC_ERR_ARG; }
  std::lock_guard<std::mutex> lk(b->mu);
  if (param == GC_PARAM_SMALL_N_MAX) *value = b->cfg.small_n_max;
  else if (param >= GC_PARAM_BLOCK_N64 && param < GC_PARAM_BLOCK_N64 + kSmallClasses)
    *value = b->cfg.class_block[param - GC_PARAM_BLOCK_N64];
  else if (param == GC_PARAM_USE_GRAPH) *value = b->cfg.use_graph;
  else if (param == GC_PARAM_MAX_INFLIGHT) *value = b->cfg.max_inflight;
  else { set_error("unknown parameter"); return GC_ERR_ARG; }
  return GC_OK;
}

gc_status gc_batch_last_stats(gc_batch b, double* out) {
  if (!b || !out) { set_error("NULL argument"); return GC_ERR_ARG; }
  std::lock_guard<std::mutex> lk(b->mu);
  for (int i = 0; i < GC_BATCH_STATS; ++i) out[i] = b->last_stats[i];
  return GC_OK;
}

gc_status gc_batch_submit(gc_batch b, int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                          uint64_t* ticket_out) {
  if (!b || !ticket_out || !row_ptr || n < 0) { set_error("bad arguments"); return GC_ERR_ARG; }
  gc_status st = validate_csr(n, row_ptr, col_idx);
  if (st != GC_OK) return st;
  const int64_t m = row_ptr[n] / 2;
  const int64_t bytes = footprint(n, m);
  if (bytes > b->budget) {
    set_error("graph needs more device memory than the whole budget");
    return GC_ERR_NOMEM;
  }
  PendingGraph pg;
  pg.n = n;
  pg.m = m;
  pg.bytes = bytes;
  try {
    pg.owner = std::shared_ptr<int32_t>(new int32_t[(size_t)n + 1 + 2 * (size_t)m], std::default_delete<int32_t[]>());
  } catch (...) {
    set_error("host allocation failed");
    return GC_ERR_NOMEM;
  }
  std::memcpy(pg.owner.get(), row_ptr, sizeof(int32_t) * ((size_t)n + 1));
  if (m > 0) std::memcpy(pg.owner.get() + n + 1, col_idx, sizeof(int32_t) * 2 * (size_t)m);
  pg.rp = pg.owner.get();
  pg.ci = pg.owner.get() + n + 1;
  {
    std::lock_guard<std::mutex> lk(b->mu);
    if (b->in_use + bytes > b->budget) {
      set_error("device-memory budget is full");
      return GC_ERR_BUSY;
    }
    pg.ticket = b->next_ticket++;
    *ticket_out = pg.ticket;
    b->in_use += bytes;
    b->live.insert(pg.ticket);
    b->pending.push_back(std::move(pg));
  }
  b->cv.notify_all();
  return GC_OK;
}

gc_status gc_batch_submit_many(gc_batch b, int64_t G, const int32_t* nvert, const int64_t* voff, const int64_t* eoff,
                               const int32_t* row_ptr, const int32_t* col_idx, uint64_t* tickets_out) {
  if (!b || G < 0 || (G > 0 && (!nvert || !voff || !eoff || !row_ptr || !tickets_out))) {
    set_error("bad arguments");
    return GC_ERR_ARG;
  }
  if (G == 0) return GC_OK;
  // the library's copy: one buffer for all graphs, rows then columns, each
  // graph at its own offset (own_v, own_e), filled while validating
  std::vector<int64_t> own_v((size_t)G + 1), own_e((size_t)G + 1);
  own_v[0] = own_e[0] = 0;
  for (int64_t g = 0; g < G; ++g) {
    const int32_t n = nvert[g];
    if (n < 0 || eoff[g + 1] < eoff[g]) {
      set_error("graph " + std::to_string(g) + ": negative size or decreasing offsets");
      return GC_ERR_ARG;
    }
    own_v[g + 1] = own_v[g] + n + 1;
    own_e[g + 1] = own_e[g] + (eoff[g + 1] - eoff[g]);
  }
  std::shared_ptr<int32_t> owner;
  try {
    owner = host_buffer(b->host, (size_t)(own_v[G] + own_e[G]));
  } catch (...) {
    set_error("host allocation failed");
    return GC_ERR_NOMEM;
  }
  int32_t* own_rp = owner.get();
  int32_t* own_ci = owner.get() + own_v[G];
  std::vector<PendingGraph> pgs((size_t)G);
  unsigned hw = std::thread::hardware_concurrency();
  const int nt = (int)std::min<int64_t>(std::max(1u, std::min(hw, 32u)), G);
  std::vector<gc_status> res(nt, GC_OK);
  std::vector<std::string> msg(nt);
  auto work = [&](int t) {  // the graphs whose entries start in this thread's share
    std::vector<int32_t> fill;  // symmetry-walk scratch of this thread
    const int64_t e0 = own_e[G] * t / nt, e1 = own_e[G] * (t + 1) / nt;
    int64_t g = std::lower_bound(own_e.begin(), own_e.begin() + G, e0) - own_e.begin();
    for (; g < G && (own_e[g] < e1 || t == nt - 1); ++g) {
      if (t > 0 && own_e[g] < e0) continue;
      const int32_t n = nvert[g];
      const int32_t* rp = row_ptr + voff[g];
      const int32_t* ci = col_idx ? col_idx + eoff[g] : nullptr;
      if ((int64_t)rp[n] != eoff[g + 1] - eoff[g]) {
        res[t] = GC_ERR_ARG;
        msg[t] = "graph " + std::to_string(g) + ": offsets disagree with row_ptr";
        return;
      }
      gc_status st = (int64_t)rp[n] < (1 << 20) ? validate_csr_small(n, rp, ci, &fill) : validate_csr(n, rp, ci);
      if (st != GC_OK) {
        res[t] = st;
        msg[t] = "graph " + std::to_string(g) + ": " + gc_last_error();
        return;
      }
      PendingGraph& pg = pgs[(size_t)g];
      pg.n = n;
      pg.m = rp[n] / 2;
      pg.bytes = footprint(n, pg.m);
      std::memcpy(own_rp + own_v[g], rp, sizeof(int32_t) * ((size_t)n + 1));
      if (pg.m > 0) std::memcpy(own_ci + own_e[g], ci, sizeof(int32_t) * 2 * (size_t)pg.m);
      pg.rp = own_rp + own_v[g];
      pg.ci = own_ci + own_e[g];
      pg.owner = owner;
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < nt; ++t) th.emplace_back(work, t);
  work(0);
  for (auto& x : th) x.join();
  for (int t = 0; t < nt; ++t)
    if (res[t] != GC_OK) {
      set_error(msg[t]);
      return res[t];
    }
  int64_t bytes = 0;
  for (auto& pg : pgs) bytes += pg.bytes;
  {
    std::lock_guard<std::mutex> lk(b->mu);
    if (bytes > b->budget) {
      set_error("graphs need more device memory than the whole budget");
      return GC_ERR_NOMEM;
    }
    if (b->in_use + bytes > b->budget) {
      set_error("device-memory budget is full");
      return GC_ERR_BUSY;
    }
    b->in_use += bytes;
    for (int64_t g = 0; g < G; ++g) {
      pgs[(size_t)g].ticket = b->next_ticket++;
      tickets_out[g] = pgs[(size_t)g].ticket;
      b->live.insert(pgs[(size_t)g].ticket);
      b->pending.push_back(std::move(pgs[(size_t)g]));
    }
  }
  b->cv.notify_all();
  return GC_OK;
}

gc_status gc_batch_flush(gc_batch b) {
  if (!b) { set_error("batch is NULL"); return GC_ERR_ARG; }
  if (b->flags & GC_BATCH_MANUAL) {
    while (launch_pending(b)) {
    }
  } else {
    b->cv.notify_all();
  }
  return GC_OK;
}

gc_status gc_batch_poll(gc_batch b, uint64_t ticket, uint64_t* global_out, uint64_t* global_hi,
                        int32_t timeout_us) {
  if (!b || !global_out) { set_error("NULL argument"); return GC_ERR_ARG; }
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us > 0 ? timeout_us : 0);
  std::unique_lock<std::mutex> lk(b->mu);
  if (!b->live.count(ticket)) {
    set_error("unknown or retired ticket");
    return GC_ERR_ARG;
  }
  for (;;) {
    if (b->flags & GC_BATCH_MANUAL) retire_locked(b);
    auto it = b->done.find(ticket);
    if (it != b->done.end()) {
      Result r = it->second;
      b->done.erase(it);
      b->live.erase(ticket);
      if (r.status != GC_OK) {
        set_error("batch launch failed");
        return r.status;
      }
      bool need_hi = false;
      for (int i = 0; i < 17; ++i) {
        global_out[i] = r.x[2 * i];
        if (global_hi) global_hi[i] = r.x[2 * i + 1];
        if (r.x[2 * i + 1]) need_hi = true;
      }
      if (need_hi && !global_hi) {
        set_error("a global count exceeds 64 bits and global_hi is NULL");
        return GC_ERR_OVERFLOW;
      }
      return GC_OK;
    }
    if (timeout_us == 0) return GC_PENDING;
    if (timeout_us > 0 && std::chrono::steady_clock::now() >= deadline) return GC_PENDING;
    b->cv.wait_for(lk, std::chrono::microseconds(50));
  }
}

gc_status gc_batch_poll_many(gc_batch b, int64_t G, const uint64_t* tickets, uint64_t* global_out,
                             uint64_t* global_hi, int32_t timeout_us) {
  if (!b || G < 0 || (G > 0 && (!tickets || !global_out))) { set_error("bad arguments"); return GC_ERR_ARG; }
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us > 0 ? timeout_us : 0);
  std::unique_lock<std::mutex> lk(b->mu);
  for (int64_t i = 0; i < G; ++i)
    if (!b->live.count(tickets[i])) {
      set_error("ticket " + std::to_string(i) + " is unknown or retired");
      return GC_ERR_ARG;
    }
  int64_t ready = 0;  // tickets[0 .. ready) are known to be done
  for (;;) {
    if (b->flags & GC_BATCH_MANUAL) retire_locked(b);
    while (ready < G && b->done.count(tickets[ready])) ++ready;
    if (ready == G) break;
    if (timeout_us == 0) return GC_PENDING;
    if (timeout_us > 0 && std::chrono::steady_clock::now() >= deadline) return GC_PENDING;
    b->cv.wait_for(lk, std::chrono::microseconds(50));
  }
  gc_status first = GC_OK;
  bool need_hi = false;
  for (int64_t i = 0; i < G; ++i) {
    auto it = b->done.find(tickets[i]);
    const Result r = it->second;
    b->done.erase(it);
    b->live.erase(tickets[i]);
    if (r.status != GC_OK && first == GC_OK) {
      first = r.status;
      set_error("the launch of ticket " + std::to_string(i) + " failed");
    }
    for (int k = 0; k < 17; ++k) {
      global_out[17 * i + k] = r.x[2 * k];
      if (global_hi) global_hi[17 * i + k] = r.x[2 * k + 1];
      if (r.x[2 * k + 1]) need_hi = true;
    }
  }
  if (first != GC_OK) return first;
  if (need_hi && !global_hi) {
    set_error("a global count exceeds 64 bits and global_hi is NULL");
    return GC_ERR_OVERFLOW;
  }
  return GC_OK;
}

gc_status gc_batch_destroy(gc_batch b) {
  if (!b) return GC_OK;
  {
    std::lock_guard<std::mutex> lk(b->mu);
    b->stop = true;
  }
  b->cv.notify_all();
  if (b->dispatcher.joinable()) b->dispatcher.join();
  for (auto& s : b->streams) cudaStreamSynchronize(s);
  {
    std::lock_guard<std::mutex> lk(b->mu);
    retire_locked(b);
  }
  for (auto& sb : b->small) free_small_bufs(&sb);
  for (auto& s : b->streams) cudaStreamDestroy(s);
  delete b;
  return GC_OK;
}

}  // extern "C"
