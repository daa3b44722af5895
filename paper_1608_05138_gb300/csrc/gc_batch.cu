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

struct PendingGraph {
  uint64_t ticket;
  int32_t n;
  int64_t m;
  int64_t bytes;
  std::vector<int32_t> rp, ci;
};

struct Result {
  uint64_t x[34];
  gc_status status;
};

struct Launch {
  std::vector<uint64_t> tickets;
  std::vector<int32_t> slot;          // ticket k's row in h_x
  int64_t bytes = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  unsigned long long* h_x = nullptr;  // pinned [G][17][2]
  int32_t* h_status = nullptr;        // pinned
  gc_status launch_status = GC_OK;
  std::string error;
};

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
  cudaStream_t streams[2] = {nullptr, nullptr};
  int next_stream = 0;
  int device = 0;
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
      if (pg.m > 0) std::memcpy(h_ci.data() + eo, pg.ci.data(), sizeof(int32_t) * 2 * pg.m);
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
  GB_TRY(cudaMallocAsync(&d_rp, sizeof(int32_t) * ((size_t)n + 1), s), "batch alloc");
  GB_TRY(cudaMallocAsync(&d_ci, sizeof(int32_t) * h_ci.size(), s), "batch alloc");
  GB_TRY(cudaMallocAsync(&d_vgid, sizeof(int32_t) * h_vgid.size(), s), "batch alloc");
  GB_TRY(cudaMallocAsync(&d_desc, sizeof(int32_t) * h_desc.size(), s), "batch alloc");
  GB_TRY(cudaMallocAsync(&d_gm, sizeof(int64_t) * G, s), "batch alloc");
  GB_TRY(cudaMallocAsync(&d_csum, sizeof(unsigned long long) * (size_t)G * 26, s), "batch alloc");
  GB_TRY(cudaMallocAsync(&d_x, sizeof(unsigned long long) * (size_t)G * 34, s), "batch alloc");
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
    ku.chash_w = prep.chash_w;
    ku.n_chash = prep.n_chash;
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

// Graphs of at most kSmallN vertices: packed as they are (local ids) and
// counted one CTA per graph on a shared-memory bitmatrix.
gc_status run_small(std::vector<PendingGraph*>& graphs, cudaStream_t s, Launch* L, unsigned long long* h_x_dst) {
  const int32_t G = (int32_t)graphs.size();
  std::vector<int64_t> h_voff((size_t)G + 1), h_eoff((size_t)G + 1), h_gm((size_t)G);
  std::vector<int32_t> h_gn((size_t)G), h_order((size_t)G);
  h_voff[0] = h_eoff[0] = 0;
  for (int32_t gi = 0; gi < G; ++gi) {
    h_voff[gi + 1] = h_voff[gi] + graphs[gi]->n + 1;
    h_eoff[gi + 1] = h_eoff[gi] + 2 * graphs[gi]->m;
    h_gn[gi] = graphs[gi]->n;
    h_gm[gi] = graphs[gi]->m;
    h_order[gi] = gi;
  }
  std::sort(h_order.begin(), h_order.end(), [&](int32_t a, int32_t b) { return h_gm[a] > h_gm[b]; });
  // packed on all host cores into buffers that are not zeroed first (every
  // entry is copied over)
  struct Packed {
    std::unique_ptr<int32_t[]> p;
    size_t n;
    int32_t* data() { return p.get(); }
    size_t size() const { return n; }
  } h_rp{std::unique_ptr<int32_t[]>(new int32_t[(size_t)h_voff[G] + 1]), (size_t)h_voff[G] + 1},
    h_ci{std::unique_ptr<int32_t[]>(new int32_t[(size_t)(h_eoff[G] > 0 ? h_eoff[G] : 1)]),
         (size_t)(h_eoff[G] > 0 ? h_eoff[G] : 1)};
  {
    const unsigned hw = std::thread::hardware_concurrency();
    const int nt = h_eoff[G] < (1 << 22) ? 1 : (int)std::min<unsigned>(hw ? hw : 1, 32);
    auto pack = [&](int t) {  // the graphs whose entries start in this thread's share
      const int64_t e0 = h_eoff[G] * t / nt, e1 = h_eoff[G] * (t + 1) / nt;
      int32_t gi = (int32_t)(std::lower_bound(h_eoff.begin(), h_eoff.begin() + G, e0) - h_eoff.begin());
      for (; gi < G && (h_eoff[gi] < e1 || t == nt - 1); ++gi) {
        std::memcpy(h_rp.data() + h_voff[gi], graphs[gi]->rp.data(), sizeof(int32_t) * (graphs[gi]->n + 1));
        if (graphs[gi]->m > 0)
          std::memcpy(h_ci.data() + h_eoff[gi], graphs[gi]->ci.data(), sizeof(int32_t) * 2 * graphs[gi]->m);
      }
    };
    std::vector<std::thread> th;
    for (int t = 1; t < nt; ++t) th.emplace_back(pack, t);
    pack(0);
    for (auto& x : th) x.join();
  }
  int32_t *d_rp = nullptr, *d_ci = nullptr, *d_gn = nullptr, *d_order = nullptr, *d_misc = nullptr;
  int64_t *d_voff = nullptr, *d_eoff = nullptr, *d_gm = nullptr;
  unsigned long long *d_csum = nullptr, *d_x = nullptr;
  cudaError_t e = cudaSuccess;
  gc_status st = GC_OK;
#define GS_TRY(call, what)                   \
  do {                                       \
    e = (call);                              \
    if (e != cudaSuccess) {                  \
      st = cuda_fail(e, what);               \
      L->error = gc_last_error();            \
      goto out;                              \
    }                                        \
  } while (0)
  GS_TRY(cudaMallocAsync(&d_rp, sizeof(int32_t) * h_rp.size(), s), "small alloc");
  GS_TRY(cudaMallocAsync(&d_ci, sizeof(int32_t) * h_ci.size(), s), "small alloc");
  GS_TRY(cudaMallocAsync(&d_voff, sizeof(int64_t) * h_voff.size(), s), "small alloc");
  GS_TRY(cudaMallocAsync(&d_eoff, sizeof(int64_t) * h_eoff.size(), s), "small alloc");
  GS_TRY(cudaMallocAsync(&d_gn, sizeof(int32_t) * G, s), "small alloc");
  GS_TRY(cudaMallocAsync(&d_gm, sizeof(int64_t) * G, s), "small alloc");
  GS_TRY(cudaMallocAsync(&d_order, sizeof(int32_t) * G, s), "small alloc");
  GS_TRY(cudaMallocAsync(&d_misc, sizeof(int32_t) * 2, s), "small alloc");
  GS_TRY(cudaMallocAsync(&d_csum, sizeof(unsigned long long) * (size_t)G * 26, s), "small alloc");
  GS_TRY(cudaMallocAsync(&d_x, sizeof(unsigned long long) * (size_t)G * 34, s), "small alloc");
  GS_TRY(cudaMemcpyAsync(d_rp, h_rp.data(), sizeof(int32_t) * h_rp.size(), cudaMemcpyHostToDevice, s), "small copy");
  GS_TRY(cudaMemcpyAsync(d_ci, h_ci.data(), sizeof(int32_t) * h_ci.size(), cudaMemcpyHostToDevice, s), "small copy");
  GS_TRY(cudaMemcpyAsync(d_voff, h_voff.data(), sizeof(int64_t) * h_voff.size(), cudaMemcpyHostToDevice, s),
         "small copy");
  GS_TRY(cudaMemcpyAsync(d_eoff, h_eoff.data(), sizeof(int64_t) * h_eoff.size(), cudaMemcpyHostToDevice, s),
         "small copy");
  GS_TRY(cudaMemcpyAsync(d_gn, h_gn.data(), sizeof(int32_t) * G, cudaMemcpyHostToDevice, s), "small copy");
  GS_TRY(cudaMemcpyAsync(d_gm, h_gm.data(), sizeof(int64_t) * G, cudaMemcpyHostToDevice, s), "small copy");
  GS_TRY(cudaMemcpyAsync(d_order, h_order.data(), sizeof(int32_t) * G, cudaMemcpyHostToDevice, s), "small copy");
  GS_TRY(cudaMemsetAsync(d_misc, 0, sizeof(int32_t) * 2, s), "small memset");
  GS_TRY(cudaMemsetAsync(d_csum, 0, sizeof(unsigned long long) * (size_t)G * 26, s), "small memset");
  if ((st = run_small_graphs(d_rp, d_voff, d_ci, d_eoff, d_order, G, d_misc, d_csum, s)) != GC_OK) {
    L->error = gc_last_error();
    goto out;
  }
  {
    DevGraph dg = DevGraph();
    dg.G = G;
    dg.gn = d_gn;
    dg.gm = d_gm;
    if ((st = run_derive(dg, d_csum, d_x, d_misc + 1, s)) != GC_OK) {
      L->error = gc_last_error();
      goto out;
    }
  }
  GS_TRY(cudaMemcpyAsync(h_x_dst, d_x, sizeof(unsigned long long) * (size_t)G * 34, cudaMemcpyDeviceToHost, s),
         "small copy out");
out:
#undef GS_TRY
  for (void* p : {(void*)d_rp, (void*)d_ci, (void*)d_voff, (void*)d_eoff, (void*)d_gn, (void*)d_gm, (void*)d_order,
                  (void*)d_misc, (void*)d_csum, (void*)d_x})
    if (p) cudaFreeAsync(p, s);
  return st;
}

// Counts `graphs` as one launch on `s`: small graphs on the bitmatrix kernel,
// the others as one disjoint union. Results land in L->h_x when L->done
// completes. Runs in the dispatcher thread (or the flushing thread in manual
// mode) without holding the batch lock.
void run_launch(std::vector<PendingGraph>& graphs, cudaStream_t s, Launch* L) {
  std::vector<PendingGraph*> small, large;
  for (auto& pg : graphs) (pg.n <= kSmallN ? small : large).push_back(&pg);
  L->slot.resize(graphs.size());
  {
    int32_t is = 0, il = (int32_t)small.size();
    for (size_t k = 0; k < graphs.size(); ++k) L->slot[k] = graphs[k].n <= kSmallN ? is++ : il++;
  }
  gc_status st = GC_OK;
  L->h_status[0] = 0;
  if (!small.empty()) st = run_small(small, s, L, L->h_x);
  if (st == GC_OK && !large.empty()) st = run_union(large, s, L, L->h_x + 34 * small.size(), L->h_status);
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
    for (size_t k = 0; k < L->tickets.size(); ++k) {
      Result r;
      if (L->launch_status == GC_OK) {
        std::memcpy(r.x, L->h_x + 34 * (size_t)L->slot[k], sizeof(r.x));
        int32_t dst = *L->h_status;
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
    L->stream = b->streams[b->next_stream];
    b->next_stream ^= 1;
  }
  cudaSetDevice(b->device);
  cudaError_t e1 = cudaMallocHost(&L->h_x, sizeof(unsigned long long) * 34 * take.size());
  cudaError_t e2 = cudaMallocHost(&L->h_status, sizeof(int32_t));
  cudaError_t e3 = cudaEventCreateWithFlags(&L->done, cudaEventDisableTiming);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
    L->launch_status = GC_ERR_NOMEM;
  } else {
    run_launch(take, L->stream, L);
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
    if (!b->pending.empty() && b->inflight.size() < 2) {
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
  if (!(flags & GC_BATCH_MANUAL)) b->dispatcher = std::thread(dispatcher_main, b);
  *out = b;
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
  pg.rp.assign(row_ptr, row_ptr + n + 1);
  if (m > 0) pg.ci.assign(col_idx, col_idx + 2 * m);
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
  std::vector<PendingGraph> pgs((size_t)G);
  unsigned hw = std::thread::hardware_concurrency();
  const int nt = (int)std::min<int64_t>(std::max(1u, std::min(hw, 32u)), G);
  std::vector<gc_status> res(nt, GC_OK);
  std::vector<std::string> msg(nt);
  auto work = [&](int t) {
    for (int64_t g = t; g < G; g += nt) {
      const int32_t n = nvert[g];
      const int32_t* rp = row_ptr + voff[g];
      const int32_t* ci = col_idx ? col_idx + eoff[g] : nullptr;
      if (n < 0 || (int64_t)rp[n] != eoff[g + 1] - eoff[g]) {
        res[t] = GC_ERR_ARG;
        msg[t] = "graph " + std::to_string(g) + ": offsets disagree with row_ptr";
        return;
      }
      gc_status st = validate_csr(n, rp, ci);
      if (st != GC_OK) {
        res[t] = st;
        msg[t] = "graph " + std::to_string(g) + ": " + gc_last_error();
        return;
      }
      PendingGraph& pg = pgs[(size_t)g];
      pg.n = n;
      pg.m = rp[n] / 2;
      pg.bytes = footprint(n, pg.m);
      pg.rp.assign(rp, rp + n + 1);
      if (pg.m > 0) pg.ci.assign(ci, ci + 2 * pg.m);
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
  for (auto& s : b->streams) cudaStreamDestroy(s);
  delete b;
  return GC_OK;
}

}  // extern "C"
