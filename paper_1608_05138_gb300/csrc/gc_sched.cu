// gc_sched.cu -- balanced work units for the clique/cycle pass.
//
// Per-edge work is power-law distributed (Fig. 1): on skewed graphs a few
// v-groups (hub high endpoints) carry several times a CTA's fair share, and a
// persistent grid that hands out whole groups waits on them. The paper splits
// heavy jobs into finer independent sub-jobs (Sec. 4.5, splitting T or S_u).
// Here, once pass A has produced |T| for every edge, each v-group is cut into
// contiguous slot ranges of Gamma(v) with about equal estimated work; every
// chunk rebuilds Psi for v (cost about 2 d_v), so a group is cut into at most
// W_v / (2 d_v) chunks. Chunks keep the heaviest-first order
// of the groups (the queue Pi).
#include <cuda_runtime.h>

#include <cstdlib>
#include <cstring>

#include "gc_internal.h"

namespace gc {
namespace {

// Estimated pass-B work of one edge: the scan of Gamma(u) plus the 4-clique
// intersections over T (about |T| * min(|T|, out-degree)).
__device__ __forceinline__ long long edge_cost(int32_t du, int32_t t) {
  return 16LL + (long long)du + (long long)t * (long long)min(t, 64);
}

__device__ __forceinline__ bool rank_less(const int32_t* __restrict__ deg, int32_t a, int32_t b) {
  int32_t da = deg[a], db = deg[b];
  return da < db || (da == db && a < b);
}

__global__ void k_group_work(DevGraph g, const int32_t* __restrict__ units, int32_t n_units,
                             const int32_t* __restrict__ tri, long long* __restrict__ W,
                             unsigned long long* __restrict__ total, int32_t* __restrict__ n_big, int32_t big_t) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int32_t k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n_units; k += warps) {
    const int32_t v = units[k];
    long long w = 0;
    int big = 0;
    for (int32_t p = g.rp[v] + lane; p < g.rp[v + 1]; p += 32) {
      const int32_t u = g.ci[p];
      if (rank_less(g.deg, u, v)) {
        const int32_t t = tri[g.eid[p]];
        if (t > big_t) ++big; else w += edge_cost(g.deg[u], t);  // large-T edges go to their own pass
      }
    }
    for (int o = 16; o; o >>= 1) {
      w += __shfl_xor_sync(0xffffffffu, w, o);
      big += __shfl_xor_sync(0xffffffffu, big, o);
    }
    w += 16;
    if (lane == 0) {
      W[k] = w;
      atomicAdd(total, (unsigned long long)w);
      if (big) atomicAdd(n_big, big);
    }
  }
}

__global__ void k_chunk_count(const int32_t* __restrict__ units, int32_t n_units,
                              const long long* __restrict__ W, const int32_t* __restrict__ deg,
                              long long U, int32_t* __restrict__ nch) {
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n_units; k += gridDim.x * blockDim.x) {
    const long long w = W[k];
    const long long sv = 2LL * deg[units[k]] + 64;  // Psi rebuild + clear per chunk
    long long c = (w + U - 1) / U;
    long long cap = w / sv;
    if (cap < 1) cap = 1;
    if (c > cap) c = cap;
    if (c > 4096) c = 4096;
    nch[k] = (int32_t)(c < 1 ? 1 : c);
  }
}

// Warp per group: cut its slots where the running cost crosses j * W / nc.
__global__ void k_chunk_emit(DevGraph g, const int32_t* __restrict__ units, int32_t n_units,
                             const int32_t* __restrict__ tri, const long long* __restrict__ W,
                             const int32_t* __restrict__ off, int32_t* __restrict__ chunks, int32_t big_t) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int32_t k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n_units; k += warps) {
    const int32_t v = units[k];
    const int32_t b = g.rp[v], e = g.rp[v + 1];
    const int32_t base = off[k];
    const long long nc = off[k + 1] - base;
    if (lane == 0) {
      chunks[3 * base] = v;
      chunks[3 * base + 1] = b;
      chunks[3 * (base + nc - 1) + 2] = e;
    }
    if (nc == 1) continue;
    const long long Wk = W[k];
    for (int32_t j = 1 + lane; j < nc; j += 32) chunks[3 * (base + j)] = v;
    long long running = 0;
    for (int32_t p0 = b; p0 < e; p0 += 32) {
      const int32_t p = p0 + lane;
      long long c = 0;
      if (p < e) {
        const int32_t u = g.ci[p];
        if (rank_less(g.deg, u, v)) {
          const int32_t t = tri[g.eid[p]];
          c = t > big_t ? 0 : edge_cost(g.deg[u], t);
        }
      }
      if (p == e - 1) c += 16;  // matches the constant added to W
      long long incl = c;
      for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const long long X = running + incl, Y = running + incl - c;
      // boundaries j with Y < floor(j W / nc) <= X end chunk j-1 after slot p
      long long jlo = ((Y + 1) * nc + Wk - 1) / Wk;
      long long jhi = ((X + 1) * nc + Wk - 1) / Wk - 1;
      if (jlo < 1) jlo = 1;
      if (jhi > nc - 1) jhi = nc - 1;
      for (long long j = jlo; j <= jhi; ++j) {
        chunks[3 * (base + j) + 1] = p + 1;
        chunks[3 * (base + j - 1) + 2] = p + 1;
      }
      running += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
}

}  // namespace

int chunk_factor() {
  static int v = [] {
    const char* e = getenv("GC_CHUNK_FACTOR");
    int x = e ? atoi(e) : 8;
    return x < 1 ? 1 : (x > 256 ? 256 : x);
  }();
  return v;
}

int order_key() {
  static int v = [] {
    const char* e = getenv("GC_ORDER");
    if (!e) return 0;
    if (!strcmp(e, "deg")) return 1;
    if (!strcmp(e, "none")) return 2;
    return 0;
  }();
  return v;
}

namespace {

int blocks_for(long long threads) {
  long long b = (threads + 255) / 256;
  if (b < 1) b = 1;
  if (b > 65535LL * 8) b = 65535LL * 8;
  return (int)b;
}

}  // namespace

gc_status run_make_chunks(const DevGraph& g, const int32_t* units, int32_t n_units,
                          const int32_t* tri, int32_t* chunks, int32_t* off,
                          unsigned long long* total_dev, int32_t* n_big_dev, int32_t big_t, cudaStream_t s) {
  long long* W = nullptr;
  int32_t* nch = nullptr;
  cudaError_t e = cudaMallocAsync(&W, sizeof(long long) * (n_units > 0 ? n_units : 1), s);
  if (e != cudaSuccess) return cuda_fail(e, "alloc chunk scratch");
  e = cudaMallocAsync(&nch, sizeof(int32_t) * (n_units > 0 ? n_units : 1), s);
  if (e != cudaSuccess) {
    cudaFreeAsync(W, s);
    return cuda_fail(e, "alloc chunk scratch");
  }
  gc_status st = GC_OK;
  unsigned long long total = 0;
  const int grid = count_grid_size();
  cudaMemsetAsync(total_dev, 0, sizeof(unsigned long long), s);
  k_group_work<<<blocks_for((long long)n_units * 32), 256, 0, s>>>(g, units, n_units, tri, W, total_dev,
                                                                    n_big_dev, big_t);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&total, total_dev, sizeof(total), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    st = cuda_fail(e, "chunk work");
  } else {
    // ceil so that sum_k ceil(W_k / U) <= n_units + chunk_factor * grid
    const unsigned long long per = (unsigned long long)chunk_factor() * (unsigned long long)grid;
    long long U = (long long)((total + per - 1) / per);
    if (U < 1) U = 1;
    k_chunk_count<<<blocks_for(n_units), 256, 0, s>>>(units, n_units, W, g.deg, U, nch);
    e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_fail(e, "k_chunk_count");
    if (st == GC_OK) st = exclusive_scan(n_units, nch, off, s);  // off[n_units] = number of chunks
    if (st == GC_OK) {
      k_chunk_emit<<<blocks_for((long long)n_units * 32), 256, 0, s>>>(g, units, n_units, tri, W,
                                                                       off, chunks, big_t);
      e = cudaGetLastError();
      if (e != cudaSuccess) st = cuda_fail(e, "k_chunk_emit");
    }
  }
  cudaFreeAsync(W, s);
  cudaFreeAsync(nch, s);
  return st;
}

}  // namespace gc
