// gc_prep.cu -- one-time device preparation of an uploaded graph.
//
//   * degrees d_x and the P3 orientation of every edge (Sec. 4.3): the "low"
//     endpoint u has the smaller (degree, id) pair, the "high" endpoint v the
//     larger, so d_v >= d_u;
//   * edge ids (rank of (u, v), u < v, in row-major upper-triangle order) and
//     the slot -> edge id map of both CSR directions;
//   * degree-oriented out-lists: out(x) = neighbours of higher (degree, id)
//     rank, ascending ids. Each pair {a, b} of adjacent vertices appears in
//     exactly one out-list; the 4-clique step uses this to count each pair
//     of T once (the role of the Psi reset in Alg. 5);
//   * the work units of the counting passes: every vertex v that is the high
//     endpoint of at least one edge forms one "v-group" (its low neighbours);
//     groups are binned by floor(log2(estimated work)) and listed heaviest
//     bin first -- the difficulty-ordered edge queue Pi of Sec. 4.4 at group
//     granularity, with d_v + sum_{r in Gamma(v)} d_r as the work estimate
//     (a vertex analogue of the vol ordering of Table 4).
#include <cuda_runtime.h>

#include <cmath>

#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <vector>

#include "gc_internal.h"

namespace gc {
namespace {

constexpr int kScanTile = 2048;  // elements per scan tile (256 threads x 8)

__device__ __forceinline__ bool rank_less(const int32_t* deg, int32_t a, int32_t b) {
  int32_t da = deg[a], db = deg[b];
  return da < db || (da == db && a < b);
}

// first index in [lo, hi) with a[i] >= key
__device__ __forceinline__ int32_t lower_bound_i32(const int32_t* a, int32_t lo, int32_t hi,
                                                   int32_t key) {
  while (lo < hi) {
    int32_t mid = lo + ((hi - lo) >> 1);
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void k_deg_up(int32_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                         int32_t* __restrict__ deg, int32_t* __restrict__ up) {
  for (int32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
    int32_t b = rp[x], e = rp[x + 1];
    deg[x] = e - b;
    up[x] = e - lower_bound_i32(ci, b, e, x + 1);
  }
}

// Warp per vertex: number of higher-rank neighbours, sum of neighbour degrees,
// maximum degree.
__global__ void k_out_cnt(int32_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                          const int32_t* __restrict__ deg, int32_t* __restrict__ out_cnt,
                          long long* __restrict__ S, int32_t* __restrict__ dmax, int32_t* __restrict__ kmax) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int32_t x = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n; x += warps) {
    int32_t b = rp[x], e = rp[x + 1];
    int32_t c = 0;
    long long s = 0;
    for (int32_t p = b + lane; p < e; p += 32) {
      int32_t y = ci[p];
      c += rank_less(deg, x, y) ? 1 : 0;
      s += deg[y];
    }
    for (int o = 16; o; o >>= 1) {
      c += __shfl_xor_sync(0xffffffffu, c, o);
      s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    if (lane == 0) {
      out_cnt[x] = c;
      S[x] = s;
      if (e - b > 0) atomicMax(dmax, e - b);
      if (c > 0) atomicMax(kmax, c);
    }
  }
}

// Warp per vertex: edge ids of every slot, edge list, out-lists, and the
// out-slot of every edge id.
__global__ void k_edges(int32_t n, int32_t m, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                        const int32_t* __restrict__ deg, const int32_t* __restrict__ up,
                        const int32_t* __restrict__ upoff, const int32_t* __restrict__ out_ptr,
                        int32_t* __restrict__ eid, int32_t* __restrict__ uv,
                        int32_t* __restrict__ out_idx, int32_t* __restrict__ ocsr, int32_t* __restrict__ rev,
                        int32_t* __restrict__ e2o, bool write_ids, const int32_t* __restrict__ perm) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int32_t x = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n; x += warps) {
    const int32_t b = rp[x], e = rp[x + 1];
    const int32_t first_up = e - up[x];
    int32_t o = out_ptr[x];
    for (int32_t base = b; base < e; base += 32) {
      int32_t p = base + lane;
      bool valid = p < e;
      int32_t y = valid ? ci[p] : 0;
      bool is_out = valid && rank_less(deg, x, y);
      int32_t qr = -1;  // ids given: the reverse slot, once found
      if (valid && write_ids) {  // the slot of (y, x); the ids below take the same search
        const int32_t yb = rp[y], ye = rp[y + 1];
        const int32_t q = lower_bound_i32(ci, yb, ye, x);
        rev[p] = (q < ye && ci[q] == x) ? q : p;  // p itself only for invalid input
      } else if (valid && y > x) {  // ids given: one search per edge, from its lower end, sets both
        const int32_t yb = rp[y], ye = rp[y + 1];
        const int32_t q = lower_bound_i32(ci, yb, ye, x);
        if (q < ye && ci[q] == x) {
          rev[p] = q;
          rev[q] = p;
          qr = q;
        }  // else both keep rev = self (k_rev_init): no reverse, invalid input
      }
      int32_t id = 0;
      if (valid && write_ids) {
        if (y > x) {
          id = upoff[x] + (p - first_up);
          uv[2 * (int64_t)id] = x;
          uv[2 * (int64_t)id + 1] = y;
        } else {
          int32_t yb = rp[y], ye = rp[y + 1];
          int32_t q = lower_bound_i32(ci, yb, ye, x);  // x is in row y (symmetry)
          id = (q < ye && ci[q] == x) ? upoff[y] + (q - (ye - up[y])) : 0;  // 0 only for invalid input
        }
        eid[p] = id;
      }
      unsigned mask = __ballot_sync(0xffffffffu, is_out);
      if (is_out) {
        const int32_t os = o + __popc(mask & ((1u << lane) - 1u));
        out_idx[os] = y;
        ocsr[os] = p;
        // ids given (ids are ranks, so an out-slot is the slot searched from):
        // the relabel wrote the id of the slot whose caller labels ascend;
        // the other slot of the edge takes it here
        int32_t ide = id;
        if (!write_ids) {
          if (qr >= 0 && perm[x] > perm[y]) {
            ide = eid[qr];
            eid[p] = ide;
          } else {
            ide = eid[p];
            if (qr >= 0) eid[qr] = ide;
          }
        }
        if ((uint32_t)ide < (uint32_t)m) e2o[ide] = os;  // out of range only for invalid input
      }
      o += __popc(mask);
    }
  }
}

// rev[p] = p for every slot, before k_edges searches each edge once: a slot
// that no search reaches keeps it (it has no reverse).
__global__ void k_rev_init(int64_t nnz, int32_t* __restrict__ rev) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x)
    rev[p] = (int32_t)p;
}

// Edge list in the caller's labels when the graph was relabelled.
__global__ void k_uv_perm(int32_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                          const int32_t* __restrict__ eid, const int32_t* __restrict__ perm,
                          int32_t* __restrict__ uv) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int32_t x = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n; x += warps) {
    const int32_t px = perm[x];
    for (int32_t p = rp[x] + lane; p < rp[x + 1]; p += 32) {
      const int32_t y = ci[p];
      if (y < x) continue;
      const int32_t py = perm[y];
      const int64_t e = eid[p];
      uv[2 * e] = px < py ? px : py;
      uv[2 * e + 1] = px < py ? py : px;
    }
  }
}

__device__ __forceinline__ int bin_of(long long cost) {
  return cost <= 1 ? 0 : 63 - __clzll(cost);
}

// Bin key of a v-group under the chosen ordering (0 vol, 1 degree, 2 none).
__device__ __forceinline__ int unit_bin(int key, long long S, int32_t d) {
  return key == 0 ? bin_of(S + d) : (key == 1 ? bin_of(d) : 0);
}

__global__ void k_bin_hist(int32_t n, const int32_t* __restrict__ deg,
                           const int32_t* __restrict__ out_cnt, const long long* __restrict__ S,
                           int32_t* __restrict__ hist, int key) {
  __shared__ int32_t h[64];
  if (threadIdx.x < 64) h[threadIdx.x] = 0;
  __syncthreads();
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    if (deg[v] - out_cnt[v] > 0) atomicAdd(&h[unit_bin(key, S[v], deg[v])], 1);
  }
  __syncthreads();
  if (threadIdx.x < 64 && h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

__global__ void k_bin_scatter(int32_t n, const int32_t* __restrict__ deg,
                              const int32_t* __restrict__ out_cnt,
                              const long long* __restrict__ S, int32_t* __restrict__ cursor,
                              int32_t* __restrict__ units, int key) {
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    if (deg[v] - out_cnt[v] > 0) {
      int32_t pos = atomicAdd(&cursor[unit_bin(key, S[v], deg[v])], 1);
      units[pos] = v;
    }
  }
}

// Pass K units: every vertex a with |out(a)| = k >= 2 (a triangle needs two
// higher-rank neighbours), binned by ceil(log2 k) and listed largest bin
// first, so that the tiers of pass K (k > 1024, <= 1024, <= 512, <= 256,
// <= 32) are contiguous ranges of the list.
__device__ __forceinline__ int kbin_of(int32_t k) { return 32 - __clz(k - 1); }

__global__ void k_kbin_hist(int32_t n, const int32_t* __restrict__ out_cnt, int32_t* __restrict__ hist) {
  __shared__ int32_t h[32];
  if (threadIdx.x < 32) h[threadIdx.x] = 0;
  __syncthreads();
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    if (out_cnt[v] >= 2) atomicAdd(&h[kbin_of(out_cnt[v])], 1);
  __syncthreads();
  if (threadIdx.x < 32 && h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

__global__ void k_kbin_scatter(int32_t n, const int32_t* __restrict__ out_cnt, int32_t* __restrict__ cursor,
                               int32_t* __restrict__ units) {
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    if (out_cnt[v] >= 2) units[atomicAdd(&cursor[kbin_of(out_cnt[v])], 1)] = v;
}

// Wedges of every pass-C unit h of a ranked graph: W_h = sum over the
// lower-rank neighbours x of h of |{o in Gamma(x) : o < h}| (warp per unit).
// Wedges W and lower neighbours NX of every pass-C unit h of a ranked graph.
// Ids are ranks and rows ascend, so the o < h of Gamma(x) are the entries
// before the slot of (x, h), the reverse of the slot of (h, x): no search per
// lower neighbour (the reverse is clamped into the row, as the hub kernel does,
// so that W is what the kernels count even before symmetry is checked).
__global__ void k_cwork(int32_t n_units, const int32_t* __restrict__ units, const int32_t* __restrict__ rp,
                        const int32_t* __restrict__ ci, const int32_t* __restrict__ rev, long long* __restrict__ W,
                        int32_t* __restrict__ NX) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int32_t k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n_units; k += warps) {
    const int32_t h = units[k];
    const int32_t hb = rp[h];
    const int32_t nx = lower_bound_i32(ci, hb, rp[h + 1], h) - hb;
    long long w = 0;
    for (int32_t i = lane; i < nx; i += 32) {
      const int32_t x = ci[hb + i];
      const int32_t xb = rp[x];
      w += min(max(rev[hb + i], xb), rp[x + 1]) - xb;
    }
    for (int o = 16; o; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (lane == 0) {
      W[k] = w;
      NX[k] = nx;
    }
  }
}

// Smallest slot whose reverse was not found (rev[p] == p): the input is not
// symmetric exactly when there is one.
__global__ void k_first_unreversed(int64_t nnz, const int32_t* __restrict__ rev, int32_t* __restrict__ first) {
  int32_t best = 0x7fffffff;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x)
    if (rev[p] == (int32_t)p) best = min(best, (int32_t)p);
  for (int o = 16; o; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0 && best != 0x7fffffff) atomicMin(first, best);
}

// ---- exclusive scan of int32 (totals fit int32) ----
__global__ void k_scan_tile_sums(int32_t n, const int32_t* __restrict__ in, int32_t* __restrict__ sums) {
  __shared__ int32_t ws[8];
  int32_t base = blockIdx.x * kScanTile;
  int32_t s = 0;
  for (int i = threadIdx.x; i < kScanTile; i += blockDim.x) {
    int32_t k = base + i;
    if (k < n) s += in[k];
  }
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    sums[blockIdx.x] = t;
  }
}

// single block: exclusive scan of the tile sums in place
__global__ void k_scan_sums(int32_t nb, int32_t* __restrict__ sums) {
  __shared__ int32_t ws[32];
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int32_t base = 0; base < nb; base += blockDim.x) {
    int32_t k = base + threadIdx.x;
    int32_t v = k < nb ? sums[k] : 0;
    int32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
      int32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
      int32_t t = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      ws[lane] = t;
    }
    __syncthreads();
    int32_t pre = (w > 0 ? ws[w - 1] : 0) + x - v + carry;
    if (k < nb) sums[k] = pre;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = pre + v;
    __syncthreads();
  }
}

// out[k] = exclusive prefix, out[n] = total
__global__ void k_scan_tiles(int32_t n, const int32_t* __restrict__ in,
                             const int32_t* __restrict__ sums, int32_t* __restrict__ out) {
  __shared__ int32_t ws[8];
  const int per = kScanTile / 256;  // 8 consecutive elements per thread
  int32_t base = blockIdx.x * kScanTile + threadIdx.x * per;
  int32_t v[per];
  int32_t t = 0;
  for (int i = 0; i < per; ++i) {
    int32_t k = base + i;
    v[i] = k < n ? in[k] : 0;
    t += v[i];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t x = t;
  for (int o = 1; o < 32; o <<= 1) {
    int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    int32_t s = lane < 8 ? ws[lane] : 0;
    for (int o = 1; o < 8; o <<= 1) {
      int32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < 8) ws[lane] = s;
  }
  __syncthreads();
  int32_t run = sums[blockIdx.x] + (w > 0 ? ws[w - 1] : 0) + x - t;
  for (int i = 0; i < per; ++i) {
    int32_t k = base + i;
    if (k < n) out[k] = run;
    run += v[i];
    if (k == n - 1) out[n] = run;
  }
}

int grid_for(int64_t work, int block) {
  int64_t g = (work + block - 1) / block;
  if (g < 1) g = 1;
  if (g > 65535LL * 16) g = 65535LL * 16;
  return (int)g;
}

}  // namespace

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

gc_status exclusive_scan(int32_t n, const int32_t* in, int32_t* out, cudaStream_t s) {
  if (n == 0) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(int32_t), s);
    return e == cudaSuccess ? GC_OK : cuda_fail(e, "scan memset");
  }
  int32_t nb = (n + kScanTile - 1) / kScanTile;
  int32_t* sums = nullptr;
  cudaError_t e = pool_alloc(&sums, sizeof(int32_t) * nb, s);
  if (e != cudaSuccess) return cuda_fail(e, "scan alloc");
  k_scan_tile_sums<<<nb, 256, 0, s>>>(n, in, sums);
  k_scan_sums<<<1, 1024, 0, s>>>(nb, sums);
  k_scan_tiles<<<nb, 256, 0, s>>>(n, in, sums, out);
  e = cudaGetLastError();
  cudaFreeAsync(sums, s);
  return e == cudaSuccess ? GC_OK : cuda_fail(e, "scan launch");
}

// Jobs per CTA of the hub kernel the hub units are cut into (environment
// GC_HUB_JOBS_PER_CTA, 0 .. 64, default 1; 0 keeps one job per hub), read
// once per process. With 1, only a hub that costs more than a whole CTA's
// share of the work is cut: a new job has to seed every lower neighbour's
// cursor with a galloping search (milliseconds for the largest hubs), and
// heaviest-first stealing already balances hubs below that size (on R-MAT
// scale 22 the CTAs' lifetimes differ by 0.1 %).
int hub_tab_words() {
  static int v = [] {
    const char* e = getenv("GC_HUB_TAB_WORDS");
    const int x = e ? atoi(e) : kHubTabDefault;
    return (x >= 4096 && x <= kHeavyTab && x % 1024 == 0) ? x : kHubTabDefault;
  }();
  return v;
}

static int hub_jobs_per_cta() {
  static int v = [] {
    const char* e = getenv("GC_HUB_JOBS_PER_CTA");
    const int x = e ? atoi(e) : 1;
    return x < 0 ? 0 : (x > 64 ? 64 : x);
  }();
  return v;
}

// The units of v (wedge counts W[v[i]] in [1, wmax]) in descending W, equal W
// in their order in v: a counting sort.
static void sort_by_wedges_desc(std::vector<int32_t>* v, const std::vector<long long>& W, long long wmax) {
  std::vector<int32_t> cnt((size_t)wmax + 2, 0);
  for (int32_t k : *v) cnt[(size_t)(wmax - W[k])]++;
  int32_t r = 0;
  for (auto& c : cnt) {
    const int32_t x = c;
    c = r;
    r += x;
  }
  std::vector<int32_t> out(v->size());
  for (int32_t k : *v) out[(size_t)cnt[(size_t)(wmax - W[k])]++] = k;
  v->swap(out);
}

gc_status classify_c_units(int32_t n, const int32_t* d_rp, const int32_t* d_ci, bool ranked, PrepBuffers* p,
                           cudaStream_t s) {
  const int32_t nu = p->n_units;
  cudaError_t e = pool_alloc(&p->cunits, sizeof(int32_t) * (nu > 0 ? nu : 1), s);
  if (e != cudaSuccess) return cuda_fail(e, "alloc cunits");
  p->n_cheavy = 0;
  p->n_chash = 0;
  p->n_chash_big = 0;
  p->n_chash_mid = 0;
  p->n_chash2 = 0;
  p->n_chash2_big = 0;
  p->n_cunits = nu;
  p->cnx_max = 0;
  if (!ranked || n <= kSmemTableMax || nu == 0) {
    e = nu > 0 ? cudaMemcpyAsync(p->cunits, p->units, sizeof(int32_t) * nu, cudaMemcpyDeviceToDevice, s) : cudaSuccess;
    return e == cudaSuccess ? GC_OK : cuda_fail(e, "copy cunits");
  }
  long long* dW = nullptr;
  int32_t* dNX = nullptr;
  std::vector<long long> W(nu);
  std::vector<int32_t> NX(nu), U(nu), out;
  e = pool_alloc(&dW, sizeof(long long) * nu, s);
  if (e == cudaSuccess) e = pool_alloc(&dNX, sizeof(int32_t) * nu, s);
  if (e == cudaSuccess) {
    k_cwork<<<grid_for((int64_t)nu * 32, 256), 256, 0, s>>>(nu, p->units, d_rp, d_ci, p->rev, dW, dNX);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(W.data(), dW, sizeof(long long) * nu, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(NX.data(), dNX, sizeof(int32_t) * nu, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(U.data(), p->units, sizeof(int32_t) * nu, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (dW) cudaFreeAsync(dW, s);
  if (dNX) cudaFreeAsync(dNX, s);
  if (e != cudaSuccess) return cuda_fail(e, "classify pass-C units");
  // A hub unit pays, per shared-memory block of the o-range, a few
  // microseconds of barriers and cursor searches (more when it has more than
  // a CTA's worth of lower neighbours), against roughly 10 ns per wedge on an
  // SM for a wedge that goes through the vertex-indexed table in DRAM; the
  // hub kernel is taken when the wedges exceed blocks x max(1024, nx), about
  // three times the break-even point. One pass over the units, in unit
  // order: the packed-key hash takes every unit it fits; the hub rule is
  // tested (with its division) only from 16384 wedges; units without wedges
  // add nothing to P and are left out.
  std::vector<int32_t> heavy, hashed, hashed2, rest;
  const long long tab = hub_tab_words();
  for (int32_t k = 0; k < nu; ++k) {
    const long long w = W[k];
    if (w <= 0) continue;
    if (w <= kHashMaxW) {
      hashed.push_back(k);
      continue;
    }
    if (w <= kHash2MaxW && NX[k] < kHash2MaxNx && n <= kHash2MaxN) {
      hashed2.push_back(k);
      continue;
    }
    if (w >= 16384 && NX[k] < (1 << 26)) {
      const long long span = (long long)hub_cpw(NX[k]) * tab;
      const long long blocks = ((long long)U[k] + span - 1) / span;
      const long long per_block = NX[k] > 1024 ? NX[k] : 1024;
      if (w >= blocks * per_block) {
        heavy.push_back(k);
        continue;
      }
    }
    rest.push_back(k);
  }
  // hub units heaviest first, then the hashed units heaviest first, the
  // packed-key hash units heaviest first, and the rest in unit order
  std::sort(heavy.begin(), heavy.end(), [&](int32_t a, int32_t b) { return W[a] > W[b]; });
  sort_by_wedges_desc(&hashed, W, kHashMaxW);
  sort_by_wedges_desc(&hashed2, W, kHash2MaxW);
  out.reserve(heavy.size() + hashed.size() + hashed2.size() + rest.size());
  std::vector<int32_t> hw;
  hw.reserve(hashed.size() + hashed2.size());
  for (int32_t k : heavy) {
    out.push_back(U[k]);
    if (NX[k] > p->cnx_max) p->cnx_max = NX[k];
  }
  for (int32_t k : hashed) {
    out.push_back(U[k]);
    hw.push_back((int32_t)W[k]);
  }
  for (int32_t k : hashed2) {
    out.push_back(U[k]);
    hw.push_back((int32_t)W[k]);
  }
  for (int32_t k : rest) out.push_back(U[k]);
  p->n_cheavy = (int32_t)heavy.size();
  p->n_chash = (int32_t)hashed.size();
  p->n_chash_big = 0;  // hashed is heaviest first
  while (p->n_chash_big < p->n_chash && W[hashed[(size_t)p->n_chash_big]] > kHashSmallW) ++p->n_chash_big;
  p->n_chash_mid = 0;
  while (p->n_chash_mid < p->n_chash_big && W[hashed[(size_t)p->n_chash_mid]] > kHashMidW) ++p->n_chash_mid;
  p->n_chash2 = (int32_t)hashed2.size();
  p->n_chash2_big = 0;  // heaviest first too
  while (p->n_chash2_big < p->n_chash2 && W[hashed2[(size_t)p->n_chash2_big]] > kHash2HalfMaxW) ++p->n_chash2_big;
  p->n_cunits = (int32_t)out.size();
  // Hub units cut into jobs of consecutive o-range blocks (the finer
  // granularity of Sec. 4.4: one hub's work spread over several CTAs), so
  // that the heaviest hubs do not end as one SM's serial tail. A unit's cost
  // is estimated as its wedges plus kSweepCost per (lower neighbour, block)
  // sweep; a unit is cut into about cost / target jobs, target = total cost
  // over jobs_per_cta x the hub kernel's CTAs (GC_HUB_JOBS_PER_CTA, default 1;
  // 0: one job per hub). Jobs are taken heaviest first.
  std::vector<int4> jobs;
  {
    constexpr double kSweepCost = 4.0;
    const int per_cta = hub_jobs_per_cta();
    std::vector<double> cost(heavy.size());
    std::vector<long long> nblk(heavy.size());
    double total = 0;
    for (size_t i = 0; i < heavy.size(); ++i) {
      const int32_t k = heavy[i];
      const long long span = (long long)hub_cpw(NX[k]) * hub_tab_words();
      nblk[i] = ((long long)U[k] + span - 1) / span;
      cost[i] = (double)W[k] + kSweepCost * (double)NX[k] * (double)nblk[i];
      total += cost[i];
    }
    const double target = per_cta > 0 ? total / ((double)(count_grid_size() / kCtasPerSm) * per_cta) : 0.0;
    std::vector<std::pair<double, int4>> cj;
    for (size_t i = 0; i < heavy.size(); ++i) {
      long long J = target > 0 ? (long long)std::ceil(cost[i] / target) : 1;
      J = std::max(1LL, std::min(J, nblk[i]));
      const long long nb = (nblk[i] + J - 1) / J;
      for (long long b0 = 0; b0 < nblk[i]; b0 += nb) {
        const long long len = std::min(nb, nblk[i] - b0);
        cj.push_back({cost[i] * (double)len / (double)nblk[i], make_int4((int)i, (int)b0, (int)len, 0)});
      }
    }
    std::stable_sort(cj.begin(), cj.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    jobs.reserve(cj.size());
    for (auto& c : cj) jobs.push_back(c.second);
  }
  p->n_cjobs = (int32_t)jobs.size();
  if (!jobs.empty()) {
    e = pool_alloc(&p->cjobs, sizeof(int4) * jobs.size(), s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->cjobs, jobs.data(), sizeof(int4) * jobs.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "hub jobs");
  }
  if (!out.empty()) e = cudaMemcpyAsync(p->cunits, out.data(), sizeof(int32_t) * out.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !hw.empty()) {
    e = pool_alloc(&p->chash_w, sizeof(int32_t) * hw.size(), s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->chash_w, hw.data(), sizeof(int32_t) * hw.size(), cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? GC_OK : cuda_fail(e, "copy cunits");
}

gc_status first_unreversed_slot(int64_t nnz, const int32_t* d_rev, int32_t* out, cudaStream_t s) {
  *out = -1;
  if (nnz <= 0) return GC_OK;
  int32_t* d = nullptr;
  cudaError_t e = pool_alloc(&d, sizeof(int32_t), s);
  const int32_t init = 0x7fffffff;
  int32_t h = init;
  if (e == cudaSuccess) e = cudaMemcpyAsync(d, &init, sizeof(int32_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    k_first_unreversed<<<grid_for(nnz, 256) > 4096 ? 4096 : grid_for(nnz, 256), 256, 0, s>>>(nnz, d_rev, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (d) cudaFreeAsync(d, s);
  if (e != cudaSuccess) return cuda_fail(e, "symmetry check");
  *out = h == init ? -1 : h;
  return GC_OK;
}

void free_prep(PrepBuffers* p, cudaStream_t s) {
  if (p->deg) cudaFreeAsync(p->deg, s);
  if (p->eid) cudaFreeAsync(p->eid, s);
  if (p->uv) cudaFreeAsync(p->uv, s);
  if (p->out_ptr) cudaFreeAsync(p->out_ptr, s);
  if (p->out_idx) cudaFreeAsync(p->out_idx, s);
  if (p->units) cudaFreeAsync(p->units, s);
  if (p->S) cudaFreeAsync(p->S, s);
  if (p->rev) cudaFreeAsync(p->rev, s);
  if (p->ocsr) cudaFreeAsync(p->ocsr, s);
  if (p->e2o) cudaFreeAsync(p->e2o, s);
  if (p->kunits) cudaFreeAsync(p->kunits, s);
  if (p->cunits) cudaFreeAsync(p->cunits, s);
  if (p->cjobs) cudaFreeAsync(p->cjobs, s);
  if (p->chash_w) cudaFreeAsync(p->chash_w, s);
  *p = PrepBuffers();
}

gc_status prepare_graph(int32_t n, int32_t m, const int32_t* d_rp, const int32_t* d_ci,
                        const int32_t* d_vgid, int32_t* d_eid_given, const int32_t* d_perm,
                        PrepBuffers* out, cudaStream_t s) {
  (void)d_vgid;
  PrepBuffers P;
  P.eid = d_eid_given;
  int32_t *up = nullptr, *upoff = nullptr, *out_cnt = nullptr, *dmax = nullptr, *hist = nullptr;
  long long* S = nullptr;
  gc_status st = GC_OK;
  cudaError_t e = cudaSuccess;
  const int64_t nnz = 2 * (int64_t)m;
#define GC_TRY(call, what)                 \
  do {                                     \
    e = (call);                            \
    if (e != cudaSuccess) {                \
      st = cuda_fail(e, what);             \
      goto fail;                           \
    }                                      \
  } while (0)
  GC_TRY(pool_alloc(&P.deg, sizeof(int32_t) * (n > 0 ? n : 1), s), "alloc deg");
  if (!P.eid) GC_TRY(pool_alloc(&P.eid, sizeof(int32_t) * (nnz > 0 ? nnz : 1), s), "alloc eid");
  GC_TRY(pool_alloc(&P.rev, sizeof(int32_t) * (nnz > 0 ? nnz : 1), s), "alloc rev");
  GC_TRY(pool_alloc(&P.uv, sizeof(int32_t) * (nnz > 0 ? nnz : 1), s), "alloc uv");
  GC_TRY(pool_alloc(&P.out_ptr, sizeof(int32_t) * ((int64_t)n + 1), s), "alloc out_ptr");
  GC_TRY(pool_alloc(&P.out_idx, sizeof(int32_t) * (m > 0 ? m : 1), s), "alloc out_idx");
  GC_TRY(pool_alloc(&P.units, sizeof(int32_t) * (n > 0 ? n : 1), s), "alloc units");
  GC_TRY(pool_alloc(&P.ocsr, sizeof(int32_t) * (m > 0 ? m : 1), s), "alloc ocsr");
  GC_TRY(pool_alloc(&P.e2o, sizeof(int32_t) * (m > 0 ? m : 1), s), "alloc e2o");
  GC_TRY(cudaMemsetAsync(P.e2o, 0, sizeof(int32_t) * (m > 0 ? m : 1), s), "memset e2o");  // in range whatever the input
  GC_TRY(pool_alloc(&P.kunits, sizeof(int32_t) * (n > 0 ? n : 1), s), "alloc kunits");
  GC_TRY(pool_alloc(&up, sizeof(int32_t) * (n > 0 ? n : 1), s), "alloc up");
  GC_TRY(pool_alloc(&upoff, sizeof(int32_t) * ((int64_t)n + 1), s), "alloc upoff");
  GC_TRY(pool_alloc(&out_cnt, sizeof(int32_t) * (n > 0 ? n : 1), s), "alloc out_cnt");
  GC_TRY(pool_alloc(&P.S, sizeof(long long) * (n > 0 ? n : 1), s), "alloc S");
  S = P.S;
  // [0] max degree, [1..64] v-group bins, [65] max out-degree, [66..97] pass-K bins
  GC_TRY(pool_alloc(&dmax, sizeof(int32_t) * 98, s), "alloc dmax");
  hist = dmax + 1;
  GC_TRY(cudaMemsetAsync(dmax, 0, sizeof(int32_t) * 98, s), "memset");
  if (n > 0) {
    k_deg_up<<<grid_for(n, 256), 256, 0, s>>>(n, d_rp, d_ci, P.deg, up);
    GC_TRY(cudaGetLastError(), "k_deg_up");
    if ((st = exclusive_scan(n, up, upoff, s)) != GC_OK) goto fail;
    k_out_cnt<<<grid_for((int64_t)n * 32, 256), 256, 0, s>>>(n, d_rp, d_ci, P.deg, out_cnt, S, dmax, dmax + 65);
    GC_TRY(cudaGetLastError(), "k_out_cnt");
    if ((st = exclusive_scan(n, out_cnt, P.out_ptr, s)) != GC_OK) goto fail;
    if (d_eid_given) {
      k_rev_init<<<grid_for(nnz, 256), 256, 0, s>>>(nnz, P.rev);
      GC_TRY(cudaGetLastError(), "k_rev_init");
    }
    k_edges<<<grid_for((int64_t)n * 32, 256), 256, 0, s>>>(n, m, d_rp, d_ci, P.deg, up, upoff,
                                                            P.out_ptr, P.eid, P.uv, P.out_idx, P.ocsr, P.rev,
                                                            P.e2o, d_eid_given == nullptr, d_perm);
    GC_TRY(cudaGetLastError(), "k_edges");
    if (d_eid_given) {
      k_uv_perm<<<grid_for((int64_t)n * 32, 256), 256, 0, s>>>(n, d_rp, d_ci, P.eid, d_perm, P.uv);
      GC_TRY(cudaGetLastError(), "k_uv_perm");
    }
    k_bin_hist<<<grid_for(n, 256), 256, 0, s>>>(n, P.deg, out_cnt, S, hist, order_key());
    GC_TRY(cudaGetLastError(), "k_bin_hist");
    k_kbin_hist<<<grid_for(n, 256), 256, 0, s>>>(n, out_cnt, dmax + 66);
    GC_TRY(cudaGetLastError(), "k_kbin_hist");
    {
      int32_t h[98];
      GC_TRY(cudaMemcpyAsync(h, dmax, sizeof(h), cudaMemcpyDeviceToHost, s), "copy hist");
      GC_TRY(cudaStreamSynchronize(s), "sync hist");
      P.dmax = h[0];
      P.kmax = h[65];
      {  // pass-K units, largest bin first; tier boundaries at k = 1024, 512, 256, 32
        int32_t kc[32];
        int32_t acc = 0;
        for (int b = 31; b >= 0; --b) {
          if (b == 10) P.ktier_off[kTier1024] = acc;
          if (b == 9) P.ktier_off[kTier512] = acc;
          if (b == 8) P.ktier_off[kTier256] = acc;
          if (b == 5) P.ktier_off[kTier32] = acc;
          kc[b] = acc;
          acc += h[66 + b];
        }
        P.ktier_off[kTierGlobal] = 0;
        P.ktier_off[kNumTiers] = acc;
        GC_TRY(cudaMemcpyAsync(dmax + 66, kc, sizeof(kc), cudaMemcpyHostToDevice, s), "copy k cursors");
        k_kbin_scatter<<<grid_for(n, 256), 256, 0, s>>>(n, out_cnt, dmax + 66, P.kunits);
        GC_TRY(cudaGetLastError(), "k_kbin_scatter");
      }
      int32_t cur[64];
      int32_t acc = 0;
      for (int b = 63; b >= 0; --b) {  // heaviest bin first
        cur[b] = acc;
        acc += h[1 + b];
      }
      P.n_units = acc;
      GC_TRY(cudaMemcpyAsync(hist, cur, sizeof(cur), cudaMemcpyHostToDevice, s), "copy cursors");
      k_bin_scatter<<<grid_for(n, 256), 256, 0, s>>>(n, P.deg, out_cnt, S, hist, P.units, order_key());
      GC_TRY(cudaGetLastError(), "k_bin_scatter");
    }
  } else {
    GC_TRY(cudaMemsetAsync(P.out_ptr, 0, sizeof(int32_t), s), "memset out_ptr");
  }
  if ((st = classify_c_units(n, d_rp, d_ci, d_perm != nullptr, &P, s)) != GC_OK) goto fail;
  cudaFreeAsync(up, s);
  cudaFreeAsync(upoff, s);
  cudaFreeAsync(out_cnt, s);
  cudaFreeAsync(dmax, s);
  *out = P;
  return GC_OK;
fail:
  cudaStreamSynchronize(s);
  if (up) cudaFreeAsync(up, s);
  if (upoff) cudaFreeAsync(upoff, s);
  if (out_cnt) cudaFreeAsync(out_cnt, s);
  if (dmax) cudaFreeAsync(dmax, s);
  free_prep(&P, s);
  return st;
#undef GC_TRY
}

}  // namespace gc
