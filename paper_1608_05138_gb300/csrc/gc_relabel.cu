// gc_relabel.cu -- preprocessing P1 (Sec. 4.3) on the device: the caller's CSR
// is renumbered by ascending degree, so that internal ids are the (degree, id)
// ranks that P3 and the degree-ordered passes compare.
//
// The host computes the permutation (a counting sort of n degrees) and the
// internal row pointers; the device
//   * writes every internal row i (caller vertex perm[i]) as 64-bit keys:
//     the internal id of each caller entry above, its position in the caller
//     row below (ids are distinct within a row, so the order is the ids'),
//   * sorts each row ascending -- bitonic networks: a warp in registers for
//     rows of up to 32 entries, a CTA in shared memory up to 4096, and for
//     longer rows a CTA over a padded copy in global memory whose strides
//     below 4096 are done tile by tile in shared memory,
//   * splits the keys: the internal ids become the row, and the caller
//     position gives, for every internal slot (u, v) with u < v in the
//     caller's labels, the caller's edge id (its rank in the caller's
//     row-major upper triangle) without a search; the reverse slot takes the
//     same id in the preparation, which finds every slot's reverse.
#include <cuda_runtime.h>

#include "gc_internal.h"

namespace gc {
namespace {

constexpr int32_t kTile = 4096;   // entries of a shared-memory tile
constexpr int kMidThreads = 256;
constexpr int kLongThreads = 1024;

constexpr long long kKeyPad = 0x7fffffffffffffffLL;  // sorts after every key

__device__ __forceinline__ void cmpswap(long long* a, int32_t i, int32_t l, bool asc) {
  const long long x = a[i], y = a[l];
  if ((x > y) == asc) {
    a[i] = y;
    a[l] = x;
  }
}

// first index in [lo, hi) with a[index] >= key
__device__ __forceinline__ int32_t lower_bound_dev(const int32_t* a, int32_t lo, int32_t hi, int32_t key) {
  while (lo < hi) {
    const int32_t mid = lo + ((hi - lo) >> 1);
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Warp per internal row: the keys (internal id, caller position) of the
// caller row, unsorted.
__global__ void k_fill_rows(int32_t n, const int32_t* __restrict__ rp0, const int32_t* __restrict__ ci0,
                            const int32_t* __restrict__ perm, const int32_t* __restrict__ newid,
                            const int32_t* __restrict__ rp, long long* __restrict__ kv) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    const int32_t x = perm[i];
    const int32_t b0 = rp0[x], len = rp0[x + 1] - b0, b = rp[i];
    for (int32_t k = lane; k < len; k += 32) kv[b + k] = ((long long)newid[ci0[b0 + k]] << 32) | k;
  }
}

// Rows of 2..32 entries: one warp each, one entry per lane.
__global__ void k_sort_short(int32_t n, const int32_t* __restrict__ rp, long long* __restrict__ ci) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    const int32_t b = rp[i], len = rp[i + 1] - b;
    if (len < 2 || len > 32) continue;  // warp-uniform
    long long v = lane < len ? ci[b + lane] : kKeyPad;
    for (int k = 2; k <= 32; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        const long long w = __shfl_xor_sync(0xffffffffu, v, j);
        const bool asc = (lane & k) == 0, lower = (lane & j) == 0;
        v = (asc == lower) ? min(v, w) : max(v, w);
      }
    if (lane < len) ci[b + lane] = v;
  }
}

// Rows of 33..4096 entries (listed): one CTA each, in shared memory.
__global__ void __launch_bounds__(kMidThreads) k_sort_mid(const int32_t* __restrict__ rows, const int32_t* __restrict__ rp,
                                                          long long* __restrict__ ci) {
  __shared__ long long sh[kTile];
  const int32_t r = rows[blockIdx.x];
  const int32_t b = rp[r], len = rp[r + 1] - b;
  int32_t P = 64;
  while (P < len) P <<= 1;
  for (int32_t i = threadIdx.x; i < P; i += kMidThreads) sh[i] = i < len ? ci[b + i] : kKeyPad;
  __syncthreads();
  for (int32_t k = 2; k <= P; k <<= 1)
    for (int32_t j = k >> 1; j > 0; j >>= 1) {
      for (int32_t t = threadIdx.x; t < P / 2; t += kMidThreads) {
        const int32_t i = 2 * t - (t & (j - 1));
        cmpswap(sh, i, i + j, (i & k) == 0);
      }
      __syncthreads();
    }
  for (int32_t i = threadIdx.x; i < len; i += kMidThreads) ci[b + i] = sh[i];
}

// Steps (k, j) of the bitonic network on one aligned tile of kTile entries of
// a, for j from j0 down to 1 (all pairs lie inside the tile when j0 < kTile).
__device__ __forceinline__ void tile_steps(long long* sh, long long* a, int32_t c0, int32_t k_lo, int32_t k_hi,
                                           int32_t j0) {
  for (int32_t i = threadIdx.x; i < kTile; i += kLongThreads) sh[i] = a[c0 + i];
  __syncthreads();
  for (int32_t k = k_lo; k <= k_hi; k <<= 1)
    for (int32_t j = (k == k_lo ? j0 : k >> 1); j > 0; j >>= 1) {
      for (int32_t t = threadIdx.x; t < kTile / 2; t += kLongThreads) {
        const int32_t i = 2 * t - (t & (j - 1));
        cmpswap(sh, i, i + j, ((c0 + i) & k) == 0);
      }
      __syncthreads();
    }
  for (int32_t i = threadIdx.x; i < kTile; i += kLongThreads) a[c0 + i] = sh[i];
  __syncthreads();
}

// Rows of more than 4096 entries (listed): one CTA each, over a padded copy
// (power-of-two length P) at tmp + toff[row].
__global__ void __launch_bounds__(kLongThreads) k_sort_long(const int32_t* __restrict__ rows,
                                                            const int64_t* __restrict__ toff,
                                                            const int32_t* __restrict__ rp, long long* __restrict__ ci,
                                                            long long* __restrict__ tmp) {
  __shared__ long long sh[kTile];
  const int32_t r = rows[blockIdx.x];
  const int32_t b = rp[r], len = rp[r + 1] - b;
  int32_t P = kTile;
  while (P < len) P <<= 1;
  long long* a = tmp + toff[blockIdx.x];
  for (int32_t i = threadIdx.x; i < P; i += kLongThreads) a[i] = i < len ? ci[b + i] : kKeyPad;
  __syncthreads();
  for (int32_t c0 = 0; c0 < P; c0 += kTile) tile_steps(sh, a, c0, 2, kTile, 1);  // k <= kTile: inside tiles
  for (int32_t k = 2 * kTile; k <= P; k <<= 1) {
    for (int32_t j = k >> 1; j >= kTile; j >>= 1) {  // pairs across tiles
      for (int32_t t = threadIdx.x; t < P / 2; t += kLongThreads) {
        const int32_t i = 2 * t - (t & (j - 1));
        cmpswap(a, i, i + j, (i & k) == 0);
      }
      __syncthreads();
    }
    for (int32_t c0 = 0; c0 < P; c0 += kTile) tile_steps(sh, a, c0, k, k, kTile / 2);
  }
  for (int32_t i = threadIdx.x; i < len; i += kLongThreads) ci[b + i] = a[i];
}

// Per caller row u: first slot with an id above u, and how many there are.
__global__ void k_upper(int32_t n, const int32_t* __restrict__ rp0, const int32_t* __restrict__ ci0,
                        int32_t* __restrict__ first_up, int32_t* __restrict__ up_cnt) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    const int32_t e = rp0[u + 1];
    const int32_t f = lower_bound_dev(ci0, rp0[u], e, (int32_t)u + 1);
    first_up[u] = f;
    up_cnt[u] = e - f;
  }
}

// Warp per internal row i (caller vertex x = perm[i]): the sorted keys split
// into the row's internal ids and, for every slot whose caller labels ascend
// (x < y), the caller's edge id from the caller position; the other slots get
// 0 here and their reverse's id in the preparation.
__global__ void k_split_eid(int32_t n, int32_t m, const int32_t* __restrict__ rp, const long long* __restrict__ kv,
                            const int32_t* __restrict__ perm, const int32_t* __restrict__ rp0,
                            const int32_t* __restrict__ first_up, const int32_t* __restrict__ up_off,
                            int32_t* __restrict__ ci, int32_t* __restrict__ eid) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    const int32_t x = perm[i];
    for (int32_t s = rp[i] + lane; s < rp[i + 1]; s += 32) {
      const long long key = kv[s];
      const int32_t j = (int32_t)(key >> 32), pos = (int32_t)(key & 0xffffffffLL);
      ci[s] = j;
      const int32_t y = perm[j];
      int32_t id = 0;
      if (x < y) id = up_off[x] + (rp0[x] + pos - first_up[x]);
      eid[s] = (id >= 0 && id < m) ? id : 0;
    }
  }
}

int blocks_for(int64_t threads, int block) {
  int64_t b = (threads + block - 1) / block;
  if (b < 1) b = 1;
  if (b > 65535LL * 16) b = 65535LL * 16;
  return (int)b;
}

}  // namespace

gc_status relabel_on_device(int32_t n, int32_t m, const int32_t* d_rp0, const int32_t* d_ci0,
                            const int32_t* d_perm, const int32_t* d_newid, const int32_t* d_rp, int32_t* d_ci,
                            int32_t* d_eid, const int32_t* d_mid_rows, int32_t n_mid, const int32_t* d_long_rows,
                            const int64_t* d_long_off, int32_t n_long, long long* d_tmp, cudaStream_t s) {
  if (n <= 0) return GC_OK;
  cudaError_t e = cudaSuccess;
  int32_t *first_up = nullptr, *up_cnt = nullptr, *up_off = nullptr;
  long long* kv = nullptr;
  const int64_t nnz = 2 * (int64_t)m;
  gc_status st = GC_OK;
#define RL_TRY(call, what)               \
  do {                                   \
    e = (call);                          \
    if (e != cudaSuccess) {              \
      st = cuda_fail(e, what);           \
      goto out;                          \
    }                                    \
  } while (0)
  RL_TRY(pool_alloc(&kv, sizeof(long long) * (size_t)(nnz > 0 ? nnz : 1), s), "alloc relabel keys");
  k_fill_rows<<<blocks_for((int64_t)n * 32, 256), 256, 0, s>>>(n, d_rp0, d_ci0, d_perm, d_newid, d_rp, kv);
  RL_TRY(cudaGetLastError(), "k_fill_rows");
  k_sort_short<<<blocks_for((int64_t)n * 32, 256), 256, 0, s>>>(n, d_rp, kv);
  RL_TRY(cudaGetLastError(), "k_sort_short");
  if (n_mid > 0) {
    k_sort_mid<<<n_mid, kMidThreads, 0, s>>>(d_mid_rows, d_rp, kv);
    RL_TRY(cudaGetLastError(), "k_sort_mid");
  }
  if (n_long > 0) {
    k_sort_long<<<n_long, kLongThreads, 0, s>>>(d_long_rows, d_long_off, d_rp, kv, d_tmp);
    RL_TRY(cudaGetLastError(), "k_sort_long");
  }
  RL_TRY(pool_alloc(&first_up, sizeof(int32_t) * (size_t)n, s), "alloc relabel");
  RL_TRY(pool_alloc(&up_cnt, sizeof(int32_t) * (size_t)n, s), "alloc relabel");
  RL_TRY(pool_alloc(&up_off, sizeof(int32_t) * ((size_t)n + 1), s), "alloc relabel");
  k_upper<<<blocks_for(n, 256), 256, 0, s>>>(n, d_rp0, d_ci0, first_up, up_cnt);
  RL_TRY(cudaGetLastError(), "k_upper");
  if ((st = exclusive_scan(n, up_cnt, up_off, s)) != GC_OK) goto out;
  k_split_eid<<<blocks_for((int64_t)n * 32, 256), 256, 0, s>>>(n, m, d_rp, kv, d_perm, d_rp0, first_up, up_off,
                                                              d_ci, d_eid);
  RL_TRY(cudaGetLastError(), "k_split_eid");
out:
#undef RL_TRY
  for (void* p : {(void*)first_up, (void*)up_cnt, (void*)up_off, (void*)kv})
    if (p) cudaFreeAsync(p, s);
  return st;
}

}  // namespace gc
