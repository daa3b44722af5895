// gc_small.cu -- small graphs (n <= kSmallN) counted on a shared-memory
// adjacency bitmatrix.
//
// For a graph of at most 512 vertices the whole adjacency fits in 32 KB of
// shared memory as bit rows. The paper's Psi marks with vertex types
// (Alg. 1: lambda1 for Gamma(v), lambda2 for S_u, lambda3 for T) become bit
// masks over the graph's vertices, and Alg. 5 / Alg. 6 become popcounts:
//   T   = row(u) & row(v)                       |T| = popc(T)
//   S_u = row(u) & ~row(v) without v            S_v = row(v) & ~row(u) without u
//   x7  = (1/2) sum_{a in T}   popc(row(a) & T)     (pairs of T counted twice)
//   x10 =       sum_{w in S_u} popc(row(w) & S_v)   (Alg. 6 with the S_v test)
// One lane holds one 32-bit word of each mask (16 words for 512 vertices);
// the members of T and S_u are listed and dealt to the lanes as (member, word)
// pairs, so an edge costs about (|T| + |S_u|) * W / 32 steps for the warp.
// One CTA per graph (work stealing over the graphs, largest first); per-edge
// terms go into the 13 unrestricted sums of the graph in 128 bits.
#include <cuda_runtime.h>

#include "gc_internal.h"

namespace gc {
namespace {

constexpr int kSmallBlock = 256;
constexpr int kSmallWarps = kSmallBlock / 32;
constexpr int kSmallWords = kSmallN / 32;  // words per bit row

__device__ __forceinline__ void add_u128(unsigned long long* p, u128 v) {
  unsigned long long lo = (unsigned long long)v;
  unsigned long long hi = (unsigned long long)(v >> 64);
  unsigned long long old = atomicAdd(p, lo);
  if (old + lo < old) hi += 1ull;
  if (hi) atomicAdd(p + 1, hi);
}

__device__ __forceinline__ uint64_t small_column(int k, int64_t t, int64_t su, int64_t sv, int64_t D,
                                                 int64_t x7, int64_t x10, int64_t m, int64_t du, int64_t dv) {
  const int64_t s = su + sv;
  switch (k) {  // unrestricted sum k: C_3 C_4 C_5 C_7 C_8 C_9 C_10 C_11 C_12 C_13 C_14 C_15 C_16
    case 0: return (uint64_t)t;
    case 1: return (uint64_t)s;
    case 2: return (uint64_t)D;
    case 3: return (uint64_t)x7;
    case 4: return (uint64_t)(t * (t - 1) / 2);
    case 5: return (uint64_t)(t * s);
    case 6: return (uint64_t)x10;
    case 7: return (uint64_t)(su * (su - 1) / 2 + sv * (sv - 1) / 2);
    case 8: return (uint64_t)(su * sv);
    case 9: return (uint64_t)(t * D);
    case 10: return (uint64_t)(m - du - dv + 1);
    case 11: return (uint64_t)(s * D);
    default: return (uint64_t)(D * (D - 1) / 2);
  }
}

// sum over the members b of `mask` (word w in lane w, words >= W are 0) of
// popc(row(b) & other), for the whole warp. The members are listed in `list`
// (the warp's shared buffer), then each lane takes one (member, word) pair:
// Wp = the power of two >= W lanes per member, 32 / Wp members per step, so
// that every lane has a word to AND whatever the graph's size.
__device__ __forceinline__ long long masked_row_popc(const uint32_t* __restrict__ bm, uint32_t mask,
                                                     uint32_t other, int lane, int Wp, int16_t* list) {
  const int c = __popc(mask);
  int incl = c;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  int pos = incl - c;
  uint32_t word = mask;
  while (word) {
    const int b = __ffs(word) - 1;
    word &= word - 1;
    list[pos++] = (int16_t)(lane * 32 + b);
  }
  __syncwarp();
  const int w = lane & (Wp - 1);
  const uint32_t ow = __shfl_sync(0xffffffffu, other, w);  // word w of the other mask
  const int per = 32 / Wp;
  long long acc = 0;
  for (int i = lane / Wp; i < total; i += per) acc += __popc(bm[list[i] * kSmallWords + w] & ow);
  __syncwarp();
  return acc;
}

__global__ void __launch_bounds__(kSmallBlock) k_small_graphs(const int32_t* __restrict__ rp,
                                                              const int64_t* __restrict__ voff,
                                                              const int32_t* __restrict__ ci,
                                                              const int64_t* __restrict__ eoff,
                                                              const int32_t* __restrict__ order, int32_t G,
                                                              int32_t* __restrict__ cursor,
                                                              unsigned long long* __restrict__ csum) {
  __shared__ uint32_t bm[kSmallN * kSmallWords];
  __shared__ int16_t s_list[kSmallWarps][kSmallN];  // members of a mask, per warp
  __shared__ int32_t s_g;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_g = atomicAdd(cursor, 1);
    __syncthreads();
    if (s_g >= G) break;
    const int32_t g = order[s_g];
    const int32_t* grp = rp + voff[g];
    const int32_t* gci = ci + eoff[g];
    const int32_t n = (int32_t)(voff[g + 1] - voff[g]) - 1;
    const int64_t m = (eoff[g + 1] - eoff[g]) / 2;
    const int W = (n + 31) / 32;
    int Wp = 1;
    while (Wp < W) Wp <<= 1;
    for (int32_t i = threadIdx.x; i < n * kSmallWords; i += kSmallBlock) bm[i] = 0u;
    __syncthreads();
    for (int32_t x = warp; x < n; x += kSmallWarps)
      for (int32_t p = grp[x] + lane; p < grp[x + 1]; p += 32) {
        const int32_t y = gci[p];
        atomicOr(&bm[x * kSmallWords + (y >> 5)], 1u << (y & 31));
      }
    __syncthreads();
    u128 acc = 0;  // lane k < 13: this warp's part of unrestricted sum k
    for (int32_t u = warp; u < n; u += kSmallWarps) {
      const int32_t ub = grp[u], ue = grp[u + 1];
      const uint32_t ru = lane < W ? bm[u * kSmallWords + lane] : 0u;
      for (int32_t p = ub; p < ue; ++p) {
        const int32_t v = gci[p];
        if (v <= u) continue;  // each edge once, from its smaller endpoint
        const uint32_t rv = lane < W ? bm[v * kSmallWords + lane] : 0u;
        const uint32_t T = ru & rv;
        uint32_t Su = ru & ~rv, Sv = rv & ~ru;
        if (lane == (v >> 5)) Su &= ~(1u << (v & 31));
        if (lane == (u >> 5)) Sv &= ~(1u << (u & 31));
        int t = __popc(T), su = __popc(Su), sv = __popc(Sv);
        for (int o = 16; o; o >>= 1) {
          t += __shfl_xor_sync(0xffffffffu, t, o);
          su += __shfl_xor_sync(0xffffffffu, su, o);
          sv += __shfl_xor_sync(0xffffffffu, sv, o);
        }
        long long x7 = masked_row_popc(bm, T, T, lane, Wp, s_list[warp]);
        long long x10 = masked_row_popc(bm, Su, Sv, lane, Wp, s_list[warp]);
        for (int o = 16; o; o >>= 1) {
          x7 += __shfl_xor_sync(0xffffffffu, x7, o);
          x10 += __shfl_xor_sync(0xffffffffu, x10, o);
        }
        x7 /= 2;
        const int64_t du = ue - ub, dv = grp[v + 1] - grp[v];
        const int64_t D = (int64_t)n - 2 - t - su - sv;
        if (lane < 13) acc += (u128)small_column(lane, t, su, sv, D, x7, x10, m, du, dv);
      }
    }
    if (lane < 13 && acc) add_u128(csum + ((size_t)g * 13 + lane) * 2, acc);  // this warp's share
  }
}

}  // namespace

// Counts graphs order[0..G) of a batch whose vertex counts are <= kSmallN;
// csum [*][13][2] must be zeroed; cursor is a zeroed device int.
gc_status run_small_graphs(const int32_t* rp, const int64_t* voff, const int32_t* ci, const int64_t* eoff,
                           const int32_t* order, int32_t G, int32_t* cursor, unsigned long long* csum,
                           cudaStream_t s) {
  if (G <= 0) return GC_OK;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_small_graphs, kSmallBlock, 0);
  int grid = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
  if (grid > G) grid = G;
  k_small_graphs<<<grid, kSmallBlock, 0, s>>>(rp, voff, ci, eoff, order, G, cursor, csum);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GC_OK : cuda_fail(e, "k_small_graphs");
}

}  // namespace gc
