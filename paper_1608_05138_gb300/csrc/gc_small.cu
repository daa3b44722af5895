// gc_small.cu -- small graphs (n <= 1024) counted on a shared-memory
// adjacency bitmatrix.
//
// For a graph of at most 1024 vertices the whole adjacency fits in at most
// 132 KB of shared memory as bit rows. The paper's Psi marks with vertex
// types (Alg. 1: lambda1 for Gamma(v), lambda2 for S_u, lambda3 for T)
// become bit masks over the graph's vertices:
//   T = row(u) & row(v),  S_u = row(u) & ~row(v) without v,  S_v likewise,
// and |T|, |S_u|, |S_v|, D_e and the per-edge summands of C_3 .. C_16 follow
// per edge as in Sec. 4.5. The batched form returns only the global counts,
// so of the two per-edge scans of Alg. 5/6 only their sums are needed:
//   C_7  = sum_e x7  = 6 #K4: every 4-clique {a < b < c < d} is met once, at
//          its edge (a, b), as an edge inside T' = the common neighbours of
//          a and b above b (sum over T' of popc(row(w) & T') counts it twice);
//   C_10 = sum_e x10 = 4 X_10 = 4 C4 - 4 C_8 + 2 C_7, with C4 the 4-cycles as
//          subgraphs, (1/2) sum over vertex pairs {u, w} of C(c_uw, 2) (c_uw
//          common neighbours; each cycle is met from both of its diagonals),
//          X_10 = C4 - X_8 - 3 X_7 and X_8 = C_8 - C_7 (Sec. 4.6).
// That is a popcount over the n^2 / 2 pairs instead of one over S_u x S_v
// per edge -- several times less work on the dense graphs of a batch -- and
// exact: the derivation of Sec. 4.6 then runs unchanged.
// One lane holds one 32-bit word of each mask; rows are stored at an odd
// word stride, so that 32 lanes reading one word index of 32 rows hit 32
// banks. One CTA per graph (work stealing over the graphs, largest first).
//
// Graphs are binned by vertex count into size classes (n <= 64, 128, 256,
// 512, 1024); each class runs its own instantiation, whose bitmatrix and
// member lists are sized for the class, so that small graphs take little
// shared memory and many CTAs fit on an SM. The block size of each class is
// a tuning parameter (BatchConfig).
#include <cuda_runtime.h>

#include "gc_internal.h"

namespace gc {
namespace {

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
// that every lane has a word to AND whatever the graph's size. kS: the row
// stride of the size class, in words.
template <int kS>
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
  for (int i = lane / Wp; i < total; i += per) acc += __popc(bm[list[i] * kS + w] & ow);
  __syncwarp();
  return acc;
}

// Row stride of a size class: the words of a row, made odd.
__host__ __device__ constexpr int small_stride(int kN) { return (kN / 32) | 1; }

// Shared memory of a size class: the bitmatrix (kN rows at the odd stride)
// and one member list of kN entries per warp.
__host__ __device__ constexpr size_t small_smem(int kN, int kBlock) {
  return (size_t)kN * (size_t)small_stride(kN) * 4 + (size_t)(kBlock / 32) * (size_t)kN * 2;
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long x) {
  for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// at least 1536 threads resident per SM (at most 42 registers a thread): the
// kernel is bound by shared-memory latency, and its time falls with the
// warps an SM holds
template <int kN, int kBlock>
__global__ void __launch_bounds__(kBlock, 1536 / kBlock) k_small_graphs(const int32_t* __restrict__ rp,
                                                         const int64_t* __restrict__ voff,
                                                         const int32_t* __restrict__ ci,
                                                         const int64_t* __restrict__ eoff,
                                                         const int32_t* __restrict__ order, int32_t G,
                                                         int32_t* __restrict__ cursor, int32_t* __restrict__ status,
                                                         unsigned long long* __restrict__ csum) {
  constexpr int kS = small_stride(kN);  // words per bit row, odd
  constexpr int kWarps = kBlock / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* bm = reinterpret_cast<uint32_t*>(smem);
  int16_t* s_list = reinterpret_cast<int16_t*>(smem + (size_t)kN * kS * 4);
  __shared__ int32_t s_g;
  // per graph: 4-cliques met twice each, C_8, sum over pairs of C(c_uw, 2)
  __shared__ unsigned long long s_k4, s_c8, s_c4;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      s_g = atomicAdd(cursor, 1);
      s_k4 = s_c8 = s_c4 = 0ull;
    }
    __syncthreads();
    if (s_g >= G) break;
    const int32_t g = order[s_g];
    const int32_t* grp = rp + voff[g];
    const int32_t* gci = ci + eoff[g];
    const int32_t n = (int32_t)(voff[g + 1] - voff[g]) - 1;
    const int64_t m = (eoff[g + 1] - eoff[g]) / 2;
    if (n > kN) {  // cannot happen: graphs are binned by n
      if (threadIdx.x == 0) atomicOr(status, (int32_t)kSpillOverflow);
      continue;
    }
    const int W = (n + 31) / 32;
    int Wp = 1;
    while (Wp < W) Wp <<= 1;
    for (int32_t i = threadIdx.x; i < n * kS; i += kBlock) bm[i] = 0u;
    __syncthreads();
    for (int32_t x = warp; x < n; x += kWarps)
      for (int32_t p = grp[x] + lane; p < grp[x + 1]; p += 32) {
        const int32_t y = gci[p];
        atomicOr(&bm[x * kS + (y >> 5)], 1u << (y & 31));
      }
    __syncthreads();
    u128 acc = 0;  // lane k < 13: this warp's part of unrestricted sum k (C_7, C_10 added per graph)
    int16_t* list = s_list + warp * kN;
    for (int32_t u = warp; u < n; u += kWarps) {
      const int32_t ub = grp[u], ue = grp[u + 1];
      const uint32_t ru = lane < W ? bm[u * kS + lane] : 0u;
      for (int32_t p = ub; p < ue; ++p) {
        const int32_t v = gci[p];
        if (v <= u) continue;  // each edge once, from its smaller endpoint
        const uint32_t rv = lane < W ? bm[v * kS + lane] : 0u;
        const uint32_t T = ru & rv;
        uint32_t Su = ru & ~rv, Sv = rv & ~ru;
        if (lane == (v >> 5)) Su &= ~(1u << (v & 31));
        if (lane == (u >> 5)) Sv &= ~(1u << (u & 31));
        // T' = the common neighbours above v
        const int vb = v >> 5, vo = v & 31;
        const uint32_t above = lane > vb ? 0xffffffffu : (lane == vb && vo < 31 ? 0xffffffffu << (vo + 1) : 0u);
        const uint32_t Tp = T & above;
        int t = __popc(T), su = __popc(Su), sv = __popc(Sv);
        for (int o = 16; o; o >>= 1) {
          t += __shfl_xor_sync(0xffffffffu, t, o);
          su += __shfl_xor_sync(0xffffffffu, su, o);
          sv += __shfl_xor_sync(0xffffffffu, sv, o);
        }
        // the edges inside T' (each met from both ends): 4-cliques with lowest edge (u, v)
        const unsigned long long k2 = warp_sum((unsigned long long)masked_row_popc<kS>(bm, Tp, Tp, lane, Wp, list));
        const int64_t du = ue - ub, dv = grp[v + 1] - grp[v];
        const int64_t D = (int64_t)n - 2 - t - su - sv;
        if (lane < 13) acc += (u128)small_column(lane, t, su, sv, D, 0, 0, m, du, dv);
        if (lane == 0) {
          if (k2) atomicAdd(&s_k4, k2);
          if (t > 1) atomicAdd(&s_c8, (unsigned long long)t * (unsigned long long)(t - 1) / 2);
        }
      }
    }
    // the 4-cycles as subgraphs: C(c_uw, 2) over every pair u < w
    unsigned long long c4 = 0;
    for (int32_t u = warp; u < n; u += kWarps) {
      const uint32_t* rowu = bm + u * kS;
      for (int32_t w0 = u + 1; w0 < n; w0 += 32) {
        const int32_t w = w0 + lane;
        if (w < n) {
          const uint32_t* roww = bm + w * kS;
          unsigned c = 0;
          for (int k = 0; k < W; ++k) c += __popc(rowu[k] & roww[k]);
          c4 += (unsigned long long)c * (c - 1) / 2;
        }
      }
    }
    c4 = warp_sum(c4);
    if (lane == 0 && c4) atomicAdd(&s_c4, c4);
    if (lane < 13 && acc) add_u128(csum + ((size_t)g * 13 + lane) * 2, acc);  // this warp's share
    __syncthreads();
    if (threadIdx.x == 0) {  // per graph: C_7 = 6 #K4, C_10 = 4 C4 - 4 C_8 + 2 C_7
      const unsigned long long c7 = 3ull * s_k4;
      const unsigned long long c10 = 2ull * s_c4 - 4ull * s_c8 + 2ull * c7;
      if (c7) add_u128(csum + ((size_t)g * 13 + 3) * 2, (u128)c7);
      if (c10) add_u128(csum + ((size_t)g * 13 + 6) * 2, (u128)c10);
    }
  }
}

typedef void (*SmallKernel)(const int32_t*, const int64_t*, const int32_t*, const int64_t*, const int32_t*, int32_t,
                            int32_t*, int32_t*, unsigned long long*);

// kSmallBlocks[j] threads per CTA for tuning choice j.
constexpr int kNumSmallBlocks = 4;
constexpr int kSmallBlocks[kNumSmallBlocks] = {64, 128, 256, 512};

template <int kN>
SmallKernel small_kernel_for(int block) {
  switch (block) {
    case 64: return k_small_graphs<kN, 64>;
    case 128: return k_small_graphs<kN, 128>;
    case 512: return k_small_graphs<kN, 512>;
    default: return k_small_graphs<kN, 256>;
  }
}

SmallKernel small_kernel(int cls, int block) {
  switch (cls) {
    case 0: return small_kernel_for<64>(block);
    case 1: return small_kernel_for<128>(block);
    case 2: return small_kernel_for<256>(block);
    case 3: return small_kernel_for<512>(block);
    default: return small_kernel_for<1024>(block);
  }
}

int valid_block(int block) {
  for (int b : kSmallBlocks)
    if (b == block) return block;
  return 256;
}

}  // namespace

int small_class_of(int32_t n) {
  for (int c = 0; c < kSmallClasses; ++c)
    if (n <= kSmallClassN[c]) return c;
  return kSmallClasses;
}

// Resident CTAs of every (size class, block) instantiation on one GPU
// (filled by small_graphs_setup, outside any stream capture).
static int g_small_ctas[kSmallClasses][kNumSmallBlocks] = {};

static int block_index(int block) {
  for (int j = 0; j < kNumSmallBlocks; ++j)
    if (kSmallBlocks[j] == block) return j;
  return 2;
}

// Grid of one size class: resident CTAs, at most one CTA per graph.
static int small_grid(int cls, int block, int32_t graphs) {
  int grid = g_small_ctas[cls][block_index(block)];
  if (grid < 1) grid = 1;
  return grid > graphs ? graphs : grid;
}

gc_status small_graphs_setup() {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "k_small_graphs setup");
  for (int c = 0; c < kSmallClasses; ++c)
    for (int j = 0; j < kNumSmallBlocks; ++j) {
      const int b = kSmallBlocks[j];
      const size_t smem = small_smem(kSmallClassN[c], b);
      e = cudaFuncSetAttribute(small_kernel(c, b), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      int per_sm = 0;
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, small_kernel(c, b), b, smem);
      if (e != cudaSuccess) return cuda_fail(e, "k_small_graphs attribute");
      g_small_ctas[c][j] = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
    }
  return GC_OK;
}

gc_status run_small_graphs(const int32_t* rp, const int64_t* voff, const int32_t* ci, const int64_t* eoff,
                           const int32_t* order, const int32_t* class_off, int32_t* cursor, int32_t* status,
                           unsigned long long* csum, const BatchConfig& cfg, cudaEvent_t* ev, cudaStream_t s) {
  for (int c = 0; c < kSmallClasses; ++c) {
    const int32_t G = class_off[c + 1] - class_off[c];
    if (ev) {
      cudaError_t e = cudaEventRecord(ev[c], s);
      if (e != cudaSuccess) return cuda_fail(e, "small event");
    }
    if (G <= 0) continue;
    const int block = valid_block(cfg.class_block[c]);
    const int grid = small_grid(c, block, G);
    small_kernel(c, block)<<<grid, block, small_smem(kSmallClassN[c], block), s>>>(
        rp, voff, ci, eoff, order + class_off[c], G, cursor + c, status, csum);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_small_graphs");
  }
  if (ev) {
    cudaError_t e = cudaEventRecord(ev[kSmallClasses], s);
    if (e != cudaSuccess) return cuda_fail(e, "small event");
  }
  return GC_OK;
}

}  // namespace gc
