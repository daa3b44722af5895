// gc_small.cu -- small graphs (n <= 1024) counted on a shared-memory
// adjacency bitmatrix.
//
// For a graph of at most 1024 vertices the whole adjacency fits in at most
// 132 KB of shared memory as bit rows. The paper's Psi marks with vertex
// types (Alg. 1: lambda1 for Gamma(v), lambda2 for S_u, lambda3 for T)
// become bit masks over the graph's vertices:
//   T = row(u) & row(v),  S_u = row(u) & ~row(v) without v,  S_v likewise,
// and |T| = popc(row(u) & row(v)), |S_u| = d_u - 1 - |T|, |S_v| and D_e
// follow per edge as in Sec. 4.5. The batched form returns only the global
// counts, so the per-edge summands of C_3 .. C_16 are needed only as sums
// over the edges: they are polynomials in |T|, d_u and d_v, and the kernel
// sums per edge only |T|, |T|^2 and |T| (d_u + d_v), per vertex d^2 and d^3,
// per entry d_x d_y, from which the columns follow in closed form
// (graph_column). Of the two per-edge scans of Alg. 5/6:
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

constexpr unsigned kFull = 0xffffffffu;

// Sums of one graph from which its unrestricted sums follow in closed form
// (graph_columns): per edge (u, v) with t = |T| and a = d_u + d_v, the sums
// of t, t^2, t a and the 4-clique term; per vertex, d^2 and d^3; per
// directed entry (x, y), d_x d_y.
enum { kQt, kQtt, kQta, kQk, kQd2, kQd3, kQdd, kQn };

// sum over the members b of `mask` (word w in lane w; the words below w0 and
// from W on are 0) of popc(row(b) & mask), this lane's part. The members are
// listed in `list` (the warp's shared buffer), then each lane takes one
// (member, word) pair over the words [w0, W): Wq = the power of two >= W - w0
// lanes per member, 32 / Wq members per step. kS: the row stride of the size
// class, in words.
template <int kS>
__device__ __forceinline__ uint32_t masked_row_popc(const uint32_t* __restrict__ bm, uint32_t mask, int lane, int w0,
                                                    int W, int16_t* list) {
  const int span = W - w0;
  const int c = __popc(mask);
  int incl = c;
  for (int o = 1; o < span; o <<= 1) {  // lanes w0 .. W-1 carry the members
    const int y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  const int total = __shfl_sync(kFull, incl, W - 1);
  int pos = incl - c;
  uint32_t word = mask;
  while (word) {
    const int b = __ffs(word) - 1;
    word &= word - 1;
    list[pos++] = (int16_t)(lane * 32 + b);
  }
  __syncwarp();
  const int lg = span <= 1 ? 0 : 32 - __clz(span - 1);
  const int w = w0 + (lane & ((1 << lg) - 1));
  const bool wv = w < W;
  const uint32_t ow = __shfl_sync(kFull, mask, w & 31);  // word w of the mask
  uint32_t acc = 0;
  for (int i = lane >> lg; i < total; i += 32 >> lg)
    if (wv) acc += __popc(bm[list[i] * kS + w] & ow);
  __syncwarp();
  return acc;
}

// The unrestricted sums of one graph (n vertices, m edges) from the sums
// q and the sum c4 over vertex pairs of C(c_uw, 2), in the column order
// C_3 C_4 C_5 C_7 C_8 C_9 C_10 C_11 C_12 C_13 C_14 C_15 C_16. Per edge
// |S_u| = d_u - 1 - t and |S_v| = d_v - 1 - t (Sec. 4.5), so s = a - 2 - 2t
// and D = n - 2 - t - s, and with A1 = sum a = sum_v d^2,
// A2 = sum a^2 = sum_v d^3 + 2P and P = sum over edges of d_u d_v:
//   C_4 = sum s = A1 - 2m - 2 sum t,       C_9 = sum t s = sum t a - 2 sum t - 2 sum t^2,
//   C_12 = sum |S_u||S_v| = P - A1 + m - sum t a + 2 sum t + sum t^2,
//   sum s^2 = A2 - 4 A1 + 4m - 4 (sum t a - 2 sum t) + 4 sum t^2,
//   C_5 = (n-2) m - sum t - C_4,            C_8 = (sum t^2 - sum t) / 2,
//   C_11 = (sum s^2 - 2 C_12 - C_4) / 2,    C_13 = (n-2) sum t - sum t^2 - C_9,
//   C_14 = m^2 + m - A1,                    C_15 = (n-2) C_4 - C_9 - sum s^2,
//   C_16 = (sum D^2 - C_5) / 2, sum D^2 = (n-2)^2 m - 2 (n-2)(sum t + C_4)
//          + sum t^2 + 2 C_9 + sum s^2,
// C_7 = 6 #K4 = 3 q_k (each 4-clique met twice), C_10 = 4 C4 - 4 C_8 + 2 C_7.
// Column k of the graph, k in 0 .. 12. Unsigned arithmetic: every result is a nonnegative count below 2^64, so
// the wrap-around of the intermediate terms cancels.
__device__ __forceinline__ unsigned long long graph_column(int k, const unsigned long long* q, unsigned long long c4,
                                                         int32_t n, int64_t m) {
  typedef unsigned long long U;
  const U N2 = (U)(long long)(n - 2), M = (U)m;
  const U St = q[kQt], Stt = q[kQtt], Sta = q[kQta], A1 = q[kQd2];
  const U C4 = A1 - 2ull * M - 2ull * St;
  const U C9 = Sta - 2ull * St - 2ull * Stt;
  const U C12 = q[kQdd] / 2ull - A1 + M - Sta + 2ull * St + Stt;
  const U Sss = q[kQd3] + q[kQdd] - 4ull * A1 + 4ull * M - 4ull * (Sta - 2ull * St) + 4ull * Stt;
  const U C5 = N2 * M - St - C4;
  switch (k) {
    case 0: return St;
    case 1: return C4;
    case 2: return C5;
    case 3: return 3ull * q[kQk];
    case 4: return (Stt - St) / 2ull;
    case 5: return C9;
    case 6: return 2ull * c4 - 2ull * (Stt - St) + 6ull * q[kQk];
    case 7: return (Sss - 2ull * C12 - C4) / 2ull;
    case 8: return C12;
    case 9: return N2 * St - Stt - C9;
    case 10: return M * M + M - A1;
    case 11: return N2 * C4 - C9 - Sss;
    default: return (N2 * N2 * M - 2ull * N2 * (St + C4) + Stt + 2ull * C9 + Sss - C5) / 2ull;
  }
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
// kernel is bound by instruction issue and shared-memory latency, and the
// more warps an SM holds, the more of its cycles issue
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
  // per graph: the per-edge sums and the sum over pairs of C(c_uw, 2)
  __shared__ unsigned long long s_q[kQn], s_c4;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_g = atomicAdd(cursor, 1);
    if (threadIdx.x < kQn) s_q[threadIdx.x] = 0ull;
    if (threadIdx.x == kQn) s_c4 = 0ull;
    __syncthreads();
    if (s_g >= G) break;
    const int32_t g = order[s_g];
    const int32_t* grp = rp + voff[g];
    const int32_t* gci = ci + eoff[g];
    const int32_t n = (int32_t)(voff[g + 1] - voff[g]) - 1;
    if (n > kN) {  // cannot happen: graphs are binned by n
      if (threadIdx.x == 0) atomicOr(status, (int32_t)kSpillOverflow);
      continue;
    }
    const int W = (n + 31) / 32;
    for (int32_t i = threadIdx.x; i < n * kS; i += kBlock) bm[i] = 0u;
    __syncthreads();
    // the bit rows, and the degree sums: lane 0 d^2 and d^3 per vertex, every
    // lane d_x d_y per entry
    unsigned long long d2 = 0, d3 = 0, dd = 0;
    for (int32_t x = warp; x < n; x += kWarps) {
      const int32_t xb = grp[x], xe = grp[x + 1];
      const uint32_t dx = (uint32_t)(xe - xb);
      if (lane == 0) {
        d2 += dx * dx;
        d3 += (unsigned long long)(dx * dx) * dx;
      }
      for (int32_t p = xb + lane; p < xe; p += 32) {
        const int32_t y = gci[p];
        atomicOr(&bm[x * kS + (y >> 5)], 1u << (y & 31));
        dd += dx * (uint32_t)(grp[y + 1] - grp[y]);
      }
    }
    dd = warp_sum(dd);
    if (lane == 0) {
      if (d2) atomicAdd(&s_q[kQd2], d2);
      if (d3) atomicAdd(&s_q[kQd3], d3);
      if (dd) atomicAdd(&s_q[kQdd], dd);
    }
    __syncthreads();
    int16_t* list = s_list + warp * kN;
    for (int32_t u = warp; u < n; u += kWarps) {
      const int32_t ub = grp[u], ue = grp[u + 1];
      const uint32_t ru = lane < W ? bm[u * kS + lane] : 0u;
      // each edge once, from its smaller endpoint: the neighbours above u
      // follow the popc(row(u) below u) ones below it in the sorted row
      const int uw = u >> 5;
      const uint32_t below = lane < uw ? ru : (lane == uw ? ru & ((1u << (u & 31)) - 1u) : 0u);
      const int32_t p1 = ub + (int32_t)__reduce_add_sync(kFull, (unsigned)__popc(below));
      // sums over the edges of u, each below 2^31 (fewer than 1024 edges,
      // every term below 2^20)
      uint32_t a_t = 0, a_tt = 0, a_tdv = 0, a_k = 0;
      for (int32_t p0 = p1; p0 < ue; p0 += 32) {
        // 32 neighbours v at a time, each with d_v (both below 2^16)
        uint32_t vd = 0;
        if (p0 + lane < ue) {
          const int32_t y = gci[p0 + lane];
          vd = (uint32_t)y | ((uint32_t)(grp[y + 1] - grp[y]) << 16);
        }
        for (int j = 0; j < 32 && p0 + j < ue; ++j) {
          const uint32_t vdj = __shfl_sync(kFull, vd, j);
          const int32_t v = (int32_t)(vdj & 0xffffu);
          const uint32_t dv = vdj >> 16;
          const uint32_t rv = lane < W ? bm[v * kS + lane] : 0u;
          const uint32_t T = ru & rv;
          const uint32_t t = __reduce_add_sync(kFull, (unsigned)__popc(T));
          a_t += t;
          a_tt += t * t;
          a_tdv += t * dv;
          if (t > 1u) {
            // T' = the common neighbours above v; the edges inside T' (each
            // met from both ends) are the 4-cliques with lowest edge (u, v)
            const int vb = (v + 1) >> 5;
            const uint32_t above = lane > vb ? 0xffffffffu : (lane == vb ? 0xffffffffu << ((v + 1) & 31) : 0u);
            const uint32_t Tp = T & above;
            const uint32_t ct = __reduce_add_sync(kFull, (unsigned)__popc(Tp));
            if (ct > 1u) a_k += __reduce_add_sync(kFull, masked_row_popc<kS>(bm, Tp, lane, vb, W, list));
          }
        }
      }
      // sum over the edges of u of t (d_u + d_v) = d_u sum t + sum t d_v
      const unsigned long long ta = (unsigned long long)(ue - ub) * a_t + a_tdv;
      const unsigned long long mine = lane == kQt ? (unsigned long long)a_t
                                      : lane == kQtt ? (unsigned long long)a_tt
                                                     : lane == kQta ? ta : (unsigned long long)a_k;
      if (lane < kQd2 && mine) atomicAdd(&s_q[lane], mine);
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
    __syncthreads();
    if (threadIdx.x < 13) {  // thread k: the graph's unrestricted sum k
      const unsigned long long c = graph_column(threadIdx.x, s_q, s_c4, n, (eoff[g + 1] - eoff[g]) / 2);
      if (c) add_u128(csum + ((size_t)g * 13 + threadIdx.x) * 2, (u128)c);
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
