// gc_count.cu -- the counting kernels of the per-edge method.
//
// Work unit: one "v-group" = a vertex v and every edge e = (u, v) for which v
// is the high endpoint (P3, Sec. 4.3: d_v >= d_u, ties to the larger id).
// One CTA owns one unit at a time and a Psi table indexed by vertex; CTAs
// take units from an atomic cursor over the difficulty-ordered unit list
// (work stealing over Pi, Sec. 4.4).
//
// Pass A -- triangle step (Alg. 1): Psi(r) = lambda1 for r in Gamma(v); for
//   every low neighbour u, |T| = #{w in Gamma(u) : Psi(w) = lambda1}.
//
// Pass B -- 4-clique and 4-cycle steps (Alg. 5 / Alg. 6), with Psi extended
//   from a type tag to a count: for the whole v-group
//       Psi(w) = [w in Gamma(v)] * 2^31 + |Gamma(w) ∩ Gamma(v)|,
//   built once by scanning Gamma(r) for every r in Gamma(v). This memoises the
//   Gamma(w) scans that Alg. 6 repeats for every edge sharing v. Per edge:
//     T       = {w in Gamma(u) \ {v} : Psi(w) has the lambda1 bit}  (Alg. 1)
//     P(e)    = sum_{w in Gamma(u)\{v}} (|Gamma(w) ∩ Gamma(v)| - 1)
//               (walks u-w-r-v with w != v, r != u: 4-cycles through e)
//     cross   = sum_{a in T} (|T_(a,u)| + |T_(a,v)| - 2)
//     x7      = sum_{a in T} |out(a) ∩ T|        (Alg. 5; out(a) = higher-rank
//               neighbours, so every adjacent pair of T is counted once --
//               the job of the Psi reset in Alg. 5)
//     x10     = P(e) - cross + 2 x7
//   The last line is Alg. 4/6's count #{(w, r) : w in S_u, r in S_v, w ~ r}:
//   for w in S_u, |Gamma(w) ∩ S_v| = |Gamma(w) ∩ Gamma(v)| - 1 - |Gamma(w) ∩ T|,
//   and sum_{w in S_u} |Gamma(w) ∩ T| = sum_{a in T} (|T_(a,u)| - 1) - 2 x7.
//   Then the per-edge columns (Sec. 4.5) are written and the unrestricted
//   counts C_3..C_16 summed in 128 bits (per warp, then global atomics: local
//   aggregation communicated once, Sec. 4.6).
//
// Derive -- X_1..X_17 from the sums (Sec. 4.6, with X_11 = (C_11 - X_9)/3 and
//   C_9 = sum |T|(|S_u| + |S_v|)), exact 128-bit division checked.
#include <cuda_runtime.h>

#include "gc_internal.h"

namespace gc {
namespace {

__device__ __forceinline__ bool rank_less(const int32_t* __restrict__ deg, int32_t a, int32_t b) {
  int32_t da = deg[a], db = deg[b];
  return da < db || (da == db && a < b);
}

__device__ __forceinline__ int warp_sum_i(int x) {
  for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
__device__ __forceinline__ long long warp_sum_ll(long long x) {
  for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// 1 if key is in the ascending array a[0..len)
__device__ __forceinline__ int contains(const int32_t* a, int32_t len, int32_t key) {
  int32_t lo = 0, hi = len;
  while (lo < hi) {
    int32_t mid = (lo + hi) >> 1;
    int32_t x = a[mid];
    if (x < key) lo = mid + 1; else hi = mid;
  }
  return (lo < len && a[lo] == key) ? 1 : 0;
}

__device__ __forceinline__ void atomic_add_u128(unsigned long long* p, u128 v) {
  unsigned long long lo = (unsigned long long)v;
  unsigned long long hi = (unsigned long long)(v >> 64);
  unsigned long long old = atomicAdd(p, lo);
  if (old + lo < old) hi += 1ull;
  if (hi) atomicAdd(p + 1, hi);
}

// Per-edge columns (Sec. 4.5): T, S_u, S_v of Fig. 2 and D_e.
__device__ __forceinline__ uint64_t edge_column(int k, int64_t t, int64_t su, int64_t sv, int64_t D,
                                                int64_t x7, int64_t x10, int64_t m_g, int64_t du,
                                                int64_t dv) {
  const int64_t s = su + sv;
  switch (k) {
    case 0: return (uint64_t)t;
    case 1: return (uint64_t)s;
    case 2: return (uint64_t)D;
    case 3: return (uint64_t)x7;
    case 4: return (uint64_t)x10;
    case 5: return (uint64_t)(t * (t - 1) / 2);
    case 6: return (uint64_t)(t * s);
    case 7: return (uint64_t)(su * (su - 1) / 2 + sv * (sv - 1) / 2);
    case 8: return (uint64_t)(su * sv);
    case 9: return (uint64_t)(t * D);
    case 10: return (uint64_t)(m_g - du - dv + 1);
    case 11: return (uint64_t)(s * D);
    default: return (uint64_t)(D * (D - 1) / 2);
  }
}

// Unrestricted count k (C_3 C_4 C_5 C_7 C_8 C_9 C_10 C_11 .. C_16) <- column
__device__ __forceinline__ int csum_column(int k) {
  // C_7 <- x7 (col 3), C_8 <- col 5, C_9 <- col 6, C_10 <- x10 (col 4)
  const int map[13] = {0, 1, 2, 3, 5, 6, 4, 7, 8, 9, 10, 11, 12};
  return map[k];
}

template <bool kSmemTable>
__device__ __forceinline__ uint32_t* table_of(const DevGraph& g, const CountArgs& a, uint32_t* smem) {
  return kSmemTable ? smem : a.tables + (size_t)blockIdx.x * (size_t)g.table_n;
}

// ---------------- pass A: |T| per edge ----------------
template <bool kSmemTable>
__global__ void __launch_bounds__(kBlock) k_pass_a(DevGraph g, CountArgs a) {
  extern __shared__ uint32_t smem[];
  __shared__ int32_t s_unit;
  uint32_t* tab = table_of<kSmemTable>(g, a, smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (kSmemTable)
    for (int32_t i = threadIdx.x; i < g.table_n; i += kBlock) tab[i] = 0;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_unit = atomicAdd(a.cursor, 1);
    __syncthreads();
    const int32_t k = s_unit;
    if (k >= a.n_units) break;
    const int32_t v = a.units[k];
    const int32_t base = g.gbase[g.vgid ? g.vgid[v] : 0];
    const int32_t vb = g.rp[v], ve = g.rp[v + 1];
    for (int32_t p = vb + threadIdx.x; p < ve; p += kBlock) tab[g.ci[p] - base] = 1u;
    __syncthreads();
    for (int32_t p = vb + warp; p < ve; p += kWarps) {
      const int32_t u = g.ci[p];
      if (!rank_less(g.deg, u, v)) continue;
      const int32_t ub = g.rp[u], ue = g.rp[u + 1];
      int c = 0;
      for (int32_t q = ub + lane; q < ue; q += 32) c += tab[g.ci[q] - base] != 0u;
      c = warp_sum_i(c);
      if (lane == 0) a.tri[g.eid[p]] = c;
    }
    __syncthreads();
    for (int32_t p = vb + threadIdx.x; p < ve; p += kBlock) tab[g.ci[p] - base] = 0u;
  }
}

// ---------------- pass B: cliques, cycles, columns, sums ----------------
template <bool kSmemTable>
__global__ void __launch_bounds__(kBlock) k_pass_b(DevGraph g, CountArgs a) {
  extern __shared__ uint32_t smem[];
  __shared__ int32_t s_unit;
  uint32_t* tab = table_of<kSmemTable>(g, a, smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t* tbuf_smem =
      reinterpret_cast<int32_t*>(smem + (kSmemTable ? ((g.table_n + 3) & ~3) : 0)) + warp * kTcap;
  int32_t* tbuf_spill =
      a.spill ? a.spill + ((size_t)blockIdx.x * kWarps + warp) * (size_t)a.spill_len : nullptr;
  const bool zero_all = kSmemTable && g.table_n <= 4096;

  u128 acc = 0;  // lane k < 13: running sum of C-sum k for graph cur_g
  int32_t cur_g = -1;

  if (kSmemTable)
    for (int32_t i = threadIdx.x; i < g.table_n; i += kBlock) tab[i] = 0;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_unit = atomicAdd(a.cursor, 1);
    __syncthreads();
    const int32_t k = s_unit;
    if (k >= a.n_units) break;
    const int32_t v = a.units[k];
    const int32_t gid = g.vgid ? g.vgid[v] : 0;
    const int32_t base = g.gbase[gid];
    const int64_t n_g = g.gn[gid], m_g = g.gm[gid];
    const int32_t vb = g.rp[v], ve = g.rp[v + 1];
    const int64_t dv = ve - vb;

    if (gid != cur_g) {  // warp-uniform
      if (cur_g >= 0 && lane < 13) atomic_add_u128(a.csum + ((size_t)cur_g * 13 + lane) * 2, acc);
      acc = 0;
      cur_g = gid;
    }

    // Build Psi for the group: lambda1 bit for Gamma(v), counts |Gamma(w) ∩ Gamma(v)|.
    for (int32_t p = vb + warp; p < ve; p += kWarps) {
      const int32_t r = g.ci[p];
      if (lane == 0) atomicOr(&tab[r - base], kFlag);
      const int32_t rb = g.rp[r], re = g.rp[r + 1];
      for (int32_t q = rb + lane; q < re; q += 32) {
        const int32_t w = g.ci[q];
        if (w != v) atomicAdd(&tab[w - base], 1u);
      }
    }
    __syncthreads();

    // One warp per edge (u, v) of the group.
    for (int32_t p = vb + warp; p < ve; p += kWarps) {
      const int32_t u = g.ci[p];
      if (!rank_less(g.deg, u, v)) continue;
      const int32_t e = g.eid[p];
      const int32_t t_expect = a.tri[e];
      int32_t* buf = t_expect <= kTcap ? tbuf_smem : tbuf_spill;
      if (buf == nullptr || (buf == tbuf_spill && t_expect > a.spill_len)) {
        if (lane == 0) atomicOr(a.status, (int32_t)kSpillOverflow);
        continue;
      }
      const int32_t ub = g.rp[u], ue = g.rp[u + 1];
      long long P = 0, cross = 0;
      int32_t t = 0;
      for (int32_t q0 = ub; q0 < ue; q0 += 32) {
        const int32_t q = q0 + lane;
        const bool valid = q < ue;
        const int32_t w = valid ? g.ci[q] : v;
        const bool use = valid && w != v;
        const uint32_t ent = use ? tab[w - base] : 0u;
        const long long W = (long long)(ent & kCount);
        const bool inT = (ent & kFlag) != 0u;
        if (use) P += W - 1;
        if (inT) cross += (long long)a.tri[g.eid[q]] + W - 2;
        const unsigned mask = __ballot_sync(0xffffffffu, inT);
        if (inT && t + __popc(mask & ((1u << lane) - 1u)) < t_expect)
          buf[t + __popc(mask & ((1u << lane) - 1u))] = w;
        t += __popc(mask);
      }
      P = warp_sum_ll(P);
      cross = warp_sum_ll(cross);
      if (t != t_expect) {  // cannot happen on a valid graph
        if (lane == 0) atomicOr(a.status, (int32_t)kSpillOverflow);
        continue;
      }
      __syncwarp();
      // 4-cliques: each adjacent pair of T counted once via the out-list of its
      // lower-rank member; per member the shorter side drives the search.
      long long x7 = 0;
      for (int32_t i = 0; i < t; ++i) {
        const int32_t aa = buf[i];
        const int32_t ob = g.out_ptr[aa], oe = g.out_ptr[aa + 1];
        const int32_t len = oe - ob;
        if (len <= t) {
          for (int32_t j = ob + lane; j < oe; j += 32) x7 += contains(buf, t, g.out_idx[j]);
        } else {
          for (int32_t j = lane; j < t; j += 32) x7 += contains(g.out_idx + ob, len, buf[j]);
        }
      }
      x7 = warp_sum_ll(x7);
      __syncwarp();
      const long long x10 = P - cross + 2 * x7;
      const int64_t du = ue - ub;
      const int64_t su = du - t - 1, sv = dv - t - 1;
      const int64_t D = n_g - 2 - t - su - sv;
      if (lane < 13) {
        const uint64_t col = edge_column(lane, t, su, sv, D, x7, x10, m_g, du, dv);
        if (a.per_edge) a.per_edge[(size_t)e * 13 + lane] = col;
        const uint64_t cs = edge_column(csum_column(lane), t, su, sv, D, x7, x10, m_g, du, dv);
        acc += (u128)cs;
      }
    }
    __syncthreads();

    // Clear what the build set.
    if (zero_all) {
      for (int32_t i = threadIdx.x; i < g.table_n; i += kBlock) tab[i] = 0;
    } else {
      for (int32_t p = vb + warp; p < ve; p += kWarps) {
        const int32_t r = g.ci[p];
        if (lane == 0) tab[r - base] = 0u;
        const int32_t rb = g.rp[r], re = g.rp[r + 1];
        for (int32_t q = rb + lane; q < re; q += 32) tab[g.ci[q] - base] = 0u;
      }
    }
  }
  if (cur_g >= 0 && lane < 13) atomic_add_u128(a.csum + ((size_t)cur_g * 13 + lane) * 2, acc);
}

// ---------------- derive X_1..X_17 per graph ----------------
__device__ __forceinline__ bool div_exact(u128 num, u128 den, u128* q) {
  if (num % den != 0) return false;
  *q = num / den;
  return true;
}

__global__ void k_derive(int32_t G, const int32_t* __restrict__ gn, const int64_t* __restrict__ gm,
                         const unsigned long long* __restrict__ csum,
                         unsigned long long* __restrict__ xout, int32_t* __restrict__ status) {
  for (int32_t gi = blockIdx.x * blockDim.x + threadIdx.x; gi < G; gi += gridDim.x * blockDim.x) {
    u128 C[17];
    const int idx[13] = {3, 4, 5, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16};
    for (int k = 0; k < 13; ++k) {
      const unsigned long long* p = csum + ((size_t)gi * 13 + k) * 2;
      C[idx[k]] = ((u128)p[1] << 64) | (u128)p[0];
    }
    const u128 n = (u128)gn[gi], m = (u128)gm[gi];
    const u128 n2 = n < 2 ? 0 : n * (n - 1) / 2;
    const u128 n3 = n < 3 ? 0 : n2 * (n - 2) / 3;
    const u128 n4 = n < 4 ? 0 : n3 * (n - 3) / 4;
    u128 X[18];
    bool ok = true;
    X[1] = m;
    X[2] = n2 - m;
    ok &= div_exact(C[3], 3, &X[3]);
    ok &= div_exact(C[4], 2, &X[4]);
    X[5] = C[5];
    X[6] = n3 - X[3] - X[4] - X[5];
    ok &= div_exact(C[7], 6, &X[7]);
    X[8] = C[8] - C[7];
    ok &= div_exact(C[9] - 4 * X[8], 2, &X[9]);
    ok &= div_exact(C[10], 4, &X[10]);
    ok &= div_exact(C[11] - X[9], 3, &X[11]);
    X[12] = C[12] - C[10];
    ok &= div_exact(C[13] - X[9], 3, &X[13]);
    ok &= div_exact(C[14] - 6 * X[7] - 4 * X[8] - 2 * X[9] - 4 * X[10] - 2 * X[12], 2, &X[14]);
    ok &= div_exact(C[15] - 2 * X[12], 2, &X[15]);
    X[16] = C[16] - 2 * X[14];
    u128 s = 0;
    for (int i = 7; i <= 16; ++i) s += X[i];
    X[17] = n4 - s;
    for (int i = 1; i <= 17; ++i) {
      xout[((size_t)gi * 17 + (i - 1)) * 2] = (unsigned long long)X[i];
      xout[((size_t)gi * 17 + (i - 1)) * 2 + 1] = (unsigned long long)(X[i] >> 64);
    }
    if (!ok) atomicOr(status, (int32_t)kInexact);
  }
}

__global__ void k_max_tri(const int32_t* __restrict__ tri, int32_t m, int32_t* __restrict__ out) {
  int32_t best = 0;
  for (int32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += gridDim.x * blockDim.x)
    best = max(best, tri[e]);
  for (int o = 16; o; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0 && best > 0) atomicMax(out, best);
}

int g_grid = 0;

size_t smem_bytes(bool smem_table, int32_t table_n, bool pass_b) {
  size_t b = 0;
  if (smem_table) b += sizeof(uint32_t) * (size_t)((table_n + 3) & ~3);
  if (pass_b) b += sizeof(int32_t) * (size_t)kWarps * kTcap;
  return b;
}

template <typename K>
gc_status launch(K kernel, size_t smem, const DevGraph& g, const CountArgs& a, cudaStream_t s,
                 const char* what) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, what);
  int grid = count_grid_size();
  if (a.n_units < grid) grid = a.n_units > 0 ? a.n_units : 1;
  kernel<<<grid, kBlock, smem, s>>>(g, a);
  e = cudaGetLastError();
  return e == cudaSuccess ? GC_OK : cuda_fail(e, what);
}

}  // namespace

// Persistent grid: two CTAs of kBlock threads per SM.
int count_grid_size() {
  if (g_grid == 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    g_grid = (sms > 0 ? sms : 1) * 2;
  }
  return g_grid;
}

gc_status run_pass_a(const DevGraph& g, const CountArgs& a, cudaStream_t s) {
  const bool sm = a.tables == nullptr;
  if (sm) return launch(k_pass_a<true>, smem_bytes(true, g.table_n, false), g, a, s, "k_pass_a");
  return launch(k_pass_a<false>, smem_bytes(false, g.table_n, false), g, a, s, "k_pass_a");
}

gc_status run_pass_b(const DevGraph& g, const CountArgs& a, cudaStream_t s) {
  const bool sm = a.tables == nullptr;
  if (sm) return launch(k_pass_b<true>, smem_bytes(true, g.table_n, true), g, a, s, "k_pass_b");
  return launch(k_pass_b<false>, smem_bytes(false, g.table_n, true), g, a, s, "k_pass_b");
}

gc_status run_derive(const DevGraph& g, const unsigned long long* csum, unsigned long long* x,
                     int32_t* status, cudaStream_t s) {
  int blocks = (g.G + 127) / 128;
  k_derive<<<blocks > 0 ? blocks : 1, 128, 0, s>>>(g.G, g.gn, g.gm, csum, x, status);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GC_OK : cuda_fail(e, "k_derive");
}

gc_status run_max_tri(const int32_t* tri, int32_t m, int32_t* d_out, cudaStream_t s) {
  int blocks = (m + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_max_tri<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(tri, m, d_out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GC_OK : cuda_fail(e, "k_max_tri");
}

}  // namespace gc
