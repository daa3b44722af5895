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
// Pass C -- 4-cycle step (Alg. 4/6) reorganised: P(e), the number of
//   4-cycles (as subgraphs) through e = #{(w, r) : w in Gamma(u)\{v},
//   r in Gamma(v)\{u}, w != r, w ~ r}, for all edges at once by counting
//   wedges from the highest-rank vertex of each cycle (see k_pass_c).
//
// Pass B -- 4-clique step (Alg. 5) and the per-edge finish. Psi for the
//   v-group holds 1 + the position of r in Gamma(v) for r in Gamma(v). Per
//   edge:
//     T       = {w in Gamma(u) \ {v} : Psi(w) != 0}          (Alg. 1)
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

#include <cstdlib>

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


// Lower bound of key in T[0..p2), p2 a power of two, T padded with INT_MAX
// from t to p2: a fixed number of halving steps, no early exit.
__device__ __forceinline__ int lower_bound_pow2(const int32_t* T, int32_t p2, int32_t key) {
  int32_t lo = 0;
  for (int32_t step = p2 >> 1; step > 0; step >>= 1)
    if (T[lo + step - 1] < key) lo += step;
  return lo;
}

// 4-clique count of one edge: sum over members a of T (ascending, t of them)
// of |out(a) ∩ T|, for one warp. Members are taken 32 at a time; the entries
// of their out-lists are laid end to end and dealt to the lanes 32 at a time
// (coalesced loads, no idle lanes), kMLP windows per round so that several
// loads are in flight; each entry's owner is found by a 5-step shuffle search
// over the 32 lists' starts. in_T(r) answers membership; a member whose
// out-list is longer than T (when long_ok) has T's members searched in its
// out-list instead.
template <int kMLP, class InT>
__device__ __forceinline__ long long warp_clique_count(const DevGraph& g, const int32_t* T, int32_t t,
                                                       int32_t i_begin, int32_t i_stride, int lane,
                                                       bool long_ok, InT in_T, long long& probes) {
  long long x7 = 0;
  for (int32_t i0 = i_begin; i0 < t; i0 += i_stride) {
    const int32_t i = i0 + lane;
    int32_t ob = 0, len = 0;
    if (i < t) {
      const int32_t aa = T[i];
      ob = g.out_ptr[aa];
      len = g.out_ptr[aa + 1] - ob;
    }
    const bool longer = long_ok && len > t;
    const int32_t L = longer ? 0 : len;
    int32_t incl = L;
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int32_t excl = incl - L;
    const int32_t total = __shfl_sync(0xffffffffu, incl, 31);
    probes += total;
    for (int32_t k0 = 0; k0 < total; k0 += 32 * kMLP) {
      int32_t r[kMLP];
#pragma unroll
      for (int j = 0; j < kMLP; ++j) {
        const int32_t kk = k0 + 32 * j + lane;
        int32_t lo = 0, hi = 31;  // owner: last lane whose range starts at or before kk
#pragma unroll
        for (int it = 0; it < 5; ++it) {
          const int32_t mid = (lo + hi + 1) >> 1;
          if (__shfl_sync(0xffffffffu, excl, mid) <= kk) lo = mid; else hi = mid - 1;
        }
        const int32_t oj = __shfl_sync(0xffffffffu, ob, lo);
        const int32_t ej = __shfl_sync(0xffffffffu, excl, lo);
        r[j] = kk < total ? g.out_idx[oj + (kk - ej)] : -1;
      }
#pragma unroll
      for (int j = 0; j < kMLP; ++j)
        if (r[j] >= 0) x7 += in_T(r[j]);
    }
    unsigned lm = __ballot_sync(0xffffffffu, longer);
    while (lm) {
      const int src = __ffs(lm) - 1;
      lm &= lm - 1;
      const int32_t oj = __shfl_sync(0xffffffffu, ob, src);
      const int32_t lj = __shfl_sync(0xffffffffu, len, src);
      probes += t;
      for (int32_t j = lane; j < t; j += 32) x7 += contains(g.out_idx + oj, lj, T[j]);
    }
  }
  return x7;
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
  __shared__ int32_t s_unit, s_next;
  uint32_t* tab = table_of<kSmemTable>(g, a, smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  long long w_units = 0;
  if (kSmemTable)
    for (int32_t i = threadIdx.x; i < g.table_n; i += kBlock) tab[i] = 0;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_unit = atomicAdd(a.cursor, 1);
    __syncthreads();
    const int32_t k = s_unit;
    if (k >= a.n_units) {
      if (lane == 0 && w_units) atomicAdd(a.work + kWorkAUnits, (unsigned long long)w_units);
      break;
    }
    const int32_t v = a.units[k];
    const int32_t base = g.gbase[g.vgid ? g.vgid[v] : 0];
    const int32_t vb = g.rp[v], ve = g.rp[v + 1];
    for (int32_t p = vb + threadIdx.x; p < ve; p += kBlock) tab[g.ci[p] - base] = 1u;
    if (threadIdx.x == 0) w_units += ve - vb;
    if (threadIdx.x == 0) s_next = vb;
    __syncthreads();
    for (;;) {  // edges of the group handed to warps one at a time
      int32_t p = 0;
      if (lane == 0) p = atomicAdd(&s_next, 1);
      p = __shfl_sync(0xffffffffu, p, 0);
      if (p >= ve) break;
      const int32_t u = g.ci[p];
      if (!rank_less(g.deg, u, v)) continue;
      const int32_t ub = g.rp[u], ue = g.rp[u + 1];
      int c = 0;
      for (int32_t q = ub + lane; q < ue; q += 32) c += tab[g.ci[q] - base] != 0u;
      c = warp_sum_i(c);
      if (lane == 0) {
        a.tri[g.eid[p]] = c;
        w_units += ue - ub;
      }
    }
    __syncthreads();
    for (int32_t p = vb + threadIdx.x; p < ve; p += kBlock) tab[g.ci[p] - base] = 0u;
  }
}

// ---------------- pass B: cliques, cycles, columns, sums ----------------
template <bool kSmemTable>
__global__ void __launch_bounds__(kBlock, kCtasPerSm) k_pass_b(DevGraph g, CountArgs a) {
  extern __shared__ uint32_t smem[];
  __shared__ int32_t s_unit, s_next;
  uint32_t* tab = table_of<kSmemTable>(g, a, smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t* buf =
      reinterpret_cast<int32_t*>(smem + (kSmemTable ? ((g.table_n + 3) & ~3) : 0)) + warp * kTcap;
  const bool zero_all = kSmemTable && g.table_n <= 4096;

  u128 acc = 0;  // lane k < 13: running sum of C-sum k for graph cur_g
  int32_t cur_g = -1;
  long long w_gdeg = 0, w_deg = 0, w_t = 0, w_probe = 0, w_edges = 0;  // warp-uniform work tallies

  const int32_t n_chunks = *a.n_chunks;
  if (kSmemTable)
    for (int32_t i = threadIdx.x; i < g.table_n; i += kBlock) tab[i] = 0;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_unit = atomicAdd(a.cursor, 1);
    __syncthreads();
    const int32_t k = s_unit;
    if (k >= n_chunks) break;
    const int32_t v = a.chunks[3 * k];
    const int32_t cb = a.chunks[3 * k + 1], ce = a.chunks[3 * k + 2];
    if (cb >= ce) continue;
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

    // Psi for the group: Psi(r) = 1 + position of r in Gamma(v) (non-zero =
    // lambda1, "neighbour of v"); the position gives the edge (r, v).
    for (int32_t p = vb + threadIdx.x; p < ve; p += kBlock) tab[g.ci[p] - base] = (uint32_t)(p - vb + 1);
    if (warp == 0) w_gdeg += dv;
    if (threadIdx.x == 0) s_next = cb;
    __syncthreads();

    // One warp per edge (u, v) of the chunk's slots of Gamma(v), handed out
    // one at a time so that heavy edges do not leave warps idle at the barrier.
    for (;;) {
      int32_t p = 0;
      if (lane == 0) p = atomicAdd(&s_next, 1);
      p = __shfl_sync(0xffffffffu, p, 0);
      if (p >= ce) break;
      const int32_t u = g.ci[p];
      if (!rank_less(g.deg, u, v)) continue;
      const int32_t e = g.eid[p];
      if (e >= g.m) continue;  // sink of an asymmetric input slot: nothing to count
      const int32_t t_expect = a.tri[e];
      if (t_expect > a.big_t) {  // large T: a whole CTA takes this edge later
        if (lane == 0) {
          const int32_t i = atomicAdd(a.n_deferred, 1);
          if (i < a.deferred_cap) {
            a.deferred[2 * i] = v;
            a.deferred[2 * i + 1] = p;
          } else {
            atomicOr(a.status, (int32_t)kSpillOverflow);
          }
        }
        continue;
      }
      const int32_t ub = g.rp[u], ue = g.rp[u + 1];
      long long cross = 0;
      int32_t t = 0;
      for (int32_t q0 = ub; q0 < ue; q0 += 32) {
        const int32_t q = q0 + lane;
        const bool valid = q < ue;
        const int32_t w = valid ? g.ci[q] : v;
        const uint32_t ent = (valid && w != v) ? tab[w - base] : 0u;
        const bool inT = ent != 0u;
        if (inT) cross += (long long)a.tri[g.eid[q]] + (long long)a.tri[g.eid[vb + (int32_t)ent - 1]] - 2;
        const unsigned mask = __ballot_sync(0xffffffffu, inT);
        if (inT && t + __popc(mask & ((1u << lane) - 1u)) < t_expect)
          buf[t + __popc(mask & ((1u << lane) - 1u))] = w;
        t += __popc(mask);
      }
      cross = warp_sum_ll(cross);
      const long long P = (long long)(a.P[p] + a.P[g.rev[p]]);
      if (t != t_expect) {  // cannot happen on a valid graph
        if (lane == 0) atomicOr(a.status, (int32_t)kSpillOverflow);
        continue;
      }
      __syncwarp();
      // 4-cliques: each adjacent pair of T is counted once, through the
      // out-list of its lower-rank member; membership by binary search in T.
      int32_t p2 = 1;
      while (p2 < t) p2 <<= 1;
      for (int32_t i = t + lane; i < p2; i += 32) buf[i] = 0x7fffffff;  // sentinels up to a power of two
      __syncwarp();
      long long x7 = warp_clique_count<4>(g, buf, t, 0, 32, lane, true, [&](int32_t r) {
        const int32_t q = lower_bound_pow2(buf, p2, r);
        return (int)(q < t && buf[q] == r);
      }, w_probe);
      x7 = warp_sum_ll(x7);
      __syncwarp();
      const long long x10 = P - cross + 2 * x7;
      const int64_t du = ue - ub;
      w_deg += du;
      w_t += t;
      w_edges += 1;
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
      for (int32_t p = vb + threadIdx.x; p < ve; p += kBlock) tab[g.ci[p] - base] = 0u;
    }
  }
  if (cur_g >= 0 && lane < 13) atomic_add_u128(a.csum + ((size_t)cur_g * 13 + lane) * 2, acc);
  if (lane == 0) {  // the tallies are warp-uniform: lane 0 holds the warp's totals
    if (w_gdeg) atomicAdd(a.work + kWorkBGroupDeg, (unsigned long long)w_gdeg);
    atomicAdd(a.work + kWorkBDeg, (unsigned long long)w_deg);
    atomicAdd(a.work + kWorkBT, (unsigned long long)w_t);
    atomicAdd(a.work + kWorkBProbe, (unsigned long long)w_probe);
    atomicAdd(a.work + kWorkBEdges, (unsigned long long)w_edges);
  }
}

// ---------------- pass B for edges with a large T ----------------
// One CTA per edge whose T has more than big_t members. T = Gamma(u) ∩ Gamma(v)
// is found by binary search of Gamma(u)'s entries in Gamma(v) (the position
// found also names the edge (a, v) for the cross term), written in order to a
// per-CTA global buffer; when its id range fits, a shared-memory bitmap over
// [min T, max T] answers "r in T" with one load in the 4-clique step
// (binary search in the buffer otherwise). Only the bitmap words set for an
// edge are cleared after it.
__global__ void __launch_bounds__(kBigBlock, 1) k_pass_big(DevGraph g, CountArgs a) {
  extern __shared__ uint32_t bm[];  // kBigWords words
  __shared__ int32_t s_k, s_wcnt[kBigWarps], s_woff[kBigWarps + 1];
  __shared__ long long s_red[kBigWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t* T = a.tbuf + (size_t)blockIdx.x * (size_t)a.tbuf_len;
  const int32_t n_def = min(*a.n_deferred, a.deferred_cap);
  for (int32_t i = threadIdx.x; i < kBigWords; i += kBigBlock) bm[i] = 0u;  // kept zero between edges
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_k = atomicAdd(a.cursor, 1);
    __syncthreads();
    const int32_t k = s_k;
    if (k >= n_def) break;
    const int32_t v = a.deferred[2 * k], p = a.deferred[2 * k + 1];
    const int32_t u = g.ci[p], e = g.eid[p];
    const int32_t gid = g.vgid ? g.vgid[v] : 0;
    const int64_t n_g = g.gn[gid], m_g = g.gm[gid];
    const int32_t vb = g.rp[v], ve = g.rp[v + 1];
    const int32_t ub = g.rp[u], ue = g.rp[u + 1];
    const int32_t t_expect = a.tri[e];
    if (t_expect > a.tbuf_len) {
      if (threadIdx.x == 0) atomicOr(a.status, (int32_t)kSpillOverflow);
      continue;
    }
    // T in order, and the cross term
    long long cross = 0;
    int32_t t = 0;
    for (int32_t q0 = ub; q0 < ue; q0 += kBigBlock) {
      const int32_t q = q0 + threadIdx.x;
      bool inT = false;
      int32_t w = 0;
      if (q < ue) {
        w = g.ci[q];
        if (w != v) {
          int32_t lo = vb, hi = ve;
          while (lo < hi) {
            const int32_t mid = (lo + hi) >> 1;
            if (g.ci[mid] < w) lo = mid + 1; else hi = mid;
          }
          if (lo < ve && g.ci[lo] == w) {
            inT = true;
            cross += (long long)a.tri[g.eid[q]] + (long long)a.tri[g.eid[lo]] - 2;
          }
        }
      }
      const unsigned mask = __ballot_sync(0xffffffffu, inT);
      if (lane == 0) s_wcnt[warp] = __popc(mask);
      __syncthreads();
      if (threadIdx.x == 0) {
        int32_t acc = 0;
        for (int i = 0; i < kBigWarps; ++i) { s_woff[i] = acc; acc += s_wcnt[i]; }
        s_woff[kBigWarps] = acc;
      }
      __syncthreads();
      const int32_t pos = t + s_woff[warp] + __popc(mask & ((1u << lane) - 1u));
      if (inT && pos < t_expect) T[pos] = w;
      t += s_woff[kBigWarps];
      __syncthreads();
    }
    cross = warp_sum_ll(cross);
    if (lane == 0) s_red[warp] = cross;
    __syncthreads();
    if (threadIdx.x == 0) {
      long long c = 0;
      for (int i = 0; i < kBigWarps; ++i) c += s_red[i];
      s_red[0] = c;
    }
    __syncthreads();
    cross = s_red[0];
    if (t != t_expect) {  // cannot happen on a valid graph
      if (threadIdx.x == 0) atomicOr(a.status, (int32_t)kSpillOverflow);
      continue;
    }
    const int32_t lo = T[0], hi = T[t - 1];
    const bool use_bm = (int64_t)hi - lo + 1 <= (int64_t)kBigWords * 32;
    if (use_bm) {
      for (int32_t i = threadIdx.x; i < t; i += kBigBlock) {
        const int32_t d = T[i] - lo;
        atomicOr(&bm[d >> 5], 1u << (d & 31));
      }
    }
    __syncthreads();
    long long x7, probes = 0;
    if (use_bm) {
      x7 = warp_clique_count<4>(g, T, t, warp * 32, kBigBlock, lane, true, [&](int32_t r) {
        const int32_t d = r - lo;
        return (r >= lo && r <= hi) ? (int)((bm[d >> 5] >> (d & 31)) & 1u) : 0;
      }, probes);
    } else {
      x7 = warp_clique_count<4>(g, T, t, warp * 32, kBigBlock, lane, true,
                                [&](int32_t r) { return contains(T, t, r); }, probes);
    }
    if (lane == 0 && probes) atomicAdd(a.work + kWorkBigProbe, (unsigned long long)probes);
    if (threadIdx.x == 0) {
      atomicAdd(a.work + kWorkBigDeg, (unsigned long long)((ve - vb) + (ue - ub)));
      atomicAdd(a.work + kWorkBigT, (unsigned long long)t);
    }
    x7 = warp_sum_ll(x7);
    __syncthreads();
    if (lane == 0) s_red[warp] = x7;
    if (use_bm)
      for (int32_t i = threadIdx.x; i < t; i += kBigBlock) bm[(T[i] - lo) >> 5] = 0u;
    __syncthreads();
    if (threadIdx.x < 13) {
      long long xs = 0;
      for (int i = 0; i < kBigWarps; ++i) xs += s_red[i];
      const long long x10 = (long long)(a.P[p] + a.P[g.rev[p]]) - cross + 2 * xs;
      const int64_t du = ue - ub, dv = ve - vb;
      const int64_t su = du - t - 1, sv = dv - t - 1;
      const int64_t D = n_g - 2 - t - su - sv;
      const int c = threadIdx.x;
      const uint64_t col = edge_column(c, t, su, sv, D, xs, x10, m_g, du, dv);
      if (a.per_edge) a.per_edge[(size_t)e * 13 + c] = col;
      const uint64_t cs = edge_column(csum_column(c), t, su, sv, D, xs, x10, m_g, du, dv);
      atomic_add_u128(a.csum + ((size_t)gid * 13 + c) * 2, (u128)cs);
    }
  }
}

// ---------------- pass C: 4-cycles through every edge ----------------
// P(e) = number of 4-cycles (as subgraphs) containing e. Each 4-cycle is
// counted from its highest-rank vertex h: with cnt_h(o) = #{x in Gamma(h) :
// x < h, o in Gamma(x), o < h}, the wedge h-x-o closes cnt_h(o) - 1 cycles
// through h, each of which contains the edges (h, x) and (x, o) once. Ranks
// are the (degree, id) order of preprocessing P1/P3, so every wedge is met
// from one h only.
template <bool kSmemTable>
__global__ void __launch_bounds__(kBlock) k_pass_c(DevGraph g, CountArgs a) {
  extern __shared__ uint32_t smem[];
  __shared__ int32_t s_unit, s_next[3];
  uint32_t* tab = table_of<kSmemTable>(g, a, smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool zero_all = kSmemTable && g.table_n <= 4096;
  long long w_wedge = 0;
  if (kSmemTable)
    for (int32_t i = threadIdx.x; i < g.table_n; i += kBlock) tab[i] = 0;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_unit = atomicAdd(a.cursor, 1);
    __syncthreads();
    const int32_t k = s_unit;
    if (k >= a.n_units) {
      if (lane == 0 && w_wedge) atomicAdd(a.work + kWorkCWedge, (unsigned long long)w_wedge);
      break;
    }
    const int32_t h = a.units[k];
    const int32_t base = g.gbase[g.vgid ? g.vgid[h] : 0];
    const int32_t hb = g.rp[h], he = g.rp[h + 1];
    if (threadIdx.x < 3) s_next[threadIdx.x] = hb;
    __syncthreads();
    // x runs over the lower-rank neighbours of h; o over those of x's
    // neighbours that rank below h (a prefix of Gamma(x) when ids are ranks).
    for (int pass = 0; pass < (zero_all ? 2 : 3); ++pass) {
      for (;;) {
        int32_t p = 0;
        if (lane == 0) p = atomicAdd(&s_next[pass], 1);
        p = __shfl_sync(0xffffffffu, p, 0);
        if (p >= he) break;
        const int32_t x = g.ci[p];
        if (!rank_less(g.deg, x, h)) continue;
        const int32_t xb = g.rp[x];
        int32_t xe = g.rp[x + 1];
        if (g.ranked) {
          int32_t lo = xb, hi = xe;
          while (lo < hi) {
            const int32_t mid = (lo + hi) >> 1;
            if (g.ci[mid] < h) lo = mid + 1; else hi = mid;
          }
          xe = lo;
        }
        unsigned long long s = 0;
        if (pass == 0 && lane == 0) w_wedge += xe - xb;
        for (int32_t q = xb + lane; q < xe; q += 32) {
          const int32_t o = g.ci[q];
          if (!g.ranked && !rank_less(g.deg, o, h)) continue;
          if (pass == 0) {
            atomicAdd(&tab[o - base], 1u);
          } else if (pass == 1) {
            const uint32_t c = tab[o - base] - 1u;
            if (c) {
              atomicAdd(&a.P[q], (unsigned long long)c);  // slot (x, o): consecutive over the lanes
              s += c;
            }
          } else {
            tab[o - base] = 0u;
          }
        }
        if (pass == 1) {
          for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
          if (lane == 0 && s) atomicAdd(&a.P[p], s);  // slot (h, x)
        }
      }
      __syncthreads();
    }
    if (zero_all) {
      for (int32_t i = threadIdx.x; i < g.table_n; i += kBlock) tab[i] = 0;
    }
  }
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

// Persistent grid: kCtasPerSm CTAs of kBlock threads per SM.
int count_grid_size() {
  if (g_grid == 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    g_grid = (sms > 0 ? sms : 1) * kCtasPerSm;
  }
  return g_grid;
}

int big_t_threshold() {
  static int v = [] {
    const char* e = getenv("GC_BIG_T");
    int x = e ? atoi(e) : 1024;
    return x < 16 ? 16 : (x > kTcap ? kTcap : x);
  }();
  return v;
}

// One CTA of kBigBlock threads per SM for the large-T edges.
int big_grid_size() { return count_grid_size() / kCtasPerSm > 0 ? count_grid_size() / kCtasPerSm : 1; }

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

gc_status run_pass_c(const DevGraph& g, const CountArgs& a, cudaStream_t s) {
  const bool sm = a.tables == nullptr;
  if (sm) return launch(k_pass_c<true>, smem_bytes(true, g.table_n, false), g, a, s, "k_pass_c");
  return launch(k_pass_c<false>, smem_bytes(false, g.table_n, false), g, a, s, "k_pass_c");
}

gc_status run_pass_big(const DevGraph& g, const CountArgs& a, int32_t n_deferred, cudaStream_t s) {
  const size_t smem = sizeof(uint32_t) * kBigWords;
  cudaError_t e = cudaFuncSetAttribute(k_pass_big, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "k_pass_big");
  int grid = big_grid_size();
  if (n_deferred < grid) grid = n_deferred > 0 ? n_deferred : 1;
  k_pass_big<<<grid, kBigBlock, smem, s>>>(g, a);
  e = cudaGetLastError();
  return e == cudaSuccess ? GC_OK : cuda_fail(e, "k_pass_big");
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
