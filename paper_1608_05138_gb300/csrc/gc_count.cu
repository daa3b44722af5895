// gc_count.cu -- the triangle and 4-cycle passes, the per-edge finish and the
// derivation of the global counts.
//
// Work unit of pass C: one "v-group" = a vertex v and every edge e = (u, v)
// for which v is the high endpoint (P3, Sec. 4.3: d_v >= d_u, ties to the
// larger id). One CTA owns one unit at a time and a count table indexed by
// vertex; CTAs take units from an atomic cursor over the difficulty-ordered
// unit list (work stealing over Pi, Sec. 4.4).
//
// Pass T (gc_clique.cu) -- triangle step (Alg. 1): |T| per edge.
//
// Pass C -- 4-cycle step (Alg. 4/6) reorganised: P(e), the number of
//   4-cycles (as subgraphs) through e = #{(w, r) : w in Gamma(u)\{v},
//   r in Gamma(v)\{u}, w != r, w ~ r}, for all edges at once by counting
//   wedges from the highest-rank vertex of each cycle (see k_pass_c).
//
// Pass K (gc_clique.cu) -- 4-cliques x7 (Alg. 3/5) and
//   cross(e) = sum_{w in T} (|T_(w,u)| + |T_(w,v)| - 2) per edge.
//
// Finish -- per edge, Alg. 4/6's count #{(w, r) : w in S_u, r in S_v, w ~ r}:
//   for w in S_u, |Gamma(w) ∩ S_v| = |Gamma(w) ∩ Gamma(v)| - 1 - |Gamma(w) ∩ T|,
//   and sum_{w in S_u} |Gamma(w) ∩ T| = sum_{a in T} (|T_(a,u)| - 1) - 2 x7, so
//     x10 = P(e) - cross(e) + 2 x7.
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
  return k == 4 ? 5 : (k == 5 ? 6 : (k == 6 ? 4 : k));
}

template <bool kSmemTable>
__device__ __forceinline__ uint32_t* table_of(const DevGraph& g, const CountArgs& a, uint32_t* smem) {
  return kSmemTable ? smem : a.tables + (size_t)blockIdx.x * (size_t)g.table_n;
}

// ---------------- finish: x10, per-edge columns, sums ----------------
// One warp per 32 consecutive edges. Each lane computes the 13 columns of its
// edge into shared memory, and lane k < 13 adds column csum_column(k) of every
// row to its 128-bit running sum, flushed whenever the graph changes.
// kByEdge: the warp's edges are 32 consecutive edge ids, whose rows leave as
// one contiguous block of 416 words (13 coalesced stores of the warp) -- the
// order for rows written over the host link into pinned host memory.
// Otherwise: 32 consecutive out-slots (coalesced reads of the pass results),
// whose rows leave one at a time (13 lanes, one 104-byte store) -- the order
// for rows in device memory.
constexpr int kFinBlock = 256;
template <bool kByEdge>
__global__ void __launch_bounds__(kFinBlock) k_finish(DevGraph g, CountArgs a) {
  __shared__ unsigned long long st[kFinBlock / 32][32][13];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned long long(*rowv)[13] = st[warp];
  const unsigned long long* flat = &st[warp][0][0];
  u128 acc = 0;
  int32_t cur_g = -1;
  long long w_edges = 0;
  const int64_t stride = (int64_t)gridDim.x * (kFinBlock / 32) * 32;
  for (int64_t e0 = ((int64_t)blockIdx.x * (kFinBlock / 32) + warp) * 32; e0 < g.m; e0 += stride) {
    const int64_t i0 = e0 + lane;  // edge id (kByEdge) or out-slot
    int32_t gid = 0, eid = 0;
    if (i0 < g.m) {
      int32_t o = kByEdge ? g.e2o[i0] : (int32_t)i0;
      if ((uint32_t)o >= (uint32_t)g.m) o = 0;  // only for invalid input
      const int32_t p = g.ocsr[o];
      if (!kByEdge) eid = g.eid[p];
      const int32_t r = g.rev[p];
      const int32_t u = g.ci[r], v = g.ci[p];
      gid = g.vgid ? g.vgid[u] : 0;
      const int64_t du = g.deg[u], dv = g.deg[v];
      const int64_t t = a.trio[o];
      const int64_t x7 = (int64_t)a.xc[2 * (size_t)o];
      const int64_t x10 = (int64_t)(a.P[p] + a.P[r]) - (int64_t)a.xc[2 * (size_t)o + 1] + 2 * x7;
      const int64_t su = du - t - 1, sv = dv - t - 1;
      const int64_t n_g = g.gn[gid], m_g = g.gm[gid];
      const int64_t D = n_g - 2 - t - su - sv;
#pragma unroll
      for (int c = 0; c < 13; ++c) rowv[lane][c] = edge_column(c, t, su, sv, D, x7, x10, m_g, du, dv);
    }
    __syncwarp();
    const int rows = (int)min((int64_t)32, (int64_t)g.m - e0);
    if (kByEdge && a.per_edge) {
      unsigned long long* dst = reinterpret_cast<unsigned long long*>(a.per_edge) + (size_t)e0 * 13;
      for (int i = lane; i < rows * 13; i += 32) dst[i] = flat[i];
    }
    for (int r = 0; r < rows; ++r) {
      const int32_t gr = __shfl_sync(0xffffffffu, gid, r);
      const int32_t er = __shfl_sync(0xffffffffu, eid, r);
      if (lane < 13) {
        if (!kByEdge && a.per_edge) a.per_edge[(size_t)er * 13 + lane] = rowv[r][lane];
        if (gr != cur_g) {
          if (cur_g >= 0) atomic_add_u128(a.csum + ((size_t)cur_g * 13 + lane) * 2, acc);
          acc = 0;
          cur_g = gr;
        }
        acc += (u128)rowv[r][csum_column(lane)];
      }
    }
    w_edges += rows;
    __syncwarp();
  }
  if (lane < 13 && cur_g >= 0) atomic_add_u128(a.csum + ((size_t)cur_g * 13 + lane) * 2, acc);
  if (lane == 0 && w_edges) atomicAdd(a.work + kWorkFinishEdges, (unsigned long long)w_edges);
}

// ---------------- per-edge induced 4-node counts ----------------
// Per vertex x: vsum[2x] = sum over Gamma(x) of |T| of the edge (twice the
// triangles at x), vsum[2x + 1] = sum over Gamma(x) of the neighbour's
// degree. One warp per vertex.
__global__ void __launch_bounds__(256) k_vertex_sums(DevGraph g, const int32_t* __restrict__ trio,
                                                     unsigned long long* __restrict__ vsum) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < g.n; x += warps) {
    unsigned long long t2 = 0, ns = 0;
    for (int32_t p = g.rp[x] + lane; p < g.rp[x + 1]; p += 32) {
      ns += (unsigned long long)g.deg[g.ci[p]];
      t2 += (unsigned long long)trio[g.e2o[g.eid[p]]];
    }
    for (int o = 16; o; o >>= 1) {
      t2 += __shfl_xor_sync(0xffffffffu, t2, o);
      ns += __shfl_xor_sync(0xffffffffu, ns, o);
    }
    if (lane == 0) {
      vsum[2 * x] = t2;
      vsum[2 * x + 1] = ns;
    }
  }
}

// For the edge e = (u, v) and the other vertices split into T, S_u, S_v (Fig.
// 2) and the rest R (|R| = D_e), the induced subgraph on {u, v, a, b} depends
// on the classes of a and b and on whether a ~ b. With A_XY the adjacent
// pairs between classes X and Y, the counts of H_7..H_16 containing e are
//   H7 = A_TT = x7            H8 = C(|T|,2) - A_TT + A_TS
//   H9 = |T||S| - A_TS + A_TR + A_SS                 H10 = A_SuSv = x10
//   H11 = C(|S_u|,2) + C(|S_v|,2) - A_SS             H12 = |S_u||S_v| - x10 + A_SR
//   H13 = |T||R| - A_TR      H14 = A_RR     H15 = |S||R| - A_SR     H16 = C(|R|,2) - A_RR
// (S = S_u + S_v, A_SS = A_SuSu + A_SvSv). The A's follow from quantities the
// passes already have, by counting incidences:
//   A_TS = cross(e) - 4 x7          (sum over T of |T_(w,u)| - 1 is 2 x7 + A_TSu)
//   A_SS = tri(u) + tri(v) - 2|T| - 2 x7 - A_TS      (triangles at u: |T| + x7 + A_TSu + A_SuSu)
//   A_TR = sum_T d_w - 2|T| - 2 x7 - A_TS            (degrees of T: u, v, T, S, R)
//   A_SR = sum_S d_w - |S| - A_TS - 2 A_SS - 2 x10   (sum_S d_w = NS(u) - d_v + NS(v) - d_u - 2 sum_T d_w)
//   A_RR = m - 1 - 2|T| - |S| - x7 - A_TS - A_SS - x10 - A_TR - A_SR
// with tri(x) the triangles at x and NS(x) the sum of the neighbours' degrees.
// Rows are staged per warp like k_finish (kByEdge: 32 consecutive edge ids).
constexpr int kIndCols = 10;
static_assert(kIndCols == GC_INDUCED_COLS, "induced columns");
template <bool kByEdge>
__global__ void __launch_bounds__(kFinBlock) k_finish_induced(DevGraph g, CountArgs a,
                                                              const unsigned long long* __restrict__ vsum,
                                                              unsigned long long* __restrict__ out) {
  __shared__ unsigned long long st[kFinBlock / 32][32][kIndCols];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned long long(*rowv)[kIndCols] = st[warp];
  const unsigned long long* flat = &st[warp][0][0];
  const int64_t stride = (int64_t)gridDim.x * (kFinBlock / 32) * 32;
  for (int64_t e0 = ((int64_t)blockIdx.x * (kFinBlock / 32) + warp) * 32; e0 < g.m; e0 += stride) {
    const int64_t i0 = e0 + lane;  // edge id (kByEdge) or out-slot
    int32_t eid = 0;
    if (i0 < g.m) {
      int32_t o = kByEdge ? g.e2o[i0] : (int32_t)i0;
      if ((uint32_t)o >= (uint32_t)g.m) o = 0;  // only for invalid input
      const int32_t p = g.ocsr[o];
      if (!kByEdge) eid = g.eid[p];
      const int32_t r = g.rev[p];
      const int32_t u = g.ci[r], v = g.ci[p];
      const int32_t gid = g.vgid ? g.vgid[u] : 0;
      const int64_t du = g.deg[u], dv = g.deg[v];
      const int64_t t = a.trio[o];
      const int64_t x7 = (int64_t)a.xc[2 * (size_t)o], cross = (int64_t)a.xc[2 * (size_t)o + 1];
      const int64_t x10 = (int64_t)(a.P[p] + a.P[r]) - cross + 2 * x7;
      const int64_t su = du - t - 1, sv = dv - t - 1, S = su + sv;
      const int64_t R = (int64_t)g.gn[gid] - 2 - t - S;
      const int64_t sdT = (int64_t)a.dsum[o];
      const int64_t aTS = cross - 4 * x7;
      const int64_t aSS = (int64_t)((vsum[2 * (size_t)u] + vsum[2 * (size_t)v]) / 2) - 2 * t - 2 * x7 - aTS;
      const int64_t aTR = sdT - 2 * t - 2 * x7 - aTS;
      const int64_t sdS = (int64_t)vsum[2 * (size_t)u + 1] - dv + (int64_t)vsum[2 * (size_t)v + 1] - du - 2 * sdT;
      const int64_t aSR = sdS - S - aTS - 2 * aSS - 2 * x10;
      const int64_t aRR = g.gm[gid] - 1 - 2 * t - S - x7 - aTS - aSS - x10 - aTR - aSR;
      unsigned long long* rw = rowv[lane];
      rw[0] = (unsigned long long)x7;
      rw[1] = (unsigned long long)(t * (t - 1) / 2 - x7 + aTS);
      rw[2] = (unsigned long long)(t * S - aTS + aTR + aSS);
      rw[3] = (unsigned long long)x10;
      rw[4] = (unsigned long long)(su * (su - 1) / 2 + sv * (sv - 1) / 2 - aSS);
      rw[5] = (unsigned long long)(su * sv - x10 + aSR);
      rw[6] = (unsigned long long)(t * R - aTR);
      rw[7] = (unsigned long long)aRR;
      rw[8] = (unsigned long long)(S * R - aSR);
      rw[9] = (unsigned long long)(R * (R - 1) / 2 - aRR);
    }
    __syncwarp();
    const int rows = (int)min((int64_t)32, (int64_t)g.m - e0);
    if (kByEdge) {
      unsigned long long* dst = out + (size_t)e0 * kIndCols;
      for (int i = lane; i < rows * kIndCols; i += 32) dst[i] = flat[i];
    } else {
      for (int r = 0; r < rows; ++r) {
        const int32_t er = __shfl_sync(0xffffffffu, eid, r);
        if (lane < kIndCols) out[(size_t)er * kIndCols + lane] = rowv[r][lane];
      }
    }
    __syncwarp();
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
  const int lane = threadIdx.x & 31;
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
        if (g.ranked) xe = min(max(g.rev[p], xb), xe);  // Gamma(x) below the slot of (x, h) is < h
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

// ---------------- pass C for hub units: the count table in shared memory ----------------
// The same wedges and attribution as k_pass_c, for the units h whose wedges
// (a few thousand hubs carry almost all of them on power-law graphs) would
// otherwise hit a vertex-indexed table in DRAM at random. Ids are ranks, so
// the lower-rank neighbours X of h are a prefix of Gamma(h) and, for x in X,
// the o < h are a prefix of Gamma(x), ascending. The o-range [0, h) is swept
// in blocks of a.hub_tab words: cnt_h(o) for the block is built in shared
// memory from each x's run of o in the block (a per-x cursor walks Gamma(x)
// once over all blocks; the end of the run is found by galloping search),
// then the wedges of the block are attributed with the block's counts.
// In both phases a warp works on a chunk of up to 32 x's: for a hub of more
// than 1024 x's it takes chunks from a shared counter, heaviest first; for a
// smaller hub each warp keeps one chunk, x = w, w + 32, ..., with its cursors
// in registers, so that the warps carry equal work. Runs of 32 or more
// entries are taken by the whole warp one
// at a time, the shorter ones are dealt to its lanes end to end, so that run
// lengths, however skewed, do not leave lanes idle, and the P atomics of
// consecutive lanes hit consecutive slots. The per-x sums of the attribution
// collect in shared memory (warp sums for long runs, shared atomics for
// short ones). The block fills shared memory: the longer the runs per block,
// the more wedges take the whole-warp path.
constexpr int kHeavyBlock = 1024;
constexpr int kHeavyWarps = kHeavyBlock / 32;

// Counters of the block, kCpw to a word: one 32-bit counter; two 16-bit
// counters when the unit has fewer than 65536 lower neighbours; three 10-bit
// counters when it has fewer than 1023 (no count exceeds the number of lower
// neighbours, so no carry crosses into the next field) -- twice or three
// times the o-range per block.
template <int kCpw>
__device__ __forceinline__ void add_count(uint32_t* tab, int32_t slot) {
  if (kCpw == 3) {
    const uint32_t w = (uint32_t)slot / 3u;
    atomicAdd(&tab[w], 1u << (((uint32_t)slot - 3u * w) * 10u));
  } else if (kCpw == 2) {
    atomicAdd(&tab[slot >> 1], 1u << ((slot & 1) << 4));
  } else {
    atomicAdd(&tab[slot], 1u);
  }
}
template <int kCpw>
__device__ __forceinline__ uint32_t read_count(const uint32_t* tab, int32_t slot) {
  if (kCpw == 3) {
    const uint32_t w = (uint32_t)slot / 3u;
    return (tab[w] >> (((uint32_t)slot - 3u * w) * 10u)) & 1023u;
  }
  if (kCpw == 2) return (tab[slot >> 1] >> ((slot & 1) << 4)) & 0xffffu;
  return tab[slot];
}

// first index in [p, e) with a[index] >= key; a ascending
__device__ __forceinline__ int32_t gallop_lower_bound(const int32_t* __restrict__ a, int32_t p, int32_t e,
                                                      int32_t key) {
  if (p >= e || a[p] >= key) return p;
  int32_t lo = p, step = 1;  // a[lo] < key throughout
  while (lo + step < e && a[lo + step] < key) {
    lo += step;
    step <<= 1;
  }
  int32_t hi = min(lo + step, e);
  ++lo;
  while (lo < hi) {
    const int32_t mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Runs of 32 lanes laid end to end: lane ranks of the non-empty runs, for
// the owner lookup of deal_owner (call with the whole warp).
struct Deal {
  int32_t excl, total;
  unsigned nz;
};
__device__ __forceinline__ Deal deal_setup(int32_t L, int32_t* comp, int lane) {
  Deal d;
  int32_t incl = L;
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  d.excl = incl - L;
  d.total = __shfl_sync(0xffffffffu, incl, 31);
  d.nz = __ballot_sync(0xffffffffu, L > 0);
  if (L > 0) comp[__popc(d.nz & ((1u << lane) - 1u))] = lane;
  __syncwarp();
  return d;
}
// Owner lane of position k0 + lane (k0 a multiple of 32, call with the whole
// warp, for the windows k0 = 0, 32, 64, ... in order): the runs starting in
// the window mark a 32-bit mask, and the owner is the last non-empty run
// starting at or before the position. `before` counts the non-empty runs that
// start before the window (0 for the first) and is advanced past it.
__device__ __forceinline__ int deal_owner(const Deal& d, int32_t L, int32_t k0, const int32_t* comp, int lane,
                                          int& before) {
  const bool in_win = L > 0 && d.excl >= k0 && d.excl < k0 + 32;
  const unsigned M = __reduce_or_sync(0xffffffffu, in_win ? 1u << (d.excl - k0) : 0u);
  const int r = before + __popc(M & (0xffffffffu >> (31 - lane))) - 1;
  before += __popc(M);
  return comp[r < 0 ? 0 : r];
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// The counts of one chunk's runs: lane l's run is [st, st + L) of Gamma(x)
// for its x (L = 0 for none); runs of 32 or more entries are taken by the
// whole warp one at a time, the shorter ones dealt to the lanes end to end.
template <int kCpw>
__device__ __forceinline__ void count_chunk(const DevGraph& g, uint32_t* tab, int32_t* comp, int32_t st, int32_t L,
                                            int32_t lo_id, int lane) {
  // runs of 32 or more entries (most of the wedges): the whole warp,
  // one run at a time, consecutive entries over the lanes
  unsigned lm = __ballot_sync(0xffffffffu, L >= 32);
  while (lm) {
    const int src = __ffs(lm) - 1;
    lm &= lm - 1;
    const int32_t s0 = __shfl_sync(0xffffffffu, st, src);
    const int32_t n0 = __shfl_sync(0xffffffffu, L, src);
    for (int32_t k0 = 0; k0 < n0; k0 += 256) {  // eight windows of loads in flight
      int32_t o[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int32_t kk = k0 + 32 * j + lane;
        o[j] = kk < n0 ? g.ci[s0 + kk] : -1;
      }
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (o[j] >= 0) add_count<kCpw>(tab, o[j] - lo_id);
    }
  }
  // shorter runs dealt to the lanes end to end
  const int32_t Ls = L < 32 ? L : 0;
  const Deal d = deal_setup(Ls, comp, lane);
  const int32_t sb = st - d.excl;  // slot of position kk of this lane's run: sb + kk
  int before = 0;
  for (int32_t k0 = 0; k0 < d.total; k0 += 128) {
    int32_t q[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int ol = deal_owner(d, Ls, k0 + 32 * j, comp, lane, before);
      const int32_t kk = k0 + 32 * j + lane;
      const int32_t bj = __shfl_sync(0xffffffffu, sb, ol);
      q[j] = kk < d.total ? bj + kk : -1;
    }
    int32_t o[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) o[j] = q[j] >= 0 ? g.ci[q[j]] : lo_id;
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (q[j] >= 0) add_count<kCpw>(tab, o[j] - lo_id);
  }
}

// The attribution of one chunk's wedges (runs as in count_chunk; lane l's x
// is the i-th lower neighbour, i < nx): cnt_h(o) - 1 to the slot (x, o) of
// each wedge, and the sum over the run to the slot (h, x).
template <int kCpw>
__device__ __forceinline__ void attr_chunk(const DevGraph& g, const CountArgs& a, uint32_t* tab,
                                           unsigned long long* sx, uint32_t* sx32, int32_t* comp, int32_t st,
                                           int32_t L, int32_t i, int32_t nx, int32_t hb, int32_t lo_id, int lane) {
  sx[lane] = 0ull;  // per x of the chunk: sum of its wedges' counts
  sx32[lane] = 0u;
  __syncwarp();
  // runs of 32 or more entries: the whole warp, one run at a time
  unsigned lm = __ballot_sync(0xffffffffu, L >= 32);
  while (lm) {
    const int src = __ffs(lm) - 1;
    lm &= lm - 1;
    const int32_t s0 = __shfl_sync(0xffffffffu, st, src);
    const int32_t n0 = __shfl_sync(0xffffffffu, L, src);
    unsigned long long acc = 0ull;
    for (int32_t k0 = 0; k0 < n0; k0 += 256) {  // eight windows of loads in flight
      int32_t o[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int32_t kk = k0 + 32 * j + lane;
        o[j] = kk < n0 ? g.ci[s0 + kk] : -1;
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (o[j] < 0) continue;
        const uint32_t cnt = read_count<kCpw>(tab, o[j] - lo_id) - 1u;
        if (cnt) {
          atomicAdd(&a.P[s0 + k0 + 32 * j + lane], (unsigned long long)cnt);  // slot (x, o)
          acc += cnt;
        }
      }
    }
    for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == src) sx[lane] += acc;
  }
  __syncwarp();
  // shorter runs dealt to the lanes end to end
  const int32_t Ls = L < 32 ? L : 0;
  const Deal d = deal_setup(Ls, comp, lane);
  const int32_t sb = st - d.excl;  // slot of position kk of this lane's run: sb + kk
  int before = 0;
  for (int32_t k0 = 0; k0 < d.total; k0 += 128) {
    int32_t q[4], ol[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      ol[j] = deal_owner(d, Ls, k0 + 32 * j, comp, lane, before);
      const int32_t kk = k0 + 32 * j + lane;
      const int32_t bj = __shfl_sync(0xffffffffu, sb, ol[j]);
      q[j] = kk < d.total ? bj + kk : -1;
    }
    int32_t o[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) o[j] = q[j] >= 0 ? g.ci[q[j]] : lo_id;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (q[j] >= 0) {
        const uint32_t cnt = read_count<kCpw>(tab, o[j] - lo_id) - 1u;
        if (cnt) {
          atomicAdd(&a.P[q[j]], (unsigned long long)cnt);  // slot (x, o)
          atomicAdd(&sx32[ol[j]], cnt);                    // the owner's sum
        }
      }
    }
  }
  __syncwarp();
  if (i < nx) {
    const unsigned long long sum = sx[lane] + sx32[lane];
    if (sum) atomicAdd(&a.P[hb + i], sum);  // slot (h, x)
  }
}

// One block [lo_id, r1) of a hub job: the counts of the block from each
// x's run in it (found by galloping search from the x's cursor), then the
// attribution of the block's wedges, for a hub of more than 1024 lower
// neighbours: chunks of 32 consecutive x's taken heaviest first (X ascends
// by degree), their cursors in the CTA's buffers (a smaller hub runs
// hub_block_small). Called by the whole CTA after the table is zeroed and
// the chunk counters reset (and a barrier).
template <int kCpw>
__device__ __forceinline__ void hub_block(const DevGraph& g, const CountArgs& a, uint32_t* tab, int32_t* s_chunk,
                                          unsigned long long* sx, uint32_t* sx32, int32_t* comp, int32_t* beg,
                                          int32_t* cur, const int32_t* endp, int32_t nx, int32_t nchunks,
                                          int32_t hb, int32_t lo_id, int32_t r1, int lane) {
  // counts of the block
  for (;;) {
    int32_t c = 0;
    if (lane == 0) c = atomicAdd(&s_chunk[0], 1);
    c = __shfl_sync(0xffffffffu, c, 0);
    if (c >= nchunks) break;
    const int32_t i = (nchunks - 1 - c) * 32 + lane;
    int32_t st = 0, L = 0;
    if (i < nx) {
      st = cur[i];
      const int32_t en = gallop_lower_bound(g.ci, st, endp[i], r1);
      L = en - st;
      beg[i] = st;
      cur[i] = en;
    }
    count_chunk<kCpw>(g, tab, comp, st, L, lo_id, lane);
    __syncwarp();
  }
  __syncthreads();
  // attribution of the block's wedges
  for (;;) {
    int32_t c = 0;
    if (lane == 0) c = atomicAdd(&s_chunk[1], 1);
    c = __shfl_sync(0xffffffffu, c, 0);
    if (c >= nchunks) break;
    const int32_t i = (nchunks - 1 - c) * 32 + lane;
    int32_t st = 0, L = 0;
    if (i < nx) {
      st = beg[i];
      L = cur[i] - st;
    }
    attr_chunk<kCpw>(g, a, tab, sx, sx32, comp, st, L, i, nx, hb, lo_id, lane);
    __syncwarp();
  }
}

// One block of a hub of at most 1024 lower neighbours: warp w always takes
// the chunk x = w, w + 32, ..., so each thread keeps its x's cursor (cur) and
// run in registers across the two phases and the blocks of the job. Called
// by the whole CTA after the table is zeroed (and a barrier).
template <int kCpw>
__device__ __forceinline__ void hub_block_small(const DevGraph& g, const CountArgs& a, uint32_t* tab,
                                                unsigned long long* sx, uint32_t* sx32, int32_t* comp,
                                                int32_t& cur, int32_t endx, int32_t i, int32_t nx, int32_t hb,
                                                int32_t lo_id, int32_t r1, int lane) {
  int32_t st = 0, L = 0, en = cur;
  if (i < nx) {
    st = cur;
    en = gallop_lower_bound(g.ci, st, endx, r1);
    L = en - st;
  }
  count_chunk<kCpw>(g, tab, comp, st, L, lo_id, lane);
  __syncwarp();
  __syncthreads();
  attr_chunk<kCpw>(g, a, tab, sx, sx32, comp, st, L, i, nx, hb, lo_id, lane);
  __syncwarp();
  cur = en;
}

__global__ void __launch_bounds__(kHeavyBlock, 1) k_pass_c_heavy(DevGraph g, CountArgs a) {
  extern __shared__ uint32_t tab[];  // a.hub_tab words of counters
  __shared__ int32_t s_unit, s_nx, s_chunk[2];
  const unsigned long long t_start = global_ns();
  __shared__ unsigned long long s_sx[kHeavyWarps][32];
  __shared__ uint32_t s_sx32[kHeavyWarps][32];  // the short runs' part (< 32 entries x counts < 2^26)
  __shared__ int32_t s_comp[kHeavyWarps][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t* beg = a.cbuf + (size_t)blockIdx.x * 3 * (size_t)a.cbuf_nx;
  int32_t* cur = beg + a.cbuf_nx;
  int32_t* endp = cur + a.cbuf_nx;
  int32_t* comp = s_comp[warp];
  long long w_wedge = 0, w_blocks = 0, w_jobs = 0;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_unit = atomicAdd(a.cursor + 8, 1);
    __syncthreads();
    const int32_t jb = s_unit;
    if (jb >= a.n_cjobs) break;
    const int4 job = a.cjobs[jb];  // hub (index into cunits), first block, blocks
    const int32_t h = a.cunits[job.x];
    const int32_t hb = g.rp[h], he = g.rp[h + 1];
    if (threadIdx.x == 0) {
      int32_t lo = hb, hi = he;  // first slot of Gamma(h) with id >= h
      while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (g.ci[mid] < h) lo = mid + 1; else hi = mid;
      }
      s_nx = lo - hb;
    }
    __syncthreads();
    const int32_t nx = s_nx;
    if (nx > a.cbuf_nx) {  // cannot happen: the buffers are sized for the largest hub
      if (threadIdx.x == 0) atomicOr(a.status, (int32_t)kSpillOverflow);
      continue;
    }
    // more than 1024 lower neighbours: chunks of 32 consecutive x's (32 of
    // them at 1024 too, the same in both readings); fewer: one per warp
    const int32_t nchunks = nx > kHeavyBlock ? (nx + 31) >> 5 : kHeavyWarps;
    const int cpw = hub_cpw(nx);
    const int32_t span = cpw * a.hub_tab;
    const int64_t job_lo = (int64_t)job.y * span;                       // the job's o-range
    const int64_t job_hi = min((int64_t)h, job_lo + (int64_t)job.z * span);
    // at most 1024 lower neighbours: this thread's x (chunk = warp) and its
    // cursor in registers; otherwise the cursors of all x in the CTA's buffers
    const bool small = nchunks == kHeavyWarps;
    const int32_t ix = warp + kHeavyWarps * lane;
    int32_t rcur = 0, rend = 0;
    if (small) {
      if (ix < nx) {
        const int32_t x = g.ci[hb + ix];
        const int32_t xb = g.rp[x];
        rend = min(max(g.rev[hb + ix], xb), g.rp[x + 1]);  // Gamma(x) below the slot of (x, h) is < h
        rcur = job.y == 0 ? xb : gallop_lower_bound(g.ci, xb, rend, (int32_t)job_lo);
        if (job.y == 0) w_wedge += rend - xb;  // the hub's wedges, counted by its first job
      }
    } else {
      for (int32_t i = threadIdx.x; i < nx; i += kHeavyBlock) {
        const int32_t x = g.ci[hb + i];
        const int32_t xb = g.rp[x];
        const int32_t lo = min(max(g.rev[hb + i], xb), g.rp[x + 1]);  // Gamma(x) below the slot of (x, h) is < h
        cur[i] = job.y == 0 ? xb : gallop_lower_bound(g.ci, xb, lo, (int32_t)job_lo);
        endp[i] = lo;
        if (job.y == 0) w_wedge += lo - xb;  // the hub's wedges, counted by its first job
      }
    }
    if (threadIdx.x == 0) ++w_jobs;
    for (int64_t lo64 = job_lo; lo64 < job_hi; lo64 += span) {
      const int32_t lo_id = (int32_t)lo64;
      const int32_t r1 = (int32_t)min(lo64 + span, job_hi);
      const int32_t words = (r1 - lo_id + cpw - 1) / cpw;
      for (int32_t i = threadIdx.x; i < words; i += kHeavyBlock) tab[i] = 0u;
      if (threadIdx.x == 0) {
        w_blocks += nx;
        s_chunk[0] = 0;
        s_chunk[1] = 0;
      }
      __syncthreads();
      if (small) {
        if (cpw == 3)
          hub_block_small<3>(g, a, tab, s_sx[warp], s_sx32[warp], comp, rcur, rend, ix, nx, hb, lo_id, r1, lane);
        else
          hub_block_small<2>(g, a, tab, s_sx[warp], s_sx32[warp], comp, rcur, rend, ix, nx, hb, lo_id, r1, lane);
      } else if (cpw == 3)
        hub_block<3>(g, a, tab, s_chunk, s_sx[warp], s_sx32[warp], comp, beg, cur, endp, nx, nchunks, hb, lo_id, r1,
                     lane);
      else if (cpw == 2)
        hub_block<2>(g, a, tab, s_chunk, s_sx[warp], s_sx32[warp], comp, beg, cur, endp, nx, nchunks, hb, lo_id, r1,
                     lane);
      else
        hub_block<1>(g, a, tab, s_chunk, s_sx[warp], s_sx32[warp], comp, beg, cur, endp, nx, nchunks, hb, lo_id, r1,
                     lane);
      __syncthreads();
    }
  }
  for (int o = 16; o; o >>= 1) w_wedge += __shfl_xor_sync(0xffffffffu, w_wedge, o);
  if (lane == 0 && w_wedge) {
    atomicAdd(a.work + kWorkCWedge, (unsigned long long)w_wedge);
    atomicAdd(a.work + kWorkCHeavyWedge, (unsigned long long)w_wedge);
  }
  if (threadIdx.x == 0) {
    if (w_blocks) atomicAdd(a.work + kWorkCBlocks, (unsigned long long)w_blocks);
    if (w_jobs) atomicAdd(a.work + kWorkCHubJobs, (unsigned long long)w_jobs);
    const unsigned long long life = global_ns() - t_start;
    atomicAdd(a.work + kWorkCHubCtas, 1ull);
    atomicAdd(a.work + kWorkCHubBusySum, life);
    atomicMax(a.work + kWorkCHubBusyMax, life);
  }
}

// ---------------- pass C for units of at most kHashMaxW wedges ----------------
// The same wedges and attribution as k_pass_c, with cnt_h(o) in a
// shared-memory hash keyed by o instead of a vertex-indexed table in DRAM
// (open addressing, linear probing; sized per unit to at least twice its
// wedges, so at most half full; 16-bit counts, since cnt_h(o) <= wedges).
// A warp takes one lower neighbour x of h at a time, its lanes the run
// {o in Gamma(x) : o < h}, which ends at the slot of (x, h) (ids are ranks
// and rows ascend).
constexpr int kHashBlock = 512;
constexpr int kHashSlots = 2 * kHashMaxW;
constexpr int kHashSmallBlock = 128;
constexpr int kHashMidBlock = 256;

__device__ __forceinline__ uint32_t o_hash(int32_t o, int bits) {
  return ((uint32_t)o * 0x9E3779B1u) >> (32 - bits);  // Fibonacci hashing
}
// slot of o (inserted if absent), or -1 if the table is full
__device__ __forceinline__ int32_t hash_insert(int32_t* keys, int32_t o, uint32_t mask, int bits) {
  uint32_t sl = o_hash(o, bits);
  for (uint32_t t = 0; t <= mask; ++t) {
    const int32_t kk = *reinterpret_cast<volatile int32_t*>(&keys[sl]);
    if (kk == o) return (int32_t)sl;
    if (kk == -1) {
      const int32_t prev = atomicCAS(&keys[sl], -1, o);
      if (prev == -1 || prev == o) return (int32_t)sl;
    }
    sl = (sl + 1) & mask;
  }
  return -1;
}
// slot of o, or -1 if absent
__device__ __forceinline__ int32_t hash_find(const int32_t* keys, int32_t o, uint32_t mask, int bits) {
  uint32_t sl = o_hash(o, bits);
  for (uint32_t t = 0; t <= mask; ++t) {
    const int32_t kk = keys[sl];
    if (kk == o) return (int32_t)sl;
    if (kk == -1) return -1;
    sl = (sl + 1) & mask;
  }
  return -1;
}

// Three instances: 512-thread CTAs, two an SM, with the table for kHashMaxW
// wedges; 256-thread CTAs, eight an SM, for units of at most kHashMidW; and,
// for the many units of at most kHashSmallW wedges (on R-MAT scale 22, 87 %
// of the hashed units and 10 % of their wedges), 128-thread CTAs with a table
// for kHashSmallW, sixteen an SM, so that a unit's barriers and latency
// chains no longer hold a large CTA. Units [k0, k1) of the hashed list
// (heaviest first), taken from *cursor.
template <int kThreads, int kMaxW>
__global__ void __launch_bounds__(kThreads, kThreads == kHashBlock ? kCtasPerSm : 2048 / kThreads)
    k_pass_c_hash(DevGraph g, CountArgs a, int32_t k0, int32_t k1, int32_t* cursor) {
  extern __shared__ int32_t hkeys[];                                  // [2 kMaxW] o, or -1
  uint32_t* hcnt = reinterpret_cast<uint32_t*>(hkeys + 2 * kMaxW);    // [kMaxW] two counts
  __shared__ int32_t s_unit, s_next[2];
  const int lane = threadIdx.x & 31;
  long long w_wedge = 0;  // lane 0
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_unit = k0 + atomicAdd(cursor, 1);
    __syncthreads();
    const int32_t k = s_unit;
    if (k >= k1) break;
    const int32_t h = a.cunits[a.n_cheavy + k];
    const int32_t wk = min(a.chash_w[k], (int32_t)kMaxW);
    int bits = 6;
    while ((1 << bits) < 2 * wk) ++bits;  // at most log2(kHashSlots)
    const uint32_t mask = (1u << bits) - 1u;
    const int32_t hb = g.rp[h], he = g.rp[h + 1];
    for (int32_t i = threadIdx.x; i <= (int32_t)mask; i += kThreads) hkeys[i] = -1;
    for (int32_t i = threadIdx.x; i <= (int32_t)(mask >> 1); i += kThreads) hcnt[i] = 0u;
    if (threadIdx.x < 2) s_next[threadIdx.x] = hb;
    __syncthreads();
    // pass 0 counts cnt_h(o); pass 1 attributes cnt_h(o) - 1 to the slots
    // (x, o) and, summed over the run, to (h, x)
    for (int pass = 0; pass < 2; ++pass) {
      for (;;) {
        int32_t p = 0;
        if (lane == 0) p = atomicAdd(&s_next[pass], 1);
        p = __shfl_sync(0xffffffffu, p, 0);
        if (p >= he) break;
        const int32_t x = g.ci[p];
        if (x >= h) break;  // the lower neighbours are a prefix of Gamma(h)
        const int32_t xb = g.rp[x];
        const int32_t xe = min(max(g.rev[p], xb), g.rp[x + 1]);  // Gamma(x) below the slot of (x, h)
        if (pass == 0 && lane == 0) w_wedge += xe - xb;
        uint32_t sx = 0u;
        for (int32_t q0 = xb; q0 < xe; q0 += 128) {  // four windows of 32 in flight
          int32_t o[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int32_t q = q0 + 32 * j + lane;
            o[j] = q < xe ? g.ci[q] : -1;
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (o[j] < 0) continue;
            if (pass == 0) {
              const int32_t sl = hash_insert(hkeys, o[j], mask, bits);
              if (sl >= 0) atomicAdd(&hcnt[sl >> 1], 1u << ((sl & 1) << 4));
              else atomicOr(a.status, (int32_t)kSpillOverflow);  // more distinct o than wedges: invalid input
            } else {
              const int32_t sl = hash_find(hkeys, o[j], mask, bits);
              const uint32_t c = sl >= 0 ? ((hcnt[sl >> 1] >> ((sl & 1) << 4)) & 0xffffu) - 1u : 0u;
              if (c) {
                atomicAdd(&a.P[q0 + 32 * j + lane], (unsigned long long)c);  // slot (x, o)
                sx += c;
              }
            }
          }
        }
        if (pass == 1) {
          for (int off = 16; off; off >>= 1) sx += __shfl_xor_sync(0xffffffffu, sx, off);
          if (lane == 0 && sx) atomicAdd(&a.P[p], (unsigned long long)sx);  // slot (h, x)
        }
      }
      __syncthreads();
    }
  }
  if (lane == 0 && w_wedge) {
    atomicAdd(a.work + kWorkCWedge, (unsigned long long)w_wedge);
    atomicAdd(a.work + kWorkCHashWedge, (unsigned long long)w_wedge);
  }
}

// ---------------- pass C for units of at most kHash2MaxW wedges ----------------
// The same counting and attribution as k_pass_c_hash, for the units whose
// wedges do not fit that hash: each slot is one 32-bit word holding the
// vertex o (22 bits; graphs of at most 2^22 vertices) and cnt_h(o) (10 bits;
// units of fewer than 1023 lower neighbours, so a count never reaches 1023
// and a word is never all ones, the empty mark). kHash2Slots words fill the
// shared memory of one 1024-thread CTA per SM; a unit uses the first
// ceil(W / 0.72) of them, so the table is at most 72 % full, and the probe
// position is a multiply-shift of the hash into that range.
constexpr int kHash2Block = 1024;
constexpr uint32_t kHash2Empty = 0xffffffffu;

__device__ __forceinline__ uint32_t h2_start(int32_t o, uint32_t size) {
  return (uint32_t)(((unsigned long long)((uint32_t)o * 0x9E3779B1u) * size) >> 32);
}
// adds 1 to the count of o (inserted with count 1 if absent); false if the
// table is full (cannot happen for a unit sized as above)
__device__ __forceinline__ bool h2_insert(uint32_t* tab, int32_t o, uint32_t size) {
  uint32_t sl = h2_start(o, size);
  for (uint32_t t = 0; t < size; ++t) {
    uint32_t w = *reinterpret_cast<volatile uint32_t*>(&tab[sl]);
    if (w == kHash2Empty) {
      w = atomicCAS(&tab[sl], kHash2Empty, ((uint32_t)o << 10) | 1u);
      if (w == kHash2Empty) return true;
    }
    if ((w >> 10) == (uint32_t)o) {
      atomicAdd(&tab[sl], 1u);
      return true;
    }
    sl = sl + 1 == size ? 0 : sl + 1;
  }
  return false;
}
__device__ __forceinline__ uint32_t h2_count(const uint32_t* tab, int32_t o, uint32_t size) {
  uint32_t sl = h2_start(o, size);
  for (uint32_t t = 0; t < size; ++t) {
    const uint32_t w = tab[sl];
    if (w == kHash2Empty) return 0u;
    if ((w >> 10) == (uint32_t)o) return w & 1023u;
    sl = sl + 1 == size ? 0 : sl + 1;
  }
  return 0u;
}

// Two instances: 1024-thread CTAs with the whole table, one an SM; and
// 512-thread CTAs with half of it, two an SM, for the units of at most
// kHash2HalfMaxW wedges. Units [k0, k1) of the packed-key list (heaviest
// first), taken from *cursor.
template <int kThreads, int kSlots>
__global__ void __launch_bounds__(kThreads, kThreads == kHash2Block ? 1 : 2)
    k_pass_c_hash2(DevGraph g, CountArgs a, int32_t k0, int32_t k1, int32_t* cursor) {
  extern __shared__ uint32_t htab[];  // kSlots packed (o, count) words
  __shared__ int32_t s_unit, s_next[2];
  const int lane = threadIdx.x & 31;
  long long w_wedge = 0;  // lane 0
  const int32_t first = a.n_cheavy + a.n_chash;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_unit = k0 + atomicAdd(cursor, 1);
    __syncthreads();
    const int32_t k = s_unit;
    if (k >= k1) break;
    const int32_t h = a.cunits[first + k];
    const int32_t wk = min(a.chash_w[a.n_chash + k], (int32_t)kHash2MaxW);
    const uint32_t size = min((uint32_t)kSlots, (uint32_t)(((long long)wk * 25 + 17) / 18) + 32u);
    const int32_t hb = g.rp[h], he = g.rp[h + 1];
    for (uint32_t i = threadIdx.x; i < size; i += kThreads) htab[i] = kHash2Empty;
    if (threadIdx.x < 2) s_next[threadIdx.x] = hb;
    __syncthreads();
    // pass 0 counts cnt_h(o); pass 1 attributes cnt_h(o) - 1 to the slots
    // (x, o) and, summed over the run, to (h, x)
    for (int pass = 0; pass < 2; ++pass) {
      for (;;) {
        int32_t p = 0;
        if (lane == 0) p = atomicAdd(&s_next[pass], 1);
        p = __shfl_sync(0xffffffffu, p, 0);
        if (p >= he) break;
        const int32_t x = g.ci[p];
        if (x >= h) break;  // the lower neighbours are a prefix of Gamma(h)
        const int32_t xb = g.rp[x];
        const int32_t xe = min(max(g.rev[p], xb), g.rp[x + 1]);  // Gamma(x) below the slot of (x, h)
        if (pass == 0 && lane == 0) w_wedge += xe - xb;
        unsigned long long sx = 0;
        for (int32_t q0 = xb; q0 < xe; q0 += 128) {  // four windows of 32 in flight
          int32_t o[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int32_t q = q0 + 32 * j + lane;
            o[j] = q < xe ? g.ci[q] : -1;
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (o[j] < 0) continue;
            if (pass == 0) {
              if (!h2_insert(htab, o[j], size)) atomicOr(a.status, (int32_t)kSpillOverflow);
            } else {
              const uint32_t c = h2_count(htab, o[j], size) - 1u;
              if (c && c < 1023u) {
                atomicAdd(&a.P[q0 + 32 * j + lane], (unsigned long long)c);  // slot (x, o)
                sx += c;
              }
            }
          }
        }
        if (pass == 1) {
          for (int off = 16; off; off >>= 1) sx += __shfl_xor_sync(0xffffffffu, sx, off);
          if (lane == 0 && sx) atomicAdd(&a.P[p], sx);  // slot (h, x)
        }
      }
      __syncthreads();
    }
  }
  if (lane == 0 && w_wedge) {
    atomicAdd(a.work + kWorkCWedge, (unsigned long long)w_wedge);
    atomicAdd(a.work + kWorkCHash2Wedge, (unsigned long long)w_wedge);
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

int g_grid = 0;

size_t smem_bytes(bool smem_table, int32_t table_n) {
  return smem_table ? sizeof(uint32_t) * (size_t)((table_n + 3) & ~3) : 0;
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

gc_status run_pass_c(const DevGraph& g, const CountArgs& a, cudaStream_t s) {
  const bool sm = a.tables == nullptr;
  if (sm) return launch(k_pass_c<true>, smem_bytes(true, g.table_n), g, a, s, "k_pass_c");
  return launch(k_pass_c<false>, smem_bytes(false, g.table_n), g, a, s, "k_pass_c");
}

gc_status run_pass_c_heavy(const DevGraph& g, const CountArgs& a, cudaStream_t s) {
  if (a.n_cheavy <= 0) return GC_OK;
  const size_t smem = sizeof(uint32_t) * (size_t)a.hub_tab;
  cudaError_t e = cudaFuncSetAttribute(k_pass_c_heavy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "k_pass_c_heavy");
  int grid = count_grid_size() / kCtasPerSm;
  if (grid > a.n_cjobs) grid = a.n_cjobs;
  if (grid < 1) return GC_OK;
  k_pass_c_heavy<<<grid, kHeavyBlock, smem, s>>>(g, a);
  e = cudaGetLastError();
  return e == cudaSuccess ? GC_OK : cuda_fail(e, "k_pass_c_heavy");
}

template <int kThreads, int kMaxW>
static gc_status launch_hash(const DevGraph& g, const CountArgs& a, int32_t k0, int32_t k1, int32_t* cursor,
                             cudaStream_t s) {
  if (k1 <= k0) return GC_OK;
  auto kern = k_pass_c_hash<kThreads, kMaxW>;
  const size_t smem = sizeof(int32_t) * 2 * kMaxW + sizeof(uint32_t) * kMaxW;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "k_pass_c_hash");
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  if (e != cudaSuccess) return cuda_fail(e, "k_pass_c_hash occupancy");
  int grid = (per_sm > 0 ? per_sm : 1) * (count_grid_size() / kCtasPerSm);
  if (grid > k1 - k0) grid = k1 - k0;
  kern<<<grid, kThreads, smem, s>>>(g, a, k0, k1, cursor);
  e = cudaGetLastError();
  return e == cudaSuccess ? GC_OK : cuda_fail(e, "k_pass_c_hash");
}

gc_status run_pass_c_hash(const DevGraph& g, const CountArgs& a, cudaStream_t s) {
  if (a.n_chash <= 0) return GC_OK;
  gc_status st = launch_hash<kHashBlock, kHashMaxW>(g, a, 0, a.n_chash_mid, a.cursor + 9, s);
  if (st != GC_OK) return st;
  st = launch_hash<kHashMidBlock, kHashMidW>(g, a, a.n_chash_mid, a.n_chash_big, a.cursor + 16, s);
  if (st != GC_OK) return st;
  return launch_hash<kHashSmallBlock, kHashSmallW>(g, a, a.n_chash_big, a.n_chash, a.cursor + 7, s);
}

template <int kThreads, int kSlots>
static gc_status launch_hash2(const DevGraph& g, const CountArgs& a, int32_t k0, int32_t k1, int32_t* cursor,
                              cudaStream_t s) {
  if (k1 <= k0) return GC_OK;
  auto kern = k_pass_c_hash2<kThreads, kSlots>;
  const size_t smem = sizeof(uint32_t) * kSlots;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "k_pass_c_hash2");
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  if (e != cudaSuccess) return cuda_fail(e, "k_pass_c_hash2 occupancy");
  int grid = (per_sm > 0 ? per_sm : 1) * (count_grid_size() / kCtasPerSm);
  if (grid > k1 - k0) grid = k1 - k0;
  kern<<<grid, kThreads, smem, s>>>(g, a, k0, k1, cursor);
  e = cudaGetLastError();
  return e == cudaSuccess ? GC_OK : cuda_fail(e, "k_pass_c_hash2");
}

gc_status run_pass_c_hash2(const DevGraph& g, const CountArgs& a, cudaStream_t s) {
  if (a.n_chash2 <= 0) return GC_OK;
  gc_status st = launch_hash2<kHash2Block, kHash2Slots>(g, a, 0, a.n_chash2_big, a.cursor + 15, s);
  if (st != GC_OK) return st;
  return launch_hash2<kHash2Block / 2, kHash2HalfSlots>(g, a, a.n_chash2_big, a.n_chash2, a.cursor + 17, s);
}

gc_status run_finish(const DevGraph& g, const CountArgs& a, cudaStream_t s) {
  if (g.m == 0) return GC_OK;
  int blocks = (int)min((int64_t)count_grid_size() * 4, ((int64_t)g.m + kFinBlock - 1) / kFinBlock);
  if (a.per_edge_host) k_finish<true><<<blocks, kFinBlock, 0, s>>>(g, a);
  else k_finish<false><<<blocks, kFinBlock, 0, s>>>(g, a);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GC_OK : cuda_fail(e, "k_finish");
}

gc_status run_induced(const DevGraph& g, const CountArgs& a, unsigned long long* vsum, uint64_t* out, bool out_host,
                      cudaStream_t s) {
  if (g.m == 0) return GC_OK;
  const int vblocks = (int)min((int64_t)count_grid_size() * 4, ((int64_t)g.n * 32 + 255) / 256);
  k_vertex_sums<<<vblocks > 0 ? vblocks : 1, 256, 0, s>>>(g, a.trio, vsum);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "k_vertex_sums");
  const int blocks = (int)min((int64_t)count_grid_size() * 4, ((int64_t)g.m + kFinBlock - 1) / kFinBlock);
  unsigned long long* o = reinterpret_cast<unsigned long long*>(out);
  if (out_host) k_finish_induced<true><<<blocks, kFinBlock, 0, s>>>(g, a, vsum, o);
  else k_finish_induced<false><<<blocks, kFinBlock, 0, s>>>(g, a, vsum, o);
  e = cudaGetLastError();
  return e == cudaSuccess ? GC_OK : cuda_fail(e, "k_finish_induced");
}

gc_status run_derive(const DevGraph& g, const unsigned long long* csum, unsigned long long* x,
                     int32_t* status, cudaStream_t s) {
  int blocks = (g.G + 127) / 128;
  k_derive<<<blocks > 0 ? blocks : 1, 128, 0, s>>>(g.G, g.gn, g.gm, csum, x, status);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GC_OK : cuda_fail(e, "k_derive");
}

}  // namespace gc
