// gc_clique.cu -- pass K: the 4-clique step (Alg. 3/5) and the cross term of
// the 4-cycle step, organised by the lowest vertex of every clique.
//
// Each 4-clique {a, b, c, d} has exactly one lowest-rank vertex a (rank =
// (degree, id), the P3 orientation), and then b, c, d all lie in out(a), the
// higher-rank neighbours of a. So the 4-cliques whose lowest vertex is a are
// exactly the triangles of H_a, the subgraph induced on out(a), and the
// triangles whose lowest vertex is a are exactly the edges of H_a. Both are
// counted per edge of the original graph:
//
//   x7(a, b_i)   += #triangles of H_a through vertex i = 1/2 sum_j c_ij
//   x7(b_i, b_j) += c_ij = |N_H(i) ∩ N_H(j)|          for every edge (i, j) of H_a
//
// and for the triangle {a, b_i, b_j} of every edge (i, j) of H_a the term
// |T_(w,x)| + |T_(w,y)| - 2 of its third vertex w goes to each of its three
// edges (x, y) -- summed, that is cross(e) = sum_{w in T_e} (|T_(w,u)| +
// |T_(w,v)| - 2), the term that turns the 4-cycles through e into Alg. 4/6's
// induced count x10 (see gc_count.cu, finish).
//
// Per unit a (one CTA): out(a) (k ids, ascending) is loaded with the |T| of
// its edges, a hash table maps an id to its position i in out(a) (Psi of
// Alg. 1 restricted to out(a)), and H_a is built as a k x k bitmatrix (rows
// padded to an odd word stride, so that lanes reading different rows hit
// different banks). Phase 1 scans out(b) for every b in out(a) and sets the
// bits of the edges found; phase 2 scans again, and for every edge (i, j) of
// H_a (met once, from its lower-rank end) counts c_ij with popcounts over the
// two rows -- Alg. 5's "count adjacent members of T" as bit operations, with
// the Psi reset of Alg. 5 replaced by counting each clique from one vertex.
// Edges of H_a found by a warp go through a 64-entry ring so that every lane
// of the popcount loop has an edge.
//
// Tiers by k: the bitmatrix (k * ((k+31)/32 | 1) words) stays in shared
// memory for k <= 1024; above that the same code runs on a per-CTA global
// buffer; units with k <= 32 run one per warp (k_pass_k_warp). The 512-thread
// CTAs run three to an SM (at most 40 registers a thread, a few bytes of
// spill in two pass-K instances): the passes wait on loads, and the third
// CTA hides more of that wait than the registers it costs (pass T 71.4 ->
// 58.1 ms, pass K 46.3 -> 45.1 ms on R-MAT scale 22). Pass T's k <= 1024 tier
// runs in 512-thread CTAs for the same reason; pass K's keeps 1024 threads,
// since its bitmatrix leaves room for one CTA an SM. Work per unit is about sum_{b in out(a)} |out(b)| (triangle
// listing) plus (#edges of H_a) * k / 32 words.
#include <cuda_runtime.h>

#include "gc_internal.h"

namespace gc {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__host__ __device__ constexpr int row_stride(int k) { return ((k + 31) >> 5) | 1; }

__device__ __forceinline__ uint32_t khash(int32_t key, int bits) {
  return ((uint32_t)key * 0x9E3779B1u) >> (32 - bits);
}
// Second hash, for the bit filter in front of the table.
__device__ __forceinline__ uint32_t fhash(int32_t key, int bits) {
  return ((uint32_t)key * 0x85EBCA6Bu) >> (32 - bits);
}

// 64-bit per-member sums kept as two 32-bit words (lo[i], hi[i]), so that
// shared-memory updates are plain 32-bit atomics.
__device__ __forceinline__ void add_split(uint32_t* lo, uint32_t* hi, int32_t i, unsigned long long v) {
  const uint32_t l = (uint32_t)v;
  uint32_t h = (uint32_t)(v >> 32);
  if (l) {
    const uint32_t old = atomicAdd(&lo[i], l);
    if (old + l < old) ++h;
  }
  if (h) atomicAdd(&hi[i], h);
}
__device__ __forceinline__ unsigned long long read_split(const uint32_t* lo, const uint32_t* hi, int32_t i) {
  return ((unsigned long long)hi[i] << 32) | lo[i];
}

// Byte offsets of the per-unit arrays for a capacity of cap members.
struct KLayout {
  size_t vx7, vcr, ids, ta, hash, filt, rows, total;
  int hcap;
  __host__ __device__ static size_t up16(size_t x) { return (x + 15) & ~(size_t)15; }
  __host__ __device__ explicit KLayout(int cap, bool with_rows = true) {
    int hb = 1;
    while ((1 << hb) < 2 * cap) ++hb;
    hcap = 1 << hb;
    size_t o = 0;
    vx7 = o; o = up16(o + 8 * (size_t)cap);
    vcr = o; o = up16(o + 8 * (size_t)cap);
    ids = o; o = up16(o + 4 * (size_t)cap);
    ta = o; o = up16(o + 4 * (size_t)cap);
    hash = o; o = up16(o + 4 * (size_t)hcap);
    filt = o; o = up16(o + (size_t)hcap);  // 8 filter bits per hash slot
    rows = o; o = with_rows ? up16(o + 4 * (size_t)cap * (size_t)row_stride(cap)) : o;
    total = o;
  }
};

// kTri: the triangle step alone (|T| per edge, Alg. 1): every triangle is an
// edge of exactly one H_a, so phase 1 adds 1 to that edge and to the two
// edges (a, b_i), (a, b_j), and nothing else runs. kDeg (with kTri): each
// triangle also adds the degree of its third vertex to each of its edges,
// so that a.dsum[e] = sum_{w in T_e} d_w (for the per-edge induced counts).
template <int kCap, int kThreads, bool kTri, bool kDeg = false>
__global__ void __launch_bounds__(kThreads, kThreads == 512 ? 3 : 65536 / (kThreads * 64)) k_pass_k(DevGraph g, CountArgs a, int tier) {
  constexpr int kW = kThreads / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int32_t s_unit, s_cur1, s_cur2, s_nhit;
  __shared__ long long s_loff;
  __shared__ int32_t s_qj[kW][64], s_qq[kW][64];
  // pass T: the warp's entries that passed the bit filter, waiting for a
  // full warp of hash probes (fewer than 32 left over + 128 of a round)
  __shared__ int32_t s_pc[kW][kTri ? 160 : 1], s_pq[kW][kTri ? 160 : 1];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cap = kCap ? kCap : a.kbuf_cap;
  const KLayout L(cap, !kTri);
  unsigned char* base = kCap ? smem : a.kbuf + (size_t)blockIdx.x * a.kbuf_stride;
  uint32_t* vx7 = reinterpret_cast<uint32_t*>(base + L.vx7);  // [cap] lo, [cap] hi
  uint32_t* vx7h = vx7 + cap;
  uint32_t* vcr = reinterpret_cast<uint32_t*>(base + L.vcr);
  uint32_t* vcrh = vcr + cap;
  int32_t* ids = reinterpret_cast<int32_t*>(base + L.ids);
  int32_t* ta = reinterpret_cast<int32_t*>(base + L.ta);
  int32_t* hash = reinterpret_cast<int32_t*>(base + L.hash);
  uint32_t* filt = reinterpret_cast<uint32_t*>(base + L.filt);
  uint32_t* rows = reinterpret_cast<uint32_t*>(base + L.rows);
  int32_t* qj = s_qj[warp];
  int32_t* qq = s_qq[warp];
  // phase-1 hits (i, j, out-slot): pass K's phase 2 needs no rescan, and
  // pass T hands them on to pass K
  int32_t* hits = (kTri && !a.tlist) ? nullptr : a.hitbuf + (size_t)blockIdx.x * 2 * (size_t)a.hitcap;

  const int32_t u0 = a.ktier_off[tier], u1 = a.ktier_off[tier + 1];
  int32_t* cursor = a.cursor + (kTri ? 10 : 2) + tier;
  long long w_members = 0, w_scan = 0, w_edges = 0, w_words = 0;  // per warp, lane 0

  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      s_unit = u0 + atomicAdd(cursor, 1);
      s_cur1 = 0;
      s_cur2 = 0;
      s_nhit = 0;
    }
    __syncthreads();
    const int32_t ui = s_unit;
    if (ui >= u1) break;
    const int32_t av = a.kunits[ui];
    const int32_t ob = g.out_ptr[av];
    const int32_t k = g.out_ptr[av + 1] - ob;
    if (k > cap) {  // cannot happen: units are binned by k
      if (threadIdx.x == 0) atomicOr(a.status, (int32_t)kSpillOverflow);
      continue;
    }
    const int W = (k + 31) >> 5, S = W | 1;
    int hbits = 1;
    while ((1 << hbits) < 2 * k) ++hbits;
    const uint32_t hmask = (1u << hbits) - 1u;
    const int fbits = hbits + 3;

    for (int32_t i = threadIdx.x; i < k; i += kThreads) {
      ids[i] = g.out_idx[ob + i];
      vx7[i] = 0u;
      vx7h[i] = 0u;
      if (!kTri || kDeg) {
        ta[i] = kTri ? g.deg[ids[i]] : a.trio[ob + i];  // kDeg: the member's degree
        vcr[i] = 0u;
        vcrh[i] = 0u;
      }
    }
    const int32_t da = kDeg ? g.deg[av] : 0;
    // pass K with the edges of H_a kept by pass T: no hash, no scan
    const int32_t lcnt = (!kTri && a.tlist) ? a.tl_cnt[ui] : -1;
    if (lcnt < 0) {
      for (int32_t i = threadIdx.x; i <= (int32_t)hmask; i += kThreads) hash[i] = 0;
      for (int32_t i = threadIdx.x; i < (1 << fbits) / 32; i += kThreads) filt[i] = 0u;
    }
    if (!kTri)
      for (int32_t i = threadIdx.x; i < k * S; i += kThreads) rows[i] = 0u;
    if (threadIdx.x == 0) w_members += k;
    __syncthreads();
    if (lcnt >= 0) {
      const int2* lst = a.tlist + a.tl_off[ui];
      for (int32_t e = threadIdx.x; e < lcnt; e += kThreads) {
        const int32_t ij = lst[e].x;
        const int32_t i = (int32_t)((uint32_t)ij >> 16), j = ij & 0xffff;
        atomicOr(&rows[i * S + (j >> 5)], 1u << (j & 31));
        atomicOr(&rows[j * S + (i >> 5)], 1u << (i & 31));
      }
      __syncthreads();
      for (int32_t e0 = warp * 32; e0 < lcnt; e0 += kThreads) {
        const int32_t e = e0 + lane;
        if (e < lcnt) {
          const int2 en = lst[e];
          const int32_t i = (int32_t)((uint32_t)en.x >> 16), j = en.x & 0xffff, q = en.y;
          const uint32_t* ri = rows + i * S;
          const uint32_t* rj = rows + j * S;
          int c4 = 0;
          for (int w = 0; w < W; ++w) c4 += __popc(ri[w] & rj[w]);
          const int32_t ti = ta[i], tj = ta[j];
          const int32_t tij = a.trio[q];
          if (c4) {
            atomicAdd(&a.xc[2 * (size_t)q], (unsigned long long)c4);
            add_split(vx7, vx7h, i, (unsigned long long)c4);
            add_split(vx7, vx7h, j, (unsigned long long)c4);
          }
          atomicAdd(&a.xc[2 * (size_t)q + 1], (unsigned long long)(ti + tj - 2));
          add_split(vcr, vcrh, i, (unsigned long long)(tj + tij - 2));
          add_split(vcr, vcrh, j, (unsigned long long)(ti + tij - 2));
        }
        if (lane == 0) {
          const int32_t cnt = min(32, lcnt - e0);
          w_edges += cnt;
          w_words += (long long)cnt * W;
        }
      }
      __syncthreads();
      for (int32_t i = threadIdx.x; i < k; i += kThreads) {
        const unsigned long long x = read_split(vx7, vx7h, i), c = read_split(vcr, vcrh, i);
        if (x) atomicAdd(&a.xc[2 * (size_t)(ob + i)], x >> 1);
        if (c) atomicAdd(&a.xc[2 * (size_t)(ob + i) + 1], c);
      }
      continue;
    }
    for (int32_t i = threadIdx.x; i < k; i += kThreads) {  // Psi: id -> 1 + position in out(a)
      uint32_t h = khash(ids[i], hbits);
      while (atomicCAS(&hash[h], 0, i + 1) != 0) h = (h + 1) & hmask;  // table at most half full
      const uint32_t f = fhash(ids[i], fbits);
      atomicOr(&filt[f >> 5], 1u << (f & 31));
    }
    __syncthreads();
    const int32_t cmax = ids[k - 1];
    auto filter_pass = [&](int32_t c) -> bool {
      const uint32_t f = fhash(c, fbits);
      return (filt[f >> 5] >> (f & 31)) & 1u;  // at most one bit in 16 set
    };
    auto probe = [&](int32_t c) -> int32_t {  // position of c in out(a), or -1
      uint32_t h = khash(c, hbits);
      for (;;) {
        const int32_t s = hash[h];
        if (s == 0) return -1;
        if (ids[s - 1] == c) return s - 1;
        h = (h + 1) & hmask;
      }
    };
    auto lookup = [&](int32_t c) -> int32_t { return filter_pass(c) ? probe(c) : -1; };

    // Phase 1: the edges of H_a, as symmetric bits.
    for (;;) {
      int32_t i = 0;
      if (lane == 0) i = atomicAdd(&s_cur1, 1);
      i = __shfl_sync(kFull, i, 0);
      if (i >= k) break;
      const int32_t b = ids[i];
      const int32_t bb = g.out_ptr[b], be = g.out_ptr[b + 1];
      if (kTri) {
        // The triangle step: four windows of 32 entries per round (four loads
        // in flight per lane); the entries that pass the bit filter are
        // compacted into the warp's buffer and looked up in the hash 32 at a
        // time, so that every lane of a probe has an entry (about one entry
        // in seven passes the filter). out(b) ascends: the scan stops at the
        // first round that reaches past max out(a).
        int32_t* pc = s_pc[warp];
        int32_t* pq = s_pq[warp];
        int32_t pend = 0;  // warp-uniform
        auto probe_batch = [&](int32_t take) {  // the last `take` buffered entries
          const int32_t c = lane < take ? pc[pend - take + lane] : 0;
          const int32_t q = lane < take ? pq[pend - take + lane] : 0;
          const int32_t j = lane < take ? probe(c) : -1;
          const unsigned hit = __ballot_sync(kFull, j >= 0);
          if (j >= 0) {
            atomicAdd(&a.trio[q], 1);  // edge (b_i, c)
            atomicAdd(&vx7[j], 1u);    // edge (a, c)
            if (kDeg) {
              atomicAdd(&a.dsum[q], (unsigned long long)da);       // edge (b_i, c): third vertex a
              add_split(vcr, vcrh, j, (unsigned long long)ta[i]);  // edge (a, c): third vertex b_i
            }
          }
          if (kDeg && hit) {  // edge (a, b_i): third vertices c
            unsigned long long sd = j >= 0 ? (unsigned long long)ta[j] : 0ull;
            for (int o = 16; o; o >>= 1) sd += __shfl_xor_sync(kFull, sd, o);
            if (lane == 0) add_split(vcr, vcrh, i, sd);
          }
          if (lane == 0 && hit) {
            atomicAdd(&vx7[i], (uint32_t)__popc(hit));  // edge (a, b_i)
            w_edges += __popc(hit);
          }
          if (hits && hit) {  // recorded for pass K
            int32_t base_h = 0;
            if (lane == 0) base_h = atomicAdd(&s_nhit, __popc(hit));
            base_h = __shfl_sync(kFull, base_h, 0);
            const int32_t slot = base_h + __popc(hit & ((1u << lane) - 1u));
            if (j >= 0 && slot < a.hitcap)
              reinterpret_cast<int2*>(hits)[slot] = make_int2((int32_t)(((uint32_t)i << 16) | (uint32_t)j), q);
          }
          pend -= take;
          __syncwarp();  // the entries are read before the buffer is refilled
        };
        for (int32_t q0 = bb; q0 < be; q0 += 128) {
          int32_t cw[4];
#pragma unroll
          for (int w4 = 0; w4 < 4; ++w4) {
            const int32_t q = q0 + 32 * w4 + lane;
            cw[w4] = q < be ? g.out_idx[q] : 0x7fffffff;
          }
          if (lane == 0) w_scan += min(128, be - q0);
          const bool past = __shfl_sync(kFull, cw[3], 31) > cmax;
#pragma unroll
          for (int w4 = 0; w4 < 4; ++w4) {
            const int32_t c = cw[w4];
            const bool pass = c <= cmax && filter_pass(c);
            const unsigned pm = __ballot_sync(kFull, pass);
            if (pass) {
              const int32_t pos = pend + __popc(pm & ((1u << lane) - 1u));
              pc[pos] = c;
              pq[pos] = q0 + 32 * w4 + lane;
            }
            pend += __popc(pm);
          }
          __syncwarp();
          const bool last = past || q0 + 128 >= be;
          while (pend >= 32) probe_batch(32);
          if (last && pend > 0) probe_batch(pend);
          if (past) break;
        }
        continue;
      }
      // pass K for a unit whose edges were not kept: four windows of 32
      // entries per round, so that four loads are in flight per lane
      for (int32_t q0 = bb; q0 < be; q0 += 128) {
        int32_t cw[4];
#pragma unroll
        for (int w4 = 0; w4 < 4; ++w4) {
          const int32_t q = q0 + 32 * w4 + lane;
          cw[w4] = q < be ? g.out_idx[q] : 0x7fffffff;
        }
        if (lane == 0) w_scan += min(128, be - q0);
        const bool past = __shfl_sync(kFull, cw[3], 31) > cmax;
#pragma unroll
        for (int w4 = 0; w4 < 4; ++w4) {
          const int32_t q = q0 + 32 * w4 + lane;
          const int32_t c = cw[w4];
          const int32_t j = c <= cmax ? lookup(c) : -1;
          const unsigned hit = __ballot_sync(kFull, j >= 0);
          if (hit) {  // pass K scanning again: the edges of H_a as bits, and their list
            int32_t base_h = 0;
            if (lane == 0) base_h = atomicAdd(&s_nhit, __popc(hit));
            base_h = __shfl_sync(kFull, base_h, 0);
            if (j >= 0) {
              atomicOr(&rows[i * S + (j >> 5)], 1u << (j & 31));
              atomicOr(&rows[j * S + (i >> 5)], 1u << (i & 31));
              const int32_t slot = base_h + __popc(hit & ((1u << lane) - 1u));
              if (slot < a.hitcap)  // read only when k <= 65535
                reinterpret_cast<int2*>(hits)[slot] = make_int2((int32_t)(((uint32_t)i << 16) | (uint32_t)j), q);
            }
          }
        }
        if (past) break;
      }
    }
    __syncthreads();
    if (kTri) {
      for (int32_t i = threadIdx.x; i < k; i += kThreads) {
        if (vx7[i]) atomicAdd(&a.trio[ob + i], (int32_t)vx7[i]);
        if (kDeg) {
          const unsigned long long sd = read_split(vcr, vcrh, i);
          if (sd) atomicAdd(&a.dsum[ob + i], sd);
        }
      }
      if (a.tlist) {  // hand the edges of H_a on to pass K, if they fit
        const int32_t nh = s_nhit;
        if (threadIdx.x == 0) {
          long long off = -1;
          if (nh <= a.hitcap && k <= 65535) {
            const unsigned long long o = atomicAdd(a.tlist_fill, (unsigned long long)nh);
            if ((long long)o + nh <= a.tlist_cap) off = (long long)o;
          }
          s_loff = off;
          a.tl_off[ui] = off < 0 ? 0 : off;
          a.tl_cnt[ui] = off < 0 ? -1 : nh;
        }
        __syncthreads();
        const long long off = s_loff;
        if (off >= 0)
          for (int32_t e = threadIdx.x; e < nh; e += kThreads)
            a.tlist[off + e] = reinterpret_cast<const int2*>(hits)[e];
      }
      continue;
    }
    const int32_t nhit = s_nhit;

    if (nhit <= a.hitcap && k <= 65535) {  // (i, j) packed in 16 bits each
      // Phase 2 over the recorded edges of H_a: lane per edge.
      for (int32_t e0 = warp * 32; e0 < nhit; e0 += kThreads) {
        const int32_t e = e0 + lane;
        if (e < nhit) {
          const int2 en = reinterpret_cast<const int2*>(hits)[e];
          const int32_t ij = en.x, q = en.y;
          const int32_t i = (int32_t)((uint32_t)ij >> 16), j = ij & 0xffff;
          const uint32_t* ri = rows + i * S;
          const uint32_t* rj = rows + j * S;
          int c4 = 0;
          for (int w = 0; w < W; ++w) c4 += __popc(ri[w] & rj[w]);
          const int32_t ti = ta[i], tj = ta[j];
          const int32_t tij = a.trio[q];
          if (c4) {
            atomicAdd(&a.xc[2 * (size_t)q], (unsigned long long)c4);
            if (kCap) {  // at most k^2 per member: no carry for k <= 1024
              atomicAdd(&vx7[i], (uint32_t)c4);
              atomicAdd(&vx7[j], (uint32_t)c4);
            } else {
              add_split(vx7, vx7h, i, (unsigned long long)c4);
              add_split(vx7, vx7h, j, (unsigned long long)c4);
            }
          }
          atomicAdd(&a.xc[2 * (size_t)q + 1], (unsigned long long)(ti + tj - 2));
          add_split(vcr, vcrh, i, (unsigned long long)(tj + tij - 2));
          add_split(vcr, vcrh, j, (unsigned long long)(ti + tij - 2));
        }
        if (lane == 0) {
          const int32_t cnt = min(32, nhit - e0);
          w_edges += cnt;
          w_words += (long long)cnt * W;
        }
      }
    } else {

    // Phase 2: per edge (i, j) of H_a, c_ij and the cross terms.
    for (;;) {
      int32_t i = 0;
      if (lane == 0) i = atomicAdd(&s_cur2, 1);
      i = __shfl_sync(kFull, i, 0);
      if (i >= k) break;
      const int32_t b = ids[i];
      const int32_t bb = g.out_ptr[b], be = g.out_ptr[b + 1];
      const int32_t ti = ta[i];
      const uint32_t* ri = rows + i * S;
      unsigned long long ax7 = 0, acr = 0;
      uint32_t head = 0, tail = 0;
      auto process = [&](int32_t j, int32_t q) {
        const uint32_t* rj = rows + j * S;
        int c4 = 0;
        for (int w = 0; w < W; ++w) c4 += __popc(ri[w] & rj[w]);
        const int32_t tj = ta[j];
        const int32_t tij = a.trio[q];
        if (c4) atomicAdd(&a.xc[2 * (size_t)q], (unsigned long long)c4);
        atomicAdd(&a.xc[2 * (size_t)q + 1], (unsigned long long)(ti + tj - 2));
        if (c4) add_split(vx7, vx7h, j, (unsigned long long)c4);
        add_split(vcr, vcrh, j, (unsigned long long)(ti + tij - 2));
        ax7 += (unsigned long long)c4;
        acr += (unsigned long long)(tj + tij - 2);
      };
      for (int32_t q0 = bb; q0 < be; q0 += 32) {
        const int32_t q = q0 + lane;
        const int32_t c = q < be ? g.out_idx[q] : 0x7fffffff;
        if (__shfl_sync(kFull, c, 0) > cmax) break;
        const int32_t j = c <= cmax ? lookup(c) : -1;
        const unsigned hit = __ballot_sync(kFull, j >= 0);
        if (j >= 0) {
          const uint32_t pos = (tail + __popc(hit & ((1u << lane) - 1u))) & 63u;
          qj[pos] = j;
          qq[pos] = q;
        }
        tail += __popc(hit);
        __syncwarp();
        if (tail - head >= 32) {
          const uint32_t pos = (head + lane) & 63u;
          process(qj[pos], qq[pos]);
          head += 32;
          if (lane == 0) {
            w_edges += 32;
            w_words += 32LL * W;
          }
          __syncwarp();
        }
      }
      const uint32_t left = tail - head;
      if (lane < (int)left) {
        const uint32_t pos = (head + lane) & 63u;
        process(qj[pos], qq[pos]);
      }
      if (lane == 0) {
        w_edges += left;
        w_words += (long long)left * W;
      }
      __syncwarp();
      for (int o = 16; o; o >>= 1) {
        ax7 += __shfl_xor_sync(kFull, ax7, o);
        acr += __shfl_xor_sync(kFull, acr, o);
      }
      if (lane == 0) {
        if (ax7) add_split(vx7, vx7h, i, ax7);
        if (acr) add_split(vcr, vcrh, i, acr);
      }
    }
    }  // phase 2
    __syncthreads();

    // Edges (a, b_i): triangles of H_a through i (each counted from both of
    // its edges at i, hence the halving) and the cross terms gathered above.
    for (int32_t i = threadIdx.x; i < k; i += kThreads) {
      const unsigned long long x = read_split(vx7, vx7h, i), c = read_split(vcr, vcrh, i);
      if (x) atomicAdd(&a.xc[2 * (size_t)(ob + i)], x >> 1);
      if (c) atomicAdd(&a.xc[2 * (size_t)(ob + i) + 1], c);
    }
  }
  if (lane == 0) {
    if (w_members) atomicAdd(a.work + (kTri ? kWorkTMembers : kWorkKMembers), (unsigned long long)w_members);
    if (w_scan) atomicAdd(a.work + (kTri ? kWorkTScan : kWorkKScan), (unsigned long long)w_scan);
    if (w_edges) atomicAdd(a.work + (kTri ? kWorkTTriangles : kWorkKLocalEdges), (unsigned long long)w_edges);
    if (w_words) atomicAdd(a.work + kWorkKWords, (unsigned long long)w_words);
  }
}

// Units with k <= 32: one warp per unit, lane i holding member b_i, its
// row of H_a as a 32-bit mask and the out-slots of the edges found from it
// (shared memory). Membership of an id in out(a) is a 5-step binary search
// over the lanes' ids (ascending). Same attribution as k_pass_k.
constexpr int kWBlock = 256;
constexpr int kWWarps = kWBlock / 32;

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x) {
  for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}

template <bool kTri, bool kDeg = false>
__global__ void __launch_bounds__(kWBlock) k_pass_k_warp(DevGraph g, CountArgs a, int tier) {
  __shared__ int32_t s_q[kWWarps][32 * 32];  // out-slot of edge (i, j) found from member i
  __shared__ uint32_t s_rowf[kWWarps][64];    // rows and found masks rebuilt from pass T's list
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t* qs = s_q[warp];
  const int32_t u0 = a.ktier_off[tier], u1 = a.ktier_off[tier + 1];
  int32_t* cursor = a.cursor + (kTri ? 10 : 2) + tier;
  long long w_members = 0, w_scan = 0, w_edges = 0;  // lane 0
  for (;;) {
    int32_t ui = 0;
    if (lane == 0) ui = u0 + atomicAdd(cursor, 1);
    ui = __shfl_sync(kFull, ui, 0);
    if (ui >= u1) break;
    const int32_t av = a.kunits[ui];
    const int32_t ob = g.out_ptr[av];
    const int32_t k = g.out_ptr[av + 1] - ob;
    if (k > 32) {  // cannot happen: units are binned by k
      if (lane == 0) atomicOr(a.status, (int32_t)kSpillOverflow);
      continue;
    }
    const int32_t id = lane < k ? g.out_idx[ob + lane] : 0x7fffffff;
    const int32_t ti = (!kTri && lane < k) ? a.trio[ob + lane] : 0;
    const int32_t dl = (kDeg && lane < k) ? g.deg[id] : 0;  // kDeg: degree of member b_lane
    const int32_t da = kDeg ? g.deg[av] : 0;
    const int32_t cmax = __shfl_sync(kFull, id, k - 1);
    unsigned row = 0u, found = 0u;
    const int32_t lcnt = (!kTri && a.tlist) ? a.tl_cnt[ui] : -1;
    if (lcnt >= 0) {  // pass K with the edges of H_a kept by pass T
      uint32_t* rw = s_rowf[warp];
      rw[lane] = 0u;
      rw[32 + lane] = 0u;
      __syncwarp();
      const int2* lst = a.tlist + a.tl_off[ui];
      for (int32_t e = lane; e < lcnt; e += 32) {
        const int2 en = lst[e];
        const int32_t i = (int32_t)((uint32_t)en.x >> 16), j = en.x & 0xffff;
        atomicOr(&rw[i], 1u << j);
        atomicOr(&rw[j], 1u << i);
        atomicOr(&rw[32 + i], 1u << j);
        qs[i * 32 + j] = en.y;
      }
      __syncwarp();
      row = rw[lane];
      found = rw[32 + lane];
      if (lane == 0) w_edges += lcnt;
    } else {
    // Phase 1: the edges of H_a.
    for (int i = 0; i < k; ++i) {
      const int32_t b = __shfl_sync(kFull, id, i);
      const int32_t bb = g.out_ptr[b], be = g.out_ptr[b + 1];
      unsigned hits = 0u;
      for (int32_t q0 = bb; q0 < be; q0 += 128) {  // four windows of 32 in flight
        int32_t cw[4];
#pragma unroll
        for (int w4 = 0; w4 < 4; ++w4) {
          const int32_t q = q0 + 32 * w4 + lane;
          cw[w4] = q < be ? g.out_idx[q] : 0x7fffffff;
        }
        if (lane == 0) w_scan += min(128, be - q0);
        const bool past = __shfl_sync(kFull, cw[3], 31) > cmax;
#pragma unroll
        for (int w4 = 0; w4 < 4; ++w4) {
          const int32_t q = q0 + 32 * w4 + lane;
          const int32_t c = cw[w4];
          int lo = 0;
#pragma unroll
          for (int step = 16; step; step >>= 1)
            if (__shfl_sync(kFull, id, lo + step) <= c) lo += step;
          const int32_t id_lo = __shfl_sync(kFull, id, lo);  // every lane takes part in the shuffle
          const bool hit = c <= cmax && id_lo == c && lo < k;  // lanes >= k hold padding ids
          if (hit) {
            if (kTri) atomicAdd(&a.trio[q], 1);  // edge (b_i, c)
            if (kDeg) atomicAdd(&a.dsum[q], (unsigned long long)da);  // its third vertex a
            qs[i * 32 + lo] = q;
          }
          hits |= __reduce_or_sync(kFull, hit ? 1u << lo : 0u);
        }
        if (past) break;
      }
      if (lane == i) {
        found = hits;
        row |= hits;
      }
      if ((hits >> lane) & 1u) row |= 1u << i;
      if (lane == 0) w_edges += __popc(hits);
    }
    }  // scan
    if (kTri) {  // edge (a, b_lane): one triangle per edge of H_a at lane
      if (lane < k && row) atomicAdd(&a.trio[ob + lane], __popc(row));
      if (kDeg) {  // and the degrees of their third vertices b_i
        unsigned long long sd = 0;
        for (int i = 0; i < k; ++i) {
          const int32_t di = __shfl_sync(kFull, dl, i);
          if ((row >> i) & 1u) sd += (unsigned long long)di;
        }
        if (lane < k && sd) atomicAdd(&a.dsum[ob + lane], sd);
      }
      if (lane == 0) w_members += k;
      if (a.tlist) {  // hand the edges of H_a on to pass K
        const int c = __popc(found);
        int incl = c;
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(kFull, incl, o);
          if (lane >= o) incl += y;
        }
        const int total = __shfl_sync(kFull, incl, 31);
        long long off = -1;
        if (lane == 0) {
          const unsigned long long o = atomicAdd(a.tlist_fill, (unsigned long long)total);
          if ((long long)o + total <= a.tlist_cap) off = (long long)o;
          a.tl_off[ui] = off < 0 ? 0 : off;
          a.tl_cnt[ui] = off < 0 ? -1 : total;
        }
        off = __shfl_sync(kFull, off, 0);
        if (off >= 0) {
          // entry e of the unit's list, lane per entry: its row r is the
          // number of rows whose inclusive prefix is <= e, its column the
          // (e - exclusive prefix of r)-th set bit of found_r
          for (int32_t e0 = 0; e0 < total; e0 += 32) {  // warp-uniform trip count
            const int32_t e = e0 + lane;
            int r = 0;
#pragma unroll
            for (int step = 16; step; step >>= 1)
              if (__shfl_sync(kFull, incl, r + step - 1) <= e) r += step;
            const unsigned fr = __shfl_sync(kFull, found, r);
            const int ir = __shfl_sync(kFull, incl, r);
            if (e < total) {
              unsigned f = fr;
              for (int t = e - (ir - __popc(fr)); t > 0; --t) f &= f - 1;
              const int j = __ffs(f) - 1;
              a.tlist[off + e] = make_int2((int32_t)(((uint32_t)r << 16) | (uint32_t)j), qs[r * 32 + j]);
            }
          }
        }
        __syncwarp();
      }
      continue;
    }
    __syncwarp();
    // Phase 2: c_ij and the cross terms of every edge (i, j) of H_a.
    unsigned long long vx = 0, vc = 0;  // for the edge (a, b_lane)
    for (int i = 0; i < k; ++i) {
      const unsigned ri = __shfl_sync(kFull, row, i);
      const unsigned fi = __shfl_sync(kFull, found, i);
      const int32_t tI = __shfl_sync(kFull, ti, i);
      if (fi == 0u) continue;  // warp-uniform
      unsigned long long cx = 0, cc = 0;
      if ((fi >> lane) & 1u) {
        const int32_t q = qs[i * 32 + lane];
        const int c4 = __popc(ri & row);
        const int32_t tij = a.trio[q];
        if (c4) atomicAdd(&a.xc[2 * (size_t)q], (unsigned long long)c4);
        atomicAdd(&a.xc[2 * (size_t)q + 1], (unsigned long long)(tI + ti - 2));
        vx += (unsigned long long)c4;
        vc += (unsigned long long)(tI + tij - 2);
        cx = (unsigned long long)c4;
        cc = (unsigned long long)(ti + tij - 2);
      }
      cx = warp_sum_u64(cx);
      cc = warp_sum_u64(cc);
      if (lane == i) {
        vx += cx;
        vc += cc;
      }
    }
    if (lane < k) {
      if (vx) atomicAdd(&a.xc[2 * (size_t)(ob + lane)], vx >> 1);
      if (vc) atomicAdd(&a.xc[2 * (size_t)(ob + lane) + 1], vc);
    }
    if (lane == 0) w_members += k;
    __syncwarp();
  }
  if (lane == 0) {
    if (w_members) atomicAdd(a.work + (kTri ? kWorkTMembers : kWorkKMembers), (unsigned long long)w_members);
    if (w_scan) atomicAdd(a.work + (kTri ? kWorkTScan : kWorkKScan), (unsigned long long)w_scan);
    if (w_edges) {
      atomicAdd(a.work + (kTri ? kWorkTTriangles : kWorkKLocalEdges), (unsigned long long)w_edges);
      if (!kTri) atomicAdd(a.work + kWorkKWords, (unsigned long long)w_edges);
    }
  }
}

template <int kCap, int kThreads, bool kTri, bool kDeg = false>
gc_status launch_tier(const DevGraph& g, const CountArgs& a, int tier, cudaStream_t s, int* launches) {
  const int32_t units = a.ktier_off[tier + 1] - a.ktier_off[tier];
  if (units <= 0) return GC_OK;
  const size_t smem = kCap ? KLayout(kCap, !kTri).total : 0;
  auto kern = k_pass_k<kCap, kThreads, kTri, kDeg>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "k_pass_k attribute");
  int grid = 0;
  if (kCap) {
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
    if (e != cudaSuccess) return cuda_fail(e, "k_pass_k occupancy");
    grid = (per_sm > 0 ? per_sm : 1) * (count_grid_size() / kCtasPerSm);
  } else {
    grid = a.kbuf_ctas;
  }
  if (grid > a.hitbuf_ctas) grid = a.hitbuf_ctas;  // one hit buffer per CTA
  if (grid > units) grid = units;
  if (grid < 1) return GC_OK;
  kern<<<grid, kThreads, smem, s>>>(g, a, tier);
  ++*launches;
  e = cudaGetLastError();
  return e == cudaSuccess ? GC_OK : cuda_fail(e, "k_pass_k");
}

template <bool kTri, bool kDeg = false>
gc_status run_tiers(const DevGraph& g, const CountArgs& a, cudaStream_t s, int* launches) {
  gc_status st;
  if (a.ktier_off[kTierGlobal + 1] > a.ktier_off[kTierGlobal]) {
    if (!a.kbuf || a.kbuf_ctas < 1) {
      set_error("internal: pass K global buffers missing");
      return GC_ERR_CUDA;
    }
    if ((st = launch_tier<0, 1024, kTri, kDeg>(g, a, kTierGlobal, s, launches)) != GC_OK) return st;
  }
  if ((st = launch_tier<1024, kTri ? 512 : 1024, kTri, kDeg>(g, a, kTier1024, s, launches)) != GC_OK) return st;
  if ((st = launch_tier<512, 512, kTri, kDeg>(g, a, kTier512, s, launches)) != GC_OK) return st;
  if ((st = launch_tier<256, 512, kTri, kDeg>(g, a, kTier256, s, launches)) != GC_OK) return st;
  const int32_t units = a.ktier_off[kTier32 + 1] - a.ktier_off[kTier32];
  if (units > 0) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pass_k_warp<kTri, kDeg>, kWBlock, 0);
    if (e != cudaSuccess) return cuda_fail(e, "k_pass_k_warp occupancy");
    int grid = (per_sm > 0 ? per_sm : 1) * (count_grid_size() / kCtasPerSm);
    const int need = (units + kWWarps - 1) / kWWarps;
    if (grid > need) grid = need;
    k_pass_k_warp<kTri, kDeg><<<grid, kWBlock, 0, s>>>(g, a, kTier32);
    ++*launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_pass_k_warp");
  }
  return GC_OK;
}

}  // namespace

size_t kbuf_bytes(int32_t cap) { return cap > 0 ? KLayout(cap).total : 0; }

gc_status run_pass_k(const DevGraph& g, const CountArgs& a, cudaStream_t s, int* launches) {
  return run_tiers<false>(g, a, s, launches);
}

gc_status run_pass_t(const DevGraph& g, const CountArgs& a, cudaStream_t s, int* launches) {
  return a.dsum ? run_tiers<true, true>(g, a, s, launches) : run_tiers<true>(g, a, s, launches);
}

}  // namespace gc
