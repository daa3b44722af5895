// oracle.cpp -- plain CPU reference for per-edge 3/4-node graphlet counts.
//
// TEST INFRASTRUCTURE ONLY. Nothing on the product path may call this code;
// only the test suite, __graft_entry__.smoke() and bench.py's cpu_baseline
// leg use it. It shares no code with the CUDA path.
//
// What it computes (Rossi & Zhou, "Hybrid CPU-GPU Framework for Network
// Motifs", arXiv 1608.05138):
//   * per edge e = (u, v), with d_v >= d_u (preprocessing step P3; ties go to
//     the smaller id as u), the sets of Fig. 2: T = common neighbours,
//     S_u = Gamma(u) \ T \ {v}, S_v = Gamma(v) \ T \ {u};
//   * |T| by Alg. 1 (neighbour marks in a hash Psi with vertex types
//     lambda1 = neighbour of v, lambda2 = S_u, lambda3 = T; the lambdas are
//     unique per edge so Psi is never reset, Sec. 4.5);
//   * x7 (4-cliques on e) by Alg. 5: for w in T scan Gamma(w) for lambda3,
//     then clear Psi(w) so each pair of T is counted once;
//   * x10 (induced 4-cycles on e) by Alg. 6 read with the membership test of
//     Alg. 4: for w in S_u scan Gamma(w) and count r in S_v, i.e. Psi(r) still
//     lambda1 (Alg. 6 as printed tests lambda2, which would count tailed
//     triangles; Alg. 4 pairs S_u with S_v);
//   * the 13 per-edge columns (the per-edge 3-graphlet equations of Sec. 4.5
//     with x5 read as D_e = n - 2 - |T| - |S_u| - |S_v|, and the summands of
//     the unrestricted counts C_3 .. C_16);
//   * C_3 .. C_16 summed in unsigned 128-bit, with C_9 read as
//     sum |T| (|S_u| + |S_v|);
//   * X_1 .. X_17 from the relations of Sec. 4.6, with X_11 read as
//     (C_11 - X_9) / 3; every division is checked to be exact.
// n is the number of CSR rows, isolated vertices included.
//
// Threads: std::thread over edges with a shared atomic chunk cursor; each
// thread owns its Psi array (O(n) per worker, Sec. 4.7).

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

typedef unsigned __int128 u128;

struct Csr {
  int32_t n;
  const int32_t* rp;
  const int32_t* ci;
  int64_t deg(int32_t x) const { return (int64_t)rp[x + 1] - rp[x]; }
};

// Per-edge raw quantities.
struct EdgeRaw {
  int64_t t, su, sv, x7, x10;
};

// Alg. 1, Alg. 5, Alg. 6 for one edge (u, v) with d_v >= d_u.
// psi is this worker's mark array; lam is a per-edge base so that
// lam + 1 = lambda1, lam + 2 = lambda2, lam + 3 = lambda3.
EdgeRaw count_edge(const Csr& g, int32_t u, int32_t v, std::vector<uint64_t>& psi,
                   uint64_t lam, std::vector<int32_t>& T, std::vector<int32_t>& Su) {
  const uint64_t L1 = lam + 1, L2 = lam + 2, L3 = lam + 3;
  T.clear();
  Su.clear();
  // Alg. 1: mark Gamma(v) \ {u} with lambda1.
  for (int32_t p = g.rp[v]; p < g.rp[v + 1]; ++p) {
    int32_t w = g.ci[p];
    if (w != u) psi[w] = L1;
  }
  // Alg. 1: classify Gamma(u) \ {v} into T (lambda3) and S_u (lambda2).
  for (int32_t p = g.rp[u]; p < g.rp[u + 1]; ++p) {
    int32_t w = g.ci[p];
    if (w == v) continue;
    if (psi[w] == L1) {
      T.push_back(w);
      psi[w] = L3;
    } else {
      Su.push_back(w);
      psi[w] = L2;
    }
  }
  EdgeRaw r;
  r.t = (int64_t)T.size();
  r.su = (int64_t)Su.size();
  r.sv = g.deg(v) - r.t - 1;  // |S_v| = d_v - |T| - 1
  // Alg. 6 (membership as in Alg. 4): r in S_v <=> Psi(r) == lambda1.
  int64_t x10 = 0;
  for (int32_t w : Su)
    for (int32_t p = g.rp[w]; p < g.rp[w + 1]; ++p)
      if (psi[g.ci[p]] == L1) ++x10;
  // Alg. 5: for w in T count neighbours still tagged lambda3, then clear w.
  int64_t x7 = 0;
  for (int32_t w : T) {
    for (int32_t p = g.rp[w]; p < g.rp[w + 1]; ++p)
      if (psi[g.ci[p]] == L3) ++x7;
    psi[w] = 0;
  }
  r.x7 = x7;
  r.x10 = x10;
  return r;
}

inline u128 choose2(u128 x) { return x < 2 ? 0 : x * (x - 1) / 2; }

// Per-edge induced 4-node counts. The paper defines per edge only x3..x5 and
// the summands of C_7..C_16 (Sec. 4.5); the number of induced copies of each
// of H_7..H_16 (Table 1) that contain the edge is this library's extension,
// read straight from the definition: every 4-set containing e = (u, v) is
// {u, v, a, b} for a pair {a, b} of the other n - 2 vertices, and its induced
// subgraph is fixed by the classes of a and b -- T, S_u, S_v of Fig. 2, or
// the rest R (the D_e vertices of Sec. 4.5) -- and by whether a ~ b:
//   a, b in T:          a~b H7  (4-clique)        else H8  (chordal cycle)
//   T, S_u or S_v:      a~b H8                    else H9  (tailed triangle)
//   T, R:               a~b H9                    else H13 (triangle + vertex)
//   both S_u / both S_v: a~b H9                   else H11 (3-star)
//   S_u, S_v:           a~b H10 (4-cycle)         else H12 (4-path)
//   S_u or S_v, R:      a~b H12                   else H15 (2-star + vertex)
//   a, b in R:          a~b H14 (2 edges)         else H16 (edge + 2 vertices)
// The adjacent pairs of every class pair are counted by scanning Gamma(w)
// for every w in T, S_u and S_v against the Psi tags of Alg. 1 (lambda1 =
// S_v, lambda2 = S_u, lambda3 = T, and one more tag for u and v themselves);
// the adjacent pairs inside R are the edges left over from m.
// out[0..9] = H7 .. H16.
void count_edge_induced(const Csr& g, int64_t m, int32_t u, int32_t v, std::vector<uint64_t>& psi,
                        uint64_t lam, std::vector<int32_t>& T, std::vector<int32_t>& Su,
                        std::vector<int32_t>& Sv, uint64_t* out) {
  const uint64_t L0 = lam + 1, L1 = lam + 2, L2 = lam + 3, L3 = lam + 4;
  T.clear();
  Su.clear();
  Sv.clear();
  for (int32_t p = g.rp[v]; p < g.rp[v + 1]; ++p)
    if (g.ci[p] != u) psi[g.ci[p]] = L1;
  for (int32_t p = g.rp[u]; p < g.rp[u + 1]; ++p) {
    int32_t w = g.ci[p];
    if (w == v) continue;
    if (psi[w] == L1) {
      T.push_back(w);
      psi[w] = L3;
    } else {
      Su.push_back(w);
      psi[w] = L2;
    }
  }
  for (int32_t p = g.rp[v]; p < g.rp[v + 1]; ++p)
    if (g.ci[p] != u && psi[g.ci[p]] == L1) Sv.push_back(g.ci[p]);
  psi[u] = L0;
  psi[v] = L0;
  // adjacent pairs per class pair; pairs inside one class are met twice
  int64_t aTT = 0, aTSu = 0, aTSv = 0, aTR = 0, aSuSu = 0, aSvSv = 0, aSuSv = 0, aSuR = 0, aSvR = 0;
  int64_t degN = g.deg(u) + g.deg(v);  // sum of degrees over N = {u, v} + T + S_u + S_v
  for (int32_t w : T) {
    degN += g.deg(w);
    for (int32_t p = g.rp[w]; p < g.rp[w + 1]; ++p) {
      const uint64_t c = psi[g.ci[p]];
      if (c == L3) ++aTT;
      else if (c == L2) ++aTSu;
      else if (c == L1) ++aTSv;
      else if (c != L0) ++aTR;
    }
  }
  for (int32_t w : Su) {
    degN += g.deg(w);
    for (int32_t p = g.rp[w]; p < g.rp[w + 1]; ++p) {
      const uint64_t c = psi[g.ci[p]];
      if (c == L2) ++aSuSu;
      else if (c == L1) ++aSuSv;
      else if (c != L3 && c != L0) ++aSuR;
    }
  }
  for (int32_t w : Sv) {
    degN += g.deg(w);
    for (int32_t p = g.rp[w]; p < g.rp[w + 1]; ++p) {
      const uint64_t c = psi[g.ci[p]];
      if (c == L1) ++aSvSv;
      else if (c != L2 && c != L3 && c != L0) ++aSvR;
    }
  }
  aTT /= 2;
  aSuSu /= 2;
  aSvSv /= 2;
  const int64_t t = (int64_t)T.size(), su = (int64_t)Su.size(), sv = (int64_t)Sv.size();
  const int64_t R = g.n - 2 - t - su - sv;
  // edges inside N: (u, v), u and v to T, u to S_u, v to S_v, and the pairs above
  const int64_t inN = 1 + 2 * t + su + sv + aTT + aTSu + aTSv + aSuSu + aSvSv + aSuSv;
  const int64_t aRR = m - degN + inN;  // m = inN + (edges from N to R = degN - 2 inN) + aRR
  const int64_t c2t = t * (t - 1) / 2, c2su = su * (su - 1) / 2, c2sv = sv * (sv - 1) / 2, c2R = R * (R - 1) / 2;
  out[0] = (uint64_t)aTT;                                                          // H7
  out[1] = (uint64_t)(c2t - aTT + aTSu + aTSv);                                    // H8
  out[2] = (uint64_t)(t * su - aTSu + t * sv - aTSv + aTR + aSuSu + aSvSv);        // H9
  out[3] = (uint64_t)aSuSv;                                                        // H10
  out[4] = (uint64_t)(c2su - aSuSu + c2sv - aSvSv);                                // H11
  out[5] = (uint64_t)(su * sv - aSuSv + aSuR + aSvR);                              // H12
  out[6] = (uint64_t)(t * R - aTR);                                                // H13
  out[7] = (uint64_t)aRR;                                                          // H14
  out[8] = (uint64_t)(su * R - aSuR + sv * R - aSvR);                              // H15
  out[9] = (uint64_t)(c2R - aRR);                                                  // H16
}

// The 13 per-edge columns, in the library's column order.
void edge_columns(const EdgeRaw& r, int64_t n, int64_t m, int64_t du, int64_t dv, uint64_t* col) {
  int64_t s = r.su + r.sv;
  int64_t D = n - 2 - r.t - s;  // x5 = D_e
  col[0] = (uint64_t)r.t;                                   // x3 = |T|
  col[1] = (uint64_t)s;                                     // x4 = |S_u| + |S_v|
  col[2] = (uint64_t)D;                                     // x5 = D_e
  col[3] = (uint64_t)r.x7;                                  // 4-cliques on e
  col[4] = (uint64_t)r.x10;                                 // induced 4-cycles on e
  col[5] = (uint64_t)choose2((u128)r.t);                    // C_8 summand
  col[6] = (uint64_t)r.t * (uint64_t)s;                     // C_9 summand
  col[7] = (uint64_t)(choose2((u128)r.su) + choose2((u128)r.sv));  // C_11 summand
  col[8] = (uint64_t)r.su * (uint64_t)r.sv;                 // C_12 summand
  col[9] = (uint64_t)r.t * (uint64_t)D;                     // C_13 summand
  col[10] = (uint64_t)(m - du - dv + 1);                    // C_14 summand
  col[11] = (uint64_t)s * (uint64_t)D;                      // C_15 summand
  col[12] = (uint64_t)choose2((u128)D);                     // C_16 summand
}

// Unrestricted count index k -> per-edge column feeding it.
// C_3 C_4 C_5 C_7 C_8 C_9 C_10 C_11 C_12 C_13 C_14 C_15 C_16
const int kCsumCol[13] = {0, 1, 2, 3, 5, 6, 4, 7, 8, 9, 10, 11, 12};

struct Edges {
  std::vector<int32_t> u, v;  // u < v, edge id = rank in row-major upper-triangle order
};

Edges list_edges(const Csr& g) {
  Edges E;
  for (int32_t x = 0; x < g.n; ++x)
    for (int32_t p = g.rp[x]; p < g.rp[x + 1]; ++p)
      if (g.ci[p] > x) {
        E.u.push_back(x);
        E.v.push_back(g.ci[p]);
      }
  return E;
}

// P3: the second endpoint returned has the larger degree (ties: larger id).
inline void orient(const Csr& g, int32_t a, int32_t b, int32_t* lo, int32_t* hi) {
  int64_t da = g.deg(a), db = g.deg(b);
  bool a_low = da < db || (da == db && a < b);
  *lo = a_low ? a : b;
  *hi = a_low ? b : a;
}

int derive_globals(int64_t n, int64_t m, const u128* C /* C[3..16] */, u128* X /* X[1..17] */) {
  auto exact = [](u128 num, u128 den, u128* q) {
    if (num % den != 0) return false;
    *q = num / den;
    return true;
  };
  u128 N = (u128)n;
  u128 cn2 = N < 2 ? 0 : N * (N - 1) / 2;
  u128 cn3 = N < 3 ? 0 : N * (N - 1) / 2 * (N - 2) / 3;
  u128 cn4 = N < 4 ? 0 : N * (N - 1) / 2 * (N - 2) / 3 * (N - 3) / 4;
  X[1] = (u128)m;
  X[2] = cn2 - (u128)m;
  if (!exact(C[3], 3, &X[3])) return -1;
  if (!exact(C[4], 2, &X[4])) return -1;
  X[5] = C[5];
  X[6] = cn3 - X[3] - X[4] - X[5];
  if (!exact(C[7], 6, &X[7])) return -1;
  X[8] = C[8] - C[7];
  if (!exact(C[9] - 4 * X[8], 2, &X[9])) return -1;
  if (!exact(C[10], 4, &X[10])) return -1;
  if (!exact(C[11] - X[9], 3, &X[11])) return -1;
  X[12] = C[12] - C[10];
  if (!exact(C[13] - X[9], 3, &X[13])) return -1;
  if (!exact(C[14] - 6 * X[7] - 4 * X[8] - 2 * X[9] - 4 * X[10] - 2 * X[12], 2, &X[14])) return -1;
  if (!exact(C[15] - 2 * X[12], 2, &X[15])) return -1;
  X[16] = C[16] - 2 * X[14];
  u128 s = 0;
  for (int i = 7; i <= 16; ++i) s += X[i];
  X[17] = cn4 - s;
  return 0;
}

}  // namespace

extern "C" {

// Number of undirected edges (row_ptr[n] / 2).
int64_t oracle_num_edges(int32_t n, const int32_t* rp) { return (int64_t)rp[n] / 2; }

// Edge list in edge-id order (u < v, row-major upper triangle): uv[2e], uv[2e+1].
void oracle_edges(int32_t n, const int32_t* rp, const int32_t* ci, int32_t* uv) {
  Csr g{n, rp, ci};
  int64_t e = 0;
  for (int32_t x = 0; x < n; ++x)
    for (int32_t p = rp[x]; p < rp[x + 1]; ++p)
      if (ci[p] > x) {
        uv[2 * e] = x;
        uv[2 * e + 1] = ci[p];
        ++e;
      }
  (void)g;
}

// Whole-graph count.
//   per_edge: [m][13] uint64 or NULL
//   csum_lo/hi: [13] (C_3 C_4 C_5 C_7 C_8 C_9 C_10 C_11 C_12 C_13 C_14 C_15 C_16)
//   x_lo/hi: [17] (X_1 .. X_17)
// Returns 0, or -1 if a division of Sec. 4.6 is not exact.
int oracle_count(int32_t n, const int32_t* rp, const int32_t* ci, int nthreads,
                 uint64_t* per_edge, uint64_t* csum_lo, uint64_t* csum_hi, uint64_t* x_lo,
                 uint64_t* x_hi) {
  Csr g{n, rp, ci};
  Edges E = list_edges(g);
  const int64_t m = (int64_t)E.u.size();
  if (nthreads < 1) nthreads = 1;
  std::vector<std::vector<u128>> part(nthreads, std::vector<u128>(13, 0));
  std::atomic<int64_t> cursor(0);
  const int64_t chunk = 64;
  auto work = [&](int tid) {
    std::vector<uint64_t> psi((size_t)n, 0);
    std::vector<int32_t> T, Su;
    uint64_t col[13];
    for (;;) {
      int64_t e0 = cursor.fetch_add(chunk);
      if (e0 >= m) break;
      int64_t e1 = std::min(m, e0 + chunk);
      for (int64_t e = e0; e < e1; ++e) {
        int32_t u, v;
        orient(g, E.u[e], E.v[e], &u, &v);
        EdgeRaw r = count_edge(g, u, v, psi, 4 * (uint64_t)e, T, Su);
        edge_columns(r, n, m, g.deg(u), g.deg(v), col);
        if (per_edge) std::memcpy(per_edge + 13 * e, col, sizeof(col));
        for (int k = 0; k < 13; ++k) part[tid][k] += (u128)col[kCsumCol[k]];
      }
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < nthreads; ++t) th.emplace_back(work, t);
  work(0);
  for (auto& t : th) t.join();
  u128 cs[13] = {0};
  for (int t = 0; t < nthreads; ++t)
    for (int k = 0; k < 13; ++k) cs[k] += part[t][k];
  u128 C[17] = {0};
  const int idx[13] = {3, 4, 5, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16};
  for (int k = 0; k < 13; ++k) {
    C[idx[k]] = cs[k];
    if (csum_lo) csum_lo[k] = (uint64_t)cs[k];
    if (csum_hi) csum_hi[k] = (uint64_t)(cs[k] >> 64);
  }
  u128 X[18] = {0};
  int rc = derive_globals(n, m, C, X);
  for (int i = 1; i <= 17; ++i) {
    if (x_lo) x_lo[i - 1] = (uint64_t)X[i];
    if (x_hi) x_hi[i - 1] = (uint64_t)(X[i] >> 64);
  }
  return rc;
}

// Per-edge columns for a sample of edge ids (for checking large graphs edge
// by edge). edge_ids[k] in [0, m); out[k][13]. Returns 0 or -2 on a bad id.
int oracle_count_sample(int32_t n, const int32_t* rp, const int32_t* ci, int nthreads,
                        const int64_t* edge_ids, int64_t k, uint64_t* out) {
  Csr g{n, rp, ci};
  Edges E = list_edges(g);
  const int64_t m = (int64_t)E.u.size();
  for (int64_t i = 0; i < k; ++i)
    if (edge_ids[i] < 0 || edge_ids[i] >= m) return -2;
  if (nthreads < 1) nthreads = 1;
  std::atomic<int64_t> cursor(0);
  auto work = [&]() {
    std::vector<uint64_t> psi((size_t)n, 0);
    std::vector<int32_t> T, Su;
    for (;;) {
      int64_t i = cursor.fetch_add(1);
      if (i >= k) break;
      int64_t e = edge_ids[i];
      int32_t u, v;
      orient(g, E.u[e], E.v[e], &u, &v);
      EdgeRaw r = count_edge(g, u, v, psi, 4 * (uint64_t)i, T, Su);
      edge_columns(r, n, m, g.deg(u), g.deg(v), out + 13 * i);
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < nthreads; ++t) th.emplace_back(work);
  work();
  for (auto& t : th) t.join();
  return 0;
}

// Per-edge induced counts of H_7..H_16 (see count_edge_induced) for the
// given edge ids (all edges when edge_ids is NULL, k = m); out[k][10].
// Returns 0 or -2 on a bad id.
int oracle_count_induced(int32_t n, const int32_t* rp, const int32_t* ci, int nthreads,
                         const int64_t* edge_ids, int64_t k, uint64_t* out) {
  Csr g{n, rp, ci};
  Edges E = list_edges(g);
  const int64_t m = (int64_t)E.u.size();
  if (!edge_ids) k = m;
  for (int64_t i = 0; edge_ids && i < k; ++i)
    if (edge_ids[i] < 0 || edge_ids[i] >= m) return -2;
  if (nthreads < 1) nthreads = 1;
  std::atomic<int64_t> cursor(0);
  auto work = [&]() {
    std::vector<uint64_t> psi((size_t)n, 0);
    std::vector<int32_t> T, Su, Sv;
    for (;;) {
      int64_t i = cursor.fetch_add(1);
      if (i >= k) break;
      int64_t e = edge_ids ? edge_ids[i] : i;
      int32_t u, v;
      orient(g, E.u[e], E.v[e], &u, &v);
      count_edge_induced(g, m, u, v, psi, 5 * (uint64_t)i, T, Su, Sv, out + 10 * i);
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < nthreads; ++t) th.emplace_back(work);
  work();
  for (auto& t : th) t.join();
  return 0;
}

// Derivation of Sec. 4.6 alone, from given unrestricted counts (13 x 128-bit,
// same order as csum above). Lets tests check the relations in isolation.
int oracle_derive(int64_t n, int64_t m, const uint64_t* csum_lo, const uint64_t* csum_hi,
                  uint64_t* x_lo, uint64_t* x_hi) {
  u128 C[17] = {0};
  const int idx[13] = {3, 4, 5, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16};
  for (int k = 0; k < 13; ++k) C[idx[k]] = ((u128)csum_hi[k] << 64) | csum_lo[k];
  u128 X[18] = {0};
  int rc = derive_globals(n, m, C, X);
  for (int i = 1; i <= 17; ++i) {
    x_lo[i - 1] = (uint64_t)X[i];
    x_hi[i - 1] = (uint64_t)(X[i] >> 64);
  }
  return rc;
}

}  // extern "C"
