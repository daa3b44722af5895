// gc_internal.h -- shared declarations of libgc's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/gc.h"

namespace gc {

typedef unsigned __int128 u128;

// Device view of a (possibly multi-graph) CSR. A batch of graphs is counted
// as their disjoint union: vertices of graph g occupy the global id range
// [gbase[g], gbase[g] + gn[g]); per-edge x3/x7/x10 of a disjoint union equal
// those of each component, while n and m in the per-edge columns and the sums
// are taken per graph.
struct DevGraph {
  int32_t n;               // vertices in total
  int32_t m;               // undirected edges in total
  const int32_t* rp;       // [n + 1] row pointers (global ids)
  const int32_t* ci;       // [2m] column ids (global ids), rows ascending
  const int32_t* deg;      // [n]
  const int32_t* eid;      // [2m] slot -> edge id
  const int32_t* out_ptr;  // [n + 1] degree-oriented out-lists (Pi order)
  const int32_t* out_idx;  // [m]
  const int32_t* rev;      // [2m] slot of (y, x) for the slot of (x, y)
  int32_t G;               // graphs in the union (>= 1)
  const int32_t* vgid;     // [n] graph of each vertex, or nullptr when G == 1
  const int32_t* gbase;    // [G] first global vertex id of each graph
  const int32_t* gn;       // [G] vertices of each graph
  const int64_t* gm;       // [G] edges of each graph
  int32_t table_n;         // max gn[g]: size of one Psi table
  bool ranked;             // ids are the (degree, id) ranks and rows ascend
};

// Counting configuration chosen on the host.
struct CountArgs {
  const int32_t* units;    // pass A: v-groups (high endpoints), heaviest bin first
  int32_t n_units;
  const int32_t* chunks;   // pass B: [n_chunks][3] = (v, first slot, end slot) of Gamma(v)
  const int32_t* n_chunks; // device count of chunks
  int32_t* cursor;         // work-stealing cursor (device int, zeroed before launch)
  uint32_t* tables;        // global Psi tables (grid x table_n) or nullptr (shared memory)
  int32_t* tri;            // [m] per-edge |T| (written by pass A, read by pass B)
  unsigned long long* P;   // [2m] per slot: 4-cycles through its edge counted at that slot
                           // (pass C, zeroed before); an edge's count = sum of its two slots
  int32_t* tbuf;           // large-T edges: per-CTA T buffer (big grid x tbuf_len)
  int32_t tbuf_len;
  int32_t* deferred;       // [deferred_cap][2] (v, slot of u in Gamma(v)) of large-T edges
  int32_t deferred_cap;
  int32_t* n_deferred;     // device counter of deferred edges
  int32_t big_t;           // |T| above which an edge is deferred to k_pass_big
  uint64_t* per_edge;      // [m][13] device pointer or nullptr
  unsigned long long* csum;  // [G][13][2] 128-bit unrestricted counts (lo, hi)
  int32_t* status;         // device status word (0 = ok)
  unsigned long long* work;  // [kNumWork] work counters of this count
};

// Work counters (units the kernels processed; bench.py turns them into
// algorithmic bytes).
enum Work {
  kWorkBGroupDeg = 0,  // pass B: sum of d_v over chunks (Psi set + clear)
  kWorkBDeg,           // pass B: sum of d_u over its edges (Gamma(u) scan)
  kWorkBT,             // pass B: sum of |T|
  kWorkBProbe,         // pass B: out-list entries tested against T
  kWorkBEdges,         // pass B: edges finished
  kWorkBigDeg,         // large-T pass: sum of d_v + d_u
  kWorkBigT,           // large-T pass: sum of |T|
  kWorkBigProbe,       // large-T pass: entries tested
  kWorkCWedge,         // pass C: wedges h-x-o
  kWorkAUnits,         // pass A: sum of d_v + sum of d_u
  kNumWork
};

enum Status : int32_t { kOk = 0, kSpillOverflow = 1, kInexact = 2, kTimeout = 4 };

constexpr int kBlock = 512;            // threads per CTA of the counting kernels
constexpr int kCtasPerSm = 2;          // resident CTAs per SM of the persistent grids
constexpr int kWarps = kBlock / 32;
constexpr int kTcap = 1024;            // per-warp T list in shared memory (entries)
constexpr int kSmallN = 512;           // graphs up to this many vertices use the bitmatrix kernel
// Edges whose |T| exceeds big_t (default 1024, environment GC_BIG_T in
// [16, kTcap]) are done by a whole CTA (k_pass_big).
int big_t_threshold();
constexpr int kSmemTableMax = 4096;    // Psi tables up to this many vertices live in shared memory
constexpr int kBigBlock = 1024;        // threads per CTA for large-T edges
constexpr int kBigWarps = kBigBlock / 32;
constexpr int kBigWords = 49152;       // shared bitmap words (1.5 M ids) for T of a large edge

// Phases timed with CUDA events.
enum Phase { kPhasePassA = 0, kPhasePassC, kPhasePassB, kPhaseBig, kPhaseDerive, kPhaseCopy, kNumPhases };

// Device scratch of one count (lazily grown; owned by a graph handle or by
// one batch launch).
struct Scratch {
  int32_t* tri = nullptr;            // [m]
  unsigned long long* P = nullptr;   // [m]
  int32_t* chunks = nullptr;         // [chunk_capacity][3]
  int32_t* off = nullptr;            // [n_units + 1]
  int32_t* misc = nullptr;           // cursor, status, max |T|, #large-T, deferred counter
  unsigned long long* total = nullptr;
  uint32_t* tables = nullptr;        // count_grid_size() x table_n
  size_t tables_n = 0;
  int32_t* tbuf = nullptr;           // big_grid_size() x tbuf_len
  int32_t tbuf_len = 0;
  int32_t* deferred = nullptr;       // [deferred_cap][2]
  int32_t deferred_cap = 0;
  unsigned long long* work = nullptr;  // [kNumWork]
};
// Allocates what does not depend on the data (stream-ordered).
gc_status scratch_init(Scratch* sc, int32_t m, int32_t n_units, int32_t table_n, cudaStream_t s);
void scratch_free(Scratch* sc, cudaStream_t s);
// The whole count: passes A, C, B (+ large-T edges), derive. csum [G][13][2]
// and x [G][17][2] are device arrays; ev (optional) receives kNumPhases + 1
// events. Returns after the derive is queued (no final sync).
gc_status run_count(const DevGraph& g, const int32_t* units, int32_t n_units, uint64_t* per_edge,
                    unsigned long long* csum, unsigned long long* x, Scratch* sc, cudaStream_t s,
                    cudaEvent_t* ev);

// ---- host helpers (gc_api.cu) ----
void set_error(const std::string& msg);
gc_status cuda_fail(cudaError_t e, const char* what);

// ---- preprocessing (gc_prep.cu) ----
struct PrepBuffers {
  int32_t* deg = nullptr;
  int32_t* eid = nullptr;
  int32_t* uv = nullptr;  // [m][2]
  int32_t* out_ptr = nullptr;
  int32_t* out_idx = nullptr;
  int32_t* units = nullptr;
  int32_t n_units = 0;
  int32_t dmax = 0;
  long long* S = nullptr;  // [n] sum of neighbour degrees (Psi build cost of a v-group)
  int32_t* rev = nullptr;  // [2m] slot of the reverse direction of every slot
};
// Builds degrees, edge ids, the edge list, degree-oriented out-lists and the
// binned unit list on `stream`. vgid may be nullptr (single graph).
// d_eid_given (optional): slot -> edge id computed by the caller (ownership
// passes to PrepBuffers); d_perm (optional, with it): internal -> caller
// vertex id, used to write the edge list in the caller's labels.
gc_status prepare_graph(int32_t n, int32_t m, const int32_t* d_rp, const int32_t* d_ci,
                        const int32_t* d_vgid, int32_t* d_eid_given, const int32_t* d_perm,
                        PrepBuffers* out, cudaStream_t stream);
void free_prep(PrepBuffers* p, cudaStream_t s);

// ---- small graphs on a shared-memory bitmatrix (gc_small.cu) ----
// rp/voff: concatenated local row pointers and their offsets ([G'+1] for the
// packed graphs); ci/eoff: concatenated local columns; order: the G graph
// indices to count, largest first; csum [G'][13][2] zeroed.
gc_status run_small_graphs(const int32_t* rp, const int64_t* voff, const int32_t* ci, const int64_t* eoff,
                           const int32_t* order, int32_t G, int32_t* cursor, unsigned long long* csum,
                           cudaStream_t s);

// ---- counting (gc_count.cu) ----
int count_grid_size();
gc_status run_pass_a(const DevGraph& g, const CountArgs& a, cudaStream_t s);
gc_status run_pass_b(const DevGraph& g, const CountArgs& a, cudaStream_t s);
gc_status run_pass_c(const DevGraph& g, const CountArgs& a, cudaStream_t s);
gc_status run_pass_big(const DevGraph& g, const CountArgs& a, int32_t n_deferred, cudaStream_t s);
int big_grid_size();
gc_status run_derive(const DevGraph& g, const unsigned long long* csum, unsigned long long* x,
                     int32_t* status, cudaStream_t s);
gc_status run_max_tri(const int32_t* tri, int32_t m, int32_t* d_out, cudaStream_t s);
// Splits v-groups into edge chunks of balanced estimated work (needs |T| per
// edge from pass A). chunks must hold (n_units + 8 * grid + 1) triples and
// off n_units + 1 ints; off[n_units] receives the number of chunks.
gc_status run_make_chunks(const DevGraph& g, const int32_t* units, int32_t n_units,
                          const int32_t* tri, int32_t* chunks, int32_t* off,
                          unsigned long long* total_dev, int32_t* n_big_dev, int32_t big_t, cudaStream_t s);
// Target chunks per CTA of the persistent grid (environment GC_CHUNK_FACTOR,
// default 8, range 1..256).
int chunk_factor();
inline size_t chunk_capacity(int32_t n_units) {
  return (size_t)n_units + (size_t)chunk_factor() * (size_t)count_grid_size() + 1;
}
// Unit ordering key (environment GC_ORDER): 0 = vol (default: d_v + sum of
// neighbour degrees, heaviest bin first), 1 = degree d_v, 2 = none (vertex id).
int order_key();
// exclusive prefix sum of n int32 into out[0..n] (out[n] = total)
gc_status exclusive_scan(int32_t n, const int32_t* in, int32_t* out, cudaStream_t s);

}  // namespace gc
