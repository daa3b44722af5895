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
  const int32_t* out_ptr;  // [n + 1] degree-oriented out-lists (P3 orientation)
  const int32_t* out_idx;  // [m] ascending ids within each list; position = out-slot
  const int32_t* ocsr;     // [m] out-slot -> CSR slot of the same direction (row of the owner)
  const int32_t* e2o;      // [m] edge id -> out-slot
  const int32_t* rev;      // [2m] slot of (y, x) for the slot of (x, y)
  int32_t G;               // graphs in the union (>= 1)
  const int32_t* vgid;     // [n] graph of each vertex, or nullptr when G == 1
  const int32_t* gbase;    // [G] first global vertex id of each graph
  const int32_t* gn;       // [G] vertices of each graph
  const int64_t* gm;       // [G] edges of each graph
  int32_t table_n;         // max gn[g]: size of one Psi table
  bool ranked;             // ids are the (degree, id) ranks and rows ascend
};

// Pass K (4-cliques and cross terms by lowest vertex) runs in tiers by the
// out-degree k of the lowest vertex: the local bitmatrix of out(a) lives in
// shared memory up to k = 1024 and in a per-CTA global buffer above.
// Units with k <= 32 are done by one warp each, with the rows in registers.
enum KTier { kTierGlobal = 0, kTier1024, kTier512, kTier256, kTier32, kNumTiers };
constexpr int kTierCap[kNumTiers] = {0, 1024, 512, 256, 32};

// Counting configuration chosen on the host.
struct CountArgs {
  const int32_t* units;    // pass C: v-groups (high endpoints), heaviest bin first
  int32_t n_units;
  const int32_t* cunits;   // pass C: hub units (blocked kernel), hashed units, then the others
  int32_t n_cheavy;        // hub units of pass C (cunits[0 .. n_cheavy))
  const int32_t* chash_w;  // wedges of the hashed units cunits[n_cheavy .. n_cheavy + n_chash + n_chash2)
  int32_t n_chash;
  int32_t n_chash_mid;     // hashed units of more than kHashMidW wedges (the first of them)
  int32_t n_chash_big;     // hashed units of more than kHashSmallW wedges (the first of them)
  int32_t n_chash2;        // units of the packed-key hash tier, after the hashed units
  int32_t n_chash2_big;    // of them, units of more than kHash2HalfMaxW wedges (the first)
  const int4* cjobs;       // pass C hub kernel: jobs (hub index into cunits, first o-range block, blocks),
                           // heaviest first
  int32_t n_cjobs;
  int32_t* cbuf;           // pass C hub kernel: per-CTA cursors (cbuf_ctas x 3 x cbuf_nx ints)
  int32_t cbuf_nx;
  int32_t hub_tab;         // pass C hub kernel: words of the count block (hub_tab_words())
  const int32_t* kunits;   // pass K: lowest vertices a with |out(a)| >= 2, tiers in KTier order
  int32_t ktier_off[kNumTiers + 1];  // tier t = kunits[ktier_off[t] .. ktier_off[t + 1])
  int32_t* cursor;         // work-stealing cursors (device ints, zeroed before each launch)
  uint32_t* tables;        // global Psi tables (grid x table_n) or nullptr (shared memory)
  int32_t* trio;           // [m] |T| by out-slot (pass T)
  unsigned long long* P;   // [2m] per slot: 4-cycles through its edge counted at that slot
                           // (pass C, zeroed before); an edge's count = sum of its two slots
  unsigned long long* xc;    // [m][2] per out-slot: 4-cliques through the edge, and the sum over T of
                             // (|T_(a,u)| + |T_(a,v)| - 2) (pass K); side by side, so that the two
                             // atomics of an edge land in one 32-byte sector
  unsigned char* kbuf;     // global-tier per-CTA buffers (kbuf_ctas x kbuf_stride bytes)
  size_t kbuf_stride;
  int32_t kbuf_ctas;
  int32_t kbuf_cap;        // largest k the global tier holds
  int32_t* hitbuf;         // passes T/K: per-CTA lists of the edges of H_a (hitbuf_ctas x hitcap x 2 ints)
  int32_t hitcap;
  int32_t hitbuf_ctas;
  // Edges of every H_a, recorded by pass T for pass K (nullptr: not kept):
  // entry = ((i << 16) | j, out-slot of (b_i, b_j)); unit ui (index into
  // kunits) has tl_cnt[ui] entries from tl_off[ui], or tl_cnt[ui] = -1.
  int2* tlist;
  long long tlist_cap;
  unsigned long long* tlist_fill;
  long long* tl_off;
  int32_t* tl_cnt;
  unsigned long long* dsum;  // [m] per out-slot: sum over T of d_w (pass T, per-edge induced counts only)
  uint64_t* per_edge;      // [m][13] device pointer or nullptr
  bool per_edge_host;      // per_edge maps pinned host memory
  unsigned long long* csum;  // [G][13][2] 128-bit unrestricted counts (lo, hi)
  int32_t* status;         // device status word (0 = ok)
  unsigned long long* work;  // [kNumWork] work counters of this count
};

// Work counters (units the kernels processed; bench.py turns them into
// algorithmic bytes).
enum Work {
  kWorkTMembers = 0,   // pass T: sum over units of |out(a)|
  kWorkCWedge,         // pass C: wedges h-x-o
  kWorkKMembers,       // pass K: sum over units of |out(a)|
  kWorkKScan,          // pass K: out-list entries scanned to build the local graphs
  kWorkKLocalEdges,    // pass K: local edges = triangles (each once)
  kWorkKWords,         // pass K: bitmatrix words ANDed (local edges x row words)
  kWorkFinishEdges,    // finish: edges written
  kWorkLaunches,       // kernels launched by the count (counted on the host)
  kWorkCHeavyWedge,    // pass C: wedges of the hub units (blocked kernel)
  kWorkCBlocks,        // pass C: lower neighbours swept, summed over the blocks of the hub units
  kWorkTScan,          // pass T: out-list entries scanned
  kWorkTTriangles,     // pass T: triangles (each once)
  kWorkCHashWedge,     // pass C: wedges of the units counted in a shared-memory hash
  kWorkCHubJobs,       // pass C: jobs of the hub kernel (hub units cut into ranges of o-range blocks)
  kWorkCHubCtas,       // pass C: CTAs of the hub kernel
  kWorkCHubBusySum,    // pass C: sum over the hub kernel's CTAs of their lifetime (ns, %globaltimer)
  kWorkCHubBusyMax,    // pass C: the longest of those lifetimes (ns)
  kWorkCHash2Wedge,    // pass C: wedges of the units counted in the packed-key hash
  kNumWork
};

// Device status bits. kSpillOverflow: a unit outgrew what it was binned for
// (a pass-T/K tier, the hub cursors, the hashed pass-C table); it cannot
// happen for a validated graph.
enum Status : int32_t { kOk = 0, kSpillOverflow = 1, kInexact = 2 };

constexpr int kBlock = 512;            // threads per CTA of passes A and C
constexpr int kCtasPerSm = 2;          // resident CTAs per SM of the persistent grids
constexpr int kWarps = kBlock / 32;
constexpr int kSmemTableMax = 4096;    // Psi tables up to this many vertices live in shared memory

// Phases timed with CUDA events.
enum Phase { kPhasePassT = 0, kPhasePassC, kPhasePassK, kPhaseFinish, kPhaseInduced, kPhaseDerive, kPhaseCopy,
             kNumPhases };

// Device scratch of one count (lazily grown; owned by a graph handle or by
// one batch launch).
struct Scratch {
  int32_t* trio = nullptr;           // [m]
  unsigned long long* P = nullptr;   // [2m]
  unsigned long long* xc = nullptr;  // [m][2]
  int32_t* misc = nullptr;           // [32] cursors, status
  int32_t* cbuf = nullptr;           // pass C hub cursors
  int32_t cbuf_nx = 0;
  uint32_t* tables = nullptr;        // count_grid_size() x table_n
  size_t tables_n = 0;
  unsigned char* kbuf = nullptr;     // pass K global tier
  size_t kbuf_stride = 0;
  int32_t kbuf_ctas = 0;
  int32_t kbuf_cap = 0;
  int32_t* hitbuf = nullptr;         // per-CTA H_a edge lists
  int32_t hitcap = 0;
  int32_t hitbuf_ctas = 0;
  int2* tlist = nullptr;             // edges of all H_a, from pass T to pass K
  long long tlist_cap = 0;           // entries
  long long tlist_want = 0;          // triangles of the last count (or a first guess): the size to keep
  long long* tl_off = nullptr;       // [units of pass K]
  int32_t* tl_cnt = nullptr;
  int32_t tl_units = 0;
  unsigned long long* tl_fill = nullptr;
  unsigned long long* work = nullptr;  // [kNumWork]
  int32_t launches = 0;              // kernels launched by the last run_count
  unsigned long long* dsum = nullptr;  // [m] per-edge induced counts: sum over T of d_w
  unsigned long long* vsum = nullptr;  // [n][2] per-edge induced counts: 2 x triangles, neighbour degrees
};
// Allocates the scratch of a graph with m edges, Psi tables of table_n
// vertices and largest out-degree kmax (stream-ordered).
gc_status scratch_init(Scratch* sc, int32_t m, int32_t table_n, int32_t kmax, int32_t cnx_max, cudaStream_t s);
void scratch_free(Scratch* sc, cudaStream_t s);
// Size of pass T's edge lists for the first count of a whole graph with m
// edges: 32 m entries within the list budget (units past it scan again).
void scratch_guess_tlist(Scratch* sc, int64_t m);
// The whole count: passes T, C, K, finish, derive. csum [G][13][2] and
// x [G][17][2] are device arrays; ev (optional) receives kNumPhases + 1
// events. Returns after the derive is queued (no host synchronisation).
struct KUnits {
  const int32_t* units;
  int32_t tier_off[kNumTiers + 1];
  const int32_t* cunits;   // pass C units: hubs, hashed units, the others
  int32_t n_cheavy;
  const int4* cjobs;       // hub jobs (see CountArgs)
  int32_t n_cjobs;
  const int32_t* chash_w;
  int32_t n_chash;
  int32_t n_chash_mid;
  int32_t n_chash_big;
  int32_t n_chash2;
  int32_t n_chash2_big;
  int32_t n_cunits;        // pass C units in all (units without wedges are left out)
};
// induced (optional): [m][10] rows of the per-edge induced counts of H_7..H_16
// (device pointer, or the device view of pinned host memory when
// induced_host), written after the finish.
gc_status run_count(const DevGraph& g, const int32_t* units, int32_t n_units, const KUnits& ku,
                    uint64_t* per_edge, unsigned long long* csum, unsigned long long* x, Scratch* sc,
                    cudaStream_t s, cudaEvent_t* ev, bool per_edge_host = false, uint64_t* induced = nullptr,
                    bool induced_host = false);

// ---- host helpers (gc_api.cu) ----
void set_error(const std::string& msg);
gc_status cuda_fail(cudaError_t e, const char* what);

// The library's stream-ordered memory pool on the current device (created on
// first use). Freed blocks stay in it, up to a limit (environment
// GC_POOL_KEEP_BYTES; default a quarter of the device's memory), so that a
// later graph or count reuses them without mapping memory again and a free
// does not unmap at the next synchronisation; gc_release_cached_memory hands
// them back. Every device buffer of the library comes from it (pool_alloc),
// and is returned with cudaFreeAsync.
cudaMemPool_t lib_pool();
template <class T>
inline cudaError_t pool_alloc(T** p, size_t bytes, cudaStream_t s) {
  cudaMemPool_t pool = lib_pool();
  if (!pool) return cudaErrorMemoryAllocation;
  return cudaMallocFromPoolAsync(reinterpret_cast<void**>(p), bytes, pool, s);
}

// ---- relabelling P1 on the device (gc_relabel.cu) ----
// Internal row i = caller row perm[i] in internal ids (newid), sorted; eid:
// caller's edge id of every internal slot. rp: internal row pointers (device);
// mid_rows / long_rows: internal rows of 33..4096 and of more entries; the
// long rows are sorted in padded copies at tmp + long_off[k].
gc_status relabel_on_device(int32_t n, int32_t m, const int32_t* d_rp0, const int32_t* d_ci0,
                            const int32_t* d_perm, const int32_t* d_newid, const int32_t* d_rp, int32_t* d_ci,
                            int32_t* d_eid, const int32_t* d_mid_rows, int32_t n_mid, const int32_t* d_long_rows,
                            const int64_t* d_long_off, int32_t n_long, long long* d_tmp, cudaStream_t s);

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
  int32_t* ocsr = nullptr;  // [m] out-slot -> CSR slot
  int32_t* e2o = nullptr;   // [m] edge id -> out-slot
  int32_t* kunits = nullptr;  // pass K units (see CountArgs::kunits)
  int32_t ktier_off[kNumTiers + 1] = {0, 0, 0, 0, 0, 0};
  int32_t kmax = 0;         // largest out-degree
  int32_t* cunits = nullptr;  // pass C units: hub units (heaviest first), hashed units (heaviest
                              // first), then the rest in unit order
  int32_t n_cheavy = 0;
  int4* cjobs = nullptr;       // hub jobs, heaviest first (see CountArgs)
  int32_t n_cjobs = 0;
  int32_t* chash_w = nullptr;  // wedges of each hashed unit (both hash tiers)
  int32_t n_chash = 0;
  int32_t n_chash_mid = 0;     // hashed units of more than kHashMidW wedges
  int32_t n_chash_big = 0;     // hashed units of more than kHashSmallW wedges
  int32_t n_chash2 = 0;        // units of the packed-key hash tier
  int32_t n_chash2_big = 0;    // of them, units of more than kHash2HalfMaxW wedges
  int32_t n_cunits = 0;
  int32_t cnx_max = 0;      // most lower neighbours of a hub unit
};
// Builds degrees, edge ids, the edge list, degree-oriented out-lists and the
// binned unit list on `stream`. vgid may be nullptr (single graph).
// d_eid_given (optional): slot -> edge id computed by the caller (ownership
// passes to PrepBuffers); d_perm (optional, with it): internal -> caller
// vertex id, used to write the edge list in the caller's labels.
gc_status prepare_graph(int32_t n, int32_t m, const int32_t* d_rp, const int32_t* d_ci,
                        const int32_t* d_vgid, int32_t* d_eid_given, const int32_t* d_perm,
                        PrepBuffers* out, cudaStream_t stream);
// Splits the pass-C units of a ranked graph (ids = ranks, rows ascending)
// into hub units for the blocked kernel, units of at most kHashMaxW wedges
// for the hashed kernel and the rest, leaving out units without wedges
// (fills cunits, n_cheavy, chash_w, n_chash, n_cunits, cnx_max; otherwise
// cunits is a copy of units).
gc_status classify_c_units(int32_t n, const int32_t* d_rp, const int32_t* d_ci, bool ranked, PrepBuffers* p,
                           cudaStream_t stream);
void free_prep(PrepBuffers* p, cudaStream_t s);
// Smallest slot p with rev[p] == p (no reverse: the input is not symmetric),
// or -1 (synchronises the stream).
gc_status first_unreversed_slot(int64_t nnz, const int32_t* d_rev, int32_t* out, cudaStream_t s);

// ---- small graphs on a shared-memory bitmatrix (gc_small.cu) ----
// Size classes of the bitmatrix kernel: class c takes graphs of at most
// kSmallClassN[c] vertices (and more than the previous class).
constexpr int kSmallClasses = 5;
constexpr int kSmallClassN[kSmallClasses] = {64, 128, 256, 512, 1024};
// Tunable parameters of the batched form (read from the tuning cache at
// gc_batch_create, or set with gc_batch_set_param).
struct BatchConfig {
  int32_t small_n_max = 512;                                  // graphs up to this many vertices: bitmatrix kernels
  int32_t class_block[kSmallClasses] = {256, 256, 256, 256, 256};  // threads per CTA of each size class
  int32_t use_graph = 1;                                      // replay each small-graph launch as a CUDA graph
  int32_t max_inflight = 2;                                   // launches the dispatcher keeps in flight
};
constexpr int kMaxInflight = 4;                                 // stream slots of a batch runtime
// Size class of a graph with n vertices (kSmallClasses if above the largest).
int small_class_of(int32_t n);
// Overrides cfg with the tuning cache's entry for the current GPU (gc_tune.cu);
// false (cfg unchanged) when there is no cache or no entry.
bool load_tuned_config(BatchConfig* cfg, std::string* source);
// Raises the dynamic shared-memory limit of every instantiation (once per
// device, before any launch or capture).
gc_status small_graphs_setup();
// rp/voff: concatenated local row pointers and their offsets; ci/eoff:
// concatenated local columns; class c counts the graphs
// order[class_off[c] .. class_off[c + 1]) (largest first within a class);
// cursor: kSmallClasses zeroed device ints; status: device status word;
// csum [*][13][2] zeroed. ev (optional): kSmallClasses + 1 events recorded
// before each class's launch and after the last.
gc_status run_small_graphs(const int32_t* rp, const int64_t* voff, const int32_t* ci, const int64_t* eoff,
                           const int32_t* order, const int32_t* class_off, int32_t* cursor, int32_t* status,
                           unsigned long long* csum, const BatchConfig& cfg, cudaEvent_t* ev, cudaStream_t s);

// ---- counting (gc_count.cu: pass C, finish, derive; gc_clique.cu: passes T and K) ----
int count_grid_size();
gc_status run_pass_c(const DevGraph& g, const CountArgs& a, cudaStream_t s);
gc_status run_pass_c_heavy(const DevGraph& g, const CountArgs& a, cudaStream_t s);
constexpr int kHeavyTab = 53248;  // largest o-range block of the hub kernel of pass C (words of shared memory)
// Words of the hub kernel's count block (environment GC_HUB_TAB_WORDS, a
// multiple of 1024 in [4096, kHeavyTab], else kHubTabDefault), read once per
// process. The block and the SM's L1 cache share one array, split in steps
// (the shared-memory carveout); kHubTabDefault is the largest block whose CTA
// (block + 16.4 KB of static arrays + 1 KB reserved) fits the 196 KB step,
// leaving about 60 KB of L1 for the rows and cursors instead of 28 KB with a
// 208 KB block (R-MAT scale 22: pass C 228.4 ms at 53248 words, 205.0 at
// 45056, 213.3 at 39936, 226.7 at 32768).
constexpr int kHubTabDefault = 45056;
int hub_tab_words();
// Counters per word of the hub kernel for a unit of nx lower neighbours
// (count fields of 32, 16 or 10 bits; no count exceeds nx): one block of
// its o-range spans hub_cpw(nx) * hub_tab_words() ids.
__host__ __device__ __forceinline__ int hub_cpw(int64_t nx) { return nx < 1023 ? 3 : nx < 65536 ? 2 : 1; }
// Units of pass C with at most kHashMaxW wedges count in a shared-memory
// hash of 2 kHashMaxW keys (at most half full: a unit has no more distinct
// o than wedges).
constexpr int kHashMaxW = 8192;
constexpr int kHashSmallW = 512;  // hashed units up to this many wedges run in small CTAs
constexpr int kHashMidW = 2048;   // and up to this many in middle-sized CTAs
gc_status run_pass_c_hash(const DevGraph& g, const CountArgs& a, cudaStream_t s);
// Units of more than kHashMaxW and at most kHash2MaxW wedges, with fewer than
// kHash2MaxNx lower neighbours, in graphs of at most 2^22 vertices: a
// shared-memory hash of kHash2Slots words, each a packed (22-bit vertex,
// 10-bit count) pair, at most 72 % full.
constexpr int kHash2Slots = 57344;
constexpr int kHash2MaxW = 41287;
constexpr int kHash2MaxNx = 1023;
// Packed-key units of at most kHash2HalfMaxW wedges fit half the table and
// run in 512-thread CTAs, two an SM.
constexpr int kHash2HalfSlots = 28672;
constexpr int kHash2HalfMaxW = 20620;  // (kHash2HalfSlots - 32) * 18 / 25
constexpr int32_t kHash2MaxN = 1 << 22;
gc_status run_pass_c_hash2(const DevGraph& g, const CountArgs& a, cudaStream_t s);
gc_status run_derive(const DevGraph& g, const unsigned long long* csum, unsigned long long* x,
                     int32_t* status, cudaStream_t s);
gc_status run_pass_t(const DevGraph& g, const CountArgs& a, cudaStream_t s, int* launches);
gc_status run_pass_k(const DevGraph& g, const CountArgs& a, cudaStream_t s, int* launches);
gc_status run_finish(const DevGraph& g, const CountArgs& a, cudaStream_t s);
// Per-edge induced counts of H_7..H_16 (needs a.dsum from pass T, and the
// results of passes C and K); vsum: [n][2] scratch.
gc_status run_induced(const DevGraph& g, const CountArgs& a, unsigned long long* vsum, uint64_t* out, bool out_host,
                      cudaStream_t s);
// Bytes of one global-tier buffer for out-degrees up to cap.
size_t kbuf_bytes(int32_t cap);
// Unit ordering key (environment GC_ORDER): 0 = vol (default: d_v + sum of
// neighbour degrees, heaviest bin first), 1 = degree d_v, 2 = none (vertex id).
int order_key();
// exclusive prefix sum of n int32 into out[0..n] (out[n] = total)
gc_status exclusive_scan(int32_t n, const int32_t* in, int32_t* out, cudaStream_t s);

}  // namespace gc
