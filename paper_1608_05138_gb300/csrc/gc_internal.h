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
  int32_t G;               // graphs in the union (>= 1)
  const int32_t* vgid;     // [n] graph of each vertex, or nullptr when G == 1
  const int32_t* gbase;    // [G] first global vertex id of each graph
  const int32_t* gn;       // [G] vertices of each graph
  const int64_t* gm;       // [G] edges of each graph
  int32_t table_n;         // max gn[g]: size of one Psi table
};

// Counting configuration chosen on the host.
struct CountArgs {
  const int32_t* units;    // v-groups to process (high endpoints), heaviest bin first
  int32_t n_units;
  int32_t* cursor;         // work-stealing cursor (device int, zeroed before launch)
  uint32_t* tables;        // global Psi tables (grid x table_n) or nullptr (shared memory)
  int32_t* tri;            // [m] per-edge |T| (written by pass A, read by pass B)
  int32_t* spill;          // per-warp T spill (grid x warps x spill_len) or nullptr
  int32_t spill_len;
  uint64_t* per_edge;      // [m][13] device pointer or nullptr
  unsigned long long* csum;  // [G][13][2] 128-bit unrestricted counts (lo, hi)
  int32_t* status;         // device status word (0 = ok)
};

enum Status : int32_t { kOk = 0, kSpillOverflow = 1, kInexact = 2, kTimeout = 4 };

constexpr int kBlock = 512;            // threads per CTA of the counting kernels
constexpr int kWarps = kBlock / 32;
constexpr int kTcap = 1024;            // per-warp shared-memory T buffer (entries)
constexpr int kSmemTableMax = 16384;   // Psi tables up to this many vertices live in shared memory
constexpr uint32_t kFlag = 0x80000000u;  // Psi: "neighbour of v"
constexpr uint32_t kCount = 0x7fffffffu; // Psi: |Gamma(w) ∩ Gamma(v)|

// Phases timed with CUDA events.
enum Phase { kPhasePassA = 0, kPhasePassB, kPhaseDerive, kPhaseCopy, kNumPhases };

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
};
// Builds degrees, edge ids, the edge list, degree-oriented out-lists and the
// binned unit list on `stream`. vgid may be nullptr (single graph).
gc_status prepare_graph(int32_t n, int32_t m, const int32_t* d_rp, const int32_t* d_ci,
                        const int32_t* d_vgid, PrepBuffers* out, cudaStream_t stream);
void free_prep(PrepBuffers* p, cudaStream_t s);

// ---- counting (gc_count.cu) ----
int count_grid_size();
gc_status run_pass_a(const DevGraph& g, const CountArgs& a, cudaStream_t s);
gc_status run_pass_b(const DevGraph& g, const CountArgs& a, cudaStream_t s);
gc_status run_derive(const DevGraph& g, const unsigned long long* csum, unsigned long long* x,
                     int32_t* status, cudaStream_t s);
gc_status run_max_tri(const int32_t* tri, int32_t m, int32_t* d_out, cudaStream_t s);

}  // namespace gc
