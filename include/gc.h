/*
 * gc.h -- exact per-edge 3/4-node graphlet counting on one GB300 GPU (sm_103a).
 *
 * C ABI of libgc.so. Implements the data-parallel hot path of Rossi & Zhou,
 * "Hybrid CPU-GPU Framework for Network Motifs" (arXiv 1608.05138):
 *   Problem 1 (global graphlet counting): for the 17 graphlets H_1..H_17 of
 *   Table 1 (all connected and disconnected induced subgraphs on 2, 3 and 4
 *   vertices) count their induced embeddings in G;
 *   the edge-centric method of Sec. 4: per edge e = (u, v) the triangle set T
 *   and star sets S_u, S_v (Fig. 2, Alg. 1/2), the 4-cliques over T
 *   (Alg. 3/5) and the induced 4-cycles over S_u x S_v (Alg. 4/6), the
 *   per-edge 3-graphlet equations and unrestricted counts C_3..C_16
 *   (Sec. 4.5), and the global counts X_1..X_17 (Sec. 4.6).
 *
 * General conventions
 *   - No C++ exception crosses this boundary; every call returns a gc_status.
 *     On failure gc_last_error() returns a thread-local message.
 *   - Inputs are owned by the caller and are copied during the call; the
 *     library keeps no pointer to them. Outputs are caller-owned. Handles are
 *     library-owned until gc_graph_free / gc_batch_destroy.
 *   - A handle must not be used from two threads at the same time.
 *   - Graphs are CSR with int32 indices: row_ptr[n + 1] with row_ptr[0] = 0,
 *     col_idx[row_ptr[n]]; each row sorted strictly ascending, the graph
 *     undirected (symmetric), without self-loops. n counts every vertex,
 *     isolated ones included (they change X_2, X_5, X_6, X_13..X_17).
 *     2m = row_ptr[n] must be below 2^31.
 *   - Edge ids: edge e is the e-th pair (u, v), u < v, met in row-major order
 *     of the upper triangle of the CSR.
 *   - Counts are exact integers. Global counts are 128-bit: global_out[i-1]
 *     holds the low 64 bits of X_i, global_hi[i-1] the high 64 bits.
 */
#ifndef GC_H
#define GC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gc_graph_s* gc_graph;
typedef struct gc_batch_s* gc_batch;
typedef int gc_status;

enum {
  GC_OK = 0,
  GC_PENDING = 1,          /* gc_batch_poll: not finished yet */
  GC_ERR_ARG = -1,         /* NULL handle/pointer, negative size, bad flag */
  GC_ERR_UNSORTED = -2,    /* a row of col_idx is not ascending, or row_ptr decreases */
  GC_ERR_DUPLICATE = -3,   /* a neighbour appears twice in one row */
  GC_ERR_SELF_LOOP = -4,   /* col_idx of row x contains x */
  GC_ERR_ASYMMETRIC = -5,  /* (x, y) present without (y, x) */
  GC_ERR_RANGE = -6,       /* column index outside [0, n), row_ptr[0] != 0 */
  GC_ERR_NOMEM = -7,       /* device or host allocation failed */
  GC_ERR_CUDA = -8,        /* a CUDA call failed (message has the CUDA error) */
  GC_ERR_OVERFLOW = -9,    /* 2m >= 2^31, or a high word is needed but global_hi is NULL */
  GC_ERR_TIMEOUT = -10,    /* reserved: no call returns it (no kernel of this library waits
                              on another CTA, stream or device) */
  GC_ERR_BUSY = -11        /* gc_batch_submit: the device-memory budget is full */
};

#define GC_EDGE_COLS 13      /* per-edge columns, see gc_count_edge_graphlets */
#define GC_NUM_GRAPHLETS 17  /* X_1 .. X_17 */
#define GC_NUM_CSUMS 13      /* C_3 C_4 C_5 C_7 .. C_16 */

/* gc_graph_upload flags */
#define GC_NO_VALIDATE 0x1u  /* skip the host-side CSR checks (caller guarantees them) */

/* Thread-local message describing the last failed call of this thread. */
const char* gc_last_error(void);

/*
 * Validate a CSR graph on the host, copy it to the device and prepare it
 * (Problem 1 input; preprocessing P3 of Sec. 4.3; edge ordering Pi of Sec. 4.4).
 *   n        number of vertices, 0 <= n < 2^31
 *   row_ptr  host pointer, n + 1 int32
 *   col_idx  host pointer, row_ptr[n] int32
 *   flags    0 or GC_NO_VALIDATE
 *   stream   cudaStream_t (as void*) on which all work of this graph runs;
 *            NULL = the legacy default stream
 *   out      receives the new handle
 * Errors: GC_ERR_ARG, GC_ERR_RANGE, GC_ERR_UNSORTED, GC_ERR_DUPLICATE,
 * GC_ERR_SELF_LOOP, GC_ERR_ASYMMETRIC, GC_ERR_OVERFLOW (2m >= 2^31),
 * GC_ERR_NOMEM, GC_ERR_CUDA. On error *out is NULL and nothing is leaked.
 * The call returns after the device data is ready.
 */
gc_status gc_graph_upload(int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                          uint32_t flags, void* stream, gc_graph* out);

/*
 * The host checks of gc_graph_upload alone, with no device work: row_ptr[0]
 * == 0, row_ptr ascending, row_ptr[n] even, every column in [0, n), rows
 * strictly ascending without self-loops, and every entry (x, y) matched by
 * (y, x). Host pointers, read only. Graphs of fewer than 2^20 entries get the
 * single-threaded checks that every graph of gc_batch_submit_many gets, larger
 * ones the multi-threaded checks of gc_graph_upload; both return the same
 * code and message for the same graph. The message names the first failing
 * entry in row order -- for GC_ERR_ASYMMETRIC, the first entry (x, y) whose
 * reverse (y, x) is absent.
 * Errors: GC_ERR_ARG, GC_ERR_RANGE, GC_ERR_UNSORTED, GC_ERR_DUPLICATE,
 * GC_ERR_SELF_LOOP, GC_ERR_ASYMMETRIC.
 */
gc_status gc_validate_csr(int32_t n, const int32_t* row_ptr, const int32_t* col_idx);

/* n and the number of undirected edges m = row_ptr[n] / 2. Either pointer may be NULL. */
gc_status gc_graph_info(gc_graph g, int64_t* n, int64_t* m);

/* Edge list in edge-id order: uv[2e] = u, uv[2e+1] = v, u < v. uv is a host
 * pointer to 2m int32. */
gc_status gc_graph_edges(gc_graph g, int32_t* uv);

/*
 * Count every 2/3/4-node graphlet (Problem 1) by the per-edge method.
 *   per_edge_out  NULL (skip), or a host or device pointer (detected with
 *                 cudaPointerGetAttributes) to m x GC_EDGE_COLS uint64, row e
 *                 for edge id e. Device, managed and pinned host memory are
 *                 written by the device directly; pageable host memory
 *                 through a device staging buffer (kept with the graph) and
 *                 one copy. Columns (T, S_u, S_v of Fig. 2; D_e as in
 *                 Sec. 4.5):
 *                   0 x3  = |T|                     (triangles on e)
 *                   1 x4  = |S_u| + |S_v|           (2-stars on e)
 *                   2 x5  = D_e = n-2-|T|-|S_u|-|S_v| (3-node-1-edge on e)
 *                   3 x7  = 4-cliques containing e
 *                   4 x10 = induced 4-cycles containing e
 *                   5 C(|T|,2)        6 |T|(|S_u|+|S_v|)
 *                   7 C(|S_u|,2)+C(|S_v|,2)            8 |S_u||S_v|
 *                   9 |T| D_e        10 m - d_u - d_v + 1
 *                  11 (|S_u|+|S_v|) D_e               12 C(D_e,2)
 *                 (columns 5..12 are the per-edge summands of C_8, C_9,
 *                 C_11..C_16; all columns are symmetric in u and v).
 *   global_out    host pointer, 17 uint64: low 64 bits of X_1..X_17 (Table 1
 *                 numbering, Sec. 4.6); must not be NULL.
 *   global_hi     host pointer, 17 uint64 for the high 64 bits, or NULL. If
 *                 NULL and some X_i >= 2^64 the call writes the low words and
 *                 returns GC_ERR_OVERFLOW.
 * Runs on the graph's stream and returns when the results are written.
 * Errors: GC_ERR_ARG, GC_ERR_CUDA, GC_ERR_NOMEM, GC_ERR_OVERFLOW.
 */
gc_status gc_count_edge_graphlets(gc_graph g, uint64_t* per_edge_out, uint64_t* global_out,
                                  uint64_t* global_hi);

/*
 * The count of gc_count_edge_graphlets, plus per-edge induced 4-node counts.
 * The paper defines per edge only x3..x5 and the summands of C_7..C_16
 * (Sec. 4.5); this call adds, for every edge e, the number of 4-vertex sets
 * containing e whose induced subgraph is H_i (Table 1), for the ten
 * 4-node graphlets that have an edge:
 *   induced_out   host or device pointer (as per_edge_out) to
 *                 m x GC_INDUCED_COLS uint64, row e for edge id e, columns
 *                   0 H7 4-clique (= x7)     1 H8 chordal cycle
 *                   2 H9 tailed triangle     3 H10 4-cycle (= x10)
 *                   4 H11 3-star             5 H12 4-path
 *                   6 H13 triangle + vertex  7 H14 two disjoint edges
 *                   8 H15 2-star + vertex    9 H16 edge + two vertices
 *                 Summed over the edges, column i is |E(H_{i+7})| X_{i+7}
 *                 (6, 5, 4, 4, 3, 3, 3, 2, 2, 1 edges); every row sums to
 *                 C(n-2, 2). Must not be NULL when m > 0.
 *   per_edge_out, global_out, global_hi: as in gc_count_edge_graphlets.
 * The extra work is the degree sum of the third vertex of every triangle
 * (pass T), the per-vertex triangle and neighbour-degree sums, and one more
 * per-edge pass; the scratch (16 bytes per vertex, 8 per edge) is kept with
 * the graph. Errors: as gc_count_edge_graphlets.
 */
#define GC_INDUCED_COLS 10
gc_status gc_count_edge_induced(gc_graph g, uint64_t* induced_out, uint64_t* per_edge_out, uint64_t* global_out,
                                uint64_t* global_hi);

/* The 13 unrestricted counts C_3, C_4, C_5, C_7, C_8, ..., C_16 (Sec. 4.5) of
 * the last gc_count_edge_graphlets on g, as low/high 64-bit words (host
 * pointers, 13 each; hi may be NULL). GC_ERR_ARG if g was never counted. */
gc_status gc_graph_csums(gc_graph g, uint64_t* lo, uint64_t* hi);

/* Device time of each phase of the last gc_count_edge_graphlets, measured
 * with CUDA events on the graph's stream. ms: host array of
 * gc_phase_count() doubles. Phases, in order: "pass_t_triangles" (Alg. 1),
 * "pass_c_cycles" (4-cycles through each edge, Alg. 4/6), "pass_k_cliques"
 * (4-cliques and cross terms, Alg. 3/5), "finish_columns" (Sec. 4.5 columns
 * and sums), "induced_columns" (gc_count_edge_induced only; empty otherwise),
 * "derive" (Sec. 4.6), "copy_out". */
int gc_phase_count(void);
const char* gc_phase_name(int i);
gc_status gc_graph_phase_ms(gc_graph g, double* ms);

/* Units of work the kernels processed in the last gc_count_edge_graphlets on
 * g (host pointer, GC_NUM_WORK uint64), in this order:
 *   0 pass T (triangles): sum over lowest vertices a of |out(a)|
 *   1 pass C (4-cycles): wedges h-x-o
 *   2 pass K (4-cliques): sum over lowest vertices a of |out(a)|
 *   3 pass K: out-list entries scanned to build the induced subgraphs H_a
 *   4 pass K: edges of the H_a (= triangles, each once)
 *   5 pass K: bitmatrix words ANDed (edges of H_a x row words)
 *   6 finish: edges whose columns were written
 *   7 kernels launched by the count
 *   8 pass C: wedges of the hub units (counted in shared-memory blocks)
 *   9 pass C: lower neighbours swept, summed over the blocks of the hub units
 *  10 pass T: out-list entries scanned
 *  11 pass T: triangles (each once)
 *  12 pass C: wedges of the units counted in a shared-memory hash
 *  13 pass C: jobs of the hub kernel (hub units cut into ranges of o-range
 *     blocks, Sec. 4.4's finer granularity)
 *  14 pass C: CTAs of the hub kernel
 *  15 pass C: sum over those CTAs of their lifetime, ns (%globaltimer)
 *  16 pass C: the longest of those lifetimes, ns (15 / 14 against 16 is the
 *     kernel's tail)
 *  17 pass C: wedges of the units counted in the packed-key shared-memory hash
 * Used to turn kernel times into algorithmic bytes per second. */
#define GC_NUM_WORK 18
gc_status gc_graph_work_counts(gc_graph g, uint64_t* out);

/* Release the graph and all its device memory. NULL is accepted. The device
 * buffers go back to the library's memory pool (freed in the graph's stream
 * order), where later graphs, counts and batches reuse them; the pool keeps up
 * to GC_POOL_KEEP_BYTES bytes (environment, read when the pool is created on
 * first use; default a quarter of the device's memory) and returns the rest
 * to the device. */
gc_status gc_graph_free(gc_graph g);

/* Return every unused block of the library's memory pool on the current
 * device to the device (like a caching allocator's empty-cache call). Waits
 * for all work on the device first (cudaDeviceSynchronize). Live graphs and
 * batches keep their memory. Errors: GC_ERR_CUDA (no device). */
gc_status gc_release_cached_memory(void);

/*
 * Batched and served counting of many graphs (global counts only).
 *
 * gc_batch_create: a runtime with its own CUDA stream that keeps admitted
 *   graphs resident on the device and counts them in shared launches (one
 *   persistent kernel per pass over all graphs of a launch, with work
 *   stealing over the graphs' vertex groups). device_mem_budget_bytes bounds
 *   the device memory the admitted graphs may hold at once (> 0).
 *   flags: 0, or GC_BATCH_MANUAL (launch only on gc_batch_flush; otherwise a
 *   dispatcher thread launches pending graphs as soon as the device is free:
 *   continuous batching).
 * gc_batch_submit: validates and copies one CSR graph (same rules as
 *   gc_graph_upload), admits it if it fits in the budget, and returns a
 *   ticket. GC_ERR_BUSY if it does not fit now (retry after polling), or
 *   GC_ERR_NOMEM if it could never fit.
 * gc_batch_flush: launch everything pending now (returns without waiting).
 * gc_batch_poll: waits up to timeout_us microseconds (0 = just test, < 0 =
 *   forever) for the ticket. GC_OK: global_out/global_hi (17 words each, hi
 *   may be NULL as above) hold X_1..X_17 and the ticket is retired; GC_PENDING:
 *   not finished; GC_ERR_ARG: unknown or already retired ticket;
 *   GC_ERR_CUDA: the launch that held the ticket failed (message says how).
 * gc_batch_destroy: waits for outstanding work and frees everything.
 */
#define GC_BATCH_MANUAL 0x1u
gc_status gc_batch_create(int64_t device_mem_budget_bytes, uint32_t flags, gc_batch* out);
gc_status gc_batch_submit(gc_batch b, int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                          uint64_t* ticket_out);
/* Submit G graphs at once from one concatenated buffer (the batched form's
 * input): graph g has nvert[g] vertices, local row pointers
 * row_ptr[voff[g] .. voff[g] + nvert[g]] (starting at 0) and local columns
 * col_idx[eoff[g] .. eoff[g + 1]). All graphs are validated (in parallel)
 * and admitted together, or none is: the first invalid graph's error is
 * returned (message names its index), GC_ERR_BUSY if they do not fit in the
 * budget now. tickets_out receives G tickets. Host pointers; copied into a
 * host buffer that the batch keeps for reuse once the graphs retire (at most
 * four such buffers, the smallest given back first; all freed by
 * gc_batch_destroy once no graph holds them). */
gc_status gc_batch_submit_many(gc_batch b, int64_t G, const int32_t* nvert, const int64_t* voff, const int64_t* eoff,
                               const int32_t* row_ptr, const int32_t* col_idx, uint64_t* tickets_out);
gc_status gc_batch_flush(gc_batch b);
gc_status gc_batch_poll(gc_batch b, uint64_t ticket, uint64_t* global_out, uint64_t* global_hi,
                        int32_t timeout_us);
/* Waits (as gc_batch_poll) until all G tickets are done, then writes their
 * X_1..X_17 to global_out[17 g .. 17 g + 16] (and the high words to
 * global_hi, which may be NULL as above) and retires them. GC_PENDING: not
 * all done within timeout_us, nothing retired; GC_ERR_ARG: a ticket unknown
 * or retired; a failed launch's status if one of them failed (all are
 * retired). Host pointers. */
gc_status gc_batch_poll_many(gc_batch b, int64_t G, const uint64_t* tickets, uint64_t* global_out,
                             uint64_t* global_hi, int32_t timeout_us);
gc_status gc_batch_destroy(gc_batch b);

/*
 * Tuning of the batched form. Graphs of at most GC_PARAM_SMALL_N_MAX vertices
 * are counted one CTA per graph on a shared-memory bitmatrix (Alg. 1/5/6 as
 * bit operations), binned by vertex count into size classes n <= 64, 128,
 * 256, 512 and 1024, each class with its own block size; larger graphs go
 * through the general passes as one disjoint union. The small-graph sequence
 * of a launch (copies in, kernels, Sec. 4.6 derivation, copy out) is
 * captured into a CUDA graph and replayed (GC_PARAM_USE_GRAPH = 1), or
 * issued eagerly with a timer per size class (0). gc_batch_create takes the
 * defaults (512; 256 threads per class; 1), then the tuning cache's entry for
 * the GPU if there is one: the JSON file named by the environment variable
 * GC_TUNE_CACHE, else tune_cache.json beside libgc.so, written by the tuner
 * (paper_1608_05138_gb300/tune.py). Results are identical under every
 * setting. A parameter applies to launches taken after the call.
 *   GC_PARAM_SMALL_N_MAX   0 .. 1024
 *   GC_PARAM_BLOCK_N64 + c threads per CTA of size class c (n <= 64, 128,
 *                          256, 512, 1024): 64, 128, 256 or 512
 *   GC_PARAM_USE_GRAPH     0 or 1
 *   GC_PARAM_MAX_INFLIGHT  1 .. 4: launches the dispatcher of a continuous
 *                          batch keeps in flight, each on its own stream
 *                          (default 2)
 * Errors: GC_ERR_ARG (unknown parameter or value out of range).
 */
#define GC_PARAM_SMALL_N_MAX 0
#define GC_PARAM_BLOCK_N64 1
#define GC_PARAM_USE_GRAPH 6
#define GC_PARAM_MAX_INFLIGHT 7
gc_status gc_batch_set_param(gc_batch b, int32_t param, int32_t value);
gc_status gc_batch_get_param(gc_batch b, int32_t param, int32_t* value);

/* Device times (ms, CUDA events) of the last launch the batch retired, as
 * GC_BATCH_STATS doubles: [0..4] the bitmatrix kernel of each size class
 * (eager launches only, else 0), [5] the whole small-graph sequence, [6] the
 * larger graphs' passes, [7] 1 if the small-graph sequence was replayed from
 * a CUDA graph. */
#define GC_BATCH_STATS 8
gc_status gc_batch_last_stats(gc_batch b, double* out);

/*
 * Triangle counts per CSR slot without any memory allocation.
 *
 * For callers that cannot allocate device memory (a fixed arena, an
 * allocator callback, a budget that forbids growth). The
 * paper has no counterpart: it is a variant of the triangle step that reads
 * the caller's device CSR in place and uses, as its only scratch, a 32 MiB
 * file-scope device array (256 bitmaps of 2^20 bits) that every GPU loading
 * libgc.so holds until the process exits.
 *   n        vertices, 0 <= n <= 1,048,576; larger n returns GC_ERR_OVERFLOW
 *   row_ptr  device pointer, n + 1 int32 (same CSR rules as gc_graph_upload;
 *            not validated here: a column index outside [0, n) is skipped,
 *            and a slot whose column is outside gets 0)
 *   col_idx  device pointer, row_ptr[n] int32
 *   tri_out  device pointer, row_ptr[n] int32: tri_out[p] = |Gamma(x) ∩ Gamma(y)|
 *            for the slot p = (x, y) (both directions of an edge get its |T|)
 *   stream   cudaStream_t (as void*), NULL = legacy default stream
 * Asynchronous on `stream`; calls no cudaMalloc/cudaFree. The first call on a
 * device, with that device current, looks up the array's device address
 * (cudaGetSymbolAddress) -- make that first call before any stream capture.
 * The address is kept per device ordinal for the life of the process: it
 * assumes the runtime's primary context and no cudaDeviceReset afterwards.
 * All calls share the array and each call clears it first: calls whose
 * kernels overlap on the GPU (other streams, other threads) race and give
 * wrong results.
 */
gc_status gc_edge_triangles_noalloc(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t* tri_out,
                                    void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GC_H */
