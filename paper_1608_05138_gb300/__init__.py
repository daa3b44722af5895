"""Python binding of libgc.so -- exact per-edge 3/4-node graphlet counts on GB300.

Thin ctypes marshalling over the C ABI declared in include/gc.h; every step
of the computation runs in the library's CUDA kernels. The functions keep the
C names. Arrays may be numpy arrays (host) or torch tensors (host or CUDA);
torch streams are passed as ``torch.cuda.Stream`` objects or raw handles.

There is no CPU fallback: importing works anywhere, but the first call raises
``RuntimeError`` if libgc.so has not been built (``__graft_entry__.build()``)
or cannot be loaded.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libgc.so")
_lock = threading.Lock()
_lib = None

GC_OK, GC_PENDING = 0, 1
STATUS_NAMES = {
    0: "GC_OK", 1: "GC_PENDING", -1: "GC_ERR_ARG", -2: "GC_ERR_UNSORTED", -3: "GC_ERR_DUPLICATE",
    -4: "GC_ERR_SELF_LOOP", -5: "GC_ERR_ASYMMETRIC", -6: "GC_ERR_RANGE", -7: "GC_ERR_NOMEM",
    -8: "GC_ERR_CUDA", -9: "GC_ERR_OVERFLOW", -10: "GC_ERR_TIMEOUT", -11: "GC_ERR_BUSY",
}
GC_EDGE_COLS = 13
GC_INDUCED_COLS = 10
INDUCED_NAMES = ["H7", "H8", "H9", "H10", "H11", "H12", "H13", "H14", "H15", "H16"]
GC_NUM_GRAPHLETS = 17
GC_NO_VALIDATE = 0x1
GC_BATCH_MANUAL = 0x1
GC_PARAM_SMALL_N_MAX, GC_PARAM_BLOCK_N64, GC_PARAM_USE_GRAPH, GC_PARAM_MAX_INFLIGHT = 0, 1, 6, 7
SMALL_CLASS_N = [64, 128, 256, 512, 1024]      # size classes of the bitmatrix kernels
SMALL_BLOCKS = [64, 128, 256, 512]
BATCH_STATS = ["class_n64_ms", "class_n128_ms", "class_n256_ms", "class_n512_ms", "class_n1024_ms",
               "small_sequence_ms", "union_ms", "replayed"]
EXPORTED = ["gc_last_error", "gc_graph_upload", "gc_graph_info", "gc_graph_edges",
            "gc_count_edge_graphlets", "gc_graph_csums", "gc_phase_count", "gc_phase_name",
            "gc_graph_phase_ms", "gc_graph_free", "gc_batch_create", "gc_batch_submit",
            "gc_batch_flush", "gc_batch_poll", "gc_batch_destroy", "gc_edge_triangles_noalloc",
            "gc_graph_work_counts", "gc_batch_submit_many", "gc_count_edge_induced", "gc_batch_set_param",
            "gc_batch_get_param", "gc_batch_last_stats", "gc_batch_poll_many", "gc_release_cached_memory",
            "gc_validate_csr"]
WORK_NAMES = ["t_members", "c_wedges", "k_members", "k_scan", "k_local_edges", "k_words", "finish_edges", "launches",
              "c_heavy_wedges", "c_heavy_sweeps", "t_scan", "t_triangles", "c_hash_wedges", "c_hub_jobs",
              "c_hub_ctas", "c_hub_busy_sum_ns", "c_hub_busy_max_ns", "c_hash2_wedges"]


class GcError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")


def library_path() -> str:
    return _SO


def lib():
    """Load libgc.so (raises if it is missing: there is no fallback path)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_SO):
                raise RuntimeError(f"{_SO} is not built; run __graft_entry__.build()")
            L = C.CDLL(_SO)
            vp, i32, i64, u32 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32
            L.gc_last_error.restype = C.c_char_p
            L.gc_graph_upload.argtypes = [i32, vp, vp, u32, vp, C.POINTER(vp)]
            L.gc_graph_info.argtypes = [vp, C.POINTER(i64), C.POINTER(i64)]
            L.gc_graph_edges.argtypes = [vp, vp]
            L.gc_count_edge_graphlets.argtypes = [vp, vp, vp, vp]
            L.gc_count_edge_induced.argtypes = [vp, vp, vp, vp, vp]
            L.gc_graph_csums.argtypes = [vp, vp, vp]
            L.gc_phase_name.restype = C.c_char_p
            L.gc_phase_name.argtypes = [C.c_int]
            L.gc_graph_phase_ms.argtypes = [vp, vp]
            L.gc_graph_free.argtypes = [vp]
            L.gc_batch_create.argtypes = [i64, u32, C.POINTER(vp)]
            L.gc_batch_submit.argtypes = [vp, i32, vp, vp, C.POINTER(C.c_uint64)]
            L.gc_batch_flush.argtypes = [vp]
            L.gc_batch_poll.argtypes = [vp, C.c_uint64, vp, vp, i32]
            L.gc_batch_destroy.argtypes = [vp]
            L.gc_edge_triangles_noalloc.argtypes = [i32, vp, vp, vp, vp]
            L.gc_graph_work_counts.argtypes = [vp, vp]
            L.gc_batch_submit_many.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp]
            L.gc_batch_set_param.argtypes = [vp, i32, i32]
            L.gc_batch_get_param.argtypes = [vp, i32, C.POINTER(i32)]
            L.gc_batch_last_stats.argtypes = [vp, vp]
            L.gc_batch_poll_many.argtypes = [vp, i64, vp, vp, vp, i32]
            L.gc_release_cached_memory.argtypes = []
            for name in ("gc_graph_upload", "gc_graph_info", "gc_graph_edges", "gc_count_edge_graphlets",
                         "gc_count_edge_induced",
                         "gc_graph_csums", "gc_graph_phase_ms", "gc_graph_free", "gc_batch_create",
                         "gc_batch_submit", "gc_batch_flush", "gc_batch_poll", "gc_batch_destroy",
                         "gc_edge_triangles_noalloc", "gc_graph_work_counts", "gc_batch_submit_many",
                         "gc_batch_set_param", "gc_batch_get_param", "gc_batch_last_stats", "gc_batch_poll_many",
                         "gc_release_cached_memory", "gc_validate_csr"):
                getattr(L, name).restype = C.c_int
            _lib = L
    return _lib


def _check(status: int, where: str):
    if status not in (GC_OK, GC_PENDING):
        raise GcError(status, where, lib().gc_last_error().decode(errors="replace"))
    return status


def _ptr(a):
    """Raw address of a contiguous numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr())
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return C.c_void_p(a.ctypes.data)


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _host_i32(a):
    if hasattr(a, "cpu"):
        a = a.cpu().numpy()
    return np.ascontiguousarray(a, dtype=np.int32)


def _join(lo, hi):
    return [int(l) | (int(h) << 64) for l, h in zip(lo, hi)]


# ---------------- plain whole-graph API ----------------

def gc_last_error() -> str:
    return lib().gc_last_error().decode(errors="replace")


def gc_validate_csr(row_ptr, col_idx):
    """The host checks of gc_graph_upload alone (no device work); raises
    GcError with the code and message of the first failing entry."""
    rp, ci = _host_i32(row_ptr), _host_i32(col_idx)
    _check(lib().gc_validate_csr(len(rp) - 1, _ptr(rp), _ptr(ci) if len(ci) else None), "gc_validate_csr")


def gc_graph_upload(row_ptr, col_idx, flags: int = 0, stream=None):
    """Validate, copy and prepare a host CSR graph; returns the handle."""
    rp, ci = _host_i32(row_ptr), _host_i32(col_idx)
    h = C.c_void_p()
    _check(lib().gc_graph_upload(len(rp) - 1, _ptr(rp), _ptr(ci) if len(ci) else None, flags,
                                 _stream_handle(stream), C.byref(h)), "gc_graph_upload")
    return h


def gc_graph_info(g):
    n, m = C.c_int64(), C.c_int64()
    _check(lib().gc_graph_info(g, C.byref(n), C.byref(m)), "gc_graph_info")
    return n.value, m.value


def gc_graph_edges(g):
    _, m = gc_graph_info(g)
    uv = np.zeros((m, 2), np.int32)
    if m:
        _check(lib().gc_graph_edges(g, _ptr(uv)), "gc_graph_edges")
    return uv


def gc_count_edge_graphlets(g, per_edge_out=None, wide: bool = True):
    """Count; fills per_edge_out ([m, 13] uint64 numpy array, or int64/uint64
    CUDA tensor) if given and returns X_1..X_17 as Python ints."""
    lo = np.zeros(17, np.uint64)
    hi = np.zeros(17, np.uint64)
    _check(lib().gc_count_edge_graphlets(g, _ptr(per_edge_out), _ptr(lo), _ptr(hi) if wide else None),
           "gc_count_edge_graphlets")
    return _join(lo, hi)


def gc_count_edge_induced(g, induced_out, per_edge_out=None, wide: bool = True):
    """Count with per-edge induced 4-node counts: fills induced_out ([m, 10]
    uint64 numpy array, or int64/uint64 CUDA tensor; columns H7..H16) and
    per_edge_out if given; returns X_1..X_17 as Python ints."""
    lo = np.zeros(17, np.uint64)
    hi = np.zeros(17, np.uint64)
    _check(lib().gc_count_edge_induced(g, _ptr(induced_out), _ptr(per_edge_out), _ptr(lo), _ptr(hi) if wide else None),
           "gc_count_edge_induced")
    return _join(lo, hi)


def gc_graph_csums(g):
    lo = np.zeros(13, np.uint64)
    hi = np.zeros(13, np.uint64)
    _check(lib().gc_graph_csums(g, _ptr(lo), _ptr(hi)), "gc_graph_csums")
    return _join(lo, hi)


def gc_phase_names():
    L = lib()
    return [L.gc_phase_name(i).decode() for i in range(L.gc_phase_count())]


def gc_graph_phase_ms(g):
    ms = np.zeros(lib().gc_phase_count(), np.float64)
    _check(lib().gc_graph_phase_ms(g, _ptr(ms)), "gc_graph_phase_ms")
    return dict(zip(gc_phase_names(), ms.tolist()))


def gc_graph_work_counts(g):
    out = np.zeros(len(WORK_NAMES), np.uint64)
    _check(lib().gc_graph_work_counts(g, _ptr(out)), "gc_graph_work_counts")
    return dict(zip(WORK_NAMES, (int(x) for x in out)))


def gc_graph_free(g):
    if g is not None:
        _check(lib().gc_graph_free(g), "gc_graph_free")


class Graph:
    """Context-managed handle: ``with Graph(rp, ci) as g: X = g.count()``."""

    def __init__(self, row_ptr, col_idx, flags: int = 0, stream=None):
        self.handle = gc_graph_upload(row_ptr, col_idx, flags, stream)
        self.n, self.m = gc_graph_info(self.handle)

    def count(self, per_edge_out=None, wide: bool = True):
        return gc_count_edge_graphlets(self.handle, per_edge_out, wide)

    def count_induced(self, induced_out, per_edge_out=None, wide: bool = True):
        return gc_count_edge_induced(self.handle, induced_out, per_edge_out, wide)

    def edges(self):
        return gc_graph_edges(self.handle)

    def csums(self):
        return gc_graph_csums(self.handle)

    def phase_ms(self):
        return gc_graph_phase_ms(self.handle)

    def work_counts(self):
        return gc_graph_work_counts(self.handle)

    def close(self):
        if self.handle is not None:
            gc_graph_free(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------- batched / served API ----------------

def gc_batch_create(device_mem_budget_bytes: int, flags: int = 0):
    h = C.c_void_p()
    _check(lib().gc_batch_create(int(device_mem_budget_bytes), flags, C.byref(h)), "gc_batch_create")
    return h


def gc_batch_submit(b, row_ptr, col_idx):
    """Returns the ticket, or raises GcError (status GC_ERR_BUSY when the budget is full)."""
    rp, ci = _host_i32(row_ptr), _host_i32(col_idx)
    t = C.c_uint64()
    _check(lib().gc_batch_submit(b, len(rp) - 1, _ptr(rp), _ptr(ci) if len(ci) else None, C.byref(t)),
           "gc_batch_submit")
    return t.value


def gc_batch_try_submit(b, row_ptr, col_idx):
    """Like gc_batch_submit but returns None instead of raising on GC_ERR_BUSY."""
    rp, ci = _host_i32(row_ptr), _host_i32(col_idx)
    t = C.c_uint64()
    st = lib().gc_batch_submit(b, len(rp) - 1, _ptr(rp), _ptr(ci) if len(ci) else None, C.byref(t))
    if st == -11:
        return None
    _check(st, "gc_batch_submit")
    return t.value


def gc_batch_submit_many(b, nvert, voff, eoff, row_ptr, col_idx):
    """Submit many graphs from one concatenated CSR (int32 local ids, int64
    offsets; see include/gc.h). Returns the tickets as a uint64 array."""
    nv = np.ascontiguousarray(nvert, np.int32)
    vo = np.ascontiguousarray(voff, np.int64)
    eo = np.ascontiguousarray(eoff, np.int64)
    rp = np.ascontiguousarray(row_ptr, np.int32)
    ci = np.ascontiguousarray(col_idx, np.int32)
    t = np.zeros(len(nv), np.uint64)
    _check(lib().gc_batch_submit_many(b, len(nv), _ptr(nv), _ptr(vo), _ptr(eo), _ptr(rp),
                                      _ptr(ci) if len(ci) else None, _ptr(t)), "gc_batch_submit_many")
    return t


def gc_batch_flush(b):
    _check(lib().gc_batch_flush(b), "gc_batch_flush")


def gc_batch_poll(b, ticket: int, timeout_us: int = -1):
    """X_1..X_17 as Python ints, or None while pending."""
    lo = np.zeros(17, np.uint64)
    hi = np.zeros(17, np.uint64)
    st = _check(lib().gc_batch_poll(b, ticket, _ptr(lo), _ptr(hi), int(timeout_us)), "gc_batch_poll")
    if st == GC_PENDING:
        return None
    return _join(lo, hi)


def gc_batch_poll_many(b, tickets, timeout_us: int = -1):
    """X_1..X_17 of every ticket as a uint64 array [G, 17, 2] of (low, high)
    words, or None while not all are done (nothing is retired then)."""
    t = np.ascontiguousarray(tickets, np.uint64)
    lo = np.zeros((len(t), 17), np.uint64)
    hi = np.zeros((len(t), 17), np.uint64)
    st = _check(lib().gc_batch_poll_many(b, len(t), _ptr(t), _ptr(lo), _ptr(hi), int(timeout_us)),
                "gc_batch_poll_many")
    if st == GC_PENDING:
        return None
    return np.stack([lo, hi], axis=-1)


def gc_batch_set_param(b, param: int, value: int):
    _check(lib().gc_batch_set_param(b, int(param), int(value)), "gc_batch_set_param")


def gc_batch_get_param(b, param: int) -> int:
    v = C.c_int32()
    _check(lib().gc_batch_get_param(b, int(param), C.byref(v)), "gc_batch_get_param")
    return v.value


def gc_batch_config(b) -> dict:
    """The batch's parameters: small_n_max, block per size class, use_graph."""
    return {"small_n_max": gc_batch_get_param(b, GC_PARAM_SMALL_N_MAX),
            "block": {str(n): gc_batch_get_param(b, GC_PARAM_BLOCK_N64 + c) for c, n in enumerate(SMALL_CLASS_N)},
            "use_graph": gc_batch_get_param(b, GC_PARAM_USE_GRAPH),
            "max_inflight": gc_batch_get_param(b, GC_PARAM_MAX_INFLIGHT)}


def gc_batch_configure(b, config: dict):
    """Set the parameters of a dict shaped like gc_batch_config's (keys may be missing)."""
    if "small_n_max" in config:
        gc_batch_set_param(b, GC_PARAM_SMALL_N_MAX, config["small_n_max"])
    for c, n in enumerate(SMALL_CLASS_N):
        if str(n) in config.get("block", {}):
            gc_batch_set_param(b, GC_PARAM_BLOCK_N64 + c, config["block"][str(n)])
    if "use_graph" in config:
        gc_batch_set_param(b, GC_PARAM_USE_GRAPH, config["use_graph"])
    if "max_inflight" in config:
        gc_batch_set_param(b, GC_PARAM_MAX_INFLIGHT, config["max_inflight"])


def gc_batch_last_stats(b) -> dict:
    out = np.zeros(len(BATCH_STATS), np.float64)
    _check(lib().gc_batch_last_stats(b, _ptr(out)), "gc_batch_last_stats")
    return dict(zip(BATCH_STATS, out.tolist()))


def gc_release_cached_memory():
    """Return the unused blocks of the library's device memory pool to the
    device (waits for all device work first)."""
    _check(lib().gc_release_cached_memory(), "gc_release_cached_memory")


def gc_batch_destroy(b):
    if b is not None:
        _check(lib().gc_batch_destroy(b), "gc_batch_destroy")


# ---------------- allocation-free triangle step ----------------

def _noalloc_args(row_ptr, col_idx, tri_out):
    """The C entry point takes raw device pointers and cannot see sizes or
    types, so a wrong tensor here would make its kernel read or write past a
    buffer: every check happens before the call. Returns n."""
    import torch
    named = (("row_ptr", row_ptr), ("col_idx", col_idx), ("tri_out", tri_out))
    for name, t in named:
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{name} must be a torch tensor")
        if t.dtype != torch.int32:
            raise ValueError(f"{name} must be int32, not {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if row_ptr.dim() != 1 or row_ptr.numel() < 1:
        raise ValueError("row_ptr must be a 1-D tensor of n + 1 >= 1 entries")
    if tri_out.numel() < col_idx.numel():
        raise ValueError(f"tri_out holds {tri_out.numel()} entries, fewer than the {col_idx.numel()} slots of col_idx")
    devs = {t.device for _, t in named}
    if len(devs) != 1 or next(iter(devs)).type != "cuda":
        raise ValueError("row_ptr, col_idx and tri_out must be on the same CUDA device")
    nnz = int(row_ptr[-1].item())  # one 4-byte read back; allocates no device memory
    if nnz < 0 or nnz > col_idx.numel():
        raise ValueError(f"row_ptr[n] = {nnz} does not fit col_idx of {col_idx.numel()} entries")
    return row_ptr.numel() - 1


def gc_edge_triangles_noalloc(row_ptr, col_idx, tri_out, stream=None):
    """Per-slot triangle counts from a device CSR into a device int32 buffer,
    with no memory allocation (see include/gc.h). row_ptr, col_idx and
    tri_out are contiguous int32 tensors on one CUDA device, tri_out with at
    least col_idx.numel() entries (ValueError otherwise); the library reads
    row_ptr[n] entries of col_idx, so row_ptr must describe col_idx. Runs
    asynchronously on `stream`."""
    n = _noalloc_args(row_ptr, col_idx, tri_out)
    _check(lib().gc_edge_triangles_noalloc(n, _ptr(row_ptr), _ptr(col_idx), _ptr(tri_out),
                                           _stream_handle(stream)), "gc_edge_triangles_noalloc")
