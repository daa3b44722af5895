"""CPU oracle for per-edge graphlet counts -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package. The product path (the ``gc_*`` library and its
Python binding) never touches it, and it shares no code with the CUDA path.

``oracle.cpp`` follows the paper's CPU method (Alg. 1 / 5 / 6 with Psi tags,
the per-edge equations of Sec. 4.5 and the global relations of Sec. 4.6,
with the corrections documented there); ``brute.py`` is an independent
full-enumeration census used to pin it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CSUM_NAMES = ["C3", "C4", "C5", "C7", "C8", "C9", "C10", "C11", "C12", "C13", "C14", "C15", "C16"]
COLUMNS = ["x3", "x4", "x5", "x7", "x10", "c8", "c9", "c11", "c12", "c13", "c14", "c15", "c16"]


def build(force: bool = False) -> str:
    """Compile liboracle.so in-tree with g++ -O3 (portable flags only)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O3", "-std=c++17", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            vp = C.c_void_p
            L.oracle_num_edges.restype = C.c_int64
            L.oracle_num_edges.argtypes = [C.c_int32, vp]
            L.oracle_edges.argtypes = [C.c_int32, vp, vp, vp]
            L.oracle_count.argtypes = [C.c_int32, vp, vp, C.c_int, vp, vp, vp, vp, vp]
            L.oracle_count_sample.argtypes = [C.c_int32, vp, vp, C.c_int, vp, C.c_int64, vp]
            L.oracle_derive.argtypes = [C.c_int64, C.c_int64, vp, vp, vp, vp]
            L.oracle_count_induced.argtypes = [C.c_int32, vp, vp, C.c_int, vp, C.c_int64, vp]
            _lib = L
    return _lib


def _p(a):
    return C.c_void_p(a.ctypes.data)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def _join(lo, hi):
    return [int(l) | (int(h) << 64) for l, h in zip(lo, hi)]


def edges(row_ptr, col_idx):
    rp = np.ascontiguousarray(row_ptr, np.int32)
    ci = np.ascontiguousarray(col_idx, np.int32)
    n = len(rp) - 1
    m = int(rp[-1]) // 2
    uv = np.zeros((m, 2), np.int32)
    lib().oracle_edges(n, _p(rp), _p(ci), _p(uv))
    return uv


def count(row_ptr, col_idx, per_edge: bool = True, threads: int | None = None):
    """Whole-graph oracle. Returns dict with
    per_edge (uint64 [m, 13] or None), csum (13 Python ints), X (17 Python ints)."""
    rp = np.ascontiguousarray(row_ptr, np.int32)
    ci = np.ascontiguousarray(col_idx, np.int32)
    n = len(rp) - 1
    m = int(rp[-1]) // 2
    pe = np.zeros((m, 13), np.uint64) if per_edge else None
    clo, chi = np.zeros(13, np.uint64), np.zeros(13, np.uint64)
    xlo, xhi = np.zeros(17, np.uint64), np.zeros(17, np.uint64)
    rc = lib().oracle_count(n, _p(rp), _p(ci), threads or default_threads(),
                            _p(pe) if pe is not None else None, _p(clo), _p(chi), _p(xlo), _p(xhi))
    if rc != 0:
        raise ArithmeticError("oracle: a division of the global relations was not exact")
    return {"per_edge": pe, "csum": _join(clo, chi), "X": _join(xlo, xhi)}


def count_sample(row_ptr, col_idx, edge_ids, threads: int | None = None):
    """Per-edge columns (uint64 [k, 13]) for the given edge ids."""
    rp = np.ascontiguousarray(row_ptr, np.int32)
    ci = np.ascontiguousarray(col_idx, np.int32)
    ids = np.ascontiguousarray(edge_ids, np.int64)
    out = np.zeros((len(ids), 13), np.uint64)
    rc = lib().oracle_count_sample(len(rp) - 1, _p(rp), _p(ci), threads or default_threads(),
                                   _p(ids), len(ids), _p(out))
    if rc != 0:
        raise IndexError("oracle: edge id out of range")
    return out


INDUCED = ["H7", "H8", "H9", "H10", "H11", "H12", "H13", "H14", "H15", "H16"]


def count_induced(row_ptr, col_idx, edge_ids=None, threads: int | None = None):
    """Per-edge induced 4-node counts (uint64 [k, 10], columns H7..H16 of
    Table 1): for each edge, the number of 4-vertex sets containing it whose
    induced subgraph is H_i. All edges in edge-id order, or the given ids."""
    rp = np.ascontiguousarray(row_ptr, np.int32)
    ci = np.ascontiguousarray(col_idx, np.int32)
    m = int(rp[-1]) // 2
    ids = None if edge_ids is None else np.ascontiguousarray(edge_ids, np.int64)
    k = m if ids is None else len(ids)
    out = np.zeros((k, 10), np.uint64)
    if k == 0:
        return out
    rc = lib().oracle_count_induced(len(rp) - 1, _p(rp), _p(ci), threads or default_threads(),
                                    _p(ids) if ids is not None else None, k, _p(out))
    if rc != 0:
        raise IndexError("oracle: edge id out of range")
    return out


def derive(n: int, m: int, csum):
    """Global relations of Sec. 4.6 alone, from 13 unrestricted counts."""
    lo = np.array([c & (2**64 - 1) for c in csum], np.uint64)
    hi = np.array([c >> 64 for c in csum], np.uint64)
    xlo, xhi = np.zeros(17, np.uint64), np.zeros(17, np.uint64)
    rc = lib().oracle_derive(n, m, _p(lo), _p(hi), _p(xlo), _p(xhi))
    return rc, _join(xlo, xhi)
