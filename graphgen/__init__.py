"""Seeded synthetic graph generators shared by the CPU oracle and the GPU path.

This package draws graphs; it contains none of the graphlet-counting
arithmetic. All randomness comes from one counter-based generator
(SplitMix64, Steele/Lea/Flood 2014) implemented in ``graphgen.c``, so the
same seed gives the same graph on x86_64 and aarch64.

Every generator returns a CSR graph ``(row_ptr, col_idx)`` as int32 numpy
arrays: ``row_ptr`` has n + 1 entries starting at 0, each row of
``col_idx`` is sorted ascending, the graph is symmetric and simple.

The named workloads stand in for the paper's graphs (power-law social, web
and technological networks with skewed per-edge work, Sec. 5 / Fig. 1, and
the random graphs of its GPU comparison); the real datasets are not used.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_SO = os.path.join(_HERE, "libgraphgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile libgraphgen.so in-tree with gcc (no FMA contraction)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            P32 = C.POINTER(C.POINTER(C.c_int32))
            P64 = C.POINTER(C.POINTER(C.c_int64))
            L.gg_free.argtypes = [C.c_void_p]
            L.gg_splitmix_at.restype = C.c_uint64
            L.gg_splitmix_at.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64]
            L.gg_er.argtypes = [C.c_int32, C.c_double, C.c_uint64, C.POINTER(C.c_int64), P32, P32]
            L.gg_chung_lu.argtypes = [C.c_int32, C.c_int64, C.c_double, C.c_double, C.c_double,
                                      C.c_uint64, C.POINTER(C.c_int64), P32, P32]
            L.gg_rmat.argtypes = [C.c_int, C.c_int64, C.c_double, C.c_double, C.c_double,
                                  C.c_uint64, C.POINTER(C.c_int32), C.POINTER(C.c_int64), P32, P32]
            L.gg_batch.argtypes = [C.c_int64, C.c_int32, C.c_int32, C.c_double, C.c_double,
                                   C.c_double, C.c_double, C.c_uint64,
                                   P32, P64, P64, P32, P32, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
            L.gg_serving_params.argtypes = [C.c_int64, C.c_int64, C.c_int64, C.c_double, C.c_double,
                                            C.c_uint64, C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                            C.POINTER(C.c_double), C.POINTER(C.c_double),
                                            C.POINTER(C.c_uint64)]
            _lib = L
    return _lib


def _take(ptr, count, dtype):
    """Copy a malloc'd C array into numpy and free it."""
    if count == 0:
        out = np.zeros(0, dtype=dtype)
    else:
        ctype = np.ctypeslib.as_ctypes_type(dtype)
        arr = np.ctypeslib.as_array(C.cast(ptr, C.POINTER(ctype)), shape=(count,))
        out = np.array(arr, dtype=dtype, copy=True)
    lib().gg_free(C.cast(ptr, C.c_void_p))
    return out


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"graphgen.{what} failed with code {rc}")


def splitmix_at(seed: int, stream: int, i: int) -> int:
    return int(lib().gg_splitmix_at(seed, stream, i))


def er(n: int, p: float, seed: int = 1):
    """G(n, p): each pair i < j (lexicographic rank k) present iff u(k) < p."""
    L = lib()
    m = C.c_int64()
    rp = C.POINTER(C.c_int32)()
    ci = C.POINTER(C.c_int32)()
    _check(L.gg_er(n, p, seed, C.byref(m), C.byref(rp), C.byref(ci)), "er")
    return _take(rp, n + 1, np.int32), _take(ci, 2 * m.value, np.int32)


def chung_lu(n: int, m_target: int, gamma: float, sum_w: float, w_cap: float, seed: int = 1):
    """Chung-Lu: weights (i+1)^(-1/(gamma-1)) scaled to sum_w, capped at w_cap;
    pairs drawn from an alias table until m_target distinct non-loop pairs."""
    L = lib()
    m = C.c_int64()
    rp = C.POINTER(C.c_int32)()
    ci = C.POINTER(C.c_int32)()
    _check(L.gg_chung_lu(n, m_target, gamma, sum_w, w_cap, seed, C.byref(m), C.byref(rp),
                         C.byref(ci)), "chung_lu")
    return _take(rp, n + 1, np.int32), _take(ci, 2 * m.value, np.int32)


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1):
    """R-MAT (Chakrabarti, Zhan, Faloutsos 2004), no noise, no permutation;
    symmetrised, deduplicated, self-loops dropped, isolated vertices kept."""
    L = lib()
    n = C.c_int32()
    m = C.c_int64()
    rp = C.POINTER(C.c_int32)()
    ci = C.POINTER(C.c_int32)()
    _check(L.gg_rmat(scale, edge_factor, a, b, c, seed, C.byref(n), C.byref(m), C.byref(rp),
                     C.byref(ci)), "rmat")
    return _take(rp, n.value + 1, np.int32), _take(ci, 2 * m.value, np.int32)


class Batch:
    """A batch of small graphs in concatenated CSR form.

    Graph g has ``nvert[g]`` vertices; its local row pointers are
    ``row_ptr[voff[g] : voff[g] + nvert[g] + 1]`` (starting at 0) and its local
    column ids are ``col_idx[eoff[g] : eoff[g + 1]]``.
    """

    def __init__(self, nvert, voff, eoff, row_ptr, col_idx):
        self.nvert, self.voff, self.eoff = nvert, voff, eoff
        self.row_ptr, self.col_idx = row_ptr, col_idx

    def __len__(self):
        return len(self.nvert)

    def graph(self, g: int):
        n = int(self.nvert[g])
        v0 = int(self.voff[g])
        return self.row_ptr[v0:v0 + n + 1], self.col_idx[int(self.eoff[g]):int(self.eoff[g + 1])]

    @property
    def total_edges(self) -> int:
        return int(self.eoff[-1]) // 2


def batch(G: int, n_lo: int = 20, n_hi: int = 500, p_lo: float = 0.05, p_hi: float = 0.5,
          g_lo: float = 2.0, g_hi: float = 3.0, seed: int = 1) -> Batch:
    """Mixed batch: even ids ER(n, p), odd ids Chung-Lu(n, gamma, mean degree)."""
    L = lib()
    nv = C.POINTER(C.c_int32)()
    vo = C.POINTER(C.c_int64)()
    eo = C.POINTER(C.c_int64)()
    rp = C.POINTER(C.c_int32)()
    ci = C.POINTER(C.c_int32)()
    rows = C.c_int64()
    nnz = C.c_int64()
    _check(L.gg_batch(G, n_lo, n_hi, p_lo, p_hi, g_lo, g_hi, seed, C.byref(nv), C.byref(vo),
                      C.byref(eo), C.byref(rp), C.byref(ci), C.byref(rows), C.byref(nnz)), "batch")
    return Batch(_take(nv, G, np.int32), _take(vo, G + 1, np.int64), _take(eo, G + 1, np.int64),
                 _take(rp, rows.value, np.int32), _take(ci, nnz.value, np.int32))


def serving_params(R: int, m_lo: int = 1000, m_hi: int = 2_000_000, g_lo: float = 2.1,
                   g_hi: float = 2.5, seed: int = 1):
    """Per-request sizes of the serving stream: dict of numpy arrays
    m, n, gamma, gap (unit-rate exponential inter-arrival), seed."""
    L = lib()
    m = np.zeros(R, np.int64)
    n = np.zeros(R, np.int32)
    gam = np.zeros(R, np.float64)
    gap = np.zeros(R, np.float64)
    sd = np.zeros(R, np.uint64)
    _check(L.gg_serving_params(R, m_lo, m_hi, g_lo, g_hi, seed,
                               m.ctypes.data_as(C.POINTER(C.c_int64)),
                               n.ctypes.data_as(C.POINTER(C.c_int32)),
                               gam.ctypes.data_as(C.POINTER(C.c_double)),
                               gap.ctypes.data_as(C.POINTER(C.c_double)),
                               sd.ctypes.data_as(C.POINTER(C.c_uint64))), "serving_params")
    return {"m": m, "n": n, "gamma": gam, "gap": gap, "seed": sd}


def serving_graph(params: dict, r: int):
    m = int(params["m"][r])
    n = int(params["n"][r])
    return chung_lu(n, m, float(params["gamma"][r]), 2.0 * m, float(min(50000, n - 1)),
                    int(params["seed"][r]))


# ---- the named workloads ----

def config_er2000(seed: int = 1):
    """Erdos-Renyi G(n=2000, p=0.01), about 20k edges."""
    return er(2000, 0.01, seed)


def config_chung_lu(seed: int = 1, n: int = 1_000_000, m: int = 10_000_000):
    """Chung-Lu, n = 1M, m = 10M distinct edges, exponent 2.1, weights scaled to
    sum 2m and capped at 50k."""
    return chung_lu(n, m, 2.1, 2.0 * m, 50000.0, seed)


def config_rmat(scale: int = 22, seed: int = 1):
    """R-MAT scale 22, edge factor 16, (0.57, 0.19, 0.19, 0.05)."""
    return rmat(scale, 16, 0.57, 0.19, 0.19, seed)


def config_er_dense(seed: int = 1):
    """Dense Erdos-Renyi G(n=1000, p=0.3), about 150k edges: the 1K-vertex /
    150K-edge shape of the paper's single-GPU comparison (Sec. 5, Fig. 3)."""
    return er(1000, 0.3, seed)
