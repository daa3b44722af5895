"""Small named graphs for tests (pure Python, CSR int32)."""
from itertools import combinations

import numpy as np


def csr(n, edges):
    """CSR (row_ptr, col_idx) of an undirected simple graph on n vertices."""
    adj = [set() for _ in range(n)]
    for a, b in edges:
        if a == b:
            raise ValueError("self-loop")
        adj[a].add(b)
        adj[b].add(a)
    rp = np.zeros(n + 1, np.int32)
    for i in range(n):
        rp[i + 1] = rp[i] + len(adj[i])
    ci = np.array([c for i in range(n) for c in sorted(adj[i])], dtype=np.int32)
    return rp, ci


def complete(n):
    return csr(n, combinations(range(n), 2))


def star(k):
    return csr(k + 1, [(0, i) for i in range(1, k + 1)])


def cycle(n):
    return csr(n, [(i, (i + 1) % n) for i in range(n)])


def complete_bipartite(a, b):
    return csr(a + b, [(i, a + j) for i in range(a) for j in range(b)])


def empty(n):
    return csr(n, [])


def petersen():
    outer = [(i, (i + 1) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    return csr(10, outer + spokes + inner)


def cube():
    return csr(8, [(a, b) for a in range(8) for b in range(a + 1, 8) if bin(a ^ b).count("1") == 1])


def wheel(k):
    """Hub 0 joined to a k-cycle 1..k."""
    rim = [(1 + i, 1 + (i + 1) % k) for i in range(k)]
    return csr(k + 1, rim + [(0, i) for i in range(1, k + 1)])


def edges_of(rp, ci):
    n = len(rp) - 1
    return [(u, int(v)) for u in range(n) for v in ci[rp[u]:rp[u + 1]] if v > u]


def csr_large(n, edges):
    """csr() for large n with few edges (numpy; no per-vertex Python objects)."""
    e = np.asarray(list(edges), np.int64).reshape(-1, 2)
    if len(e) and (e[:, 0] == e[:, 1]).any():
        raise ValueError("self-loop")
    a = np.concatenate([e[:, 0], e[:, 1]])
    b = np.concatenate([e[:, 1], e[:, 0]])
    key = np.unique(a * n + b)
    rows, cols = key // n, key % n
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, rows + 1, 1)
    return np.cumsum(rp).astype(np.int32), cols.astype(np.int32)
