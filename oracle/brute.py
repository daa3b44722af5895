"""Brute-force graphlet census -- test infrastructure, independent of everything else.

TEST INFRASTRUCTURE ONLY (tests, smoke, bench's CPU baseline). This module
does not use the per-edge machinery of the paper at all: it enumerates every
2-, 3- and 4-vertex subset of a small graph and classifies the induced
subgraph by its number of edges and sorted degree sequence, which identifies
each of the 17 graphlets of Table 1 uniquely:

  k=2: H1 edge, H2 non-edge
  k=3: H3 triangle (3 edges), H4 2-star (2), H5 one edge (1), H6 empty (0)
  k=4: H7 4-clique (6 edges), H8 chordal cycle (5), H9 tailed triangle
       (4; degrees 3,2,2,1), H10 4-cycle (4; 2,2,2,2), H11 3-star
       (3; 3,1,1,1), H12 4-path (3; 2,2,1,1), H13 triangle + isolated
       vertex (3; 2,2,2,0), H14 two disjoint edges (2; 1,1,1,1), H15 2-star +
       isolated vertex (2; 2,1,1,0), H16 one edge (1), H17 empty (0).

It also gives per-edge quantities straight from their definitions (Problem 1
and Fig. 2): T, S_u, S_v, D_e as set operations, x7 = number of 4-sets
{u, v, a, b} inducing a 4-clique and x10 = number inducing a 4-cycle.
Only for small graphs (pure Python loops).
"""
from __future__ import annotations

from itertools import combinations
from math import comb

import numpy as np

# (edge count, sorted degree tuple) -> graphlet index 1..17
_CLASS4 = {
    (6, (3, 3, 3, 3)): 7,
    (5, (2, 2, 3, 3)): 8,
    (4, (1, 2, 2, 3)): 9,
    (4, (2, 2, 2, 2)): 10,
    (3, (1, 1, 1, 3)): 11,
    (3, (1, 1, 2, 2)): 12,
    (3, (0, 2, 2, 2)): 13,
    (2, (1, 1, 1, 1)): 14,
    (2, (0, 1, 1, 2)): 15,
    (1, (0, 0, 1, 1)): 16,
    (0, (0, 0, 0, 0)): 17,
}
_CLASS3 = {3: 3, 2: 4, 1: 5, 0: 6}


def adjacency_sets(row_ptr, col_idx):
    n = len(row_ptr) - 1
    return [set(int(c) for c in col_idx[row_ptr[i]:row_ptr[i + 1]]) for i in range(n)]


def census(row_ptr, col_idx):
    """Global counts X_1..X_17 (list index 0 -> X_1) by full enumeration."""
    adj = adjacency_sets(row_ptr, col_idx)
    n = len(adj)
    X = [0] * 18
    m = sum(len(a) for a in adj) // 2
    X[1] = m
    X[2] = comb(n, 2) - m
    for s in combinations(range(n), 3):
        e = sum(1 for a, b in combinations(s, 2) if b in adj[a])
        X[_CLASS3[e]] += 1
    for s in combinations(range(n), 4):
        deg = {x: 0 for x in s}
        e = 0
        for a, b in combinations(s, 2):
            if b in adj[a]:
                e += 1
                deg[a] += 1
                deg[b] += 1
        X[_CLASS4[(e, tuple(sorted(deg.values())))]] += 1
    return X[1:]


def per_edge(row_ptr, col_idx):
    """Per-edge rows (edge-id order: u < v, row-major), each a dict of
    t, su, sv, D, x7, x10 from the set definitions."""
    adj = adjacency_sets(row_ptr, col_idx)
    n = len(adj)
    rows = []
    for u in range(n):
        for v in sorted(adj[u]):
            if v <= u:
                continue
            T = adj[u] & adj[v]
            Su = adj[u] - T - {v}
            Sv = adj[v] - T - {u}
            D = n - 2 - len(T) - len(Su) - len(Sv)
            others = [x for x in range(n) if x != u and x != v]
            x7 = x10 = 0
            for a, b in combinations(others, 2):
                s = (u, v, a, b)
                deg = {x: 0 for x in s}
                e = 0
                for p, q in combinations(s, 2):
                    if q in adj[p]:
                        e += 1
                        deg[p] += 1
                        deg[q] += 1
                cls = _CLASS4[(e, tuple(sorted(deg.values())))]
                if cls == 7:
                    x7 += 1
                elif cls == 10:
                    x10 += 1
            rows.append(dict(u=u, v=v, t=len(T), su=len(Su), sv=len(Sv), D=D, x7=x7, x10=x10))
    return rows


def per_edge_columns(row_ptr, col_idx, m=None):
    """The 13 per-edge columns computed from the brute-force sets."""
    rows = per_edge(row_ptr, col_idx)
    n = len(row_ptr) - 1
    if m is None:
        m = len(rows)
    adj = adjacency_sets(row_ptr, col_idx)
    out = np.zeros((len(rows), 13), dtype=np.uint64)
    for i, r in enumerate(rows):
        t, su, sv, D = r["t"], r["su"], r["sv"], r["D"]
        s = su + sv
        du, dv = len(adj[r["u"]]), len(adj[r["v"]])
        out[i] = [t, s, D, r["x7"], r["x10"], comb(t, 2), t * s, comb(su, 2) + comb(sv, 2),
                  su * sv, t * D, m - du - dv + 1, s * D, comb(D, 2)]
    return out


def per_edge_induced(row_ptr, col_idx):
    """Per edge (edge-id order), the number of 4-vertex sets containing it
    whose induced subgraph is H_7 .. H_16: int64 [m, 10], by enumerating
    every pair {a, b} of the other vertices and classifying {u, v, a, b}."""
    adj = adjacency_sets(row_ptr, col_idx)
    n = len(adj)
    rows = []
    for u in range(n):
        for v in sorted(adj[u]):
            if v <= u:
                continue
            row = [0] * 10
            others = [x for x in range(n) if x != u and x != v]
            for a, b in combinations(others, 2):
                s = (u, v, a, b)
                deg = {x: 0 for x in s}
                e = 0
                for p, q in combinations(s, 2):
                    if q in adj[p]:
                        e += 1
                        deg[p] += 1
                        deg[q] += 1
                row[_CLASS4[(e, tuple(sorted(deg.values())))] - 7] += 1
            rows.append(row)
    return np.array(rows, dtype=np.int64).reshape(-1, 10)
