"""Pins for the CPU oracle against things other than itself.

The oracle (oracle/oracle.cpp) follows the paper's CPU method. Here it is
checked against:
  * an independent brute-force census of every 2/3/4-subset (oracle/brute.py)
    on many small random graphs, per edge and globally;
  * closed forms for K_n, stars, cycles, complete bipartite graphs, empty
    graphs and a single edge, derived by hand from Problem 1;
  * hand-derived values for the 3-cube and the Petersen graph;
  * per-edge x7 and x10 recomputed as quadratic forms of 0/1 indicator
    vectors with numpy (a different computation of the same definitions);
  * counting identities that do not use the per-edge machinery (paths,
    stars and 4-cycles as non-induced subgraphs, converted to induced counts).
"""
from math import comb

import numpy as np
import pytest

import graphgen
import oracle
from oracle import brute
from tests import graphs


def X_of(rp, ci):
    return oracle.count(rp, ci, per_edge=False, threads=2)["X"]


def expect(**nonzero):
    X = [0] * 17
    for k, v in nonzero.items():
        X[int(k[1:]) - 1] = v
    return X


# ---------------- brute force on small random graphs ----------------

@pytest.mark.parametrize("seed", range(1, 41))
def test_oracle_equals_brute_force(seed):
    rng_n = 4 + (seed * 7) % 11          # n in [4, 14]
    for p in (0.15, 0.35, 0.6, 0.9):
        rp, ci = graphgen.er(rng_n, p, seed)
        o = oracle.count(rp, ci, threads=2)
        assert o["X"] == brute.census(rp, ci), (seed, p)
        np.testing.assert_array_equal(o["per_edge"], brute.per_edge_columns(rp, ci))


def test_brute_force_power_law_small():
    for seed in range(1, 6):
        rp, ci = graphgen.chung_lu(14, 30, 2.1, 60.0, 13.0, seed)
        o = oracle.count(rp, ci, threads=2)
        assert o["X"] == brute.census(rp, ci)
        np.testing.assert_array_equal(o["per_edge"], brute.per_edge_columns(rp, ci))


# ---------------- closed forms ----------------

@pytest.mark.parametrize("n", range(2, 13))
def test_complete_graph(n):
    rp, ci = graphs.complete(n)
    o = oracle.count(rp, ci, threads=2)
    assert o["X"] == expect(X1=comb(n, 2), X3=comb(n, 3), X7=comb(n, 4))
    for row in o["per_edge"]:
        assert row[0] == n - 2 and row[1] == 0 and row[2] == 0
        assert row[3] == comb(n - 2, 2) and row[4] == 0


@pytest.mark.parametrize("k", range(1, 12))
def test_star(k):
    rp, ci = graphs.star(k)
    assert X_of(rp, ci) == expect(X1=k, X2=comb(k, 2), X4=comb(k, 2), X6=comb(k, 3),
                                   X11=comb(k, 3), X17=comb(k, 4))


@pytest.mark.parametrize("n", range(6, 16))
def test_cycle(n):
    rp, ci = graphs.cycle(n)
    o = oracle.count(rp, ci, threads=2)
    X = expect(X1=n, X2=comb(n, 2) - n, X4=n, X5=n * (n - 4), X6=comb(n, 3) - n - n * (n - 4),
               X12=n, X14=n * (n - 5) // 2, X15=n * (n - 5),
               X16=n * (comb(n - 4, 2) - (n - 5)))
    X[16] = comb(n, 4) - sum(X[6:16])
    assert o["X"] == X
    for row in o["per_edge"]:
        assert list(row[:5]) == [0, 2, n - 4, 0, 0]


def test_small_cycles():
    # C_4 is itself an induced 4-cycle, C_5 has five induced 4-paths.
    assert X_of(*graphs.cycle(4)) == expect(X1=4, X2=2, X4=4, X10=1)
    assert X_of(*graphs.cycle(5)) == expect(X1=5, X2=5, X4=5, X5=5, X12=5)


@pytest.mark.parametrize("a,b", [(1, 1), (1, 4), (2, 2), (2, 3), (3, 3), (3, 5), (4, 4), (5, 5), (2, 7)])
def test_complete_bipartite(a, b):
    rp, ci = graphs.complete_bipartite(a, b)
    o = oracle.count(rp, ci, threads=2)
    assert o["X"] == expect(X1=a * b, X2=comb(a, 2) + comb(b, 2),
                            X4=a * comb(b, 2) + b * comb(a, 2), X6=comb(a, 3) + comb(b, 3),
                            X10=comb(a, 2) * comb(b, 2), X11=a * comb(b, 3) + b * comb(a, 3),
                            X17=comb(a, 4) + comb(b, 4))
    for row in o["per_edge"]:
        assert row[4] == (a - 1) * (b - 1)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 7, 50])
def test_empty_graph(n):
    assert X_of(*graphs.empty(n)) == expect(X2=comb(n, 2), X6=comb(n, 3), X17=comb(n, 4))


def test_empty_graph_128bit():
    # C(2^20, 4) ~ 4.8e22 exceeds 64 bits: the sums and X_17 are 128-bit.
    n = 1 << 20
    X = X_of(np.zeros(n + 1, np.int32), np.zeros(0, np.int32))
    assert X[16] == comb(n, 4) and X[16] >= 2**64
    assert X == expect(X2=comb(n, 2), X6=comb(n, 3), X17=comb(n, 4))


@pytest.mark.parametrize("n", [2, 3, 4, 9])
def test_single_edge_with_isolated_vertices(n):
    rp, ci = graphs.csr(n, [(0, 1)])
    assert X_of(rp, ci) == expect(X1=1, X2=comb(n, 2) - 1, X5=n - 2, X6=comb(n, 3) - (n - 2),
                                   X16=comb(n - 2, 2), X17=comb(n, 4) - comb(n - 2, 2))


def test_hand_derived_cube_and_petersen():
    # 3-cube: bipartite cubic, 12 edges, its 4-cycles are its 6 faces.
    X = X_of(*graphs.cube())
    assert X[0] == 12 and X[2] == 0 and X[3] == 24 and X[9] == 6 and X[10] == 8
    assert X[6] == X[7] == X[8] == 0 and X[11] == 48 - 24
    # Petersen: cubic, girth 5 (no triangles, no 4-cycles), 15 edges.
    X = X_of(*graphs.petersen())
    assert X[:6] == [15, 30, 0, 30, 60, 30]
    assert X[6:11] == [0, 0, 0, 0, 10] and X[11] == 60 and X[12] == 0
    assert X[13] == 75 - 60 and X[14] == 30 * 2


# ---------------- independent per-edge definitions and identities ----------------

def dense(rp, ci):
    n = len(rp) - 1
    A = np.zeros((n, n), np.int64)
    for u in range(n):
        A[u, ci[rp[u]:rp[u + 1]]] = 1
    return A


def per_edge_linear_algebra(rp, ci):
    """x3, x7, x10 per edge as quadratic forms of indicator vectors."""
    A = dense(rp, ci)
    n = A.shape[0]
    rows = []
    for u, v in graphs.edges_of(rp, ci):
        t = A[u] * A[v]
        su = A[u] * (1 - A[v])
        su[v] = 0
        sv = A[v] * (1 - A[u])
        sv[u] = 0
        rows.append((int(t.sum()), int(t @ A @ t) // 2, int(su @ A @ sv)))
    return np.array(rows, np.int64).reshape(-1, 3)


@pytest.mark.parametrize("maker", [
    lambda: graphgen.er(120, 0.12, 3),
    lambda: graphgen.er(80, 0.45, 4),
    lambda: graphgen.chung_lu(200, 900, 2.1, 1800.0, 60.0, 5),
    lambda: graphgen.rmat(7, 8, 0.57, 0.19, 0.19, 6),
])
def test_per_edge_against_linear_algebra(maker):
    rp, ci = maker()
    o = oracle.count(rp, ci, threads=2)
    la = per_edge_linear_algebra(rp, ci)
    pe = o["per_edge"].astype(np.int64)
    np.testing.assert_array_equal(pe[:, 0], la[:, 0])  # x3
    np.testing.assert_array_equal(pe[:, 3], la[:, 1])  # x7
    np.testing.assert_array_equal(pe[:, 4], la[:, 2])  # x10


@pytest.mark.parametrize("maker", [
    lambda: graphgen.er(400, 0.05, 7),
    lambda: graphgen.er(150, 0.3, 8),
    lambda: graphgen.chung_lu(1500, 8000, 2.1, 16000.0, 400.0, 9),
    lambda: graphgen.rmat(10, 16, 0.57, 0.19, 0.19, 10),
])
def test_subgraph_to_induced_identities(maker):
    rp, ci = maker()
    n = len(rp) - 1
    m = int(rp[-1]) // 2
    X = [0] + X_of(rp, ci)
    A = dense(rp, ci)
    d = A.sum(1)
    A2 = A @ A
    E = np.array(graphs.edges_of(rp, ci), np.int64).reshape(-1, 2)
    tri = int(A2[E[:, 0], E[:, 1]].sum()) // 3
    assert X[3] == tri
    assert X[4] == sum(comb(int(x), 2) for x in d) - 3 * X[3]
    assert X[11] == sum(comb(int(x), 3) for x in d) - X[9] - 2 * X[8] - 4 * X[7]
    iu = np.triu_indices(n, 1)
    c4 = int((A2[iu] * (A2[iu] - 1) // 2).sum()) // 2
    assert X[10] == c4 - X[8] - 3 * X[7]
    p4 = int(((d[E[:, 0]] - 1) * (d[E[:, 1]] - 1)).sum()) - 3 * X[3]
    assert X[12] == p4 - 2 * X[9] - 4 * X[10] - 6 * X[8] - 12 * X[7]
    # totals per size
    assert X[1] + X[2] == comb(n, 2)
    assert sum(X[3:7]) == comb(n, 3)
    assert sum(X[7:18]) == comb(n, 4)
    assert X[1] == m


def test_per_edge_sums_are_multiples():
    rp, ci = graphgen.rmat(11, 16, 0.57, 0.19, 0.19, 11)
    o = oracle.count(rp, ci, threads=4)
    pe = o["per_edge"]
    X = o["X"]
    assert int(pe[:, 0].sum()) == 3 * X[2]
    assert int(pe[:, 3].sum()) == 6 * X[6]
    assert int(pe[:, 4].sum()) == 4 * X[9]


def test_derive_rejects_inexact_division():
    rp, ci = graphs.complete(5)
    o = oracle.count(rp, ci, threads=1)
    rc, X = oracle.derive(5, 10, o["csum"])
    assert rc == 0 and X == o["X"]
    bad = list(o["csum"])
    bad[0] += 1          # C_3 no longer a multiple of 3
    rc, _ = oracle.derive(5, 10, bad)
    assert rc != 0


def test_sample_matches_whole_graph():
    rp, ci = graphgen.chung_lu(3000, 20000, 2.1, 40000.0, 500.0, 12)
    full = oracle.count(rp, ci, threads=4)["per_edge"]
    ids = np.array([0, 5, 17, 1000, 19999, 12345], np.int64)
    np.testing.assert_array_equal(oracle.count_sample(rp, ci, ids, threads=3), full[ids])


def test_edge_order_is_upper_triangle_row_major():
    rp, ci = graphs.wheel(6)
    uv = oracle.edges(rp, ci)
    assert [tuple(x) for x in uv] == graphs.edges_of(rp, ci)
