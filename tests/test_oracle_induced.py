"""Pins of the oracle's per-edge induced 4-node counts (H_7..H_16 of Table 1
per edge; the paper defines per edge only x3..x5 and the summands of
C_7..C_16, Sec. 4.5, so these counts are read straight from the definition of
an induced subgraph). Pinned by brute-force enumeration of every 4-set
containing each edge, by hand-derived closed forms, and by invariants that
tie them to the pinned global counts and per-edge columns."""
from math import comb

import numpy as np
import pytest

import graphgen
import oracle
from oracle import brute
from tests import graphs

EDGES_OF = [6, 5, 4, 4, 3, 3, 3, 2, 2, 1]  # edges of H7 .. H16


def induced(rp, ci):
    return oracle.count_induced(rp, ci, threads=2).astype(np.int64)


@pytest.mark.parametrize("seed", range(8))
def test_induced_equals_brute_force(seed):
    rng = np.random.default_rng(seed)
    for _ in range(20):
        n = int(rng.integers(4, 15))
        p = float(rng.uniform(0.15, 0.9))
        rp, ci = graphgen.er(n, p, int(rng.integers(1, 1 << 30)))
        np.testing.assert_array_equal(induced(rp, ci), brute.per_edge_induced(rp, ci))


def test_induced_brute_force_power_law_and_named():
    for rp, ci in (graphgen.chung_lu(14, 30, 2.1, 60.0, 13.0, 3), graphgen.rmat(4, 4, 0.57, 0.19, 0.19, 2),
                   graphs.petersen(), graphs.cube(), graphs.wheel(7),
                   graphs.csr(12, [(0, 1), (1, 2), (5, 6)])):
        np.testing.assert_array_equal(induced(rp, ci), brute.per_edge_induced(rp, ci))


def test_induced_sample_matches_whole_graph():
    rp, ci = graphgen.chung_lu(3000, 20000, 2.1, 40000.0, 500.0, 12)
    full = induced(rp, ci)
    ids = np.array([0, 5, 17, 1000, 19999, 12345], np.int64)
    np.testing.assert_array_equal(oracle.count_induced(rp, ci, ids, threads=3).astype(np.int64), full[ids])


@pytest.mark.parametrize("maker", [
    lambda: graphgen.er(300, 0.05, 7),
    lambda: graphgen.er(120, 0.4, 8),
    lambda: graphgen.chung_lu(1500, 8000, 2.1, 16000.0, 400.0, 9),
    lambda: graphgen.rmat(10, 16, 0.57, 0.19, 0.19, 10),
])
def test_induced_sums_and_rows(maker):
    rp, ci = maker()
    n = len(rp) - 1
    h = induced(rp, ci)
    o = oracle.count(rp, ci, threads=2)
    X = o["X"]
    # every induced copy of H_i is met once from each of its edges
    for i in range(10):
        assert int(h[:, i].sum()) == EDGES_OF[i] * X[6 + i], i
    # every pair of the other n - 2 vertices is classified exactly once
    assert (h.sum(1) == comb(n - 2, 2)).all()
    # 4-cliques and induced 4-cycles on e are per-edge columns x7 and x10
    np.testing.assert_array_equal(h[:, 0], o["per_edge"][:, 3].astype(np.int64))
    np.testing.assert_array_equal(h[:, 3], o["per_edge"][:, 4].astype(np.int64))


def row(**nz):
    r = np.zeros(10, np.int64)
    for k, v in nz.items():
        r[int(k[1:]) - 7] = v
    return r


@pytest.mark.parametrize("n", [4, 5, 9])
def test_induced_complete_graph(n):
    # K_n: every 4-set is a 4-clique
    assert (induced(*graphs.complete(n)) == row(H7=comb(n - 2, 2))).all()


@pytest.mark.parametrize("k", [2, 3, 7])
def test_induced_star(k):
    # K_{1,k}: the other vertices are leaves; two leaves with the edge form a 3-star
    assert (induced(*graphs.star(k)) == row(H11=comb(k - 1, 2))).all()


@pytest.mark.parametrize("n", [6, 7, 12])
def test_induced_cycle(n):
    # C_n, edge (i, i+1): the 4-paths {i-2..i+1}, {i-1..i+2}, {i..i+3}; a
    # neighbour i-1 or i+2 with a vertex adjacent to none of the three (2-star
    # + vertex); another edge at distance >= 2 (two edges); any other pair
    # (edge + two vertices)
    assert (induced(*graphs.cycle(n)) == row(H12=3, H15=2 * (n - 5), H14=n - 5,
                                            H16=comb(n - 4, 2) - (n - 5))).all()


@pytest.mark.parametrize("a,b", [(2, 3), (3, 5), (4, 4)])
def test_induced_complete_bipartite(a, b):
    # K_{a,b}, edge (x, y): two other vertices on x's side form a 3-star at y,
    # two on y's side a 3-star at x, one on each side a 4-cycle
    assert (induced(*graphs.complete_bipartite(a, b)) == row(H10=(a - 1) * (b - 1),
                                                             H11=comb(a - 1, 2) + comb(b - 1, 2))).all()


@pytest.mark.parametrize("n", [2, 3, 8])
def test_induced_single_edge(n):
    assert (induced(*graphs.csr(n, [(0, 1)])) == row(H16=comb(n - 2, 2))).all()


def test_induced_empty_and_edgeless():
    assert induced(*graphs.empty(5)).shape == (0, 10)
