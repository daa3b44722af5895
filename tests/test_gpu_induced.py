"""Per-edge induced 4-node counts (gc_count_edge_induced) against the oracle,
bit-exact.

The GPU derives each edge's counts of H_7..H_16 from the quantities the
passes already have (|T|, x7, the cross term, the 4-cycles through the edge)
plus the degree sum of T, the triangles and the neighbour-degree sums of the
two endpoints; the oracle classifies every neighbour of T, S_u and S_v
directly (oracle.count_induced, pinned by brute force). Integer counts: zero
tolerance. Large graphs: sampled edges, computed one by one by the oracle,
plus the invariants sum_e H_i(e) = |E(H_i)| X_i and row sums C(n-2, 2).
"""
from math import comb

import numpy as np
import pytest

import graphgen
import oracle
import paper_1608_05138_gb300 as gcb
from tests import graphs

pytestmark = pytest.mark.gpu

EDGES_OF = [6, 5, 4, 4, 3, 3, 3, 2, 2, 1]  # edges of H7 .. H16


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1608_05138_gb300 import build
    build.build()


def gpu_induced(rp, ci):
    with gcb.Graph(rp, ci) as g:
        ind = np.zeros((g.m, 10), np.uint64)
        pe = np.zeros((g.m, 13), np.uint64)
        X = g.count_induced(ind, pe)
        return X, ind, pe


def assert_induced_parity(rp, ci):
    X, ind, pe = gpu_induced(rp, ci)
    np.testing.assert_array_equal(ind, oracle.count_induced(rp, ci))
    o = oracle.count(rp, ci)
    np.testing.assert_array_equal(pe, o["per_edge"])
    assert X == o["X"]
    return X, ind


def test_er2000_induced():
    assert_induced_parity(*graphgen.config_er2000())


def test_dense_er_induced():
    # every pass-T tier of the dense 1K/150K graph (warp tier to k <= 512)
    X, ind = assert_induced_parity(*graphgen.config_er_dense())
    for i in range(10):
        assert int(ind[:, i].sum()) == EDGES_OF[i] * X[6 + i]


@pytest.mark.parametrize("seed", range(1, 5))
def test_random_graphs_induced(seed):
    for n, p in ((7, 0.5), (40, 0.3), (150, 0.08), (300, 0.02), (64, 0.9)):
        assert_induced_parity(*graphgen.er(n, p, seed * 100 + n))


@pytest.mark.parametrize("seed", range(1, 3))
def test_power_law_induced(seed):
    assert_induced_parity(*graphgen.chung_lu(3000, 15000, 2.1, 30000.0, 800.0, seed))
    assert_induced_parity(*graphgen.rmat(11, 16, 0.57, 0.19, 0.19, seed))


def test_closed_form_families_induced():
    for rp, ci in (graphs.complete(30), graphs.cycle(17), graphs.complete_bipartite(7, 9),
                   graphs.star(3000), graphs.petersen(), graphs.cube(), graphs.wheel(12),
                   graphs.csr(2, [(0, 1)]), graphs.csr(9, [(3, 7)])):
        assert_induced_parity(rp, ci)
    X, ind, _ = gpu_induced(*graphs.empty(5))
    assert ind.shape == (0, 10)


def test_global_tier_and_hubs_induced():
    # out-degrees above 1024 (pass T's global-memory tier) and hub units
    rp, ci = graphs.complete(1100)
    X, ind, _ = gpu_induced(rp, ci)
    assert (ind[:, 0] == comb(1098, 2)).all() and (ind[:, 1:] == 0).all()
    assert_induced_parity(*graphgen.chung_lu(60000, 400000, 2.1, 8e5, 3000.0, 11))


def test_device_output_and_repeat_induced():
    import torch
    rp, ci = graphgen.rmat(12, 16, 0.57, 0.19, 0.19, 23)
    expect = oracle.count_induced(rp, ci)
    with gcb.Graph(rp, ci) as g:
        X0 = g.count()  # a plain count first: the induced scratch is added on demand
        dev = torch.zeros((g.m, 10), dtype=torch.int64, device="cuda")
        X1 = g.count_induced(dev)
        pinned = torch.zeros((g.m, 10), dtype=torch.int64, pin_memory=True)
        X2 = g.count_induced(pinned.numpy().view(np.uint64))
        host = np.zeros((g.m, 10), np.uint64)
        X3 = g.count_induced(host)
        assert X0 == X1 == X2 == X3
        assert g.phase_ms()["induced_columns"] >= 0
    np.testing.assert_array_equal(dev.cpu().numpy().view(np.uint64), expect)
    np.testing.assert_array_equal(pinned.numpy().view(np.uint64), expect)
    np.testing.assert_array_equal(host, expect)


def _sampled_induced(rp, ci, k, seed):
    import torch
    n = len(rp) - 1
    with gcb.Graph(rp, ci) as g:
        dev = torch.zeros((g.m, 10), dtype=torch.int64, device="cuda")
        X = g.count_induced(dev)
        m = g.m
        ids = np.unique(np.concatenate([np.random.default_rng(seed).integers(0, m, k), [0, m - 1]])).astype(np.int64)
        rows = dev[torch.from_numpy(ids).cuda()].cpu().numpy().view(np.uint64)
        np.testing.assert_array_equal(rows, oracle.count_induced(rp, ci, ids))
        for i in range(10):  # exact column sums: the high and low 32-bit halves summed apart
            col = dev[:, i]
            s = (int((col >> 32).sum().item()) << 32) + int((col & 0xFFFFFFFF).sum().item())
            assert s == EDGES_OF[i] * X[6 + i], i
        assert bool((dev.sum(1) == comb(n - 2, 2)).all().item())


def test_chung_lu_1m_induced_sampled():
    _sampled_induced(*graphgen.config_chung_lu(), k=1000, seed=5)


def test_rmat22_induced_sampled():
    _sampled_induced(*graphgen.config_rmat(22), k=300, seed=6)
