"""GPU path (libgc.so through the C ABI) against the CPU oracle, bit-exact.

Counts are integers, so the tolerance is zero: every per-edge column and
every global count must be equal. Small and medium graphs are compared in
full; the full-size power-law graphs are compared on sampled edges computed
one by one by the oracle, plus the exact relation between the GPU's own
per-edge rows and its global counts.
"""
import numpy as np
import pytest

import graphgen
import oracle
import paper_1608_05138_gb300 as gcb
from tests import graphs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1608_05138_gb300 import build
    build.build()


def gpu_count(rp, ci, per_edge=True):
    with gcb.Graph(rp, ci) as g:
        pe = np.zeros((g.m, 13), np.uint64) if per_edge else None
        X = g.count(pe)
        return X, pe, g.csums(), g.edges()


def assert_parity(rp, ci):
    X, pe, cs, uv = gpu_count(rp, ci)
    o = oracle.count(rp, ci)
    np.testing.assert_array_equal(uv, oracle.edges(rp, ci))
    np.testing.assert_array_equal(pe, o["per_edge"])
    assert cs == o["csum"]
    assert X == o["X"]
    return X, pe


def test_er2000_config_bit_exact():
    rp, ci = graphgen.config_er2000()
    X, pe = assert_parity(rp, ci)
    assert X[0] == len(ci) // 2


def test_dense_er_1k_150k_bit_exact():
    # the 1K-vertex / 150K-edge dense shape of the paper's GPU comparison
    rp, ci = graphgen.config_er_dense()
    X, _ = assert_parity(rp, ci)
    assert 140000 < X[0] < 160000


@pytest.mark.parametrize("seed", range(1, 13))
def test_random_graphs(seed):
    for n, p in ((7, 0.5), (40, 0.3), (150, 0.08), (300, 0.02), (64, 0.9)):
        assert_parity(*graphgen.er(n, p, seed * 100 + n))


@pytest.mark.parametrize("seed", range(1, 5))
def test_power_law_graphs(seed):
    assert_parity(*graphgen.chung_lu(3000, 15000, 2.1, 30000.0, 800.0, seed))
    assert_parity(*graphgen.rmat(11, 16, 0.57, 0.19, 0.19, seed))


def test_closed_form_families():
    for rp, ci in (graphs.complete(30), graphs.cycle(17), graphs.complete_bipartite(7, 9),
                   graphs.star(3000), graphs.petersen(), graphs.cube(), graphs.wheel(12)):
        assert_parity(rp, ci)


def test_degenerate_graphs():
    for n in (0, 1, 2, 5):
        X, pe, _, _ = gpu_count(*graphs.empty(n))
        assert X == oracle.count(*graphs.empty(n))["X"] and pe.shape == (0, 13)
    assert_parity(*graphs.csr(2, [(0, 1)]))
    assert_parity(*graphs.csr(9, [(3, 7)]))          # single edge, 7 isolated vertices
    assert_parity(*graphs.csr(40, [(0, 1), (1, 2), (0, 2), (30, 31)]))


def test_asymmetric_input_rejected():
    # symmetry is checked on the device from the reverse slots of the
    # preparation; nothing is counted for an asymmetric input
    def status(rp, ci):
        with pytest.raises(gcb.GcError) as ei:
            gcb.Graph(np.asarray(rp, np.int32), np.asarray(ci, np.int32))
        return ei.value.status, str(ei.value)
    st, msg = status([0, 2, 4, 5, 6], [1, 2, 0, 2, 3, 0])  # (0,2), (1,2), (2,3), (3,0) have no reverse
    assert st == -5 and "no reverse" in msg
    rp, ci = graphgen.chung_lu(5000, 40000, 2.1, 80000.0, 900.0, 9)
    E = graphs.edges_of(rp, ci)
    arcs = [(a, b) for a, b in E] + [(b, a) for a, b in E]
    a, b = E[len(E) // 2]
    arcs.remove((b, a))            # one direction dropped ...
    nbr_a = set(int(x) for x in ci[rp[a]:rp[a + 1]])
    c = next(x for x in range(len(rp) - 1) if x not in (a, b) and x not in nbr_a)
    arcs.append((min(a, c), max(a, c)))  # ... and one arc added, so the entry count stays even
    n = len(rp) - 1
    order = sorted(arcs)
    rp2 = np.zeros(n + 1, np.int64)
    for x, _ in order:
        rp2[x + 1] += 1
    rp2 = np.cumsum(rp2).astype(np.int32)
    ci2 = np.array([y for _, y in order], np.int32)
    st, msg = status(rp2, ci2)
    assert st == -5
    # the graph handle of a valid graph still works after rejected uploads
    assert_parity(rp, ci)


def test_wide_counts_need_high_words():
    n = 200000  # C(n, 4) > 2^64
    rp, ci = graphs.csr(n, [(0, 1), (1, 2)])
    with gcb.Graph(rp, ci) as g:
        X = g.count()
        assert X == oracle.count(rp, ci, per_edge=False)["X"] and X[16] >= 2**64
        with pytest.raises(gcb.GcError) as ei:
            g.count(wide=False)
        assert ei.value.status == -9


def test_large_common_neighbourhood():
    # book graph: two adjacent hubs sharing 1500 neighbours (|T| = 1500), with
    # a matching and a few triangles among the shared neighbours.
    k = 1500
    edges = [(0, 1)] + [(0, 2 + i) for i in range(k)] + [(1, 2 + i) for i in range(k)]
    edges += [(2 + i, 3 + i) for i in range(0, k - 1, 2)]
    edges += [(2 + i, 4 + i) for i in range(0, 60, 3)]
    edges += [(2 + k + j, 2 + j) for j in range(50)]
    assert_parity(*graphs.csr(2 + k + 50, edges))


def test_global_psi_tables():
    # more vertices than the shared-memory table holds
    assert_parity(*graphgen.chung_lu(60000, 300000, 2.1, 600000.0, 3000.0, 21))


def test_hub_units_of_the_cycle_pass():
    # n > 2 x 45056 and ~100 hub vertices whose wedges are counted in
    # shared-memory blocks of the vertex range (several blocks each)
    assert_parity(*graphgen.chung_lu(120000, 600000, 2.1, 1.2e6, 4000.0, 7))


def wedges_by_highest_vertex(rp, ci):
    """Wedges h-x-o with x and o both below h in the (degree, id) order,
    summed per h (numpy; independent of the library)."""
    n = len(rp) - 1
    deg = np.diff(rp).astype(np.int64)
    key = deg * (n + 1) + np.arange(n)  # (degree, id) order
    rows = np.repeat(np.arange(n), deg)
    cols = ci.astype(np.int64)
    below = key[cols] < key[rows]  # slot (r, c) with c below r
    nb = np.bincount(rows[below], minlength=n)  # neighbours below each vertex
    # for h and x below h: the o in Gamma(x) below h (o != h automatically)
    W = np.zeros(n, np.int64)
    for r, c in zip(rows[below], cols[below]):
        nbr = ci[rp[c]:rp[c + 1]].astype(np.int64)
        W[r] += int(np.count_nonzero(key[nbr] < key[r]))
    return W, nb


def test_hashed_units_of_the_cycle_pass():
    # A unit h with 160 lower neighbours x of 50 lower neighbours o each
    # (8000 wedges, hash at its full 16384 slots), the o drawn from a pool
    # of 2000 so that cnt_h(o) > 1 often; a 2400-cycle so that n exceeds the
    # shared-memory table size and the graph is ranked.
    rng = np.random.default_rng(3)
    h = 0
    xs = np.arange(1, 161)
    pool = np.arange(161, 2161)
    E = [(h, int(x)) for x in xs]
    for x in xs:
        for o in rng.choice(pool, 50, replace=False):
            E.append((int(x), int(o)))
    filler = np.arange(2161, 4561)
    E += [(int(a), int(b)) for a, b in zip(filler, np.roll(filler, 1))]
    rp, ci = graphs.csr(4561, E)
    W, _ = wedges_by_highest_vertex(rp, ci)
    assert W.max() == 8000 and W.sum() > 8000
    with gcb.Graph(rp, ci) as g:
        pe = np.zeros((g.m, 13), np.uint64)
        X = g.count(pe)
        w = g.work_counts()
    o = oracle.count(rp, ci)
    np.testing.assert_array_equal(pe, o["per_edge"])
    assert X == o["X"]
    assert w["c_wedges"] == W.sum() and w["c_heavy_wedges"] == 0 and w["c_hash_wedges"] == W.sum()


def test_cycle_pass_unit_kinds_on_a_power_law_graph():
    # hubs (shared-memory blocks), hashed units (at most 8192 wedges), the
    # packed-key hash and vertex-indexed tables take part; the wedge counters
    # add up to the wedges counted on the host
    rp, ci = graphgen.chung_lu(60000, 400000, 2.1, 8e5, 3000.0, 11)
    with gcb.Graph(rp, ci) as g:
        g.count(None)
        w = g.work_counts()
    W, nb = wedges_by_highest_vertex(rp, ci)
    assert w["c_wedges"] == W.sum()
    assert 0 < w["c_heavy_wedges"] and w["c_hash_wedges"] == W[W <= 8192].sum()
    assert 0 < w["c_hash2_wedges"] <= W[(W > 8192) & (W <= 41287)].sum()
    assert w["c_heavy_wedges"] + w["c_hash_wedges"] + w["c_hash2_wedges"] <= w["c_wedges"]
    assert_parity(rp, ci)


def _count_with_work(rp, ci):
    with gcb.Graph(rp, ci) as g:
        pe = np.zeros((g.m, 13), np.uint64)
        X = g.count(pe)
        w = g.work_counts()
    o = oracle.count(rp, ci)
    np.testing.assert_array_equal(pe, o["per_edge"])
    assert X == o["X"]
    return w


def test_hub_counts_near_the_10_bit_field_limit():
    # h joined to 900 vertices x and 50 pendant vertices; every x joined to the
    # same 60 vertices o: 54000 wedges on 60 distinct o, each of count 900
    # (a hub of fewer than 1023 lower neighbours keeps 10-bit counters); the o
    # (degree 900) rank below h (degree 950) and are hubs of that kind too
    n = 100_000
    h, xs, os_, pend = 0, np.arange(1, 901), np.arange(901, 961), np.arange(961, 1011)
    E = [(h, int(x)) for x in xs] + [(h, int(p)) for p in pend]
    E += [(int(x), int(o)) for x in xs for o in os_]
    rp, ci = graphs.csr_large(n, E)
    W, nb = wedges_by_highest_vertex(rp, ci)
    assert W[h] == 54000 and nb[h] == 950
    w = _count_with_work(rp, ci)
    assert w["c_heavy_wedges"] >= 54000 and w["c_wedges"] == W.sum()


def test_hub_over_a_skewed_o_range():
    # 3M vertices, almost all isolated (the lowest ranks): h has 620 lower
    # neighbours, 600 of them with 150 o each, drawn with weights 1/(i + 100)
    # from a pool of 50000, so the o crowd the top of [0, h): 19 blocks of
    # the o-range, the wedges in the last one
    rng = np.random.default_rng(17)
    n = 3_000_000
    h, xs = 0, np.arange(1, 601)
    pool = np.arange(1000, 51000)
    wt = 1.0 / (np.arange(len(pool)) + 100.0)
    wt /= wt.sum()
    E = [(h, int(x)) for x in xs] + [(h, int(p)) for p in range(601, 621)]
    for x in xs:
        for o in rng.choice(pool, 150, replace=False, p=wt):
            E.append((int(x), int(o)))
    rp, ci = graphs.csr_large(n, E)
    W, nb = wedges_by_highest_vertex(rp, ci)
    assert W[h] == 90000 and nb[h] == 620
    w = _count_with_work(rp, ci)
    assert w["c_heavy_wedges"] >= 90000 and w["c_wedges"] == W.sum()


def test_hubs_of_few_lower_neighbours_rmat14():
    # R-MAT scale 14: 91 hubs of more than 41287 wedges and fewer than 1023
    # lower neighbours (10-bit counters), half of all wedges
    rp, ci = graphgen.rmat(14, 16, 0.57, 0.19, 0.19, 1)
    W, nb = wedges_by_highest_vertex(rp, ci)
    few = (W > 41287) & (nb < 1023)
    w = _count_with_work(rp, ci)
    assert few.sum() == 91 and w["c_heavy_wedges"] >= W[few].sum()


def _unit_of_18000_wedges(n):
    # A unit of 18000 wedges (above the first hash) whose rank spans 19 or
    # more blocks of the hub kernel's o-range (not a hub); the n vertices are
    # mostly isolated.
    rng = np.random.default_rng(4)
    h = 0
    xs = np.arange(1, 201)
    pool = np.arange(201, 8201)
    E = [(h, int(x)) for x in xs]
    for x in xs:
        for o in rng.choice(pool, 90, replace=False):
            E.append((int(x), int(o)))
    rp, ci = graphs.csr_large(n, E)
    sub_rp, sub_ci = graphs.csr(8201, E)
    W, _ = wedges_by_highest_vertex(sub_rp, sub_ci)
    assert W.max() == 18000
    return rp, ci, W


def test_packed_hash_units_of_the_cycle_pass():
    # 2M vertices (ids fit 22 bits), 200 lower neighbours: the packed-key
    # shared-memory hash counts the unit
    rp, ci, W = _unit_of_18000_wedges(2_000_000)
    with gcb.Graph(rp, ci) as g:
        pe = np.zeros((g.m, 13), np.uint64)
        X = g.count(pe)
        w = g.work_counts()
    o = oracle.count(rp, ci)
    np.testing.assert_array_equal(pe, o["per_edge"])
    assert X == o["X"]
    assert w["c_wedges"] == W.sum() and w["c_heavy_wedges"] == 0
    assert w["c_hash2_wedges"] == 18000 and w["c_hash_wedges"] == W.sum() - 18000


def test_table_units_of_the_cycle_pass():
    # the same unit among 4.4M vertices: ids above 2^22 do not fit the packed
    # hash, so it is counted on the vertex-indexed tables
    rp, ci, W = _unit_of_18000_wedges(4_400_000)
    with gcb.Graph(rp, ci) as g:
        pe = np.zeros((g.m, 13), np.uint64)
        X = g.count(pe)
        w = g.work_counts()
    o = oracle.count(rp, ci)
    np.testing.assert_array_equal(pe, o["per_edge"])
    assert X == o["X"]
    assert w["c_wedges"] == W.sum() and w["c_heavy_wedges"] == 0 and w["c_hash2_wedges"] == 0
    assert w["c_hash_wedges"] == W.sum() - 18000


def test_clique_pass_rescan_when_edge_list_is_full():
    # pass K keeps the edges of each H_a in a per-CTA list; a unit whose list
    # overflows scans its out-lists again. Force that with a 64-entry list.
    import subprocess
    import sys
    code = ("import numpy as np, graphgen, oracle, paper_1608_05138_gb300 as gcb\n"
            "rp, ci = graphgen.rmat(12, 16, 0.57, 0.19, 0.19, 29)\n"
            "g = gcb.Graph(rp, ci); pe = np.zeros((g.m, 13), np.uint64); X = g.count(pe); g.close()\n"
            "o = oracle.count(rp, ci)\n"
            "assert X == o['X'] and (pe == o['per_edge']).all()\n"
            "print('ok')\n")
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, GC_K_LIST_CAP="64", PYTHONPATH=root)
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr


def _run_with_env(code, env_extra):
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, PYTHONPATH=root, **env_extra)
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=root, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr


_TWICE = ("import numpy as np, graphgen, oracle, paper_1608_05138_gb300 as gcb\n"
          "for rp, ci in (graphgen.rmat(13, 16, 0.57, 0.19, 0.19, 31), graphgen.config_er_dense(),\n"
          "               graphgen.chung_lu(20000, 150000, 2.1, 3e5, 2000.0, 8)):\n"
          "    o = oracle.count(rp, ci)\n"
          "    with gcb.Graph(rp, ci) as g:\n"
          "        for _ in range(2):\n"
          "            pe = np.zeros((g.m, 13), np.uint64); X = g.count(pe)\n"
          "            assert X == o['X'] and (pe == o['per_edge']).all()\n"
          "print('ok')\n")


def test_triangle_lists_that_do_not_fit():
    # a list of 5000 entries: almost every unit of pass T finds it full and
    # pass K scans its out-lists again
    _run_with_env(_TWICE, {"GC_T_LIST_CAP": "5000"})


def test_relabelling_is_metamorphic():
    rp, ci = graphgen.chung_lu(2000, 12000, 2.1, 24000.0, 500.0, 22)
    n = len(rp) - 1
    perm = np.random.default_rng(5).permutation(n)
    E = graphs.edges_of(rp, ci)
    rp2, ci2 = graphs.csr(n, [(int(perm[a]), int(perm[b])) for a, b in E])
    X1, pe1, _, uv1 = gpu_count(rp, ci)
    X2, pe2, _, uv2 = gpu_count(rp2, ci2)
    assert X1 == X2
    pos = {(int(a), int(b)): i for i, (a, b) in enumerate(uv2)}
    for i, (a, b) in enumerate(uv1):
        pa, pb = int(perm[a]), int(perm[b])
        j = pos[(min(pa, pb), max(pa, pb))]
        np.testing.assert_array_equal(pe1[i], pe2[j])


def test_repeated_count_reuses_the_triangle_lists():
    # from the second count on a handle, pass T keeps the edges of every H_a
    # and pass K rebuilds its bitmatrices from them instead of scanning; both
    # counts must equal the oracle, in every tier (k <= 32 warp tier, 256, 512,
    # 1024 and the global tier above 1024)
    for rp, ci in (graphgen.chung_lu(3000, 15000, 2.1, 30000.0, 800.0, 5), graphgen.rmat(12, 16, 0.57, 0.19, 0.19, 6),
                   graphgen.config_er_dense()):
        o = oracle.count(rp, ci)
        with gcb.Graph(rp, ci) as g:
            for _ in range(3):
                pe = np.zeros((g.m, 13), np.uint64)
                assert g.count(pe) == o["X"]
                np.testing.assert_array_equal(pe, o["per_edge"])
            assert g.work_counts()["t_triangles"] == g.work_counts()["k_local_edges"]
    rp, ci = graphgen.er(1200, 0.92, 41)  # out-degrees up to ~1100
    with gcb.Graph(rp, ci) as g:
        pe1 = np.zeros((g.m, 13), np.uint64)
        X1 = g.count(pe1)
        pe2 = np.zeros((g.m, 13), np.uint64)
        X2 = g.count(pe2)
    assert X1 == X2
    np.testing.assert_array_equal(pe1, pe2)


def test_device_output_and_repeat():
    import torch
    rp, ci = graphgen.rmat(12, 16, 0.57, 0.19, 0.19, 23)
    with gcb.Graph(rp, ci) as g:
        host = np.zeros((g.m, 13), np.uint64)
        X1 = g.count(host)
        dev = torch.zeros((g.m, 13), dtype=torch.int64, device="cuda")
        X2 = g.count(dev)
        X3 = g.count()
        # pinned host memory: the rows are written by the device directly
        pinned = torch.zeros((g.m, 13), dtype=torch.int64, pin_memory=True)
        X4 = g.count(pinned.numpy().view(np.uint64))
        assert X1 == X2 == X3 == X4
        np.testing.assert_array_equal(dev.cpu().numpy().view(np.uint64), host)
        np.testing.assert_array_equal(pinned.numpy().view(np.uint64), host)
        ms = g.phase_ms()
        assert set(ms) == set(gcb.gc_phase_names()) and all(v >= 0 for v in ms.values())
    np.testing.assert_array_equal(host, oracle.count(rp, ci)["per_edge"])


def _sampled_check(rp, ci, k=1500, seed=0):
    """Full-size graph: sampled rows against the oracle one by one, and the
    GPU's global counts against the derivation from its own per-edge rows."""
    import torch
    with gcb.Graph(rp, ci) as g:
        dev = torch.zeros((g.m, 13), dtype=torch.int64, device="cuda")
        X = g.count(dev)
        cs = g.csums()
        m = g.m
        rng = np.random.default_rng(seed)
        deg = np.diff(rp)
        uv = g.edges()
        heavy = np.argsort(-(deg[uv[:, 0]].astype(np.int64) * deg[uv[:, 1]]))[:20]
        ids = np.unique(np.concatenate([rng.integers(0, m, k), heavy, [0, m - 1]])).astype(np.int64)
        rows = dev[torch.from_numpy(ids).cuda()].cpu().numpy().view(np.uint64)
        np.testing.assert_array_equal(rows, oracle.count_sample(rp, ci, ids))
        # column sums of the GPU's per-edge rows (exact, in Python ints) equal
        # its unrestricted counts, and the derivation reproduces its globals
        colsum = [int(dev[:, c].sum(dtype=torch.int64).item()) for c in range(13)]
        order = [0, 1, 2, 3, 5, 6, 4, 7, 8, 9, 10, 11, 12]
        for kk, c in enumerate(order):
            assert colsum[c] % (1 << 64) == cs[kk] % (1 << 64) or colsum[c] == cs[kk]
        rc, Xd = oracle.derive(len(rp) - 1, m, cs)
        assert rc == 0 and Xd == X
        n = len(rp) - 1
        from math import comb
        assert sum(X[6:17]) == comb(n, 4) and sum(X[2:6]) == comb(n, 3)
        assert X[3] == int(sum(comb(int(d), 2) for d in deg)) - 3 * X[2]


def test_dense_graph_reaches_every_clique_tier():
    # out-degrees up to ~1100: the 4-clique pass runs its shared-memory tiers
    # (k <= 256, 512, 1024) and its global-memory tier (k > 1024)
    rp, ci = graphgen.er(1200, 0.92, 41)
    deg = np.diff(rp)
    assert deg.max() > 1024
    _sampled_check(rp, ci, k=150, seed=3)


def test_complete_graph_every_clique_tier():
    # K_n: |T| = n - 2, x7 = C(n-2, 2), no S_u, S_v or D_e (Table 1 / Sec. 4.5)
    from math import comb
    n = 1100
    rp, ci = graphs.complete(n)
    m = n * (n - 1) // 2
    with gcb.Graph(rp, ci) as g:
        pe = np.zeros((g.m, 13), np.uint64)
        X = g.count(pe)
    row = np.array([n - 2, 0, 0, comb(n - 2, 2), 0, comb(n - 2, 2), 0, 0, 0, 0, m - 2 * (n - 1) + 1, 0, 0],
                   np.uint64)
    assert (pe == row).all()
    assert X == [m, 0, comb(n, 3), 0, 0, 0, comb(n, 4)] + [0] * 10
    np.testing.assert_array_equal(pe[[0, m // 2, m - 1]], oracle.count_sample(rp, ci, np.array([0, m // 2, m - 1])))


def test_chung_lu_1m_config_sampled():
    rp, ci = graphgen.config_chung_lu()
    _sampled_check(rp, ci, k=1000, seed=1)


def test_rmat22_config_sampled():
    rp, ci = graphgen.config_rmat(22)
    _sampled_check(rp, ci, k=300, seed=2)


# ---------------- batched / served form ----------------

def _oracle_X(rp, ci):
    return oracle.count(rp, ci, per_edge=False, threads=4)["X"]


@pytest.mark.parametrize("manual", [True, False])
def test_batch_matches_plain_and_oracle(manual):
    B = graphgen.batch(300, n_lo=20, n_hi=200, seed=31)
    b = gcb.gc_batch_create(8 << 30, gcb.GC_BATCH_MANUAL if manual else 0)
    try:
        tickets = [gcb.gc_batch_submit(b, *B.graph(i)) for i in range(len(B))]
        gcb.gc_batch_flush(b)
        res = [gcb.gc_batch_poll(b, t, timeout_us=60_000_000) for t in tickets]
    finally:
        gcb.gc_batch_destroy(b)
    for i in range(len(B)):
        assert res[i] == _oracle_X(*B.graph(i)), i


def test_batch_large_graphs_in_one_launch():
    gs = [graphgen.chung_lu(30000, 150000, 2.2, 300000.0, 2000.0, 40 + i) for i in range(3)]
    gs.append(graphgen.er(500, 0.3, 44))
    b = gcb.gc_batch_create(16 << 30, gcb.GC_BATCH_MANUAL)
    try:
        ts = [gcb.gc_batch_submit(b, *g) for g in gs]
        gcb.gc_batch_flush(b)
        res = [gcb.gc_batch_poll(b, t, timeout_us=120_000_000) for t in ts]
    finally:
        gcb.gc_batch_destroy(b)
    for g, r in zip(gs, res):
        assert r == _oracle_X(*g)


def test_batch_budget_and_tickets():
    rp, ci = graphgen.er(300, 0.2, 50)
    b = gcb.gc_batch_create(1 << 20, gcb.GC_BATCH_MANUAL)  # 1 MiB: a few small graphs
    try:
        t1 = gcb.gc_batch_submit(b, rp, ci)
        busy = None
        for _ in range(100):
            busy = gcb.gc_batch_try_submit(b, rp, ci)
            if busy is None:
                break
        assert busy is None, "budget never filled"
        big = graphgen.er(3000, 0.5, 51)
        with pytest.raises(gcb.GcError) as ei:
            gcb.gc_batch_submit(b, *big)
        assert ei.value.status == -7
        assert gcb.gc_batch_poll(b, t1, timeout_us=0) is None  # nothing launched yet
        gcb.gc_batch_flush(b)
        assert gcb.gc_batch_poll(b, t1, timeout_us=120_000_000) == _oracle_X(rp, ci)
        with pytest.raises(gcb.GcError):
            gcb.gc_batch_poll(b, t1, timeout_us=0)  # retired
        t2 = gcb.gc_batch_try_submit(b, rp, ci)     # budget freed after retirement
        assert t2 is not None
        gcb.gc_batch_flush(b)
        assert gcb.gc_batch_poll(b, t2, timeout_us=120_000_000) == _oracle_X(rp, ci)
    finally:
        gcb.gc_batch_destroy(b)


@pytest.mark.parametrize("inflight", [1, 2, 4])
def test_served_result_same_alone_and_in_mix(inflight):
    params = graphgen.serving_params(12, m_lo=1000, m_hi=60000, seed=7)
    gs = [graphgen.serving_graph(params, r) for r in range(12)]
    alone = []
    for g in gs:
        b = gcb.gc_batch_create(4 << 30, 0)
        try:
            alone.append(gcb.gc_batch_poll(b, gcb.gc_batch_submit(b, *g), timeout_us=120_000_000))
        finally:
            gcb.gc_batch_destroy(b)
    b = gcb.gc_batch_create(4 << 30, 0)
    try:
        gcb.gc_batch_set_param(b, gcb.GC_PARAM_MAX_INFLIGHT, inflight)
        assert gcb.gc_batch_config(b)["max_inflight"] == inflight
        ts = [gcb.gc_batch_submit(b, *g) for g in gs]
        mix = [gcb.gc_batch_poll(b, t, timeout_us=120_000_000) for t in ts]
    finally:
        gcb.gc_batch_destroy(b)
    assert mix == alone
    for g, r in zip(gs[:4], mix[:4]):
        assert r == _oracle_X(*g)



def test_batch_rejects_asymmetric_graph_and_keeps_the_others():
    good = [graphgen.er(60, 0.2, 70 + i) for i in range(3)]
    bad_rp = np.array([0, 2, 3, 4], np.int32)
    bad_ci = np.array([1, 2, 2, 0], np.int32)   # 0:{1,2} 1:{2} 2:{0}: (0,1) has no reverse
    b = gcb.gc_batch_create(1 << 30, gcb.GC_BATCH_MANUAL)
    try:
        t0 = gcb.gc_batch_submit(b, *good[0])
        with pytest.raises(gcb.GcError) as ei:
            gcb.gc_batch_submit(b, bad_rp, bad_ci)
        assert ei.value.status == -5
        ts = [t0, gcb.gc_batch_submit(b, *good[1]), gcb.gc_batch_submit(b, *good[2])]
        gcb.gc_batch_flush(b)
        res = [gcb.gc_batch_poll(b, t, timeout_us=120_000_000) for t in ts]
    finally:
        gcb.gc_batch_destroy(b)
    assert res == [_oracle_X(*g) for g in good]


def test_batch_submit_many_matches_single_submits():
    B = graphgen.batch(200, n_lo=20, n_hi=700, seed=33)   # small and large (n > 512) graphs
    b = gcb.gc_batch_create(8 << 30, gcb.GC_BATCH_MANUAL)
    try:
        ts = gcb.gc_batch_submit_many(b, B.nvert, B.voff, B.eoff, B.row_ptr, B.col_idx)
        gcb.gc_batch_flush(b)
        res = [gcb.gc_batch_poll(b, int(t), timeout_us=120_000_000) for t in ts]
    finally:
        gcb.gc_batch_destroy(b)
    for i in range(0, len(B), 7):
        assert res[i] == _oracle_X(*B.graph(i)), i


def _batch_results(B, config):
    b = gcb.gc_batch_create(16 << 30, gcb.GC_BATCH_MANUAL)
    try:
        gcb.gc_batch_configure(b, config)
        assert gcb.gc_batch_config(b)["small_n_max"] == config.get("small_n_max", 512)
        res, stats = [], []
        for _ in range(2):  # the second launch replays (or updates) the captured graph
            ts = gcb.gc_batch_submit_many(b, B.nvert, B.voff, B.eoff, B.row_ptr, B.col_idx)
            gcb.gc_batch_flush(b)
            res.append([gcb.gc_batch_poll(b, int(t), timeout_us=120_000_000) for t in ts])
            stats.append(gcb.gc_batch_last_stats(b))
    finally:
        gcb.gc_batch_destroy(b)
    assert res[0] == res[1]
    return res[0], stats


def test_batch_results_identical_under_every_setting():
    # every size class of the bitmatrix kernels (n up to 1024) and graphs on
    # both sides of every cut; the counts must not depend on the parameters
    B = graphgen.batch(240, n_lo=20, n_hi=1024, seed=35)
    base = {"small_n_max": 1024, "use_graph": 1, "block": {str(n): 256 for n in gcb.SMALL_CLASS_N}}
    ref, st = _batch_results(B, base)
    assert st[1]["replayed"] == 1.0 and st[1]["small_sequence_ms"] > 0
    configs = [dict(base, small_n_max=0), dict(base, small_n_max=64), dict(base, small_n_max=300),
               dict(base, use_graph=0, block={str(n): 64 for n in gcb.SMALL_CLASS_N}),
               dict(base, block={str(n): 512 for n in gcb.SMALL_CLASS_N}),
               dict(base, use_graph=0, small_n_max=512, block={"64": 128, "128": 64, "256": 512, "512": 128})]
    for cfg in configs:
        res, st = _batch_results(B, cfg)
        assert res == ref, cfg
        if cfg["use_graph"] == 0:
            assert st[1]["replayed"] == 0.0
            assert sum(st[1][f"class_n{n}_ms"] for n in gcb.SMALL_CLASS_N) > 0
        if cfg["small_n_max"] < 1024:
            assert st[1]["union_ms"] > 0
    checked = 0
    for i in range(len(B)):
        rp, ci = B.graph(i)
        if len(ci) // 2 <= 40000 and i % 4 == 0:
            assert ref[i] == _oracle_X(rp, ci), i
            checked += 1
    assert checked >= 20


def test_batch_parameters_and_tuning_cache(tmp_path, monkeypatch):
    import json
    import torch
    b = gcb.gc_batch_create(1 << 30, gcb.GC_BATCH_MANUAL)
    try:
        for param, value in ((gcb.GC_PARAM_SMALL_N_MAX, 2000), (gcb.GC_PARAM_BLOCK_N64, 96),
                             (gcb.GC_PARAM_USE_GRAPH, 2), (gcb.GC_PARAM_MAX_INFLIGHT, 5), (99, 1)):
            with pytest.raises(gcb.GcError) as ei:
                gcb.gc_batch_set_param(b, param, value)
            assert ei.value.status == -1
        gcb.gc_batch_set_param(b, gcb.GC_PARAM_BLOCK_N64 + 2, 128)
        assert gcb.gc_batch_get_param(b, gcb.GC_PARAM_BLOCK_N64 + 2) == 128
    finally:
        gcb.gc_batch_destroy(b)
    # a cache entry for this GPU is read at gc_batch_create
    entry = {"small_n_max": 300, "use_graph": 0, "block": {"64": 64, "128": 512, "256": 128, "512": 64, "1024": 512},
             "max_inflight": 3}
    path = tmp_path / "cache.json"
    path.write_text(json.dumps({"some other GPU": {"small_n_max": 7}, torch.cuda.get_device_name(0): entry}))
    monkeypatch.setenv("GC_TUNE_CACHE", str(path))
    b = gcb.gc_batch_create(1 << 30, gcb.GC_BATCH_MANUAL)
    try:
        assert gcb.gc_batch_config(b) == entry
    finally:
        gcb.gc_batch_destroy(b)
    path.write_text("{ not json")
    b = gcb.gc_batch_create(1 << 30, gcb.GC_BATCH_MANUAL)  # a broken cache leaves the defaults
    try:
        assert gcb.gc_batch_config(b)["small_n_max"] == 512
    finally:
        gcb.gc_batch_destroy(b)


_HUB_JOBS = ("import numpy as np, os, graphgen, oracle, paper_1608_05138_gb300 as gcb\n"
             "rp, ci = graphgen.chung_lu(120000, 600000, 2.1, 1.2e6, 4000.0, 7)\n"
             "o = oracle.count(rp, ci)\n"
             "with gcb.Graph(rp, ci) as g:\n"
             "    pe = np.zeros((g.m, 13), np.uint64); X = g.count(pe); w = g.work_counts()\n"
             "assert X == o['X'] and (pe == o['per_edge']).all()\n"
             "assert w['c_hub_ctas'] > 0 and 0 < w['c_hub_busy_max_ns'] and w['c_hub_busy_sum_ns'] >= w['c_hub_busy_max_ns']\n"
             "print('ok', w['c_hub_jobs'])\n")


def test_hub_jobs_split_or_whole_give_the_same_counts():
    # hub units cut into many jobs of o-range blocks (Sec. 4.4's finer
    # granularity), or kept whole: the same exact counts either way
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    jobs = {}
    for per_cta in ("0", "64"):
        env = dict(os.environ, PYTHONPATH=root, GC_HUB_JOBS_PER_CTA=per_cta)
        r = subprocess.run([sys.executable, "-c", _HUB_JOBS], env=env, cwd=root, capture_output=True, text=True,
                           timeout=900)
        assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr
        jobs[per_cta] = int(r.stdout.split()[-1])
    assert jobs["64"] > jobs["0"] > 0


def test_serving_under_a_nearly_full_budget():
    # a budget that holds about two of the requests at once: submissions are
    # refused (GC_ERR_BUSY) until earlier ones retire, and every result equals
    # the graph's own whole-graph count
    import time
    params = graphgen.serving_params(16, m_lo=200000, m_hi=800000, seed=9)
    gs = [graphgen.serving_graph(params, r) for r in range(16)]
    expect = []
    for g in gs:
        with gcb.Graph(*g) as h:
            expect.append(h.count())
    grid = 2 * 152

    def footprint(rp, ci):  # the runtime's estimate of a graph's device memory
        n, m = len(rp) - 1, len(ci) // 2
        return 44 * n + 32 * m + 1024 + (grid * n * 4 if n > 4096 else 0)

    budget = 2 * max(footprint(*g) for g in gs)
    b = gcb.gc_batch_create(budget, 0)
    tickets, results, busy, nxt = {}, {}, 0, 0
    t_end = time.time() + 300
    try:
        while len(results) < len(gs) and time.time() < t_end:
            while nxt < len(gs):  # submit until the runtime refuses
                t = gcb.gc_batch_try_submit(b, *gs[nxt])
                if t is None:
                    busy += 1
                    break
                tickets[nxt] = t
                nxt += 1
            for r, t in list(tickets.items()):
                x = gcb.gc_batch_poll(b, t, timeout_us=0)
                if x is not None:
                    results[r] = x
                    del tickets[r]
            time.sleep(0.0005)
    finally:
        gcb.gc_batch_destroy(b)
    assert busy > 0
    assert [results.get(r) for r in range(len(gs))] == expect


def test_batch_submit_many_rejects_a_malformed_graph():
    # the bulk path validates each graph on its own thread: the codes and
    # messages are those of a single submission, and nothing is admitted
    good = [graphgen.er(60, 0.2, 80 + i) for i in range(4)]
    bad = {-5: (np.array([0, 2, 3, 4], np.int32), np.array([1, 2, 2, 0], np.int32)),   # (0,1) without (1,0)
           -4: (np.array([0, 1, 2], np.int32), np.array([0, 0], np.int32)),             # self-loop
           -3: (np.array([0, 2, 4], np.int32), np.array([1, 1, 0, 0], np.int32)),       # duplicate
           -6: (np.array([0, 1, 2], np.int32), np.array([7, 0], np.int32))}             # out of range
    for code, (brp, bci) in bad.items():
        gs = good[:2] + [(brp, bci)] + good[2:]
        nvert = np.array([len(r) - 1 for r, _ in gs], np.int32)
        voff = np.concatenate([[0], np.cumsum([len(r) for r, _ in gs])]).astype(np.int64)
        eoff = np.concatenate([[0], np.cumsum([len(c) for _, c in gs])]).astype(np.int64)
        rp = np.concatenate([r for r, _ in gs]).astype(np.int32)
        ci = np.concatenate([c for _, c in gs]).astype(np.int32)
        b = gcb.gc_batch_create(1 << 30, gcb.GC_BATCH_MANUAL)
        try:
            with pytest.raises(gcb.GcError) as ei:
                gcb.gc_batch_submit_many(b, nvert, voff, eoff, rp, ci)
            assert ei.value.status == code and "graph 2" in str(ei.value)
            x = gcb.gc_batch_poll_many(b, np.zeros(0, np.uint64), timeout_us=0)  # nothing was admitted
            assert x is not None and x.shape == (0, 17, 2)
        finally:
            gcb.gc_batch_destroy(b)


def test_memory_pool_keeps_blocks_until_released():
    # a freed graph's blocks stay in the library pool (not zeroed) and serve
    # the next graph, whose counts must not depend on their old contents;
    # gc_release_cached_memory hands them back to the device
    import torch
    torch.cuda.synchronize()
    gcb.gc_release_cached_memory()
    free0, _ = torch.cuda.mem_get_info()
    rp, ci = graphgen.rmat(16, 16, 0.57, 0.19, 0.19, 3)
    with gcb.Graph(rp, ci) as g:
        g.count(np.zeros((g.m, 13), np.uint64))
    free1, _ = torch.cuda.mem_get_info()
    assert free0 - free1 > 50 << 20  # kept by the pool
    rp2, ci2 = graphgen.chung_lu(60000, 400000, 2.1, 8e5, 3000.0, 5)
    assert_parity(rp2, ci2)          # counted in reused blocks
    gcb.gc_release_cached_memory()
    free2, _ = torch.cuda.mem_get_info()
    assert free2 > free1 and free0 - free2 < 64 << 20


def test_batch_submit_many_randomized_corruptions():
    # one graph of a bulk submission corrupted at random (range, self-loop,
    # duplicate, order): refused with the code and message of its first
    # failing entry in row order, naming that graph; nothing is admitted
    from tests.test_abi import _first_violation
    rng = np.random.default_rng(21)
    gs = [graphgen.er(int(rng.integers(40, 400)), 0.1, 300 + i) for i in range(12)]
    for trial in range(10):
        k = int(rng.integers(0, len(gs)))
        rp, ci = gs[k][0], gs[k][1].copy()
        n = len(rp) - 1
        x = int(rng.choice(np.flatnonzero(np.diff(rp) >= 3)))
        p = int(rng.integers(rp[x] + 1, rp[x + 1] - 1))
        kind = trial % 4
        if kind == 0:
            ci[p] = n + 2
        elif kind == 1:
            ci[p] = x
        elif kind == 2:
            ci[p] = ci[p - 1]
        else:
            ci[p], ci[p + 1] = ci[p + 1], ci[p]
        code, msg = _first_violation(rp, ci)
        parts = [(r, c) for r, c in gs]
        parts[k] = (rp, ci)
        nvert = np.array([len(r) - 1 for r, _ in parts], np.int32)
        voff = np.concatenate([[0], np.cumsum([len(r) for r, _ in parts])]).astype(np.int64)
        eoff = np.concatenate([[0], np.cumsum([len(c) for _, c in parts])]).astype(np.int64)
        b = gcb.gc_batch_create(1 << 30, gcb.GC_BATCH_MANUAL)
        try:
            with pytest.raises(gcb.GcError) as ei:
                gcb.gc_batch_submit_many(b, nvert, voff, eoff, np.concatenate([r for r, _ in parts]),
                                         np.concatenate([c for _, c in parts]))
            assert ei.value.status == code and str(ei.value).endswith(f"graph {k}: {msg}"), (str(ei.value), code, msg)
            assert gcb.gc_batch_poll_many(b, np.zeros(0, np.uint64), timeout_us=0).shape == (0, 17, 2)
        finally:
            gcb.gc_batch_destroy(b)
