"""Whole configurations, GPU against the oracle, bit-exact (integer counts,
zero tolerance).

The oracle needs minutes to an hour of host time on the full-size workloads,
so its results are stored once by tests/golden/make_large_digests.py (which
calls only oracle/ and graphgen/) as SHA-256 digests of the complete arrays:
  * Chung-Lu n = 1M, m = 10M: the digest of all m x 13 per-edge rows, the
    13 unrestricted counts and X_1..X_17 (Problem 1, Sec. 4.5/4.6);
  * the 100 000-graph batch: X_1..X_17 of every graph;
  * every serving request of at least 10^6 edges: X_1..X_17.
R-MAT scale 22 would need about half a day of host time: it is checked on
more than 20 000 edges drawn from every kind of work unit of the GPU path
(each counted one by one by the oracle), over a first count (whose list of
pass-T edges is sized by a guess and overflows) and a second one, and its
global counts against three subgraph identities that share nothing with the
per-edge machinery.
"""
import hashlib
import json
import os
from math import comb

import numpy as np
import pytest

import graphgen
import oracle
import paper_1608_05138_gb300 as gcb

pytestmark = pytest.mark.gpu

with open(os.path.join(os.path.dirname(__file__), "golden", "large_configs.json")) as f:
    GOLDEN = json.load(f)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1608_05138_gb300 import build
    build.build()


def sha(*arrays):
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).astype(a.dtype.newbyteorder("<"), copy=False).tobytes())
    return h.hexdigest()


def lohi(xs):
    return np.array([[x & (2**64 - 1), x >> 64] for x in xs], np.uint64).reshape(-1, 2)


def test_chung_lu_1m_whole_config_equals_oracle():
    import torch
    gold = GOLDEN["chung_lu"]
    rp, ci = graphgen.config_chung_lu()
    assert sha(rp, ci) == gold["csr_sha256"]  # the same graph the oracle counted
    with gcb.Graph(rp, ci) as g:
        dev = torch.zeros((g.m, 13), dtype=torch.int64, device="cuda")
        X = g.count(dev)
        cs = g.csums()
        host = dev.cpu().numpy().view(np.uint64)
    assert X == gold["X"]
    assert cs == gold["csum"]
    assert sha(host) == gold["per_edge_sha256"]


@pytest.mark.parametrize("name,make", [("er2000", graphgen.config_er2000), ("er_dense", graphgen.config_er_dense)])
def test_er_configs_equal_stored_oracle(name, make):
    gold = GOLDEN[name]
    rp, ci = make()
    assert sha(rp, ci) == gold["csr_sha256"]
    with gcb.Graph(rp, ci) as g:
        pe = np.zeros((g.m, 13), np.uint64)
        X = g.count(pe)
    assert X == gold["X"] and sha(pe) == gold["per_edge_sha256"]


def test_batched_100k_whole_config_equals_oracle():
    gold = GOLDEN["batched"]
    B = graphgen.batch(100_000)
    assert sha(B.nvert, B.voff, B.eoff, B.row_ptr, B.col_idx) == gold["csr_sha256"]
    b = gcb.gc_batch_create(200 << 30, gcb.GC_BATCH_MANUAL)
    try:
        tickets = gcb.gc_batch_submit_many(b, B.nvert, B.voff, B.eoff, B.row_ptr, B.col_idx)
        gcb.gc_batch_flush(b)
        X = gcb.gc_batch_poll_many(b, tickets, timeout_us=600_000_000)  # [G][17] (lo, hi)
        # the single-ticket poll agrees on a few graphs submitted again
        t2 = gcb.gc_batch_submit_many(b, B.nvert[:3], B.voff[:4], B.eoff[:4], B.row_ptr, B.col_idx)
        gcb.gc_batch_flush(b)
        for k in range(3):
            x = gcb.gc_batch_poll(b, int(t2[k]), timeout_us=60_000_000)
            assert np.array_equal(lohi(x), X[k])
    finally:
        gcb.gc_batch_destroy(b)
    c = gold["chunk"]
    bad = [k for k, d in enumerate(gold["chunk_sha256"]) if sha(X[k * c:(k + 1) * c]) != d]
    assert not bad, f"graphs differ in chunks {bad[:10]} (of {c} graphs each)"
    assert sha(X) == gold["X_sha256"]
    totals = [sum(int(v) for v in X[:, i, 0]) + (sum(int(v) for v in X[:, i, 1]) << 64) for i in range(17)]
    assert totals == gold["X_totals"]


def test_serving_requests_of_a_million_edges_equal_oracle():
    gold = GOLDEN["serving"]
    P = graphgen.serving_params(gold["requests"])
    reqs = gold["graphs"]
    assert len(reqs) >= 10
    graphs_ = []
    for q in reqs:
        rp, ci = graphgen.serving_graph(P, q["request"])
        assert len(ci) // 2 >= gold["min_edges"] and sha(rp, ci) == q["csr_sha256"]
        graphs_.append((rp, ci))
    # served together by the continuous-batching runtime ...
    b = gcb.gc_batch_create(120 << 30, 0)
    try:
        ts = [gcb.gc_batch_submit(b, *g) for g in graphs_]
        served = [gcb.gc_batch_poll(b, t, timeout_us=600_000_000) for t in ts]
    finally:
        gcb.gc_batch_destroy(b)
    # ... and one by one through the whole-graph path
    for q, g, s in zip(reqs, graphs_, served):
        with gcb.Graph(*g) as h:
            assert h.count() == q["X"] == s, q["request"]


# ---------------- R-MAT scale 22: stratified sample and identities ----------------

K_TIERS = [(2, 32), (33, 256), (257, 512), (513, 1024), (1025, 1 << 30)]
HASH_MAX_W = 8192          # pass-C units of at most this many wedges: shared-memory hash
HUB_BLOCK = 45056          # words of an o-range block of the hub kernel (1, 2 or 3 counters a word)


def unit_strata(rp, ci):
    """Per edge (edge-id order), the kind of work unit of the GPU path that
    owns it, computed on the host with numpy: the pass-C unit of its
    higher-rank end (hub, hashed, vertex-indexed table, or no wedges) and
    the pass-K tier of its lower-rank end (|out(a)|), rank = (degree, id)."""
    n = len(rp) - 1
    deg = np.diff(rp).astype(np.int64)
    order = np.lexsort((np.arange(n), deg))
    rank = np.empty(n, np.int64)
    rank[order] = np.arange(n)
    rows = np.repeat(np.arange(n, dtype=np.int64), deg)
    cols = ci.astype(np.int64)
    X, Y = rank[rows], rank[cols]
    key = np.sort(X * n + Y)                      # relabelled CSR, rows ascending
    Xs, Ys = key // n, key % n
    rps = np.concatenate([[0], np.cumsum(np.bincount(Xs, minlength=n))])
    pos = np.arange(len(key)) - rps[Xs]           # o below Ys in row Xs
    up = Ys > Xs                                  # slot (x, h), h above x
    W = np.bincount(Ys[up], weights=pos[up], minlength=n).astype(np.int64)
    NX = np.bincount(Ys[up], minlength=n).astype(np.int64)   # lower neighbours of h
    span = np.where(NX < 1023, 3 * HUB_BLOCK, np.where(NX < 65536, 2 * HUB_BLOCK, HUB_BLOCK))
    blocks = (np.arange(n) + span - 1) // span
    hub = (W >= 16384) & (W >= blocks * np.maximum(1024, NX))
    ckind = np.where(hub, 0, np.where(W == 0, 3, np.where(W <= HASH_MAX_W, 1, 2)))  # by rank
    out = deg[order] - NX                                                          # |out(a)| by rank
    e = rows < cols                                # edge-id order: upper triangle, row-major
    a, b = X[e], Y[e]
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    kout = out[lo]
    ktier = np.full(len(lo), -1)
    for t, (k0, k1) in enumerate(K_TIERS):
        ktier[(kout >= k0) & (kout <= k1)] = t
    return ckind[hi], ktier, deg


def test_rmat22_stratified_sample_and_identities():
    import torch
    rp, ci = graphgen.config_rmat(22)
    n, m = len(rp) - 1, len(ci) // 2
    ck, kt, deg = unit_strata(rp, ci)
    rng = np.random.default_rng(22)
    picks = [rng.integers(0, m, 2000)]
    sizes = {}
    for name, mask in [("c_hub", ck == 0), ("c_hash", ck == 1), ("c_table", ck == 2), ("c_none", ck == 3)] + \
                      [(f"k_tier{t}", kt == t) for t in range(len(K_TIERS))]:
        ids = np.flatnonzero(mask)
        sizes[name] = len(ids)
        if len(ids):
            picks.append(rng.choice(ids, min(len(ids), 2200), replace=False))
    ids = np.unique(np.concatenate(picks + [[0, m - 1]])).astype(np.int64)
    assert len(ids) >= 20000, (len(ids), sizes)
    assert all(sizes[k] > 1000 for k in ("c_hub", "c_hash", "c_table", "k_tier0", "k_tier1", "k_tier2")), sizes
    expect = oracle.count_sample(rp, ci, ids)
    sel = torch.from_numpy(ids).cuda()
    with gcb.Graph(rp, ci) as g:
        dev = torch.zeros((m, 13), dtype=torch.int64, device="cuda")
        for _ in range(2):  # the first count's list of pass-T edges is a guess; the second is sized by it
            X = g.count(dev)
            np.testing.assert_array_equal(dev[sel].cpu().numpy().view(np.uint64), expect)
        cs = g.csums()
        colsum = [int(dev[:, c].sum(dtype=torch.int64).item()) % (1 << 64) for c in range(13)]
    order = [0, 1, 2, 3, 5, 6, 4, 7, 8, 9, 10, 11, 12]
    assert [cs[k] % (1 << 64) for k in range(13)] == [colsum[c] for c in order]
    rc, Xd = oracle.derive(n, m, cs)
    assert rc == 0 and Xd == X
    X = [0] + X
    E_u = np.repeat(np.arange(n), np.diff(rp))
    up = E_u < ci
    du, dv = deg[E_u[up]], deg[ci[up]]

    def exact_sum(v):  # int64 partial sums of 2^20 terms each, added as Python ints
        return sum(int(v[i:i + (1 << 20)].sum()) for i in range(0, len(v), 1 << 20))

    assert X[1] + X[2] == comb(n, 2) and sum(X[3:7]) == comb(n, 3) and sum(X[7:18]) == comb(n, 4)
    # 2-paths, 3-stars and 3-paths as subgraphs, from degrees alone
    assert X[4] == exact_sum(deg * (deg - 1) // 2) - 3 * X[3]
    assert X[11] == exact_sum(deg * (deg - 1) * (deg - 2) // 6) - X[9] - 2 * X[8] - 4 * X[7]
    p4 = exact_sum((du - 1) * (dv - 1)) - 3 * X[3]
    assert X[12] == p4 - 2 * X[9] - 4 * X[10] - 6 * X[8] - 12 * X[7]
