"""The allocation-free triangle entry point against the regular one.

gc_edge_triangles_noalloc serves callers that cannot allocate device memory:
it reads a device CSR in place and keeps its only scratch in a fixed
file-scope device array. Here it is called through the C ABI twice in a row
(the array keeps the previous call's contents, so the second call checks that
each call starts clean) and its per-slot counts must equal column 0 (|T|) of
gc_count_edge_graphlets for the same edges, and |T| of the CPU oracle,
exactly (integer counts). A call after the first one must leave the device's
free memory and torch's allocated bytes unchanged. This file is collected
last on purpose.
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


def _slot_edge_ids(rp, ci, uv):
    """Edge id (row of the edge list uv, u < v) behind every CSR slot."""
    n = len(rp) - 1
    key = uv[:, 0].astype(np.int64) * n + uv[:, 1]
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    cols = ci.astype(np.int64)
    return np.searchsorted(key, np.minimum(rows, cols) * n + np.maximum(rows, cols))


def _oracle_per_slot(rp, ci):
    """|T| of the edge behind every CSR slot, from the CPU oracle."""
    t = oracle.count(rp, ci)["per_edge"][:, 0]
    return t[_slot_edge_ids(rp, ci, oracle.edges(rp, ci))].astype(np.int32)


def _expected_per_slot(rp, ci):
    """|T| of the edge behind every CSR slot, from the regular entry point."""
    with gcb.Graph(rp, ci) as g:
        pe = np.zeros((g.m, 13), np.uint64)
        g.count(pe)
        uv = g.edges()
    return pe[_slot_edge_ids(rp, ci, uv), 0].astype(np.int32)


@pytest.mark.parametrize("make", [
    lambda: graphgen.chung_lu(50000, 400000, 2.1, 800000.0, 4000.0, 61),
    lambda: graphgen.er(3000, 0.05, 62),
    lambda: graphs.complete(40),
    lambda: graphs.star(500),
])
def test_noalloc_matches_regular_entry_point_twice(make):
    import torch
    rp, ci = make()
    expect = _expected_per_slot(rp, ci)
    np.testing.assert_array_equal(expect, _oracle_per_slot(rp, ci))
    d_rp = torch.from_numpy(rp).cuda()
    d_ci = torch.from_numpy(ci).cuda()
    stream = torch.cuda.current_stream()
    for _ in range(2):
        out = torch.full((len(ci),), -1, dtype=torch.int32, device="cuda")
        gcb.gc_edge_triangles_noalloc(d_rp, d_ci, out, stream=stream)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), expect)


def test_noalloc_rejects_graphs_above_its_limit():
    import torch
    n = (1 << 20) + 1
    d_rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    d_ci = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(gcb.GcError) as ei:
        gcb.gc_edge_triangles_noalloc(d_rp, d_ci, out)
    assert ei.value.status == -9
    assert "limit" in str(ei.value)


def test_noalloc_call_allocates_nothing():
    import torch
    rp, ci = graphgen.er(3000, 0.05, 63)
    d_rp = torch.from_numpy(rp).cuda()
    d_ci = torch.from_numpy(ci).cuda()
    out = torch.zeros(len(ci), dtype=torch.int32, device="cuda")
    gcb.gc_edge_triangles_noalloc(d_rp, d_ci, out)  # first call: module and symbol set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    gcb.gc_edge_triangles_noalloc(d_rp, d_ci, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == alloc0
    assert free1 == free0
    np.testing.assert_array_equal(out.cpu().numpy(), _oracle_per_slot(rp, ci))
