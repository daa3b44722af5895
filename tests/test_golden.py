"""Oracle against stored brute-force censuses of small named graphs
(tests/golden/named_graphs.json, written by tests/golden/make_golden.py,
which calls only the brute-force enumerator of Problem 1)."""
import json
import os

import numpy as np
import pytest

import oracle
from tests import graphs

with open(os.path.join(os.path.dirname(__file__), "golden", "named_graphs.json")) as f:
    GOLDEN = json.load(f)


@pytest.mark.parametrize("name", sorted(GOLDEN))
def test_named_graph(name):
    g = GOLDEN[name]
    rp, ci = graphs.csr(g["n"], [tuple(e) for e in g["edges"]])
    o = oracle.count(rp, ci, threads=1)
    assert o["X"] == g["X"]
    np.testing.assert_array_equal(o["per_edge"], np.array(g["per_edge"], np.uint64).reshape(-1, 13))
