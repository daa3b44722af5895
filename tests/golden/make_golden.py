"""Writes tests/golden/named_graphs.json: brute-force censuses of small named
graphs (the 3-cube, the Petersen graph, wheels, a bowtie, K5 minus an edge,
the 5-prism). Calls only oracle/brute.py (full enumeration of Problem 1).

    python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import brute  # noqa: E402
from tests import graphs  # noqa: E402

NAMED = {
    "cube": graphs.cube,
    "petersen": graphs.petersen,
    "wheel5": lambda: graphs.wheel(5),
    "wheel8": lambda: graphs.wheel(8),
    "bowtie": lambda: graphs.csr(5, [(0, 1), (1, 2), (0, 2), (2, 3), (3, 4), (2, 4)]),
    "k5_minus_edge": lambda: graphs.csr(5, [(a, b) for a in range(5) for b in range(a + 1, 5)
                                             if (a, b) != (0, 1)]),
    "prism5": lambda: graphs.csr(10, [(i, (i + 1) % 5) for i in range(5)]
                                 + [(5 + i, 5 + (i + 1) % 5) for i in range(5)]
                                 + [(i, i + 5) for i in range(5)]),
}


def main():
    out = {}
    for name, make in NAMED.items():
        rp, ci = make()
        out[name] = {
            "n": len(rp) - 1,
            "edges": graphs.edges_of(rp, ci),
            "X": brute.census(rp, ci),
            "per_edge": brute.per_edge_columns(rp, ci).astype(int).tolist(),
        }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "named_graphs.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
