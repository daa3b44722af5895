"""Writes tests/golden/large_configs.json: the CPU oracle's results on the
full-size workloads, stored as SHA-256 digests (and the global counts in the
clear), so that the GPU tests can compare whole configurations bit for bit
without re-running the oracle (minutes to an hour of host time each).

Calls only oracle/ (the paper's CPU Alg. 1/5/6 and the Sec. 4.5/4.6
relations) and graphgen/ (the seeded generators):

    python tests/golden/make_large_digests.py er chung_lu batched serving

  er        ER-2000 (G(2000, 0.01)) and the dense ER G(1000, 0.3), seed 1:
            the same fields as chung_lu.
  chung_lu  Chung-Lu n = 1M, m = 10M, gamma 2.1, cap 50k, seed 1: digest of
            the CSR, digest of the full uint64 [m][13] per-edge array, the 13
            unrestricted counts and X_1..X_17.
  batched   the 100 000-graph batch (n uniform in [20, 500], seed 1): X_1..X_17
            of every graph as (lo, hi) uint64 pairs, digested per chunk of
            1000 graphs and as a whole, plus the column totals.
  serving   every request of at least 10^6 edges in the 300-request serving
            stream (seed 1): its CSR digest and X_1..X_17.

Digests: SHA-256 of the little-endian bytes of the C-contiguous arrays.
"""
import hashlib
import json
import os
import sys
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import graphgen  # noqa: E402
import oracle  # noqa: E402

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "large_configs.json")
BATCH_CHUNK = 1000
SERVING_REQUESTS = 300
SERVING_MIN_EDGES = 1_000_000


def sha(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).astype(a.dtype.newbyteorder("<"), copy=False).tobytes())
    return h.hexdigest()


def lohi(xs) -> np.ndarray:
    """Python ints (< 2^128) -> uint64 [len][2] (lo, hi)."""
    return np.array([[x & (2**64 - 1), x >> 64] for x in xs], np.uint64).reshape(-1, 2)


def chung_lu():
    rp, ci = graphgen.config_chung_lu()
    t0 = time.time()
    o = oracle.count(rp, ci)
    return {"n": len(rp) - 1, "m": len(ci) // 2, "csr_sha256": sha(rp, ci),
            "per_edge_sha256": sha(o["per_edge"]), "csum": o["csum"], "X": o["X"],
            "oracle_seconds": round(time.time() - t0, 1), "threads": oracle.default_threads()}


def er_configs():
    """ER-2000 (the small configuration) and the dense ER 1K/150K graph: the
    same digests as chung_lu."""
    out = {}
    for name, make in (("er2000", graphgen.config_er2000), ("er_dense", graphgen.config_er_dense)):
        rp, ci = make()
        o = oracle.count(rp, ci)
        out[name] = {"n": len(rp) - 1, "m": len(ci) // 2, "csr_sha256": sha(rp, ci),
                     "per_edge_sha256": sha(o["per_edge"]), "csum": o["csum"], "X": o["X"]}
    return out


def batched():
    B = graphgen.batch(100_000)
    G = len(B)
    X = np.zeros((G, 17, 2), np.uint64)

    def one(g):  # ctypes releases the GIL: one oracle call per thread
        X[g] = lohi(oracle.count(*B.graph(g), per_edge=False, threads=1)["X"])

    t0 = time.time()
    with ThreadPoolExecutor(oracle.default_threads()) as ex:
        list(ex.map(one, range(G), chunksize=64))
    totals = [int(sum(int(X[g, i, 0]) | (int(X[g, i, 1]) << 64) for g in range(G))) for i in range(17)]
    return {"graphs": G, "edges": B.total_edges,
            "csr_sha256": sha(B.nvert, B.voff, B.eoff, B.row_ptr, B.col_idx),
            "chunk": BATCH_CHUNK, "X_sha256": sha(X),
            "chunk_sha256": [sha(X[c:c + BATCH_CHUNK]) for c in range(0, G, BATCH_CHUNK)],
            "X_totals": totals, "oracle_seconds": round(time.time() - t0, 1),
            "threads": oracle.default_threads()}


def serving():
    P = graphgen.serving_params(SERVING_REQUESTS)
    out = []
    t0 = time.time()
    for r in range(SERVING_REQUESTS):
        if int(P["m"][r]) < SERVING_MIN_EDGES:
            continue
        rp, ci = graphgen.serving_graph(P, r)
        out.append({"request": r, "n": len(rp) - 1, "m": len(ci) // 2, "csr_sha256": sha(rp, ci),
                    "X": oracle.count(rp, ci, per_edge=False)["X"]})
    return {"requests": SERVING_REQUESTS, "min_edges": SERVING_MIN_EDGES, "graphs": out,
            "oracle_seconds": round(time.time() - t0, 1), "threads": oracle.default_threads()}


def main(which):
    data = {}
    if os.path.exists(PATH):
        with open(PATH) as f:
            data = json.load(f)
    for w in which:
        print("computing", w, flush=True)
        if w == "er":
            data.update(er_configs())
        else:
            data[w] = {"chung_lu": chung_lu, "batched": batched, "serving": serving}[w]()
        with open(PATH, "w") as f:
            json.dump(data, f, indent=1)
        print("wrote", w, "to", PATH, flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["er", "chung_lu", "batched", "serving"])
