"""The closed forms by which the batched small-graph kernel forms the
unrestricted sums C_3 .. C_16 (Sec. 4.5) from a few per-edge, per-vertex and
per-entry sums, checked against the per-edge definitions on random graphs
(brute force, independent of the oracle and of the kernel). Per edge (u, v):
T = Gamma(u) & Gamma(v), S_u = Gamma(u) \\ (Gamma(v) + {v}), S_v likewise,
s = |S_u| + |S_v|, D = n - 2 - |T| - s."""
import itertools
import random

import pytest

M64 = (1 << 64) - 1


def per_edge_sums(n, adj):
    """C_3 C_4 C_5 . C_8 C_9 . C_11 .. C_16 summed edge by edge (Sec. 4.5);
    the C_7 and C_10 slots hold 0 (they come from the 4-clique and 4-cycle
    terms, not from a polynomial in |T|, |S_u|, |S_v|)."""
    E = [(u, v) for u in range(n) for v in adj[u] if u < v]
    m = len(E)
    out = [0] * 13
    for u, v in E:
        t = len(adj[u] & adj[v])
        su = len(adj[u] - adj[v] - {v})
        sv = len(adj[v] - adj[u] - {u})
        s = su + sv
        D = n - 2 - t - s
        du, dv = len(adj[u]), len(adj[v])
        vals = [t, s, D, 0, t * (t - 1) // 2, t * s, 0, su * (su - 1) // 2 + sv * (sv - 1) // 2, su * sv, t * D,
                m - du - dv + 1, s * D, D * (D - 1) // 2]
        out = [a + b for a, b in zip(out, vals)]
    return out


def closed_forms(n, adj):
    """The same columns from sum t, sum t^2, sum t (d_u + d_v) over the edges,
    sum d^2 and sum d^3 over the vertices and sum d_x d_y over the directed
    entries, in 64-bit unsigned arithmetic as the kernel does them."""
    E = [(u, v) for u in range(n) for v in adj[u] if u < v]
    M = len(E)
    St = sum(len(adj[u] & adj[v]) for u, v in E)
    Stt = sum(len(adj[u] & adj[v]) ** 2 for u, v in E)
    Sta = sum(len(adj[u] & adj[v]) * (len(adj[u]) + len(adj[v])) for u, v in E)
    d = [len(adj[x]) for x in range(n)]
    A1 = sum(x * x for x in d)
    d3 = sum(x ** 3 for x in d)
    dd = sum(d[x] * d[y] for x in range(n) for y in adj[x])

    def U(x):
        return x & M64

    N2 = U(n - 2)
    C4 = U(A1 - 2 * M - 2 * St)
    C9 = U(Sta - 2 * St - 2 * Stt)
    C12 = U(dd // 2 - A1 + M - Sta + 2 * St + Stt)
    Sss = U(d3 + dd - 4 * A1 + 4 * M - 4 * (Sta - 2 * St) + 4 * Stt)
    C5 = U(N2 * M - St - C4)
    SD2 = U(N2 * N2 * M - 2 * N2 * (St + C4) + Stt + 2 * C9 + Sss)
    return [St, C4, C5, 0, U(Stt - St) // 2, C9, 0, U(Sss - 2 * C12 - C4) // 2, C12, U(N2 * St - Stt - C9),
            U(M * M + M - A1), U(N2 * C4 - C9 - Sss), U(SD2 - C5) // 2]


@pytest.mark.parametrize("seed", range(4))
def test_closed_forms_equal_per_edge_sums(seed):
    rng = random.Random(seed)
    for _ in range(60):
        n = rng.randint(0, 36)
        p = rng.random()
        adj = [set() for _ in range(n)]
        for u, v in itertools.combinations(range(n), 2):
            if rng.random() < p:
                adj[u].add(v)
                adj[v].add(u)
        assert closed_forms(n, adj) == per_edge_sums(n, adj), (n, p)


def test_closed_forms_on_special_graphs():
    for n in range(0, 9):
        complete = [set(range(n)) - {x} for x in range(n)]
        star = [set(range(1, n)) if x == 0 else ({0} if n > 1 else set()) for x in range(n)]
        empty = [set() for _ in range(n)]
        for adj in (complete, star, empty):
            assert closed_forms(n, adj) == per_edge_sums(n, adj)
