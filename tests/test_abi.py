"""The C-ABI library builds, loads and exports every entry point that
include/gc.h declares; host-side CSR validation returns the documented error
codes before any device work (no GPU needed)."""
import os
import re

import numpy as np
import pytest

import paper_1608_05138_gb300 as gcb
from tests import graphs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "gc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gc_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1608_05138_gb300 import build
    build.build()
    return gcb.lib()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(gcb.EXPORTED) == names


def test_library_is_built_for_sm103a(lib):
    import subprocess
    out = subprocess.run(["cuobjdump", "--list-elf", gcb.library_path()], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


def _err(rp, ci):
    with pytest.raises(gcb.GcError) as ei:
        gcb.gc_graph_upload(np.asarray(rp, np.int32), np.asarray(ci, np.int32))
    return ei.value.status


def test_validation_error_codes(lib):
    # unsorted row
    assert _err([0, 2, 3, 4], [2, 1, 0, 0]) == -2
    # duplicate neighbour
    assert _err([0, 2, 4], [1, 1, 0, 0]) == -3
    # self-loop
    assert _err([0, 2, 4], [0, 1, 0, 1]) == -4
    # asymmetric: 0-1 present, 1-0 missing, 1-2 / 2-1 present
    assert _err([0, 1, 2, 3], [1, 2, 1]) == -5
    # out of range
    assert _err([0, 1, 2], [5, 0]) == -6
    # row_ptr[0] != 0
    assert _err([1, 2, 3], [1, 0]) == -6
    # decreasing row_ptr
    assert _err([0, 2, 1, 4], [1, 2, 0, 0]) == -2


def test_valid_graph_passes_host_validation_first(lib):
    # a valid graph gets past validation; without a GPU the next step fails
    # with a CUDA error, never a validation code.
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present: covered by the GPU tests")
    rp, ci = graphs.complete(4)
    with pytest.raises(gcb.GcError) as ei:
        gcb.gc_graph_upload(rp, ci)
    assert ei.value.status in (-7, -8)


def test_no_fallback_when_library_missing(monkeypatch, tmp_path):
    monkeypatch.setattr(gcb, "_SO", str(tmp_path / "missing.so"))
    monkeypatch.setattr(gcb, "_lib", None)
    with pytest.raises(RuntimeError):
        gcb.lib()


def test_noalloc_wrapper_rejects_bad_tensors_before_the_call():
    # the C entry point takes raw device pointers, so the binding checks
    # type, contiguity, sizes and device before calling it (no GPU needed:
    # every case below is refused before the library is touched)
    import torch
    rp = torch.tensor([0, 1, 2], dtype=torch.int32)
    ci = torch.tensor([1, 0], dtype=torch.int32)
    out = torch.zeros(2, dtype=torch.int32)
    cases = [
        ((rp.numpy(), ci, out), "torch tensor"),
        ((rp.long(), ci, out), "int32"),
        ((rp, ci.long(), out), "int32"),
        ((rp, ci, out.long()), "int32"),
        ((rp, torch.zeros(4, dtype=torch.int32)[::2], out), "contiguous"),
        ((torch.zeros(0, dtype=torch.int32), ci, out), "n + 1"),
        ((rp, ci, torch.zeros(1, dtype=torch.int32)), "fewer than"),
        ((rp, ci, out), "same CUDA device"),
    ]
    for args, words in cases:
        with pytest.raises(ValueError, match=re.escape(words)):
            gcb.gc_edge_triangles_noalloc(*args)


def _first_violation(rp, ci):
    """The code and message of the first entry (in row order) that breaks a
    linear check, range, self-loop, duplicate, order in that priority, the
    contract of include/gc.h (numpy)."""
    n = len(rp) - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    ci64 = ci.astype(np.int64)
    start = np.zeros(len(ci), bool)
    start[rp[:-1][np.diff(rp) > 0]] = True
    prev = np.concatenate([[0], ci64[:-1]])
    rng = (ci64 < 0) | (ci64 >= n)
    loop = ci64 == rows
    dup = ~start & (prev == ci64)
    desc = ~start & (prev > ci64)
    bad = np.flatnonzero(rng | loop | dup | desc)
    if len(bad) == 0:
        return None
    p = bad[0]
    x, y = int(rows[p]), int(ci[p])
    if rng[p]:
        return -6, f"column {y} out of range in row {x}"
    if loop[p]:
        return -4, f"self-loop at vertex {x}"
    if dup[p]:
        return -3, f"duplicate neighbour {y} in row {x}"
    return -2, f"row {x} not ascending"


def test_validation_of_corrupted_large_graphs(lib):
    # more than 2^20 entries (the checks run in threads, with a branch-free
    # pass per row and the entry-by-entry checks on a failing row): random
    # corruptions, one or two rows at a time, give the first failure in row
    # order with its code and message
    import graphgen
    rp0, ci0 = graphgen.er(20000, 0.003, 5)
    assert len(ci0) > (1 << 20)
    n = len(rp0) - 1
    rng = np.random.default_rng(11)
    deg = np.diff(rp0)
    rows_ok = np.flatnonzero(deg >= 3)

    def corrupt(ci, kind):
        x = int(rng.choice(rows_ok))
        b, e = int(rp0[x]), int(rp0[x + 1])
        p = int(rng.integers(b + 1, e - 1))
        if kind == 0:
            ci[p] = n + int(rng.integers(0, 5))
        elif kind == 1:
            ci[p] = -1 - int(rng.integers(0, 5))
        elif kind == 2:
            ci[p] = x
        elif kind == 3:
            ci[p] = ci[p - 1]
        else:
            ci[p], ci[p + 1] = ci[p + 1], ci[p]

    for trial in range(24):
        ci = ci0.copy()
        corrupt(ci, trial % 5)
        if trial % 3 == 0:
            corrupt(ci, int(rng.integers(0, 5)))
        want = _first_violation(rp0, ci)
        assert want is not None
        with pytest.raises(gcb.GcError) as ei:
            gcb.gc_graph_upload(rp0, ci)
        assert ei.value.status == want[0], (trial, str(ei.value), want)
        assert str(ei.value).endswith(want[1]), (trial, str(ei.value), want)


def _first_without_reverse(rp, ci):
    """The first entry (x, y) in row order whose reverse (y, x) is absent, or
    None (numpy, on a graph that passes the linear checks)."""
    n = len(rp) - 1
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    key = rows * n + ci.astype(np.int64)           # (x, y), ascending in row order
    rev = ci.astype(np.int64) * n + rows           # (y, x)
    pos = np.searchsorted(key, rev)
    present = (pos < len(key)) & (key[np.minimum(pos, len(key) - 1)] == rev)
    bad = np.flatnonzero(~present)
    return None if len(bad) == 0 else (int(rows[bad[0]]), int(ci[bad[0]]))


@pytest.mark.parametrize("n,p,seed", [(300, 0.1, 1), (20000, 0.003, 5)])
def test_validate_csr_names_the_first_failing_entry(lib, n, p, seed):
    # gc_validate_csr on corrupted graphs below 2^20 entries (the checks of a
    # bulk submission's graphs) and above (the threaded checks of an upload):
    # the code and message of the first failing entry in row order; for an
    # asymmetric graph, the first entry whose reverse is absent -- also where
    # an extra entry of another row shifts a walk's alignment
    import graphgen
    rp0, ci0 = graphgen.er(n, p, seed)
    assert (len(ci0) < (1 << 20)) == (n == 300)
    gcb.gc_validate_csr(rp0, ci0)
    rng = np.random.default_rng(seed)
    deg = np.diff(rp0)
    rows_ok = np.flatnonzero(deg >= 3)

    def drop(rp, ci, x, k):
        """row x without its entry k (row pointers shifted)."""
        ci = np.delete(ci, rp[x] + k)
        rp = rp.copy()
        rp[x + 1:] -= 1
        return rp, ci

    for trial in range(30):
        rp, ci = rp0.copy(), ci0.copy()
        kind = trial % 3
        if kind == 0:    # two entries dropped: their reverses left alone
            for _ in range(2):
                x = int(rng.choice(rows_ok))
                rp, ci = drop(rp, ci, x, int(rng.integers(0, rp[x + 1] - rp[x])))
        elif kind == 1:  # an entry moved to an absent column between its neighbours
            x = int(rng.choice(rows_ok))
            b, e = int(rp[x]), int(rp[x + 1])
            k = int(rng.integers(b + 1, e - 1))
            free = [y for y in range(int(ci[k - 1]) + 1, int(ci[k + 1])) if y != x and y != ci[k]]
            if not free:
                continue
            ci[k] = int(rng.choice(free))
        else:            # a linear violation (range, self-loop, duplicate, order)
            x = int(rng.choice(rows_ok))
            k = int(rng.integers(rp[x] + 1, rp[x + 1] - 1))
            v = trial % 4
            if v == 0:
                ci[k] = n + 3
            elif v == 1:
                ci[k] = x
            elif v == 2:
                ci[k] = ci[k - 1]
            else:
                ci[k], ci[k + 1] = ci[k + 1], ci[k]
        want = _first_violation(rp, ci)
        if want is None and rp[-1] % 2:
            want = (-5, "row_ptr[n] is odd: the graph cannot be symmetric")
        if want is None:
            e = _first_without_reverse(rp, ci)
            want = None if e is None else (-5, f"edge ({e[0]},{e[1]}) has no reverse")
        if want is None:
            gcb.gc_validate_csr(rp, ci)
            continue
        with pytest.raises(gcb.GcError) as ei:
            gcb.gc_validate_csr(rp, ci)
        assert ei.value.status == want[0], (trial, str(ei.value), want)
        assert str(ei.value).endswith(want[1]), (trial, str(ei.value), want)


def test_validate_csr_extra_entry_names_the_entry_without_reverse(lib):
    # rows 0:{1,3} 1:{0,2} 2:{0,1} 3:{0,1}: (2,0) and (3,1) have no reverse,
    # (2,0) first in row order. Matching row 2's lower part in order, (1,2)
    # meets the slot of the extra entry 0 first, though (2,1) exists: the
    # message names the entry that really lacks its reverse.
    rp = np.array([0, 2, 4, 6, 8], np.int32)
    ci = np.array([1, 3, 0, 2, 0, 1, 0, 1], np.int32)
    assert _first_without_reverse(rp, ci) == (2, 0)
    with pytest.raises(gcb.GcError) as ei:
        gcb.gc_validate_csr(rp, ci)
    assert ei.value.status == -5 and str(ei.value).endswith("edge (2,0) has no reverse")
    # an odd number of entries is refused before any walk
    with pytest.raises(gcb.GcError) as ei:
        gcb.gc_validate_csr(np.array([0, 1, 2, 3], np.int32), np.array([1, 2, 1], np.int32))
    assert ei.value.status == -5 and str(ei.value).endswith("row_ptr[n] is odd: the graph cannot be symmetric")
