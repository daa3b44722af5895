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
