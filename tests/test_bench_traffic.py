"""bench.py's use of the committed DRAM counters: the pass-C bytes of
profiles/roofline_traffic_rmat20.txt are reported only for the workload they
were taken on (R-MAT scale 20) and only while the kernel sources have the
SHA-256 digests the file records."""
import os
import shutil

import bench


def test_counters_used_for_their_own_workload_only():
    v = bench.measured_traffic("pass_c_cycles", "rmat22", bench.TRAFFIC_SCALE)
    assert isinstance(v, int) and v > 0
    assert bench.measured_traffic("pass_c_cycles", "rmat22", 22) is None
    assert bench.measured_traffic("pass_c_cycles", "chung_lu", bench.TRAFFIC_SCALE) is None
    assert bench.measured_traffic("no_such_phase", "rmat22", bench.TRAFFIC_SCALE) is None


def test_counters_dropped_when_a_kernel_source_changes(tmp_path, monkeypatch):
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    shutil.copy(os.path.join(bench.ROOT, bench.TRAFFIC_FILE), root / bench.TRAFFIC_FILE)
    src = root / "paper_1608_05138_gb300" / "csrc"
    src.mkdir(parents=True)
    names = [line.split()[1] for line in open(root / bench.TRAFFIC_FILE) if line.startswith("source ")]
    assert len(names) >= 4
    for f in names:
        shutil.copy(os.path.join(bench.ROOT, "paper_1608_05138_gb300", "csrc", f), src / f)
    monkeypatch.setattr(bench, "ROOT", str(root))
    want = bench.measured_traffic("pass_c_cycles", "rmat22", bench.TRAFFIC_SCALE)
    assert want is not None
    with open(src / names[0], "a") as fh:  # a one-byte edit, even outside the code
        fh.write("\n")
    assert bench.measured_traffic("pass_c_cycles", "rmat22", bench.TRAFFIC_SCALE) is None
    (src / names[0]).unlink()
    assert bench.measured_traffic("pass_c_cycles", "rmat22", bench.TRAFFIC_SCALE) is None
