"""Host logic of bench.py that needs no GPU: the recorded DRAM traffic of a kernel is
reported only while the sources it was captured on are unchanged."""

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _tree(tmp_path):
    csrc = tmp_path / "paper_1607_04245_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES["lap"]:
        (csrc / f).write_text(f"// {f}\n")
    (tmp_path / "profiles").mkdir()
    return csrc


def test_recorded_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    csrc = _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.src_hash(bench.KERNEL_SOURCES["lap"])
    (tmp_path / "profiles" / "dram_traffic.txt").write_text(
        f"other src={h} bytes=1\nlap3d_mixed src={h} bytes=59903232 read=1 write=2 note=x\n")
    assert bench.recorded_traffic("lap3d_mixed") == 59903232.0
    assert bench.recorded_traffic("missing") is None
    # any edit of a listed source invalidates the record
    f = csrc / bench.KERNEL_SOURCES["lap"][-1]
    f.write_text(f.read_text() + "// edited\n")
    assert bench.src_hash(bench.KERNEL_SOURCES["lap"]) != h
    assert bench.recorded_traffic("lap3d_mixed") is None


def test_recorded_traffic_without_a_summary(tmp_path, monkeypatch):
    _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("lap3d_mixed") is None


def test_committed_record_names_the_headline_kernel():
    """The committed summary has a line for the headline kernel with a source hash and a
    byte count (it is reported by the bench only while that hash is current)."""
    lines = open(os.path.join(ROOT, "profiles", "dram_traffic.txt")).read().split("\n")
    rec = [ln for ln in lines if ln.startswith("lap3d_mixed ")]
    assert len(rec) == 1
    kv = dict(x.split("=", 1) for x in rec[0].split()[1:])
    assert len(kv["src"]) == 16 and int(kv["bytes"]) == int(kv["read"]) + int(kv["write"])


def test_rotating_copies_keep_each_step_out_of_the_l2():
    """The timed steps cycle through input copies: between two uses of one copy the other
    copies move at least 3 L2 sizes; too small a workload (over 128 copies) is timed with
    a flush instead (None)."""
    l2 = 126 << 20
    for set_bytes in (83_186_972, 135 << 20, 3 << 20, 1 << 30):
        n = bench.rotating_sets(set_bytes, l2)
        assert n is not None and n >= 2
        assert (n - 1) * set_bytes >= bench.ROTATE_L2_MULT * l2
        assert n == 2 or (n - 2) * set_bytes < bench.ROTATE_L2_MULT * l2  # no more copies than needed
    assert bench.rotating_sets(83_186_972, l2) == 6
    assert bench.rotating_sets(600_000, l2) is None
