"""Host-side logic of bench.py that needs no GPU: the recorded DRAM traffic
is used only for the walk-kernel source it was measured on, and the digest
that keys it ignores comments and layout but not code."""
import os

import bench
from paper_2512_00705_gb300 import _build


def _traffic_file(tmp_path, digest, values=(164.0, 273.0, 473.0)):
    p = tmp_path / "traffic.md"
    p.write_text("# traffic\n\n"
                 f"- source_digest: {digest}\n"
                 f"- dram_bytes_per_hop_p1_q1: {values[0]}\n"
                 f"- dram_bytes_per_hop_p4_q0.25: {values[1]}\n"
                 f"- dram_bytes_per_hop_p0.25_q4: {values[2]}\n")
    return str(p)


def test_traffic_used_only_for_the_recorded_source(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "TRAFFIC_FILE", _traffic_file(tmp_path, bench.source_digest()))
    t = bench.read_traffic()
    assert t == {(1.0, 1.0): 164.0, (4.0, 0.25): 273.0, (0.25, 4.0): 473.0}
    monkeypatch.setattr(bench, "TRAFFIC_FILE", _traffic_file(tmp_path, "0" * 16))
    assert bench.read_traffic() is None
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.md"))
    assert bench.read_traffic() is None


def test_traffic_file_with_a_missing_value_is_not_used(tmp_path, monkeypatch):
    p = tmp_path / "traffic.md"
    p.write_text(f"- source_digest: {bench.source_digest()}\n- dram_bytes_per_hop_p1_q1: 164.0\n")
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(p))
    assert bench.read_traffic() is None


def test_committed_traffic_file_names_a_digest_and_three_values():
    txt = open(bench.TRAFFIC_FILE).read()
    assert "source_digest:" in txt
    for key in ("p1_q1", "p4_q0.25", "p0.25_q4"):
        assert f"dram_bytes_per_hop_{key}:" in txt


def test_digest_ignores_comments_and_layout_but_not_code():
    src = "int f(int x) {\n  return x + 1;  // add one\n}\n/* block\n comment */\n"
    same = "int f(int x) { return x + 1; }\n"
    other = "int f(int x) { return x + 2; }\n"
    assert _build._code_only(src) == _build._code_only(same)
    assert _build._code_only(src) != _build._code_only(other)


def test_digest_covers_the_walk_kernel_sources():
    for f in _build.WALK_KERNEL_FILES:
        assert os.path.exists(os.path.join(_build.CSRC, f)), f
    assert len(bench.source_digest()) == 16
