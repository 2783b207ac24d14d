"""Host logic of bench.py's committed traffic record (no GPU): the record is keyed on
the step kernels' code, so rewording a comment keeps it while any change of code voids
it."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_comments_and_blank_lines_do_not_change_the_code_key():
    a = "int f(int x) {\n  return x + 1;  // one more\n}\n"
    b = "/* a block\n   comment */\nint f(int x) {\n\n  return x + 1;\n}   \n// trailing\n"
    assert bench._code_only(a) == bench._code_only(b)


def test_a_change_of_code_changes_the_code_key():
    a = "int f(int x) {\n  return x + 1;  // one more\n}\n"
    c = "int f(int x) {\n  return x + 2;  // one more\n}\n"
    assert bench._code_only(a) != bench._code_only(c)


def test_traffic_record_is_reported_only_for_the_code_it_was_taken_from(monkeypatch):
    """profiles/ncu_traffic.json holds the DRAM bytes per launch of the dominant kernels at
    full size; bench.py reports them only while the kernels' code is the one they were
    taken from (else the roofline's `traffic` is null)."""
    import json
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
        rec = json.load(f)
    for k in ("collide_move", "scatter_spans"):
        t = rec["kernels"][k]["dram_bytes_per_launch_full_size"]
        # both kernels move about their algorithmic 32 B per particle of the 5e7 workload
        assert 0.9 * 32 * 5e7 < t < 1.1 * 32 * 5e7, (k, t)
    monkeypatch.setattr(bench, "sources_hash", lambda: rec["sources_sha256"])
    assert bench.ncu_traffic("collide_move") == rec["kernels"]["collide_move"][
        "dram_bytes_per_launch_full_size"]
    monkeypatch.setattr(bench, "sources_hash", lambda: "0" * 64)
    assert bench.ncu_traffic("collide_move") is None
