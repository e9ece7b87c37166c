"""Host-side arithmetic of bench.py's roofline object: the algorithmic bytes
of one k_step launch per fluid node, and the recorded DRAM traffic, which must
turn null as soon as the kernel source it was measured on changes."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("Q,D,moving,contrast,want", [
    (19, 3, 4, True, 260),    # 18*4 pulled + 2*76 written + phi 4 + u_in 12 + u 12 + p 4 + mask 4
    (19, 3, 4, False, 248),   # without the previous velocity's stencil
    (19, 3, 2, True, 152),    # FP16 moving populations: 18*2 + 2*(4 + 36) + 36
    (9, 2, 4, True, 132),     # 8*4 + 2*36 + 4 + 8 + 8 + 4 + 4
    (9, 2, 2, False, 76),     # 8*2 + 2*(4 + 16) + 4 + 8 + 4 + 4
])
def test_k_step_algorithmic_bytes(Q, D, moving, contrast, want):
    """The float step pulls the Q - 1 moving populations of N (no rest
    population: the deviation form takes every moment from the moving ones)
    and writes N* and B* whole (float rest plane)."""
    assert bench.k_step_bytes_per_fluid_node(Q, D, 4, contrast, moving) == want


def test_recorded_traffic_follows_the_kernel_source(monkeypatch, tmp_path):
    rec = {"kernel_hash": "abc", "dram_bytes_per_fluid_node": 250.0,
           "k_step_fp16_storage": {"dram_bytes_per_fluid_node": 150.0}}
    path = tmp_path / "traffic.json"
    path.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "abc")
    assert bench.recorded_traffic(1000) == 250000.0
    assert bench.recorded_traffic(1000, fp16=True) == 150000.0
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "changed")
    assert bench.recorded_traffic(1000) is None
    assert bench.recorded_traffic(1000, fp16=True) is None
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.json"))
    assert bench.recorded_traffic(1000) is None


def test_committed_traffic_record_is_well_formed():
    """Per fluid node, the DRAM bytes of each recorded kernel lie near its
    algorithmic bytes (some reads hit L2, so a little below is expected; far
    above would be wasted re-reads)."""
    with open(bench.TRAFFIC_FILE) as f:
        rec = json.load(f)
    for r in (rec, rec["k_phi"], rec["k_step_fp16_storage"]):
        assert 0.9 <= r["dram_bytes_per_fluid_node"] / r["algorithmic_bytes_per_fluid_node"] <= 1.1
