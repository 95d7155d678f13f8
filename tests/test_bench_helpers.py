"""The benchmark's bookkeeping on CPU: algorithmic bytes of the operator kernel (every energy
evaluation reads the reference and template level once: 2 s P_l bytes), and the hash gate that
keeps a stale ncu traffic figure out of the JSON line."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_algorithmic_bytes_counts_two_levels_per_evaluation():
    stats = [{"evals": [10, 4]}, {"evals": [3, 0]}]
    # 512^2 at level 0 and 256^2 at level 1, fp32 (4 bytes)
    want = (10 + 3) * 2 * 4 * 512 * 512 + 4 * 2 * 4 * 256 * 256
    assert bench.algorithmic_bytes(stats, 512, 512, 2, 4, "rigid") == want
    # odd sizes round the coarser level up, 2-byte storage halves the bytes
    assert bench.algorithmic_bytes([{"evals": [1, 1]}], 5, 7, 2, 2, "rigid") == 2 * 2 * 35 + 2 * 2 * 12


def test_pyramid_bytes_by_hand():
    # rigid, fp32, 2 levels of 4 x 6: frame read 4*24, levels 4*24 + 4*6 (2 x 3) written
    assert bench.pyramid_bytes(1, 4, 6, 2, 4, "rigid") == 4 * 24 + 4 * 24 + 4 * 6
    # nonrigid, 2-byte storage, one level of 5 x 7 on 3 frames: frame read 4*35, the level with its
    # 3-sample border (11 x 13) and the model at the pixel centres (5 x 7) written
    assert bench.pyramid_bytes(3, 5, 7, 1, 2, "nonrigid") == 3 * (4 * 35 + 2 * 11 * 13 + 2 * 35)
    # odd sizes round the coarser level up: 5 x 7 -> 3 x 4
    assert bench.pyramid_bytes(1, 5, 7, 2, 4, "rigid") == 4 * 35 + 4 * 35 + 4 * 12


def test_profile_traffic_is_used_only_for_the_profiled_source(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    src = tmp_path / "paper_2010_12478_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "k.cu").write_text("kernel v1")
    (tmp_path / "profiles").mkdir()
    h = bench.kernel_hash("k.cu")
    (tmp_path / "profiles" / "p.md").write_text(f"kernel source sha256: {h}\ndram bytes per call (scaled): 1.5e8\n")
    assert bench.profile_traffic("p", "k.cu", "dram bytes per call (scaled)") == pytest.approx(1.5e8)
    (src / "k.cu").write_text("kernel v2")   # the kernel changed since the capture
    assert bench.profile_traffic("p", "k.cu", "dram bytes per call (scaled)") is None
    assert bench.profile_traffic("missing", "k.cu", "dram bytes per call (scaled)") is None


def test_the_committed_profiles_name_their_command_and_source():
    for name in os.listdir(os.path.join(ROOT, "profiles")):
        text = open(os.path.join(ROOT, "profiles", name)).read()
        assert "kernel source sha256:" in text and "ncu " in text and "--clock-control none" in text, name


def test_imbalance_metric_by_hand():
    # 8 operators with work 1..8 in 2 segments: T = (10, 26), mean 18, imbalance (26 - 18) / 18
    m = bench.imbalance_metric(list(range(1, 9)), [2, 4, 16])
    assert m["segments"]["2"] == pytest.approx(8 / 18, abs=1e-4)
    # 4 segments: T = (3, 7, 11, 15), mean 9
    assert m["segments"]["4"] == pytest.approx(6 / 9, abs=1e-4)
    assert "16" not in m["segments"]            # more segments than operators
    assert bench.imbalance_metric([5] * 12, [3])["segments"]["3"] == 0.0   # equal work: balanced


def test_paper_bounds_formulas():
    # scan: (N-1) / (2N/P - 1 + C1 log2 P); full: (2N-1) / (3N/P - 1 + C1 log2 P)
    b = bench.paper_bounds(4096, 1024, 1.0)
    assert b["scan"] == pytest.approx(4095 / (8 - 1 + 10), abs=0.01)
    assert b["full"] == pytest.approx(8191 / (12 - 1 + 10), abs=0.01)
    one = bench.paper_bounds(16, 1, 1.0)      # one worker: no speedup on either
    assert one["scan"] == pytest.approx(15 / 31, abs=0.01) and one["full"] == pytest.approx(31 / 47, abs=0.01)
