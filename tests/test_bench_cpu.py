"""Host-side pieces of bench.py (no GPU): the committed ncu traffic record is
used only while the render kernels' sources match it, the peak table is read
with its provenance, and the workloads name what their lines claim."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_record_is_used_for_matching_sources(tmp_path, monkeypatch):
    """A record taken on the current render sources is reported for its
    workload and batch size only."""
    sys.path.insert(0, os.path.join(ROOT, "paper_2412_10084_gb300"))
    import build as _b
    rec = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))
    rec["render_digest"] = _b.render_digest()
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "dram_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    w = rec["object256"]
    got = bench.captured_traffic("object256", "render_backward_kernel", w["rays"])
    assert got == w["render_backward_kernel"]["read"] + w["render_backward_kernel"]["write"]
    # another batch size or workload has no record
    assert bench.captured_traffic("object256", "render_backward_kernel", 12345) is None
    assert bench.captured_traffic("human384", "render_backward_kernel", w["rays"]) is None


def test_traffic_record_is_ignored_for_other_sources(tmp_path, monkeypatch):
    rec = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))
    rec["render_digest"] = "0" * 64
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "dram_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the build module is still found beside the real package
    monkeypatch.syspath_prepend(os.path.join(ROOT, "paper_2412_10084_gb300"))
    assert bench.captured_traffic("object256", "render_backward_kernel",
                                  rec["object256"]["rays"]) is None


def test_algorithmic_bytes_per_sample():
    # FP32 node records: 8 x 16 B gathered, 8 x 16 B of gradient read and written
    assert bench.bytes_per_sample("f32") == (128, 384)
    # BF16 features: 8 x (4 + 6) B gathered
    assert bench.bytes_per_sample("bf16") == (80, 336)
    # tile tri-planes: the SDF array only (the planes stay in L2)
    assert bench.bytes_per_sample("f32", triplane=True) == (32, 96)


def test_workloads_state_their_shapes():
    for name, wl in bench.WORKLOADS.items():
        assert wl["desc"] and wl["dtype"]
    assert bench.WORKLOADS["object1024_sparse"]["R"] == 1024
    assert bench.INFER_METRIC.startswith("ms per 1080p frame")
