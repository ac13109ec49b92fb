"""The benchmark's per-launch DRAM traffic (`bench.transform_traffic`): the ncu
figures in profiles/transform_traffic.json are used only while the transform
section of the kernel source is the one that was profiled (its SHA-1 matches);
any other state of the file reads as "no figure" (null in the JSON line)."""
import json
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _with_file(monkeypatch, tmp_path, text):
    p = tmp_path / "traffic.json"
    p.write_text(text)
    monkeypatch.setattr(bench, "TRAFFIC_JSON", str(p))


def test_record_used_when_the_source_matches(monkeypatch, tmp_path):
    rec = {"dram_bytes_per_launch": 123, "transform_source_sha1": bench.transform_source_sha1()}
    _with_file(monkeypatch, tmp_path, json.dumps({"w": rec}))
    assert bench.transform_traffic("w") == rec
    assert bench.transform_traffic("other") is None


def test_no_figure_after_a_source_change_or_a_bad_file(monkeypatch, tmp_path):
    stale = {"dram_bytes_per_launch": 123, "transform_source_sha1": "0" * 40}
    _with_file(monkeypatch, tmp_path, json.dumps({"w": stale}))
    assert bench.transform_traffic("w") is None
    _with_file(monkeypatch, tmp_path, "{ not json")
    assert bench.transform_traffic("w") is None
    monkeypatch.setattr(bench, "TRAFFIC_JSON", str(tmp_path / "missing.json"))
    assert bench.transform_traffic("w") is None


def test_source_hash_is_a_stable_sha1():
    h = bench.transform_source_sha1()
    assert re.fullmatch(r"[0-9a-f]{40}", h)
    assert bench.transform_source_sha1() == h   # stable


def test_committed_900hz_figure_is_the_pair_capture_scaled_to_a_launch():
    """The 64-direction step's launches hold 32 directions (16 pairs) on
    average; the committed figure is 16 x the bytes of the one-pair capture
    that its note names."""
    recs = json.load(open(os.path.join(ROOT, "profiles", "transform_traffic.json")))
    rec = recs["highfreq_T1024_1yr_900Hz_64dir"]
    pair = int(re.search(r"one pair, (\d+) bytes", rec["how"]).group(1))
    assert rec["dram_bytes_per_launch"] == 16 * pair
    for r in recs.values():
        assert r["dram_bytes_per_launch"] > 0
        assert re.fullmatch(r"[0-9a-f]{40}", r["transform_source_sha1"])
