"""The width-tuning cache (host logic, no GPU): a graph's policy is tuned once
per GPU name and graph class and read back from the JSON cache afterwards."""
import json

import paper_1708_01159_gb300 as bfs


def test_cache_miss_tunes_and_hit_sets(tmp_path, monkeypatch):
    calls = {"tune": 0, "set": []}

    def fake_tune(g, roots, stream=None):
        calls["tune"] += 1
        return {"policy": 3, "name": "w4", "ms": {w: 1.0 + i for i, w in enumerate(bfs.WARP_WIDTHS)}}

    monkeypatch.setattr(bfs, "bfs_tune_warp_width", fake_tune)
    monkeypatch.setattr(bfs, "bfs_set_warp_width", lambda g, p: calls["set"].append(p))
    info = {"n": 100, "m": 400, "deg_summary": [1, 2, 4, 6, 9]}
    path = str(tmp_path / "vw.json")
    r1 = bfs.tune_warp_width_cached(7, [0, 1], path, "GB300", info)
    assert r1["cached"] is False and r1["policy"] == 3 and calls["tune"] == 1 and calls["set"] == []
    key = bfs.warp_width_cache_key("GB300", info)
    assert json.load(open(path))[key]["policy"] == 3
    r2 = bfs.tune_warp_width_cached(7, [0, 1], path, "GB300", info)
    assert r2["cached"] is True and calls["tune"] == 1 and calls["set"] == [3]
    # another graph class or another GPU tunes again
    bfs.tune_warp_width_cached(7, [0], path, "GB300", dict(info, m=402))
    bfs.tune_warp_width_cached(7, [0], path, "B200", info)
    assert calls["tune"] == 3 and len(json.load(open(path))) == 3
