"""Host-side logic that needs no GPU: the serving driver's request plans and
the autotuner table cache (with the two library calls it makes replaced by
fakes)."""
import json
import types

import numpy as np

from paper_2106_12655_gb300 import serving, tuning


def _scenes(sizes):
    out = []
    for k, n in enumerate(sizes):
        pairs = np.stack([np.arange(n, dtype=np.int32), np.arange(n, dtype=np.int32) + 1 + k], 1)
        out.append(types.SimpleNamespace(geometry=types.SimpleNamespace(pairs=pairs)))
    return out


def test_request_plan_windows():
    scenes = _scenes([30_000, 5_000, 800])
    plan = serving.request_plan(scenes, 400, seed=3, min_pairs=1000, max_pairs=20000)
    assert len(plan) == 400
    seen = set()
    for k, window in plan:
        seen.add(k)
        pairs = scenes[k].geometry.pairs
        n = pairs.shape[0]
        m = window.shape[0]
        # log-uniform size in [min, max], clipped to the scene's pair count
        assert min(1000, n) <= m <= min(20000, n)
        assert window.flags["C_CONTIGUOUS"] and window.dtype == np.int32
        # a contiguous slice of the scene's list
        lo = int(np.nonzero(pairs[:, 0] == window[0, 0])[0][0])
        assert np.array_equal(window, pairs[lo:lo + m])
    assert seen == {0, 1, 2}
    again = serving.request_plan(scenes, 400, seed=3, min_pairs=1000, max_pairs=20000)
    assert all(a[0] == b[0] and np.array_equal(a[1], b[1]) for a, b in zip(plan, again))


def test_request_plan_sizes_are_log_uniform():
    scenes = _scenes([10 ** 6])
    sizes = np.array([w.shape[0] for _, w in serving.request_plan(scenes, 4000, seed=1)])
    logs = np.log(sizes)
    # the mean of log-uniform sizes on [1k, 20k] is the midpoint of the logs
    assert abs(logs.mean() - 0.5 * (np.log(1000) + np.log(20000))) < 0.05
    assert sizes.min() >= 1000 and sizes.max() <= 20000


def test_tuning_cache_round_trip(tmp_path, monkeypatch):
    tables = {"ctx-a": np.array([0, 64, 1, 128, 2, 256], np.int32),
              "ctx-b": np.array([0, 32, 1, 32], np.int32)}
    installed = {}
    monkeypatch.setattr(tuning.lk, "lk_tune_get", lambda ctx: tables[ctx])
    monkeypatch.setattr(tuning.lk, "lk_tune_set", lambda ctx, e: installed.__setitem__(ctx, np.array(e)))
    path = str(tmp_path / "tune.json")
    tuning.save("ctx-a", "GB300 A", path)
    tuning.save("ctx-b", "GB300 B", path)
    with open(path) as f:
        data = json.load(f)
    assert sorted(data) == ["GB300 A", "GB300 B"]
    assert tuning.restore("ctx-new", "GB300 A", path)
    assert np.array_equal(installed["ctx-new"], tables["ctx-a"]) and installed["ctx-new"].dtype == np.int32
    assert not tuning.restore("ctx-other", "another GPU", path)
    assert "ctx-other" not in installed
    assert not tuning.restore("ctx-x", "GB300 A", str(tmp_path / "missing.json"))


def test_geometry_plan_whole_pile_requests():
    scenes = _scenes([10, 20, 30, 40])
    plan = serving.geometry_plan(scenes, 500, seed=4)
    assert len(plan) == 500 and all(p is None for _, p in plan)
    ks = np.array([k for k, _ in plan])
    assert set(ks.tolist()) == {0, 1, 2, 3}
    assert np.array_equal(ks, np.array([k for k, _ in serving.geometry_plan(scenes, 500, seed=4)]))


def test_tail_breakdown_separates_queueing_from_size():
    import bench

    rng = np.random.default_rng(0)
    n = 3000
    sps = rng.integers(1, 100, n).astype(np.int64)
    depth = rng.integers(0, 12, n)
    # latency made of queueing only: 1 ms per request ahead, size irrelevant
    lat = (1.0 + depth) * 1e-3
    rec = {"depth": depth, "late": np.zeros(n)}
    t = bench.tail_breakdown(lat, sps, rec)
    assert t["depth_le_2"]["n"] == int(np.sum(depth <= 2)) and t["depth_ge_8"]["n"] == int(np.sum(depth >= 8))
    assert abs(t["depth_le_2"]["p99_ms"] - 3.0) < 1e-9 and abs(t["depth_ge_8"]["p50_ms"] - 10.0) < 1.0 + 1e-9
    assert t["p99_tail_behind_8_or_more"] == 1.0
    assert abs(t["small_third"]["p99_ms"] - t["large_third"]["p99_ms"]) < 1e-9
    assert abs(t["mean_depth"] - depth.mean()) < 1e-12 and t["max_submit_late_ms"] == 0.0
