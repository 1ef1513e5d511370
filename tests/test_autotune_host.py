"""Host logic of the batched form's autotuner, on the CPU: member batches
concatenated with their offsets, the size-stratified sample, and the
coordinate descent with its cache, timed by a stand-in cost function."""
import numpy as np
import pytest

from paper_2306_08252_gb300 import autotune


def _members(rng, G):
    ms = []
    for _ in range(G):
        nv = int(rng.integers(10, 5000))
        mk = lambda k: (rng.integers(0, nv, k).astype(np.uint32), rng.integers(0, nv, k).astype(np.uint32))
        ms.append({"nv": nv, "bulk": mk(int(rng.integers(0, 50))), "insert": mk(int(rng.integers(0, 20))),
                   "delete": mk(int(rng.integers(0, 20)))})
    return ms


def test_concat_member_batches():
    rng = np.random.default_rng(1)
    ms = _members(rng, 7)
    s, d, off = autotune.concat_member_batches(ms, "insert")
    assert off[0] == 0 and off[-1] == s.size == d.size
    for i, m in enumerate(ms):
        np.testing.assert_array_equal(s[off[i]:off[i + 1]], m["insert"][0])
        np.testing.assert_array_equal(d[off[i]:off[i + 1]], m["insert"][1])


def test_sample_members_spans_sizes():
    rng = np.random.default_rng(2)
    ms = _members(rng, 100)
    sub = autotune.sample_members(ms, 10)
    assert len(sub) == 10
    sizes = sorted(m["nv"] for m in ms)
    got = [m["nv"] for m in sub]
    assert got == sorted(got) and got[0] == sizes[0] and got[-1] >= sizes[89]
    assert autotune.sample_members(ms[:5], 10) == ms[:5]


def test_coordinate_descent_and_cache(tmp_path, monkeypatch):
    torch = pytest.importorskip("torch")
    calls = []
    best = {"block_capacity": 16, "item_blocks": 16, "dense_shift": 1}

    def cost(members, cfg, reps):
        calls.append(dict(cfg))
        # separable bowl around `best` (coordinate descent finds its minimum)
        return 1.0 + sum(abs(np.log2(cfg[k]) - np.log2(best[k])) for k in best)

    monkeypatch.setattr(autotune, "_time_config", cost)
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "test-device")
    cache = str(tmp_path / "tune.json")
    ms = _members(np.random.default_rng(3), 40)
    got = autotune.tune_set(ms, sample=8, reps=1, cache=cache)
    assert {k: got[k] for k in best} == best and got["cached"] is False
    # every timed configuration obeyed the slot limit of a work item
    assert all(c["item_blocks"] <= min(32, 512 // c["block_capacity"]) for c in calls)
    n = len(calls)
    again = autotune.tune_set(ms, sample=8, reps=1, cache=cache)
    assert again["cached"] is True and len(calls) == n  # served from the cache
    fresh = autotune.tune_set(ms, sample=8, reps=1, cache=cache, refresh=True)
    assert fresh["cached"] is False and len(calls) > n
