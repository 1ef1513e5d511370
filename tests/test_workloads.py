"""The seeded generators: determinism, ranges and distribution shape."""
import numpy as np

import workloads as W


def test_xoshiro_deterministic_and_stream_separated():
    a = W.raw(1, 0, 1000)
    b = W.raw(1, 0, 1000)
    c = W.raw(1, 1, 1000)
    np.testing.assert_array_equal(a, b)
    assert (a != c).mean() > 0.99
    # roughly uniform bits
    bits = np.unpackbits(a.view(np.uint8))
    assert abs(bits.mean() - 0.5) < 0.01


def test_uniform_pairs_range():
    s, d = W.uniform_pairs(3, 0, 100_000, 1000, lo=5)
    assert s.min() >= 5 and s.max() < 1005 and d.min() >= 5 and d.max() < 1005
    h = np.bincount(s - 5, minlength=1000)
    assert h.min() > 50 and h.max() < 160


def test_rmat_bit_marginals():
    # Each bit level draws a quadrant: P(src bit = 1) = c + d, P(dst bit = 1) = b + d.
    a, b, c, d = W.RMAT_ABCD
    s, t = W.rmat_pairs(2, 0, 200_000, 12)
    assert s.max() < 4096 and t.max() < 4096
    for lvl in range(12):
        sb = ((s >> lvl) & 1).mean()
        tb = ((t >> lvl) & 1).mean()
        assert abs(sb - (c + d)) < 0.01
        assert abs(tb - (b + d)) < 0.01
    both = (((s & 1) == 1) & ((t & 1) == 1)).mean()
    assert abs(both - d) < 0.01


def test_rmat_limit_redraws():
    s, t = W.rmat_pairs(4, 0, 10_000, 10, limit=700)
    assert s.max() < 700 and t.max() < 700


def test_shuffle_is_permutation():
    x = np.arange(1000, dtype=np.uint32)
    y = W.shuffled(5, 0, x)
    assert not np.array_equal(x, y)
    np.testing.assert_array_equal(np.sort(y), x)


def test_tiny_config_shape():
    cfg = W.tiny_uniform()
    assert cfg["nv"] == 1024 and cfg["bulk"][0].size == 8192
    assert len(cfg["ops"]) == 20
    seen = set(zip(*[a.tolist() for a in cfg["bulk"]]))
    base = set(seen)
    for op in cfg["ops"]:
        if op.kind == "insert":
            assert len(op) == 1024
            seen |= set(zip(op.src.tolist(), op.dst.tolist()))
        else:
            pairs = list(zip(op.src.tolist(), op.dst.tolist()))
            assert len(pairs) == 1024
            existing = [p for p in pairs if p in base]
            absent = [p for p in pairs if p not in seen]
            assert len(existing) == 512 and len(absent) == 512


def test_unique_and_membership_helpers_match_numpy():
    rng = np.random.default_rng(3)
    for n in (0, 1, 7, 5000):
        a = rng.integers(0, 900, n).astype(np.uint64)
        np.testing.assert_array_equal(W.unique_sorted(a), np.unique(a))
        b = rng.integers(0, 1200, 2000).astype(np.uint64)
        np.testing.assert_array_equal(W.in_sorted(b, W.unique_sorted(a)), np.isin(b, a))
