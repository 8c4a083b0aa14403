"""The mixed-batch tile recipe: counts, orders, parameter ranges, clipping, determinism (CPU)."""
import collections
import math

from paper_2608_25203_b300 import seas


def test_batch_recipe():
    T = seas.batch_tiles()
    assert len(T) == 96
    c = collections.Counter(t["nx"] for t in T)
    assert c == {128: 40, 256: 32, 512: 16, 1024: 8}
    per = collections.Counter((t["nx"], t["M"]) for t in T)
    assert per[(128, 3)] == per[(128, 6)] == 10 and per[(1024, 4)] == 2
    for t in T:
        assert t["nx"] == t["nz"] and abs(t["Lx"] / t["nx"] - 0.78125) < 1e-12
        assert 10 <= t["h"] <= 100 and 6 <= t["Tp"] <= 12 and 0 < t["Hs"] <= 4
        kref = max(seas.peak_wavenumber(t["Tp"], t["h"]), 2 * math.pi / t["Lx"])
        assert kref * t["Hs"] / 2 <= 0.1 + 1e-12
    assert [t["seed"] for t in T] == list(range(1000, 1096))
    assert seas.batch_tiles() == T
