"""The autotuner's host-side logic (no GPU): per-job parameters from a tuning,
the chosen method's variant and flags, and the JSON cache of tunings."""
import math

import paper_1809_07014_gb300 as pkg
from paper_1809_07014_gb300.tune import METHODS, Tuning, TuningCache


def tuning(**kw):
    base = dict(k=31, words=1, windows=10_000_000, distinct_ratio=0.4, survivor_ratio=0.1, keys_per_leaf=2000.0,
                l1_shift=0, ms_best=1.0, ms_default=1.2)
    base.update(kw)
    return Tuning(**base)


def test_params_size_the_leaves_from_the_distinct_ratio():
    t = tuning()
    for windows in (10_000, 3_000_000, 1_600_000_000):
        p = t.params(windows, min_count=2)
        distinct = max(1, int(0.4 * windows))
        want_bits = min(22, max(1, math.ceil(math.log2(max(2.0, distinct / 2000.0)))))
        assert p["leaf_bits"] == want_bits
        assert p["distinct_hint"] == int(distinct * 1.15) + 1
        assert p["survivors_hint"] == int(0.1 * windows * 1.1) + 1024
        assert p["k"] == 31 and p["min_count"] == 2
        if want_bits <= 11:
            assert p["l1_bits"] == 0
        else:  # two levels: each at most 11 bits, the level 1 near half
            l1 = p["l1_bits"]
            assert 1 <= l1 <= 11 and want_bits - l1 <= 11
    # a level-1 shift moves the split by one bit
    lo = tuning(l1_shift=-1).params(1_600_000_000)["l1_bits"]
    mid = t.params(1_600_000_000)["l1_bits"]
    assert lo == mid - 1


def test_method_params():
    assert tuning().method_params() == {}
    assert tuning(method="gate").method_params() == {"flags": pkg.KMER_FLAG_BLOOM_GATE}
    assert tuning(method="hbm_table").method_params() == {"variant": pkg.KMER_VARIANT_HBM_TABLE}
    assert set(METHODS) == {"partitioned", "gate", "hbm_table"}


def test_cache_round_trip_and_nearest_size_class(tmp_path):
    path = str(tmp_path / "tunings.json")
    c = TuningCache(path)
    small = tuning(windows=2 ** 20, keys_per_leaf=1500.0)
    large = tuning(windows=2 ** 30, keys_per_leaf=2500.0, method="gate", method_ms={"partitioned": 2.0, "gate": 1.5})
    other_k = tuning(k=55, words=2, windows=2 ** 30)
    for t in (small, large, other_k):
        c.put(t)
    again = TuningCache(path)  # read back from the file
    assert again.get(31, 2 ** 21).keys_per_leaf == 1500.0   # nearest class: 20
    assert again.get(31, 2 ** 29).keys_per_leaf == 2500.0   # nearest class: 30
    assert again.get(31, 2 ** 29).method == "gate"
    assert again.get(55, 2 ** 20).k == 55
    assert again.get(21, 2 ** 20) is None
