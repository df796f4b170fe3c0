"""Autotuner selection logic, coordinate descent and cache, without a GPU
(the timers are stand-ins)."""
import json

import numpy as np
import pytest

from paper_1611_06115_gb300 import _native as N
from paper_1611_06115_gb300 import tune


class FakeText:
    n = 3_100_000_000


def test_valid_variants_follow_the_k_limits():
    assert tune.valid_variants(0) == [N.PM_VARIANT_WINDOW_SLICED, N.PM_VARIANT_PATTERN_SLICED,
                                      N.PM_VARIANT_PATTERN_SLICED_2, N.PM_VARIANT_ALL_CHUNKS]
    assert N.PM_VARIANT_WINDOW_SLICED in tune.valid_variants(8)
    assert N.PM_VARIANT_WINDOW_SLICED not in tune.valid_variants(9)
    assert tune.valid_variants(32) == [N.PM_VARIANT_PATTERN_SLICED_2, N.PM_VARIANT_ALL_CHUNKS]
    assert tune.valid_variants(64) == [N.PM_VARIANT_ALL_CHUNKS]


def model_times(ks):
    """A stand-in cost model shaped like the measured one."""
    out = {}
    for k in ks:
        t = {}
        for v in tune.valid_variants(k):
            if v == N.PM_VARIANT_WINDOW_SLICED:
                t[v] = 0.35 + 0.15 * k
            elif v == N.PM_VARIANT_PATTERN_SLICED:
                t[v] = 1.1 + (0.0 if k <= 16 else 0.6 * (k - 16))
            elif v == N.PM_VARIANT_PATTERN_SLICED_2:
                t[v] = 2.05 + (0.0 if k <= 36 else 0.8 * (k - 36))
            else:
                t[v] = 1.8 if k <= 12 else (3.1 if k <= 31 else 4.5)
        out[k] = t
    return out


def test_tune_variants_selects_fastest_and_caches(tmp_path):
    path = str(tmp_path / "tune.json")
    r = tune.tune_variants(FakeText(), kmax=64, cache=path, timer=model_times, install=False)
    table = r["table"]
    assert not r["cached"] and len(table) == 64
    assert table[:5] == [N.PM_VARIANT_WINDOW_SLICED] * 5
    assert table[5:17] == [N.PM_VARIANT_PATTERN_SLICED] * 12
    assert table[18] == N.PM_VARIANT_PATTERN_SLICED_2
    assert table[40] == N.PM_VARIANT_ALL_CHUNKS and table[63] == N.PM_VARIANT_ALL_CHUNKS
    for k, v in enumerate(table):
        assert v in tune.valid_variants(k)
    # the second call reads the cache and measures nothing
    def boom(ks):
        raise AssertionError("measured again")
    r2 = tune.tune_variants(FakeText(), kmax=64, cache=path, timer=boom, install=False)
    assert r2["cached"] and r2["table"] == table
    data = json.load(open(path))
    assert r["key"] in data and data[r["key"]]["table"] == table
    # retune measures again
    r3 = tune.tune_variants(FakeText(), kmax=20, cache=path, timer=model_times, install=False, retune=True)
    assert not r3["cached"] and r3["table"] == table[:20]


def test_select_variants_rejects_invalid_choice():
    with pytest.raises(ValueError):
        tune.select_variants({0: {N.PM_VARIANT_WINDOW_SLICED: 1.0}, 1: {N.PM_VARIANT_AUTO: 0.5}})


def test_coordinate_descent_finds_separable_minimum():
    want = {"ws_below": 3, "ps1_below": 21, "ps2_below": 45, "tiles": 2, "grid": 0}
    calls = []

    def timer(o):
        calls.append(o)
        return 1.0 + sum(abs(o[name] - want[name]) / (1 + want[name]) for name in want)

    best, t, log = tune.coordinate_descent(timer)
    assert best == want and abs(t - 1.0) < 1e-12
    # every candidate timed once
    keys = [tuple(sorted(o.items())) for o, _ in log]
    assert len(keys) == len(set(keys)) == len(calls)


def test_tune_batch_caches_by_workload_shape(tmp_path):
    path = str(tmp_path / "tune.json")

    class P:
        def __init__(self, m):
            self.m = m

    rng = np.random.default_rng(0)
    pats = [P(int(m)) for m in rng.integers(12, 512, 300)]
    ks = [int(x) for x in rng.integers(0, 40, 300)]
    timer = lambda o: 1.0 + 0.1 * abs(o["tiles"] - 4) + 0.01 * abs(o["ws_below"] - 7)
    r = tune.tune_batch(FakeText(), pats, ks, 1000, cache=path, timer=timer)
    assert not r["cached"] and r["options"]["tiles"] == 4 and r["options"]["ws_below"] == 7
    r2 = tune.tune_batch(FakeText(), pats, ks, 1000, cache=path, timer=lambda o: 1 / 0)
    assert r2["cached"] and r2["options"] == r["options"]
    # another shape of batch is another key
    r3 = tune.tune_batch(FakeText(), pats[:10], ks[:10], 1000, cache=path, timer=timer)
    assert r3["key"] != r["key"] and not r3["cached"]


def test_sample_batch_is_stratified_and_bounded():
    pats = ["A" * m for m in range(10, 1010)]
    ks = [m % 50 for m in range(10, 1010)]
    idx = tune.sample_batch(pats, ks, 100)
    assert len(idx) == 100 and len(set(idx)) == 100
    sk = sorted(ks[i] for i in idx)
    assert sk[0] == 0 and sk[-1] == 49
    assert tune.sample_batch(pats[:5], ks[:5], 100) == sorted(range(5), key=lambda i: (ks[i], len(pats[i])))


def test_probe_pattern_class_fraction():
    rng = np.random.default_rng(1)
    p = tune.probe_pattern(1000, rng)
    assert len(p) == 1000
    assert sum(c not in "ACGT" for c in p) == 100


def test_tune_batch_keeps_defaults_when_the_whole_batch_disagrees(tmp_path):
    """A sample can favour options that lose on the whole batch: the winner is
    timed on the whole batch against the defaults and the faster is kept."""
    class P:
        def __init__(self, m):
            self.m = m
    pats = [P(100)] * 50
    ks = [3] * 50
    sample_timer = lambda o: 1.0 - 0.1 * (o["tiles"] == 4)
    full_lose = lambda o: 2.0 if o["tiles"] == 4 else 1.5
    r = tune.tune_batch(FakeText(), pats, ks, 100, cache=str(tmp_path / "a.json"), timer=sample_timer,
                        full_timer=full_lose)
    assert r["options"] == tune.BATCH_DEFAULTS and r["checked"]["default_ms"] == 1.5
    full_win = lambda o: 1.0 if o["tiles"] == 4 else 1.5
    r = tune.tune_batch(FakeText(), pats, ks, 100, cache=str(tmp_path / "b.json"), timer=sample_timer,
                        full_timer=full_win)
    assert r["options"]["tiles"] == 4 and r["checked"]["tuned_ms"] == 1.0

