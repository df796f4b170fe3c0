"""The batched persistent launch: identical to per-pattern searches and to the
oracle, in one launch and under CUDA-graph replay (bit-exact)."""
import numpy as np
import pytest

import oracle
import synth
from synth import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pm():
    import torch
    assert torch.cuda.is_available()
    import paper_1611_06115_gb300 as pm
    pm.lib()
    return pm


def check_against_oracle(res, text, pats, ks):
    h, off = res.numpy()
    for i, (p, k) in enumerate(zip(pats, ks)):
        seg = h[int(off[i]):int(off[i + 1])]
        el, em = oracle.search(text, p, k)
        assert np.array_equal(seg[:, 0], el), (i, len(p), k)
        assert np.array_equal(seg[:, 1], em), (i, len(p), k)


def test_batch_mixed_patterns_vs_oracle(pm):
    import torch
    rng = np.random.default_rng(3)
    n = 3 * 4096 * 32 + 999
    text = synth.markov_text(n, seed=12)
    pats, ks = [], []
    for _ in range(37):
        m = int(rng.choice([1, 3, 12, 20, 31, 32, 33, 64, 100, 300, 600]))
        pats.append(synth.random_pattern(m, m // 10, rng))
        ks.append(int(rng.choice([0, 1, 2, 3, 4, 5, 6, 7, 9, m // 8, m, m + 2])))
    pats.append("N" * 40); ks.append(0)
    pats.append("-" * 5); ks.append(5)
    occ = synth.Occupancy()
    for p, k in zip(pats[:10], ks[:10]):
        synth.plant(text, p, 3, min(k, len(p)), rng, occ)
    t = pm.pm_encode_text(text)
    cps = [pm.pm_compile_pattern(p) for p in pats]
    cap = pm.pm_search(t, cps, ks).total + 10
    for opts in (dict(), dict(group=1, ws_below=-1), dict(group=5, ws_below=7, tiles=3),
                 dict(ws_below=1, ps1_below=-1, tiles=4), dict(ps1_below=5, ps2_below=64, tiles=2),
                 dict(ws_below=-1, ps1_below=-1, ps2_below=-1, group=16)):
        b = pm.Batch(t, cps, ks, capacity=cap, **opts)
        res = b.run()
        torch.cuda.synchronize()
        assert res.total <= cap
        check_against_oracle(res, text, pats, ks)


def test_batch_equals_per_pattern_search(pm):
    import torch
    pats, ks = workloads.batched_patterns(200, seed=5)
    text = synth.markov_text(2_000_000, seed=14)
    t = pm.pm_encode_text(text)
    cps = [pm.pm_compile_pattern(p) for p in pats]
    ref = pm.pm_search(t, cps, ks)
    b = pm.Batch(t, cps, ks, capacity=ref.total + 10)
    res = b.run()
    torch.cuda.synchronize()
    rh, ro = ref.numpy()
    bh, bo = res.numpy()
    assert np.array_equal(ro, bo)
    assert np.array_equal(rh, bh)
    # a second run over the same scratch gives the same answer
    res2 = b.run()
    torch.cuda.synchronize()
    assert np.array_equal(res2.numpy()[0], bh)


def test_batch_graph_replay(pm):
    import torch
    pats, ks = workloads.batched_patterns(64, seed=9)
    text = synth.markov_text(1_000_000, seed=15)
    t = pm.pm_encode_text(text)
    cps = [pm.pm_compile_pattern(p) for p in pats]
    ref = pm.pm_search(t, cps, ks)
    g = pm.GraphedBatch(pm.Batch(t, cps, ks, capacity=ref.total + 10))
    for _ in range(3):
        out = g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(out.numpy()[0], ref.numpy()[0])
        assert np.array_equal(out.numpy()[1], ref.numpy()[1])


def test_batch_overflow_reports_total(pm):
    import torch
    text = synth.uniform_text(50_000, seed=16)
    t = pm.pm_encode_text(text)
    cps = [pm.pm_compile_pattern("ACGTN"), pm.pm_compile_pattern("GG")]
    ks = [2, 1]
    exp = sum(oracle.search(text, p, k)[0].size for p, k in zip(["ACGTN", "GG"], ks))
    b = pm.Batch(t, cps, ks, capacity=100)
    res = b.run()
    torch.cuda.synchronize()
    assert res.total == exp > 100
    b2 = pm.Batch(t, cps, ks, capacity=exp)
    res = b2.run()
    torch.cuda.synchronize()
    check_against_oracle(res, text, ["ACGTN", "GG"], ks)


def test_batched_recipe_reduced(pm):
    """The BATCHED recipe (4096 patterns, m log-uniform 12..512, k in 0..m/8,
    planted copies) at n = 4e6, checked against the per-pattern launches for
    every pattern and against the oracle for 300 of them."""
    import torch
    w = workloads.batched(n=4_000_000, count=4096)
    t = pm.pm_encode_text(w.text)
    cps = [pm.pm_compile_pattern(p) for p in w.patterns]
    ks = [kk[0] for kk in w.ks]
    ref = pm.pm_search(t, cps, ks)
    b = pm.Batch(t, cps, ks, capacity=ref.total + 10)
    res = b.run()
    torch.cuda.synchronize()
    assert np.array_equal(res.numpy()[1], ref.numpy()[1])
    assert np.array_equal(res.numpy()[0], ref.numpy()[0])
    h, off = res.numpy()
    rng = np.random.default_rng(0)
    for i in rng.choice(len(cps), size=300, replace=False):
        seg = h[int(off[i]):int(off[i + 1])]
        el, em = oracle.search(w.text, w.patterns[i], ks[i])
        assert np.array_equal(seg[:, 0], el) and np.array_equal(seg[:, 1], em)
        found = dict(zip(seg[:, 0].tolist(), seg[:, 1].tolist()))
        for loc, s in w.planted[i]:
            assert found.get(loc) == s


def test_autotuner_on_device(pm, tmp_path):
    """The tuner measures on the device, caches, installs a valid AUTO table
    and batch options; searches under them give the oracle's hits."""
    import torch
    from paper_1611_06115_gb300 import tune
    rng = np.random.default_rng(61)
    text = synth.markov_text(4 * 4096 * 32 + 17, seed=61)
    t = pm.pm_encode_text(text)
    path = str(tmp_path / "tune.json")
    builtin = pm.pm_get_auto_variants()
    try:
        r = tune.tune_variants(t, kmax=24, ms=(40, 200), reps=1, cache=path)
        assert not r["cached"] and pm.pm_get_auto_variants(24) == r["table"]
        assert tune.tune_variants(t, kmax=24, cache=path)["cached"]
        pats = [synth.random_pattern(m, m // 10, rng) for m in (12, 40, 64, 100, 300)] * 4
        ks = [0, 3, 6, 12, 19, 25, 40, 2, 5, 8, 17, 30, 1, 4, 9, 21, 33, 45, 0, 16]
        cps = [pm.pm_compile_pattern(p) for p in pats]
        ref = pm.pm_search(t, cps, ks)
        check_against_oracle(ref, text, pats, ks)
        b = tune.tune_batch(t, cps, ks, ref.total + 10, sample=8, reps=1, cache=path)
        assert not b["cached"] and len(b["log"]) > 5
        batch = pm.Batch(t, cps, ks, capacity=ref.total + 10, **b["options"])
        res = batch.run()
        torch.cuda.synchronize()
        check_against_oracle(res, text, pats, ks)
    finally:
        pm.pm_set_auto_variants([])
    assert pm.pm_get_auto_variants() == builtin


def test_search_ex_one_launch_equals_per_pattern(pm):
    """pm_search_ex with batch options: one persistent launch, stream-ordered
    scratch; same hits as one launch per pattern, for device and host
    outputs, with `needed` and an overflow."""
    import torch
    rng = np.random.default_rng(71)
    text = synth.markov_text(3 * 4096 * 32 + 501, seed=71)
    t = pm.pm_encode_text(text)
    pats = [synth.random_pattern(int(m), int(m) // 10, rng)
            for m in rng.choice([8, 20, 33, 64, 150, 400], size=40)]
    ks = [int(x) for x in rng.integers(0, 12, size=40)]
    cps = [pm.pm_compile_pattern(p) for p in pats]
    ref = pm.pm_search(t, cps, ks)
    check_against_oracle(ref, text, pats, ks)
    for opts in ({}, {"ws_below": -1, "tiles": 2}, {"ps1_below": 3, "group": 16}):
        got = pm.pm_search_ex(t, cps, ks, batch=opts)
        assert got.total == ref.total
        assert np.array_equal(got.numpy()[0], ref.numpy()[0])
        assert np.array_equal(got.numpy()[1], ref.numpy()[1])
        host = pm.pm_search_ex(t, cps, ks, out="host", batch=opts)
        assert np.array_equal(host.numpy()[0], ref.numpy()[0])
        asyn = pm.pm_search_ex(t, cps, ks, capacity=ref.total, sync=False, batch=opts)
        torch.cuda.synchronize()
        assert asyn.total == ref.total and np.array_equal(asyn.numpy()[0], ref.numpy()[0])
    # too small a capacity: the library reports the count it needs
    small = pm.pm_search_ex(t, cps, ks, batch={}, capacity=None)
    assert small.total == ref.total
    with pytest.raises(pm.PmError) as e:
        pm.pm_search_ex(t, cps, ks, batch={}, capacity=max(ref.total // 2, 1), out="host")
    assert e.value.status == pm.PM_E_OVERFLOW
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * len(cps))]
    with pytest.raises(pm.PmError) as e:
        pm.pm_search_ex(t, cps, ks, batch={}, events=ev)
    assert e.value.status == pm.PM_E_ARG
