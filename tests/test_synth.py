"""The seeded input generators (CPU only)."""
import numpy as np

import oracle
import synth
from synth import workloads


def test_markov_reproducible_across_thread_counts():
    a = synth.markov_text(3_000_000, seed=4, threads=1)
    b = synth.markov_text(3_000_000, seed=4, threads=7)
    assert np.array_equal(a, b)
    c = synth.markov_text(3_000_000, seed=5, threads=4)
    assert not np.array_equal(a, c)
    assert set(np.unique(a).tolist()) <= set(b"ACGT")


def test_markov_range_is_a_slice():
    full = synth.markov_text(5_000_000, seed=2)
    for a, b in ((0, 10), (1_048_570, 1_048_600), (123_456, 3_210_000), (4_999_000, 5_000_000)):
        assert np.array_equal(synth.markov_text(b - a, seed=2, start=a), full[a:b])


def test_markov_gc_and_cpg():
    t = synth.markov_text(20_000_000, seed=3)
    assert abs(synth.gc_fraction(t) - 0.41) < 0.002
    # CpG is depleted relative to GpC
    s = t.tobytes()
    assert s.count(b"CG") < 0.5 * s.count(b"GC")


def test_pattern_recipe():
    rng = np.random.default_rng(0)
    p = synth.random_pattern(100, 10, rng)
    assert len(p) == 100
    assert sum(ch in synth.TWO_THREE_LETTER for ch in p) == 10
    assert all(ch in "ACGT" + synth.TWO_THREE_LETTER for ch in p)


def test_planted_copies_have_exactly_s_mismatches():
    rng = np.random.default_rng(1)
    t = synth.uniform_text(200_000, seed=1)
    pats = [synth.random_pattern(m, m // 10, rng) for m in (16, 50, 300)]
    occ = synth.Occupancy()
    for p in pats:
        pl = synth.plant(t, p, 25, min(12, len(p)), rng, occ)
        locs = [a for a, _ in pl]
        assert oracle.counts_at(t, p, locs).tolist() == [s for _, s in pl]
    iv = sorted(occ.iv)
    assert all(b <= c for (_, b), (c, _) in zip(iv, iv[1:]))


def test_pr1_recipe():
    w = workloads.pr1()
    assert w.text.size == 1_000_000 and len(w.patterns[0]) == 16
    assert sum(ch in synth.TWO_THREE_LETTER for ch in w.patterns[0]) == 4
    assert len(w.planted[0]) == 20 and all(0 <= s <= 3 for _, s in w.planted[0])
    w2 = workloads.pr1()
    assert np.array_equal(w.text, w2.text) and w.patterns == w2.patterns


def test_batched_recipe():
    pats, ks = workloads.batched_patterns(4096)
    ms = np.array([len(p) for p in pats])
    assert ms.min() >= 12 and ms.max() <= 512
    assert 100 < ms.mean() < 170
    assert all(0 <= k <= len(p) // 8 for p, k in zip(pats, ks))


def test_serving_arrivals():
    q = workloads.serving_queries(rate=2000.0, duration=1.0)
    assert 1800 < len(q) < 2200
    assert all(0 <= x.k <= 8 and 16 <= len(x.pattern) <= 4096 for x in q)
