"""Parity at the benchmark's full size, in the benchmark's launch configuration.

The GENOME workload (n = 3.1e9 Markov text, m in {32, 128, 1024}, k in
{0, 4, 16}, 100 planted copies per pattern) is searched on the GPU exactly as
bench.py does (one pm_search call, nine scan launches).  The oracle cannot
scan 3.1e9 windows nine times in a test, so the check is, per search:
  * every planted copy with s <= k is reported with count exactly s;
  * every reported window's count, recomputed by the oracle, equals the
    reported count and is <= k;
  * three slices of 6e6 windows (start, middle, end of the text) match the
    oracle's search of the same slices window for window;
  * 20,000 random unreported windows have oracle counts > k.
"""
import numpy as np
import pytest

import oracle

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N = 3_100_000_000
SLICE = 6_000_000


@pytest.fixture(scope="module")
def genome_run():
    import torch
    import paper_1611_06115_gb300 as pm
    import bench

    pats = bench.genome_patterns()
    host = torch.empty(N, dtype=torch.uint8, pin_memory=True)
    text = host.numpy()
    planted = bench.build_text(N, 0, text, pats)
    t = pm.pm_encode_text(host)
    cps = {p: pm.pm_compile_pattern(p) for p in pats}
    ents = bench.entries(pats)
    r = pm.pm_search(t, [cps[p] for p, _ in ents], [k for _, k in ents])
    res = [r.pattern(i) for i in range(len(ents))]
    del r, t
    return text, pats, planted, ents, res


def test_full_size_planted_and_reported(genome_run):
    text, pats, planted, ents, res = genome_run
    for (p, k), (loc, mm) in zip(ents, res):
        assert (np.diff(loc.astype(np.int64)) > 0).all()
        assert (mm <= k).all()
        found = dict(zip(loc.tolist(), mm.tolist()))
        for l, s in planted[pats.index(p)]:
            if s <= k:
                assert found.get(l) == s, (len(p), k, l, s)
        # every reported window, recounted by the oracle
        assert np.array_equal(oracle.counts_at(text, p, loc.astype(np.uint64)), mm)


def test_full_size_slices_window_for_window(genome_run):
    text, pats, planted, ents, res = genome_run
    for (p, k), (loc, mm) in zip(ents, res):
        m = len(p)
        nwin = N - m + 1
        for a in (0, nwin // 2 - SLICE // 2, nwin - SLICE):
            b = a + SLICE
            el, em = oracle.search(text[a:b + m - 1], p, k)
            sel = (loc >= a) & (loc < b)
            assert np.array_equal(loc[sel] - a, el), (m, k, a)
            assert np.array_equal(mm[sel], em), (m, k, a)


def test_full_size_unreported_windows_exceed_k(genome_run):
    text, pats, planted, ents, res = genome_run
    rng = np.random.default_rng(77)
    for (p, k), (loc, mm) in zip(ents, res):
        m = len(p)
        cand = rng.integers(0, N - m + 1, size=25000, dtype=np.uint64)
        cand = np.setdiff1d(cand, loc.astype(np.uint64))[:20000]
        assert (oracle.counts_at(text, p, cand) > k).all()


# ---- LARGE at full size: n = 3.1e9, m in {1e4, 1e5}, k in {0, 100, 1000} ----

@pytest.fixture(scope="module")
def large_run():
    import torch
    import paper_1611_06115_gb300 as pm
    from synth import workloads

    host = torch.empty(N, dtype=torch.uint8, pin_memory=True)
    w = workloads.large(n=N, out=host.numpy())
    t = pm.pm_encode_text(host)
    res = {}
    for p in w.patterns:
        c = pm.pm_compile_pattern(p)
        r = pm.pm_search(t, [c] * 3, list(w.meta["ks"]))
        res[p] = [r.pattern(i) for i in range(3)]
    del t
    return host.numpy(), w, res


def test_large_full_size_planted_reported_and_sampled(large_run):
    """Every planted copy with s <= k is reported with its count; every
    reported count is the oracle's; 2000 random unreported windows exceed k;
    a slice of 2e5 windows matches the oracle window for window (k = 0, 100)."""
    text, w, res = large_run
    rng = np.random.default_rng(78)
    for p, pl in zip(w.patterns, w.planted):
        m = len(p)
        for k, (loc, mm) in zip(w.meta["ks"], res[p]):
            found = dict(zip(loc.tolist(), mm.tolist()))
            for l, s in pl:
                if s <= k:
                    assert found.get(l) == s, (m, k, l, s)
            assert (mm <= k).all()
            if loc.size:
                assert np.array_equal(oracle.counts_at(text, p, loc.astype(np.uint64)), mm)
            cand = rng.integers(0, N - m + 1, size=2100, dtype=np.uint64)
            cand = np.setdiff1d(cand, loc.astype(np.uint64))[:2000]
            assert (oracle.counts_at(text, p, cand) > k).all()
            if k <= 100:
                a = int(rng.integers(0, N - m + 1 - 200_000))
                el, em = oracle.search(text[a:a + 200_000 + m - 1], p, k)
                sel = (loc >= a) & (loc < a + 200_000)
                assert np.array_equal(loc[sel] - a, el) and np.array_equal(mm[sel], em), (m, k, a)
