"""Serving scheduler (CPU): admission by memory, continuous batching, re-runs
after an output overflow, latency accounting; results equal a solo search.
A stand-in backend answers each batch with the oracle after a delay."""
import time

import numpy as np

import oracle
import synth
from paper_1611_06115_gb300 import serve


class FakeBackend:
    """Completes a batch `delay` seconds after launch, with oracle results;
    a batch whose output exceeds its capacity reports counts but no hits."""

    def __init__(self, text, delay=0.01):
        self.text = text
        self.delay = delay
        self.launched = []

    @staticmethod
    def bytes_for(reqs, n):
        return 16 * sum(r.capacity for r in reqs) + 1000 * len(reqs)

    def launch(self, reqs, slot):
        res = [oracle.search(self.text, r.pattern, r.k, threads=1) for r in reqs]
        self.launched.append([r.qid for r in reqs])
        return (time.perf_counter() + self.delay, res, sum(r.capacity for r in reqs))

    @staticmethod
    def ready(h):
        return time.perf_counter() >= h[0]

    @staticmethod
    def collect(h, reqs):
        counts = [int(x[0].size) for x in h[1]]
        if sum(counts) > h[2]:
            return counts, [None] * len(reqs)
        return counts, h[1]


def test_expected_hits_model():
    n = 10_000_000
    # k >= m: every window
    assert serve.expected_hits("ACGT", 4, n) == n - 3
    # all-N matches everywhere
    assert abs(serve.expected_hits("NNNN", 0, n) - (n - 3)) < 1e-6 * n
    # one letter, k = 0: P(letter) per window
    assert abs(serve.expected_hits("A", 0, n) - 0.295 * n) < 1e-6 * n
    # monotone in k
    e = [serve.expected_hits("ACGTACGTACGTACGT", k, n) for k in range(6)]
    assert all(a <= b for a, b in zip(e, e[1:]))


def test_expected_hits_against_enumeration():
    """The grouped-binomial form equals the probability mass of all texts of
    length m with at most k mismatches, enumerated letter by letter."""
    import itertools
    letters = "ACGT"
    n = 1000
    for pat in ("ACG", "RYKN", "AAWSB", "TTTTT", "HDVBMM"):
        m = len(pat)
        for k in range(m + 1):
            mass = 0.0
            for t in itertools.product(letters, repeat=m):
                mm = sum(1 for p, c in zip(pat, t) if c not in serve.CLASS_LETTERS[p])
                if mm <= k:
                    pr = 1.0
                    for c in t:
                        pr *= serve.LETTER_P[c]
                    mass += pr
            assert abs(serve.expected_hits(pat, k, n) - (n - m + 1) * mass) < 1e-9 * n, (pat, k)


def test_expected_hits_long_pattern_matches_position_recursion():
    """For a long pattern with classes, the grouped form agrees with the
    position-by-position Poisson-binomial recursion."""
    rng = np.random.default_rng(5)
    alphabet = list(serve.CLASS_LETTERS)
    pat = "".join(rng.choice(alphabet, size=300))
    n = 10_000_000
    for k in (0, 3, 40, 120, 200):
        dist = np.zeros(k + 1)
        dist[0] = 1.0
        for ch in pat:
            q = 1.0 - sum(serve.LETTER_P[a] for a in serve.CLASS_LETTERS[ch])
            dist[1:] = dist[1:] * (1.0 - q) + dist[:-1] * q
            dist[0] *= 1.0 - q
        want = (n - len(pat) + 1) * dist.sum()
        got = serve.expected_hits(pat, k, n)
        assert abs(got - want) <= 1e-9 * max(want, 1.0), (k, got, want)


def test_continuous_batching_and_solo_equality():
    text = synth.markov_text(200_000, seed=21)
    rng = np.random.default_rng(21)
    be = FakeBackend(text, delay=0.02)
    srv = serve.Server(be, n=text.size, slots=2, max_batch=4, mem_budget=1 << 40)
    queries = []
    for i in range(24):
        m = int(rng.integers(6, 60))
        queries.append((0.005 * i, synth.random_pattern(m, m // 10, rng), int(rng.integers(0, 5))))
    stats = serve.run_trace(srv, queries)
    assert stats["completed"] == 24
    assert stats["max_concurrent_batches"] == 2          # both slots busy at once
    assert stats["batches"] >= 24 // 4                   # batches formed as queries arrived
    for r in srv.done:
        el, em = oracle.search(text, r.pattern, r.k)
        assert np.array_equal(r.hits[0], el) and np.array_equal(r.hits[1], em)
        assert r.latency >= 0.02
    assert stats["p99_ms"] >= stats["p50_ms"] > 0


def test_memory_budget_limits_inflight():
    text = synth.uniform_text(50_000, seed=22)
    be = FakeBackend(text, delay=0.01)
    one = 16 * serve.capacity_for("ACGTACGTAC", 1, text.size) + 1000
    srv = serve.Server(be, n=text.size, slots=8, max_batch=1, mem_budget=int(2.5 * one))
    for _ in range(10):
        srv.submit("ACGTACGTAC", 1)
    peak = 0
    while not srv.idle():
        srv.step()
        peak = max(peak, len(srv.flights))
        time.sleep(0.001)
    assert peak == 2 and len(srv.done) == 10


def test_overflow_reruns_with_exact_count():
    text = synth.uniform_text(20_000, seed=23)
    be = FakeBackend(text, delay=0.0)
    srv = serve.Server(be, n=text.size, slots=1, max_batch=8, mem_budget=1 << 40)
    r = srv.submit("ACG", 1)
    r.capacity = 5  # far too small on purpose
    srv.drain()
    el, _ = oracle.search(text, "ACG", 1)
    assert r.retries == 1 and r.count == el.size and np.array_equal(r.hits[0], el)


def test_queue_depth_reported_and_grows_under_overload():
    text = synth.markov_text(100_000, seed=23)
    rng = np.random.default_rng(23)
    slow = FakeBackend(text, delay=0.05)
    srv = serve.Server(slow, n=text.size, slots=1, max_batch=1, mem_budget=1 << 40)
    qs = [(0.002 * i, synth.random_pattern(12, 1, rng), 1) for i in range(40)]
    st = serve.run_trace(srv, qs)
    assert st["completed"] == 40
    assert st["queue_depth_max"] >= 10 and st["queue_depth_mean"] > 1.0


def test_cancel_queued_and_running_queries():
    text = synth.markov_text(50_000, seed=24)
    be = FakeBackend(text, delay=0.05)
    srv = serve.Server(be, n=text.size, slots=1, max_batch=1, mem_budget=1 << 40)
    a = srv.submit("ACGTACGT", 1)
    b = srv.submit("TTGACCAA", 1)
    c = srv.submit("GGCCAATT", 0)
    srv.step()                      # a starts; b and c wait
    assert a.status == "running" and b.status == "queued"
    assert srv.cancel(b) and b.status == "cancelled"
    assert srv.cancel(a)            # running: its results will be dropped
    srv.drain(poll=0.001)
    launched = [q for batch in be.launched for q in batch]
    assert b.qid not in launched and a.qid in launched
    assert [r.qid for r in srv.done] == [c.qid]
    assert {r.qid for r in srv.cancelled} == {a.qid, b.qid}
    assert not srv.cancel(c)        # already finished


def test_queries_past_their_deadline_expire_unstarted():
    text = synth.markov_text(50_000, seed=25)
    be = FakeBackend(text, delay=0.03)
    srv = serve.Server(be, n=text.size, slots=1, max_batch=1, mem_budget=1 << 40)
    rs = [srv.submit("ACGTACGT", 1, timeout=0.05) for _ in range(8)]
    srv.drain(poll=0.001)
    launched = {q for batch in be.launched for q in batch}
    assert len(srv.expired) > 0 and len(srv.done) + len(srv.expired) == 8
    assert all(r.qid not in launched and r.status == "expired" for r in srv.expired)
    assert all(r.status == "done" for r in srv.done)


def test_expected_hits_takes_the_text_letter_frequencies():
    """The admission model uses the frequencies it is given: a text of only
    A and T makes a C or G position mismatch every window, and the
    frequencies come from letter counts in Table 1 order."""
    n = 10_000
    f = serve.letter_freqs([500, 0, 0, 500])
    assert f == {"A": 0.5, "C": 0.0, "G": 0.0, "T": 0.5}
    assert serve.expected_hits("C", 0, n, f) == 0.0
    assert abs(serve.expected_hits("A", 0, n, f) - 0.5 * n) < 1e-9 * n
    assert abs(serve.expected_hits("W", 0, n, f) - n) < 1e-9 * n   # W = A or T
    assert serve.letter_freqs([0, 0, 0, 0]) == serve.LETTER_P
    # the server takes the backend's frequencies for its capacities
    class B:
        def letter_freqs(self):
            return f
    srv = serve.Server(B(), n=n)
    r = srv.submit("SSSS", 0)   # S = C or G: never matches this text
    assert srv.freqs is f and r.capacity == serve.capacity_for("SSSS", 0, n, f) == 4096


def test_results_go_to_the_consumer_and_can_be_released():
    """on_result sees every completed query with its hits; with keep_hits
    False the server keeps counts and times only."""
    text = synth.markov_text(20_000, seed=61)
    be = FakeBackend(text, delay=0.0)
    seen = []
    srv = serve.Server(be, n=text.size, slots=2, max_batch=4, mem_budget=1 << 40,
                       on_result=lambda r: seen.append((r.qid, r.count, r.hits)), keep_hits=False)
    for p, k in (("ACGTAC", 1), ("GGATCC", 0), ("TTRYAA", 2)):
        srv.submit(p, k, arrival=0.0)
    srv.drain()
    assert sorted(q for q, _, _ in seen) == [0, 1, 2]
    for qid, count, hits in seen:
        assert hits is not None and len(hits[0]) == count
    assert all(r.hits is None and r.count >= 0 for r in srv.done)


def test_released_batches_go_back_to_the_backend():
    """With keep_hits False every finished batch is handed back (release)
    after its results were delivered; with keep_hits True only batches whose
    output did not fit are."""
    text = synth.markov_text(20_000, seed=62)

    class Releasing(FakeBackend):
        def __init__(self, *a, **k):
            super().__init__(*a, **k)
            self.released = []

        def release(self, h):
            self.released.append(h)

    for keep in (False, True):
        be = Releasing(text, delay=0.0)
        srv = serve.Server(be, n=text.size, slots=2, max_batch=2, mem_budget=1 << 40, keep_hits=keep)
        for p, k in (("ACGTAC", 1), ("GGATCC", 0), ("TTRYAA", 2), ("ACGTNN", 1)):
            srv.submit(p, k, arrival=0.0)
        srv.drain()
        assert len(srv.done) == 4
        assert len(be.released) == (len(be.launched) if not keep else 0)


def test_steady_rate_counts_completions_inside_the_arrival_period():
    """steady_qps: completions between 10 % and 100 % of the arrival period
    per second of that interval; a server that keeps up reports about the
    offered rate there."""
    text = synth.markov_text(50_000, seed=63)
    be = FakeBackend(text, delay=0.001)
    srv = serve.Server(be, n=text.size, slots=4, max_batch=2, mem_budget=1 << 40)
    queries = [(0.005 * i, "ACGTAC", 1) for i in range(60)]  # 200 q/s for 0.3 s
    st = serve.run_trace(srv, queries)
    assert st["completed"] == 60
    assert 150 <= st["steady_qps"] <= 250, st["steady_qps"]
