"""Serving on the GPU: queries that arrive while others run are admitted as
slots free up, batches overlap on the device, and every query's result in
the mix is bit-identical to a search of that query alone."""
import numpy as np
import pytest

import synth
from synth import workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("batch,to_host,keep", ((None, False, True), ({}, False, True), (None, True, True),
                                                (None, True, False)),
                         ids=("launch-per-query", "one-launch-per-batch", "hits-to-host",
                              "hits-to-host-buffers-reused"))
def test_served_results_equal_solo_searches(batch, to_host, keep):
    import torch
    import paper_1611_06115_gb300 as pm
    from paper_1611_06115_gb300 import serve

    text_np = synth.markov_text(200_000_000, seed=31)
    text = pm.pm_encode_text(text_np)
    # a burst: arrivals outpace the device, so batches queue and overlap
    qs = workloads.serving_queries(rate=20000.0, duration=0.01, seed=32, hi=600)
    queries = [(q.arrival, q.pattern, q.k) for q in qs]
    backend = serve.GpuBackend(text, slots=3, batch=batch, copy_to_host=to_host)
    # with keep_hits False the hits are valid during on_result only (their
    # pinned buffers are reused by later batches): the consumer copies them
    copies = {}
    srv = serve.Server(backend, n=text.n, slots=3, max_batch=8, mem_budget=4 << 30, keep_hits=keep,
                       on_result=None if keep else (lambda r: copies.__setitem__(r.qid, r.hits.clone())))
    # admission sizes outputs with the text's own letter frequencies
    counts = text.letter_counts()
    assert srv.freqs == serve.letter_freqs(counts) and abs(sum(srv.freqs.values()) - 1) < 1e-12
    stats = serve.run_trace(srv, queries)
    torch.cuda.synchronize()
    assert stats["completed"] == len(queries)
    assert stats["max_concurrent_batches"] >= 2
    by_pattern = {}
    for r in srv.done:
        cp = by_pattern.setdefault(r.pattern, pm.pm_compile_pattern(r.pattern))
        alone = pm.pm_search(text, [cp], [r.k]).pattern(0)
        hits = r.hits if keep else copies[r.qid]
        assert (hits.device.type == "cpu") == to_host
        got = hits.cpu().numpy().view(np.uint32).reshape(-1, 2)
        assert r.count == alone[0].size
        assert np.array_equal(got[:, 0], alone[0]) and np.array_equal(got[:, 1], alone[1])
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
