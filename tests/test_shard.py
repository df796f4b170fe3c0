"""Text sharding across ranks (CPU): shard ranges cover every window exactly
once with the m-1 overlap; a world of 2 and 3 gloo ranks, each searching
only its piece, gathers exactly the single-text result (the oracle stands in
for the per-rank GPU search)."""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
import synth
from paper_1611_06115_gb300 import shard as sh

PATTERNS = ["ACGTMRWSACGT", "GATTACA", "N" * 5 + "CG", "A"]
KS = [3, 1, 0, 0]


def oracle_fn(piece, pats, ks):
    return [oracle.search(piece, p, k) for p, k in zip(pats, ks)]


def test_shards_cover_every_window_once():
    for n in (1, 7, 100, 1001):
        for world in (1, 2, 3, 8):
            for max_m in (1, 5, 40):
                s = [sh.shard_of(n, max_m, world, r) for r in range(world)]
                assert s[0].start == 0 and s[-1].end == n
                for a, b in zip(s, s[1:]):
                    assert a.end == b.start
                for x in s:
                    assert x.piece_end == min(n, x.end + max_m - 1)


def test_sharded_equals_whole_in_process():
    text = synth.markov_text(5000, seed=41)
    whole = oracle_fn(text, PATTERNS, KS)
    max_m = max(len(p) for p in PATTERNS)
    for world in (1, 2, 3, 7):
        per_rank = []
        for r in range(world):
            s = sh.shard_of(text.size, max_m, world, r)
            per_rank.append(sh.search_shard(text[s.start:s.piece_end], s, PATTERNS, KS, oracle_fn))
        got = sh.merge(per_rank)
        for (gl, gm), (el, em) in zip(got, whole):
            assert np.array_equal(gl, el.astype(np.uint64)) and np.array_equal(gm, em)


def _worker(rank, world, port, n, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        text = synth.markov_text(n, seed=42)
        max_m = max(len(p) for p in PATTERNS)
        s = sh.shard_of(n, max_m, world, rank)
        # each rank generates only its own piece, as a GPU rank would
        piece = synth.markov_text(s.piece_len, seed=42, start=s.start)
        assert np.array_equal(piece, text[s.start:s.piece_end])
        out = sh.distributed_search(piece, s, PATTERNS, KS, oracle_fn)
        if rank == 0:
            whole = oracle_fn(text, PATTERNS, KS)
            ok = all(np.array_equal(gl, el.astype(np.uint64)) and np.array_equal(gm, em)
                     for (gl, gm), (el, em) in zip(out, whole))
            q.put(ok)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_gather_the_whole_result(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + world * 7 + (os.getpid() % 500)
    procs = [ctx.Process(target=_worker, args=(r, world, port, 1_000_000, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    assert q.get(timeout=5) is True
