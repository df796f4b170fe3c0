"""The multi-GPU path of Sec. 2.6 with the GPU search on each rank: two gloo
ranks (processes) each code and search only their own piece of the text on
the GPU (shard.gpu_search_fn), keep the windows they own, and one gather
merges the per-rank lists on rank 0, which compares them element by element
with the oracle on the whole text.  This machine has one GPU, so both ranks
share it; their kernels never wait on each other (the only exchange is the
host-side gather)."""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu

PATTERNS = ["ACGTMRWSACGT", "GATTACAGATTACA", "N" * 5 + "CG", "TTAGGGTTAGGGTTAGGGTTAGGGTTAGGGTTAGGGHH"]
KS = [3, 2, 0, 6]
N = 3_000_001


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        import synth
        from paper_1611_06115_gb300 import shard as sh
        torch.cuda.set_device(0)
        max_m = max(len(p) for p in PATTERNS)
        s = sh.shard_of(N, max_m, world, rank)
        piece = synth.markov_text(s.piece_len, seed=43, start=s.start)  # only this rank's piece
        out = sh.distributed_search(piece, s, PATTERNS, KS, sh.gpu_search_fn)
        torch.cuda.synchronize()
        if rank == 0:
            text = synth.markov_text(N, seed=43)
            ok = True
            for (gl, gm), p, k in zip(out, PATTERNS, KS):
                el, em = oracle.search(text, p, k)
                ok = ok and np.array_equal(gl, el.astype(np.uint64)) and np.array_equal(gm, em)
            q.put((ok, [int(x[0].size) for x in out]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gpu_ranks_gather_the_whole_result(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29700 + world * 11 + (os.getpid() % 400)
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    ok, sizes = q.get(timeout=5)
    assert ok, sizes
    assert sum(sizes) > 0
