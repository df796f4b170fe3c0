"""Multi-GPU search by text sharding (Sec. 2.6 across devices).

The paper parallelises by cutting the text into one piece per thread, each
piece overlapping the next by m-1 symbols.  Across GPUs the same cut is made
once: rank r of `world` owns the window starts [start_r, end_r) of the
global text and holds the text piece [start_r, end_r + max_m - 1), so every
window it owns is complete for every pattern up to max_m.  Each rank codes
and searches only its own piece (no remote reads, no collective on the data
path), keeps the hits it owns (a window starting in the overlap belongs to
the next rank) and shifts their locations by start_r.  The one collective is
a gather of the per-rank CSR lists; concatenating them in rank order gives
the global lists, already sorted by location.

`search_fn(piece_ascii, patterns, ks) -> list[(locations, mismatches)]` is
pluggable: the GPU path passes a pm_search over the piece; tests pass the
CPU oracle.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Shard:
    rank: int
    world: int
    start: int       # first owned window start (global)
    end: int         # one past the last owned window start (global)
    piece_end: int   # end of the text piece this rank holds (global, exclusive)

    @property
    def piece_len(self) -> int:
        return self.piece_end - self.start


def shard_of(n: int, max_m: int, world: int, rank: int) -> Shard:
    """Rank `rank`'s share of a text of n symbols for patterns up to max_m."""
    if world < 1 or not 0 <= rank < world or max_m < 1:
        raise ValueError("bad shard arguments")
    per = -(-n // world)
    start = min(n, rank * per)
    end = min(n, start + per)
    return Shard(rank, world, start, end, min(n, end + max_m - 1))


def owned(shard: Shard, locs: np.ndarray, mms: np.ndarray):
    """Keep the hits whose window starts inside the shard; make them global."""
    keep = (locs.astype(np.int64) + shard.start) < shard.end
    return (locs[keep].astype(np.uint64) + np.uint64(shard.start)), mms[keep]


def search_shard(text_piece, shard: Shard, patterns, ks, search_fn):
    """This rank's owned hits per pattern, with global locations."""
    res = search_fn(text_piece, patterns, ks)
    return [owned(shard, np.asarray(l), np.asarray(c)) for l, c in res]


def merge(per_rank):
    """Concatenate per-rank results (list over ranks of lists over patterns)
    in rank order: the global per-pattern lists, sorted by location."""
    npat = len(per_rank[0])
    out = []
    for p in range(npat):
        locs = np.concatenate([r[p][0] for r in per_rank]) if per_rank else np.zeros(0, np.uint64)
        mms = np.concatenate([r[p][1] for r in per_rank]) if per_rank else np.zeros(0, np.uint32)
        out.append((locs, mms))
    return out


def gpu_search_fn(piece, patterns, ks):
    """Per-rank search on this process's current GPU (pm_encode_text of the
    piece, then one pm_search)."""
    from . import api
    t = api.pm_encode_text(piece)
    cps = [api.pm_compile_pattern(p) for p in patterns]
    r = api.pm_search(t, cps, ks)
    return [r.pattern(i) for i in range(len(cps))]


def distributed_search(text_piece, shard: Shard, patterns, ks, search_fn, group=None, dst: int = 0):
    """Search this rank's piece, gather every rank's results on `dst`, return
    the merged global lists there (None elsewhere).  One collective."""
    import torch.distributed as dist
    mine = search_shard(text_piece, shard, patterns, ks, search_fn)
    gathered = [None] * shard.world if shard.rank == dst else None
    dist.gather_object(mine, gathered, dst=dst, group=group)
    return merge(gathered) if shard.rank == dst else None
