"""The named synthetic workloads (seeded), built from the generators in ``synth``.

Each builder returns plain data (ASCII text as a uint8 array, pattern strings,
k values, planted copies); nothing here knows how matching is computed.

PR1      n = 1,000,000 i.i.d. uniform text (seed 1); one m = 16 pattern with
         exactly 4 two/three-letter class positions (seed 2); 20 planted copies
         with 0-3 substitutions; k in {0, 2}.
GENOME   n = 3.1e9 order-2 Markov text, 41 % GC; patterns m in {32, 128, 1024}
         with round(0.1 m) class positions; k in {0, 4, 16}; 100 planted copies
         per pattern with s uniform in 0..16.
BATCHED  n = 1e9 Markov text; 4096 patterns, m log-uniform in 12..512,
         k uniform in 0..m//8, round(0.1 m) class positions, one planted copy
         per pattern with s uniform in 0..k.
LARGE    n = 3.1e9 Markov text; m in {10,000; 100,000}, 5 % class positions,
         k in {0, 100, 1000}; 10 planted copies per pattern, s uniform in
         0..500 (half the largest k).
SERVING  Poisson arrivals at 2000 queries/s, m log-uniform in 16..4096,
         k uniform in 0..8, over the resident GENOME text.

Every builder takes ``n`` so that tests can run the same recipe at a size the
oracle finishes in seconds.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import (Occupancy, log_uniform_lengths, markov_text, plant, poisson_arrivals,
               random_pattern, uniform_text)

GENOME_N = 3_100_000_000
BATCHED_N = 1_000_000_000


@dataclass
class Workload:
    name: str
    text: np.ndarray                      # uint8 ASCII
    patterns: list[str]
    ks: list[list[int]]                   # k values to run, per pattern
    planted: list[list[tuple[int, int]]]  # (location, substitutions) per pattern
    meta: dict = field(default_factory=dict)


def pr1(n: int = 1_000_000) -> Workload:
    text = uniform_text(n, seed=1)
    rng = np.random.default_rng(2)
    pat = random_pattern(16, 4, rng)
    pl = plant(text, pat, 20, 3, rng)
    return Workload("PR1", text, [pat], [[0, 2]], [pl],
                    {"n": n, "m": 16, "class_positions": 4, "copies": 20})


def genome_patterns(seed: int = 11, ms=(32, 128, 1024)) -> list[str]:
    rng = np.random.default_rng(seed)
    return [random_pattern(m, int(round(0.1 * m)), rng) for m in ms]


def genome(n: int = GENOME_N, seed: int = 3, copies: int = 100, s_max: int = 16,
           ms=(32, 128, 1024), ks=(0, 4, 16), out: np.ndarray | None = None) -> Workload:
    text = markov_text(n, seed, out=out)
    pats = genome_patterns(seed + 8, ms)
    rng = np.random.default_rng(seed + 16)
    occ = Occupancy()
    planted = [plant(text, p, copies, s_max, rng, occ) for p in pats]
    return Workload("GENOME", text, pats, [list(ks) for _ in pats], planted,
                    {"n": n, "ms": list(ms), "ks": list(ks), "copies": copies,
                     "s_max": s_max, "gc": 0.41})


def batched_patterns(count: int = 4096, seed: int = 21, lo: int = 12, hi: int = 512,
                     k_div: int = 8) -> tuple[list[str], list[int]]:
    rng = np.random.default_rng(seed)
    ms = log_uniform_lengths(count, lo, hi, rng)
    pats = [random_pattern(int(m), int(round(0.1 * m)), rng) for m in ms]
    ks = [int(rng.integers(0, int(m) // k_div + 1)) for m in ms]
    return pats, ks


def batched(n: int = BATCHED_N, count: int = 4096, seed: int = 5,
            out: np.ndarray | None = None) -> Workload:
    text = markov_text(n, seed, out=out)
    pats, ks = batched_patterns(count, seed + 16)
    rng = np.random.default_rng(seed + 32)
    occ = Occupancy()
    planted = [plant(text, p, 1, k, rng, occ) for p, k in zip(pats, ks)]
    return Workload("BATCHED", text, pats, [[k] for k in ks], planted,
                    {"n": n, "count": count, "m_range": [12, 512], "k": "uniform 0..m//8"})


def large(n: int = GENOME_N, seed: int = 7, ms=(10_000, 100_000), ks=(0, 100, 1000),
          copies: int = 10, out: np.ndarray | None = None) -> Workload:
    text = markov_text(n, seed, out=out)
    rng = np.random.default_rng(seed + 8)
    pats = [random_pattern(m, int(round(0.05 * m)), rng) for m in ms]
    occ = Occupancy()
    s_max = max(ks) // 2
    planted = [plant(text, p, copies, s_max, rng, occ) for p in pats]
    return Workload("LARGE", text, pats, [list(ks) for _ in pats], planted,
                    {"n": n, "ms": list(ms), "ks": list(ks), "copies": copies, "s_max": s_max})


@dataclass
class Query:
    arrival: float
    pattern: str
    k: int


def serving_queries(rate: float = 2000.0, duration: float = 10.0, seed: int = 31,
                    lo: int = 16, hi: int = 4096, k_max: int = 8) -> list[Query]:
    rng = np.random.default_rng(seed)
    times = poisson_arrivals(rate, duration, rng)
    ms = log_uniform_lengths(times.size, lo, hi, rng)
    out = []
    for t, m in zip(times, ms):
        pat = random_pattern(int(m), int(round(0.1 * m)), rng)
        out.append(Query(float(t), pat, int(rng.integers(0, k_max + 1))))
    return out
